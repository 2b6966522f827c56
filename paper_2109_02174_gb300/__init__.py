"""Python binding of libfbp (include/fbp.h): GPU filtered backprojection on GB300.

Argument marshalling only: every step of the reconstruction runs in the CUDA
kernels of libfbp.so.  PyTorch supplies device memory and streams.  There is no
CPU fallback: if libfbp.so is missing or cannot load, every call raises.

Low-level names mirror the C ABI (fbp_plan, fbp_filter, fbp_backproject,
fbp_reconstruct, radon_forward, ...); ``Plan`` wraps them for tensors.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
# FBP_LIBRARY may name another build of the library (the index-checking
# debug build, libfbp_checked.so)
LIB_PATH = os.environ.get("FBP_LIBRARY") or os.path.join(PKG, "libfbp.so")

FBP_OK, FBP_ERR_INVALID_ARG, FBP_ERR_ALIGNMENT, FBP_ERR_OUT_OF_MEMORY = 0, 1, 2, 3
FBP_ERR_BUDGET, FBP_ERR_CUDA, FBP_ERR_TIMEOUT, FBP_ERR_UNSUPPORTED = 4, 5, 6, 7
FBP_ERR_BOUNDS = 8
STATUS_NAMES = {0: "FBP_OK", 1: "FBP_ERR_INVALID_ARG", 2: "FBP_ERR_ALIGNMENT",
                3: "FBP_ERR_OUT_OF_MEMORY", 4: "FBP_ERR_BUDGET", 5: "FBP_ERR_CUDA",
                6: "FBP_ERR_TIMEOUT", 7: "FBP_ERR_UNSUPPORTED", 8: "FBP_ERR_BOUNDS"}
FBP_FILTER_RAM_LAK, FBP_FILTER_SHEPP_LOGAN, FBP_FILTER_NONE = 0, 1, 2
FBP_F32, FBP_F64, FBP_F16 = 0, 1, 2
FBP_ACC_PLAIN, FBP_ACC_KAHAN = 0, 1
FBP_PATH_AUTO, FBP_PATH_TOEPLITZ_TC, FBP_PATH_FFT, FBP_PATH_DIRECT = 0, 1, 2, 3
FBP_BATCH_FILTER, FBP_BATCH_BACKPROJECT = 1, 2


class FbpError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class fbp_batch_io(ctypes.Structure):
    _fields_ = [("sino", ctypes.c_void_p), ("ld_sino", ctypes.c_int),
                ("image", ctypes.c_void_p), ("workspace", ctypes.c_void_p)]


class fbp_request(ctypes.Structure):
    _fields_ = [("n_pix", ctypes.c_int), ("n_angles", ctypes.c_int), ("n_det", ctypes.c_int),
                ("det_spacing", ctypes.c_double), ("filter", ctypes.c_int),
                ("host_sino", ctypes.c_void_p), ("host_image", ctypes.c_void_p)]


class fbp_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("failed", ctypes.c_longlong), ("admission_stalls", ctypes.c_longlong),
                ("waves", ctypes.c_longlong), ("max_waves_in_flight", ctypes.c_int),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("span_s", ctypes.c_double), ("bytes_in_use", ctypes.c_size_t),
                ("peak_bytes", ctypes.c_size_t), ("budget_bytes", ctypes.c_size_t)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class fbp_options(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int) for name in
                ("dtype", "q_storage", "accumulate", "filter_path", "fft_len",
                 "tile_x", "tile_y", "angle_chunk")] + [("i0", ctypes.c_double),
                                                        ("point_pairs", ctypes.c_int)]


class fbp_fdk_geometry(ctypes.Structure):
    _fields_ = [("n_angles", ctypes.c_int), ("nv", ctypes.c_int), ("nu", ctypes.c_int),
                ("R", ctypes.c_double), ("du", ctypes.c_double), ("dv", ctypes.c_double),
                ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int)]


class fbp_tuning(ctypes.Structure):
    _fields_ = [("options", fbp_options), ("filter_ms", ctypes.c_double),
                ("backproject_ms", ctypes.c_double), ("from_cache", ctypes.c_int)]


_lock = threading.Lock()
_lib = None

# name -> (argtypes); every entry point returns an int status except fbp_last_error.
_P = ctypes.c_void_p
_I = ctypes.c_int
_SIGS = {
    "fbp_options_default": [ctypes.POINTER(fbp_options)],
    "fbp_plan": [ctypes.POINTER(_P), _I, _I, _I, ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                 _I, ctypes.POINTER(fbp_options)],
    "fbp_plan_destroy": [_P],
    "fbp_workspace_bytes": [_P, ctypes.POINTER(ctypes.c_size_t)],
    "fbp_plan_query": [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "fbp_filter": [_P, _P, _I, _P, _P],
    "fbp_backproject": [_P, _P, _P, _P],
    "fbp_reconstruct": [_P, _P, _I, _P, _P, _P],
    "radon_forward": [_P, _P, _P, _P],
    "fbp_device_status": [_P],
    "fbp_reconstruct_static": [_P, _P, _I, _P, _P],
    "fbp_batch_build": [ctypes.POINTER(_P), ctypes.POINTER(_P), _I, ctypes.POINTER(fbp_batch_io),
                        _P],
    "fbp_batch_build_parts": [ctypes.POINTER(_P), ctypes.POINTER(_P), _I,
                              ctypes.POINTER(fbp_batch_io), _I, _P],
    "fbp_batch_launch": [_P, _P],
    "fbp_batch_kernel_count": [_P, ctypes.POINTER(_I)],
    "fbp_quality_scratch_bytes": [_I, _I, ctypes.POINTER(ctypes.c_size_t)],
    "fbp_quality": [_P, _P, _I, _I, _I, ctypes.c_double, _P, ctypes.c_size_t, _P, _P],
    "fbp_volume_from_slices": [ctypes.POINTER(_P), _I, ctypes.POINTER(ctypes.c_double), _I,
                               ctypes.POINTER(ctypes.c_double), _I, _P, _P],
    "fbp_fdk_plan": [ctypes.POINTER(_P), ctypes.POINTER(fbp_fdk_geometry),
                     ctypes.POINTER(ctypes.c_double), _I],
    "fbp_fdk_plan_destroy": [_P],
    "fbp_fdk_workspace_bytes": [_P, ctypes.POINTER(ctypes.c_size_t)],
    "fbp_fdk_reconstruct": [_P, _P, _P, _P, _P],
    "fbp_fdk_status": [_P],
    "fbp_reconstruct_many": [ctypes.POINTER(_P), _I, ctypes.POINTER(fbp_batch_io), _P],
    "fbp_autotune": [_I, _I, _I, ctypes.c_double, _I, ctypes.POINTER(fbp_options), _I,
                     ctypes.POINTER(fbp_tuning)],
    "fbp_server_create": [ctypes.POINTER(_P), ctypes.c_size_t, _I, _I],
    "fbp_server_warm": [_P, _I, _I, _I, ctypes.c_double, _I],
    "fbp_server_submit": [_P, ctypes.POINTER(fbp_request), ctypes.POINTER(ctypes.c_longlong)],
    "fbp_server_cancel": [_P, ctypes.c_longlong],
    "fbp_server_wait": [_P, ctypes.c_longlong, ctypes.c_double],
    "fbp_server_request_info": [_P, ctypes.c_longlong, ctypes.POINTER(_I),
                                ctypes.POINTER(ctypes.c_double)],
    "fbp_server_drain": [_P, ctypes.c_double],
    "fbp_server_get_stats": [_P, ctypes.POINTER(fbp_server_stats)],
    "fbp_server_destroy": [_P],
    "fbp_batch_run_host": [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _P],
    "fbp_batch_status": [_P],
    "fbp_batch_destroy": [_P],
    "fbp_set_wait_limit": [ctypes.c_double],
    "fbp_test_withhold_arrival": [_I, _I],
    "fbp_test_shrink_window": [_I],
}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libfbp.so (built by ``paper_2109_02174_gb300.build``); raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise ImportError(f"libfbp.so not found at {path}: run __graft_entry__.build()")
            lib = ctypes.CDLL(path)
            for name, argtypes in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = argtypes
                fn.restype = ctypes.c_int
            lib.fbp_last_error.argtypes = []
            lib.fbp_last_error.restype = ctypes.c_char_p
            _lib = lib
    return _lib


def fbp_last_error() -> str:
    return load_library().fbp_last_error().decode()


def _check(status: int):
    if status != FBP_OK:
        raise FbpError(status, fbp_last_error())


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _stream(stream) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


# ------------------------------------------------------------ raw C-ABI names
def fbp_options_default() -> fbp_options:
    o = fbp_options()
    _check(load_library().fbp_options_default(ctypes.byref(o)))
    return o


def fbp_plan(n_pix, n_angles, n_det, angles=None, det_spacing=1.0, filter=FBP_FILTER_RAM_LAK,
             opt: fbp_options | None = None) -> int:
    lib = load_library()
    h = _P()
    arr = None
    if angles is not None:
        vals = [float(a) for a in angles]
        arr = (ctypes.c_double * len(vals))(*vals)
    _check(lib.fbp_plan(ctypes.byref(h), int(n_pix), int(n_angles), int(n_det),
                        arr, float(det_spacing), int(filter),
                        ctypes.byref(opt) if opt is not None else None))
    return h.value


def fbp_plan_destroy(plan: int):
    _check(load_library().fbp_plan_destroy(plan))


def fbp_workspace_bytes(plan: int) -> int:
    v = ctypes.c_size_t()
    _check(load_library().fbp_workspace_bytes(plan, ctypes.byref(v)))
    return v.value


def fbp_plan_query(plan: int) -> tuple[int, int, int]:
    a, b, c = _I(), _I(), _I()
    _check(load_library().fbp_plan_query(plan, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def fbp_filter(plan: int, sino_ptr: int, ld_sino: int, filtered_ptr: int, stream: int):
    _check(load_library().fbp_filter(plan, sino_ptr, ld_sino, filtered_ptr, stream))


def fbp_backproject(plan: int, filtered_ptr: int, image_ptr: int, stream: int):
    _check(load_library().fbp_backproject(plan, filtered_ptr, image_ptr, stream))


def fbp_reconstruct(plan: int, sino_ptr: int, ld_sino: int, image_ptr: int, workspace_ptr: int,
                    stream: int):
    _check(load_library().fbp_reconstruct(plan, sino_ptr, ld_sino, image_ptr, workspace_ptr,
                                          stream))


def radon_forward(plan: int, image_ptr: int, sino_ptr: int, stream: int):
    _check(load_library().radon_forward(plan, image_ptr, sino_ptr, stream))


def fbp_reconstruct_static(plan: int, sino_ptr: int, ld_sino: int, image_ptr: int, stream: int):
    """fbp_reconstruct with the library's static scratch array (no allocation)."""
    _check(load_library().fbp_reconstruct_static(plan, sino_ptr, ld_sino, image_ptr, stream))


def fbp_device_status(plan: int):
    _check(load_library().fbp_device_status(plan))


FBP_TEST_WITHHOLD_NONE, FBP_TEST_WITHHOLD_BACKPROJECT, FBP_TEST_WITHHOLD_FILTER_TC = 0, 1, 2


def fbp_set_wait_limit(seconds: float):
    """Limit of the kernels' bounded device waits on the current device (0 = 2 s)."""
    _check(load_library().fbp_set_wait_limit(float(seconds)))


def fbp_test_withhold_arrival(kernel: int, stage: int = 0):
    """Test-only: the first CTA of later launches of `kernel` withholds the
    arrival of pipeline stage `stage` (FBP_TEST_WITHHOLD_NONE switches it off)."""
    _check(load_library().fbp_test_withhold_arrival(int(kernel), int(stage)))


def fbp_test_shrink_window(pairs: int):
    """Test-only: in the index-checking debug build the kernels check window
    indices against the staged width minus `pairs` (0: the true width)."""
    _check(load_library().fbp_test_shrink_window(int(pairs)))


def fbp_batch_build(plans, ios, parts: int = FBP_BATCH_FILTER | FBP_BATCH_BACKPROJECT) -> int:
    n = len(plans)
    parr = (_P * n)(*plans)
    iarr = (fbp_batch_io * n)(*ios)
    h = _P()
    _check(load_library().fbp_batch_build_parts(ctypes.byref(h), parr, n, iarr, int(parts), None))
    return h.value


def fbp_reconstruct_many(plans, ios, stream: int):
    n = len(plans)
    _check(load_library().fbp_reconstruct_many((_P * n)(*plans), n, (fbp_batch_io * n)(*ios),
                                               stream))


def fbp_batch_run_host(batch: int, host_sino_ptrs, host_image_ptrs, stream: int):
    n = len(host_sino_ptrs)
    s = (_P * n)(*host_sino_ptrs)
    i = (_P * n)(*host_image_ptrs)
    _check(load_library().fbp_batch_run_host(batch, s, i, stream))


def fbp_batch_launch(batch: int, stream: int):
    _check(load_library().fbp_batch_launch(batch, stream))


def fbp_batch_status(batch: int):
    _check(load_library().fbp_batch_status(batch))


def fbp_batch_kernel_count(batch: int) -> int:
    n = _I()
    _check(load_library().fbp_batch_kernel_count(batch, ctypes.byref(n)))
    return n.value


def fbp_batch_destroy(batch: int):
    _check(load_library().fbp_batch_destroy(batch))


def fbp_autotune(n_pix, n_angles, n_det, det_spacing=1.0, filter=FBP_FILTER_RAM_LAK,
                 base: fbp_options | None = None, batch: int = 8) -> dict:
    """Tuned options for a geometry (see fbp.h): a dict of option fields plus
    filter_ms / backproject_ms (per slice) and from_cache."""
    t = fbp_tuning()
    _check(load_library().fbp_autotune(int(n_pix), int(n_angles), int(n_det), float(det_spacing),
                                       int(filter), ctypes.byref(base) if base else None,
                                       int(batch), ctypes.byref(t)))
    d = {name: getattr(t.options, name) for name, _ in fbp_options._fields_}
    d.update(filter_ms=t.filter_ms, backproject_ms=t.backproject_ms, from_cache=t.from_cache)
    return d


def fbp_quality_scratch_bytes(rows: int, cols: int) -> int:
    n = ctypes.c_size_t()
    _check(load_library().fbp_quality_scratch_bytes(int(rows), int(cols), ctypes.byref(n)))
    return n.value


def quality(image, reference, dynamic_range: float = 0.0, stream=None) -> tuple[float, float]:
    """(PSNR dB, SSIM) of a 2-D float32 device image against a reference of
    the same shape and row stride, computed on the GPU (see fbp.h: Eq. 3 with
    MAX = max|reference|; Eq. 4 with 11x11 Gaussian windows, sigma 1.5,
    K1 = 0.01, K2 = 0.03; L = dynamic_range or the reference's span).
    Synchronises the stream to return the values."""
    import torch
    assert image.shape == reference.shape and image.dim() == 2
    assert image.stride(1) == 1 and reference.stride(1) == 1
    assert image.stride(0) == reference.stride(0)
    rows, cols = image.shape
    scratch = torch.empty(fbp_quality_scratch_bytes(rows, cols), dtype=torch.uint8,
                          device=image.device)
    out = torch.empty(2, dtype=torch.float64, device=image.device)
    s = _stream(stream)
    _check(load_library().fbp_quality(_ptr(image), _ptr(reference), rows, cols, image.stride(0),
                                      float(dynamic_range), _ptr(scratch), scratch.numel(),
                                      _ptr(out), s))
    if stream is None:
        torch.cuda.current_stream().synchronize()
    else:
        stream.synchronize()
    v = out.cpu()
    return float(v[0]), float(v[1])


def volume(slices, z, z_out, out=None, stream=None):
    """3D volume [M][n][n] (float32, device) from 2-D slices (device tensors
    [n][n], e.g. Batch.images) at strictly increasing positions z, by linear
    interpolation along z onto the planes z_out (inside [z[0], z[-1]])."""
    import torch
    slices = list(slices)
    n = slices[0].shape[0]
    for t in slices:
        assert t.shape == (n, n) and t.dtype == torch.float32 and t.is_contiguous()
    zs = (ctypes.c_double * len(slices))(*[float(v) for v in z])
    zo = (ctypes.c_double * len(z_out))(*[float(v) for v in z_out])
    ptrs = (_P * len(slices))(*[_ptr(t) for t in slices])
    if out is None:
        out = torch.empty((len(z_out), n, n), dtype=torch.float32, device=slices[0].device)
    _check(load_library().fbp_volume_from_slices(ptrs, len(slices), zs, n, zo, len(z_out),
                                                 _ptr(out), _stream(stream)))
    return out


class FdkPlan:
    """FDK cone-beam plan (see fbp.h): projections [n_angles][nv][nu] on a
    virtual detector through the axis, source radius R, volume [nz][ny][nx]."""

    def __init__(self, n_angles: int, nv: int, nu: int, R: float, nx: int, ny: int, nz: int,
                 du: float = 1.0, dv: float = 1.0, beta=None, filter: int = FBP_FILTER_RAM_LAK):
        self.geometry = fbp_fdk_geometry(int(n_angles), int(nv), int(nu), float(R), float(du),
                                         float(dv), int(nx), int(ny), int(nz))
        b = None
        if beta is not None:
            assert len(beta) == n_angles
            b = (ctypes.c_double * n_angles)(*[float(v) for v in beta])
        h = _P()
        _check(load_library().fbp_fdk_plan(ctypes.byref(h), ctypes.byref(self.geometry), b,
                                           int(filter)))
        self.handle = h.value
        n = ctypes.c_size_t()
        _check(load_library().fbp_fdk_workspace_bytes(self.handle, ctypes.byref(n)))
        self.workspace_bytes = n.value

    def close(self):
        if getattr(self, "handle", None):
            load_library().fbp_fdk_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reconstruct(self, proj, out=None, workspace=None, stream=None):
        import torch
        g = self.geometry
        assert proj.shape == (g.n_angles, g.nv, g.nu) and proj.is_contiguous()
        assert proj.dtype == torch.float32
        if out is None:
            out = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float32, device=proj.device)
        if workspace is None:
            workspace = torch.empty(max(self.workspace_bytes, 16), dtype=torch.uint8,
                                    device=proj.device)
        _check(load_library().fbp_fdk_reconstruct(self.handle, _ptr(proj), _ptr(out),
                                                  _ptr(workspace), _stream(stream)))
        return out

    def device_status(self):
        _check(load_library().fbp_fdk_status(self.handle))


# ------------------------------------------------------------ tensor wrapper
class Plan:
    """A reconstruction plan bound to torch tensors on the current CUDA device."""

    def __init__(self, n_pix: int, n_angles: int, n_det: int, angles=None,
                 det_spacing: float = 1.0, filter: int = FBP_FILTER_RAM_LAK,
                 autotune: bool = False, batch_hint: int = 8, **options):
        opt = fbp_options_default()
        for k, v in options.items():
            setattr(opt, k, float(v) if k == "i0" else int(v))
        self.tuning = None
        if autotune:
            self.tuning = fbp_autotune(n_pix, n_angles, n_det, det_spacing, filter, opt,
                                       batch_hint)
            for k in ("filter_path", "fft_len", "tile_x", "tile_y", "angle_chunk"):
                setattr(opt, k, int(self.tuning[k]))
        self.n_pix, self.n_angles, self.n_det = int(n_pix), int(n_angles), int(n_det)
        self.det_spacing = float(det_spacing)
        self.filter_type = int(filter)
        self.options = opt
        self.handle = fbp_plan(n_pix, n_angles, n_det, angles, det_spacing, filter, opt)
        self.q_pitch, self.fft_len, self.filter_path = fbp_plan_query(self.handle)
        self.workspace_bytes = fbp_workspace_bytes(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            fbp_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.options.dtype == FBP_F64 else torch.float32

    @property
    def q_dtype(self):
        import torch
        if self.options.q_storage == FBP_F16:
            return torch.float16
        return self.dtype

    def empty_filtered(self):
        import torch
        return torch.empty((self.n_angles, self.q_pitch), dtype=self.q_dtype, device="cuda")

    def empty_image(self):
        import torch
        return torch.empty((self.n_pix, self.n_pix), dtype=self.dtype, device="cuda")

    def empty_workspace(self):
        import torch
        return torch.empty(max(self.workspace_bytes, 16), dtype=torch.uint8, device="cuda")

    def filter(self, sino, out=None, stream=None):
        assert sino.dim() == 2 and sino.shape[0] == self.n_angles and sino.stride(1) == 1
        out = self.empty_filtered() if out is None else out
        fbp_filter(self.handle, _ptr(sino), sino.stride(0), _ptr(out), _stream(stream))
        return out

    def backproject(self, filtered, out=None, stream=None):
        out = self.empty_image() if out is None else out
        fbp_backproject(self.handle, _ptr(filtered), _ptr(out), _stream(stream))
        return out

    def reconstruct(self, sino, out=None, workspace=None, stream=None):
        assert sino.dim() == 2 and sino.shape[0] == self.n_angles and sino.stride(1) == 1
        out = self.empty_image() if out is None else out
        ws = self.empty_workspace() if workspace is None else workspace
        fbp_reconstruct(self.handle, _ptr(sino), sino.stride(0), _ptr(out), _ptr(ws),
                        _stream(stream))
        return out

    def radon_forward(self, image, out=None, stream=None):
        import torch
        out = torch.empty((self.n_angles, self.n_det), dtype=torch.float32, device="cuda") \
            if out is None else out
        radon_forward(self.handle, _ptr(image), _ptr(out), _stream(stream))
        return out

    def device_status(self):
        fbp_device_status(self.handle)


class Batch:
    """A graph-captured batch over (plan, sinogram, image, workspace) tensors.

    The tensors are bound at construction: refill the sinograms in place and
    call ``launch()`` again for new data.  Keep plans and tensors alive.
    """

    def __init__(self, plans, sinos, images=None, workspaces=None,
                 parts: int = FBP_BATCH_FILTER | FBP_BATCH_BACKPROJECT):
        self.plans = list(plans)
        self.sinos = list(sinos)
        self.images = list(images) if images is not None else [p.empty_image() for p in self.plans]
        self.workspaces = list(workspaces) if workspaces is not None else \
            [p.empty_workspace() for p in self.plans]
        ios = [fbp_batch_io(_ptr(s), s.stride(0), _ptr(i), _ptr(w))
               for s, i, w in zip(self.sinos, self.images, self.workspaces)]
        self.handle = fbp_batch_build([p.handle for p in self.plans], ios, parts)
        self.updates = sum(p.n_pix * p.n_pix * p.n_angles for p in self.plans)

    def launch(self, stream=None):
        fbp_batch_launch(self.handle, _stream(stream))
        return self.images

    def run_host(self, host_sinos, host_images, stream=None):
        """Host sinograms in, host images out (pinned CPU tensors), one stream."""
        fbp_batch_run_host(self.handle, [_ptr(h) for h in host_sinos],
                           [_ptr(h) for h in host_images], _stream(stream))

    def status(self):
        fbp_batch_status(self.handle)

    @property
    def kernel_count(self) -> int:
        """Kernel launches per launch() (the kernel nodes of the batch graph)."""
        return fbp_batch_kernel_count(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            fbp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching reconstruction server (fbp_server_* in libfbp).

    submit() takes host tensors (pin them: the copies are asynchronous) that
    must stay alive until the request is done.
    """

    QUEUED, ADMITTED, RUNNING, DONE, FAILED, CANCELLED = range(6)

    def __init__(self, hbm_budget_bytes: int, max_wave: int = 32, n_streams: int = 2):
        h = _P()
        _check(load_library().fbp_server_create(ctypes.byref(h), int(hbm_budget_bytes),
                                                int(max_wave), int(n_streams)))
        self.handle = h.value
        self._keep = {}

    def warm(self, n_pix, n_angles, n_det, det_spacing=1.0, filter=FBP_FILTER_RAM_LAK):
        _check(load_library().fbp_server_warm(self.handle, int(n_pix), int(n_angles),
                                              int(n_det), float(det_spacing), int(filter)))

    def submit(self, sino, image, n_pix, det_spacing=1.0, filter=FBP_FILTER_RAM_LAK) -> int:
        assert sino.is_contiguous() and image.is_contiguous()
        r = fbp_request(int(n_pix), int(sino.shape[0]), int(sino.shape[1]), float(det_spacing),
                        int(filter), _ptr(sino), _ptr(image))
        rid = ctypes.c_longlong()
        _check(load_library().fbp_server_submit(self.handle, ctypes.byref(r), ctypes.byref(rid)))
        self._keep[rid.value] = (sino, image)
        return rid.value

    def cancel(self, rid: int):
        _check(load_library().fbp_server_cancel(self.handle, int(rid)))

    def wait(self, rid: int, timeout_s: float = 60.0):
        _check(load_library().fbp_server_wait(self.handle, int(rid), float(timeout_s)))
        self._keep.pop(rid, None)

    def info(self, rid: int):
        st, lat = ctypes.c_int(), ctypes.c_double()
        _check(load_library().fbp_server_request_info(self.handle, int(rid), ctypes.byref(st),
                                                      ctypes.byref(lat)))
        return st.value, lat.value

    def drain(self, timeout_s: float = 120.0):
        _check(load_library().fbp_server_drain(self.handle, float(timeout_s)))

    def stats(self) -> dict:
        out = fbp_server_stats()
        _check(load_library().fbp_server_get_stats(self.handle, ctypes.byref(out)))
        return out.as_dict()

    def close(self):
        if getattr(self, "handle", None):
            fbp_check = load_library().fbp_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()
            _check(fbp_check)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
