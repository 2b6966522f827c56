"""FP64 CPU oracle for parallel-beam FBP (arXiv 2109.02174, Eq. 2).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product package never
imports this module and this module never imports the product package; the
two share no code.

The arithmetic lives in ``fbp_oracle.c`` (plain C, double precision, explicit
loops).  This wrapper only builds it with gcc and marshals numpy arrays.

Functions (each cites the passage it follows in the C source):
  taps(kind, n_det, tau)                      filter H of Q = P * H
  filter_rows(P, kind, tau, nthreads)         Q[i][k] = tau sum_j h(k-j) P[i][j]
  backproject(Q, theta, tau, n, nthreads)     Eq. 2 with the pi/A step
  backproject_pixels(Q, theta, tau, n, r, c)  Eq. 2 at selected pixels
  forward(f, theta, n_det, tau)               transpose of the interpolation
  fbp(P, theta, tau, kind, n, nthreads)       taps + filter + backprojection
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fbp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

RAM_LAK, SHEPP_LOGAN, NONE = 0, 1, 2

# -ffp-contract=off: no fused multiply-add contraction, so the x86 and Arm
# builds round every operation the same way.
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to the source (gcc, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    """Load liboracle.so.  FBP_ORACLE_LIB may name another build of the same
    source (the mutation test points it at deliberately broken copies)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("FBP_ORACLE_LIB")
            if not path:
                build()
                path = _LIB
            lib = ctypes.CDLL(path)
            d = ctypes.POINTER(ctypes.c_double)
            i = ctypes.c_int
            ip = ctypes.POINTER(ctypes.c_int)
            lib.oracle_taps.argtypes = [i, i, ctypes.c_double, d]
            lib.oracle_taps.restype = i
            lib.oracle_filter.argtypes = [d, i, i, i, d, ctypes.c_double, d]
            lib.oracle_filter.restype = None
            lib.oracle_filter_mt.argtypes = [d, i, i, i, d, ctypes.c_double, d, i]
            lib.oracle_filter_mt.restype = None
            lib.oracle_backproject.argtypes = [d, i, i, d, ctypes.c_double, i, d, i]
            lib.oracle_backproject.restype = None
            lib.oracle_backproject_pixels.argtypes = [d, i, i, d, ctypes.c_double, i, ip, ip, i, d]
            lib.oracle_backproject_pixels.restype = None
            lib.oracle_forward.argtypes = [d, i, i, i, d, ctypes.c_double, d]
            lib.oracle_forward.restype = None
            lib.oracle_fbp.argtypes = [d, i, i, i, d, ctypes.c_double, i, i, d, i]
            lib.oracle_fbp.restype = i
            lib.oracle_lambert_beer.argtypes = [d, ctypes.c_long, ctypes.c_double, d]
            lib.oracle_lambert_beer.restype = None
            lib.oracle_psnr.argtypes = [d, d, i, i, d]
            lib.oracle_psnr.restype = None
            lib.oracle_ssim.argtypes = [d, d, i, i, ctypes.c_double]
            lib.oracle_ssim.restype = ctypes.c_double
            lib.oracle_volume.argtypes = [d, i, d, i, d, i, d]
            lib.oracle_volume.restype = i
            lib.oracle_fdk.argtypes = [d, i, i, i, d, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, i, i, i, i, d, i]
            lib.oracle_fdk.restype = i
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def default_angles(n_angles: int) -> np.ndarray:
    """theta_i = i*pi/n_angles, i = 0..n_angles-1 (uniform on [0, pi))."""
    return np.arange(n_angles, dtype=np.float64) * (np.pi / n_angles)


def lambert_beer(I, i0: float) -> np.ndarray:
    """Eq. 1: line integrals p = -ln(max(I, 1) / i0) of measured intensities or
    photon counts I (any shape)."""
    I = _f64(I)
    p = np.empty_like(I)
    _load().oracle_lambert_beer(_dp(I), int(I.size), float(i0), _dp(p))
    return p


def psnr(x, y) -> tuple[float, float, float]:
    """Eq. 3 of image x against reference y (2-D): (PSNR dB, MSE, MAX = max|y|)."""
    x = _f64(x)
    y = _f64(y)
    assert x.shape == y.shape and x.ndim == 2
    out = np.empty(3)
    _load().oracle_psnr(_dp(x), _dp(y), x.shape[0], x.shape[1], _dp(out))
    return float(out[0]), float(out[1]), float(out[2])


def ssim(x, y, dynamic_range: float = 0.0) -> float:
    """Eq. 4, mean over 11x11 Gaussian (sigma 1.5) windows, C1 = (0.01 L)^2,
    C2 = (0.03 L)^2; L <= 0 takes max(y) - min(y)."""
    x = _f64(x)
    y = _f64(y)
    assert x.shape == y.shape and x.ndim == 2
    return float(_load().oracle_ssim(_dp(x), _dp(y), x.shape[0], x.shape[1],
                                     float(dynamic_range)))


def volume(slices, z, z_out) -> np.ndarray:
    """Linear interpolation along z of a slice stack [K][n][n] at positions z
    (strictly increasing) onto planes z_out (inside [z[0], z[-1]]): [M][n][n]."""
    S = _f64(slices)
    z = _f64(z)
    zo = _f64(z_out)
    K, n, n2 = S.shape
    assert n == n2 and z.shape == (K,)
    out = np.empty((zo.size, n, n))
    if _load().oracle_volume(_dp(S), K, _dp(z), n, _dp(zo), zo.size, _dp(out)) != 0:
        raise ValueError("volume: z not increasing or a plane outside the stack")
    return out


def fdk(P, beta, R: float, du: float, dv: float, kind: int, nx: int, ny: int, nz: int,
        nthreads: int = 1) -> np.ndarray:
    """FDK cone-beam reconstruction of projections P [A][nv][nu] (virtual
    detector through the axis, source radius R) into f [nz][ny][nx]."""
    P = _f64(P)
    beta = _f64(beta)
    A, nv, nu = P.shape
    assert beta.shape == (A,)
    f = np.empty((nz, ny, nx))
    if _load().oracle_fdk(_dp(P), A, nv, nu, _dp(beta), float(R), float(du), float(dv),
                          int(kind), nx, ny, nz, _dp(f), int(nthreads)) != 0:
        raise ValueError("fdk: bad argument")
    return f


def taps(kind: int, n_det: int, tau: float = 1.0) -> np.ndarray:
    """h(m) for m = -(n_det-1)..n_det-1 (index m + n_det - 1)."""
    h = np.empty(2 * n_det - 1, dtype=np.float64)
    if _load().oracle_taps(int(kind), int(n_det), float(tau), _dp(h)) != 0:
        raise ValueError("oracle_taps: bad argument")
    return h


def filter_rows(P, kind: int, tau: float = 1.0, nthreads: int = 1) -> np.ndarray:
    P = _f64(P)
    A, D = P.shape
    h = taps(kind, D, tau)
    Q = np.empty((A, D), dtype=np.float64)
    if nthreads == 1:
        _load().oracle_filter(_dp(P), A, D, D, _dp(h), float(tau), _dp(Q))
    else:
        _load().oracle_filter_mt(_dp(P), A, D, D, _dp(h), float(tau), _dp(Q), int(nthreads))
    return Q


def backproject(Q, theta, tau: float, n: int, nthreads: int = 1) -> np.ndarray:
    Q = _f64(Q)
    theta = _f64(theta)
    A, D = Q.shape
    assert theta.shape == (A,)
    f = np.empty((n, n), dtype=np.float64)
    _load().oracle_backproject(_dp(Q), A, D, _dp(theta), float(tau), int(n), _dp(f), int(nthreads))
    return f


def backproject_pixels(Q, theta, tau: float, n: int, rows, cols) -> np.ndarray:
    Q = _f64(Q)
    theta = _f64(theta)
    A, D = Q.shape
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    out = np.empty(rows.shape[0], dtype=np.float64)
    _load().oracle_backproject_pixels(_dp(Q), A, D, _dp(theta), float(tau), int(n),
                                      _ip(rows), _ip(cols), int(rows.shape[0]), _dp(out))
    return out


def forward(f, theta, n_det: int, tau: float = 1.0) -> np.ndarray:
    f = _f64(f)
    theta = _f64(theta)
    n = f.shape[0]
    assert f.shape == (n, n)
    P = np.empty((theta.shape[0], n_det), dtype=np.float64)
    _load().oracle_forward(_dp(f), n, theta.shape[0], int(n_det), _dp(theta), float(tau), _dp(P))
    return P


def fbp(P, theta, tau: float, kind: int, n: int, nthreads: int = 1) -> np.ndarray:
    P = _f64(P)
    theta = _f64(theta)
    A, D = P.shape
    f = np.empty((n, n), dtype=np.float64)
    rc = _load().oracle_fbp(_dp(P), A, D, D, _dp(theta), float(tau), int(kind), int(n), _dp(f),
                            int(nthreads))
    if rc != 0:
        raise ValueError("oracle_fbp: bad argument")
    return f
