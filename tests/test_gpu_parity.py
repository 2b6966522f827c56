"""GPU parity: libfbp (through its C ABI) against the FP64 oracle, element by element.

Bars (FP32 path): max |f_gpu - f_oracle| <= 1e-4 * max|f_oracle| and
RMSE <= 2e-5 * max|f_oracle|.  Both sides get the same FP32-rounded sinogram.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

MAX_REL = 1e-4
RMSE_REL = 2e-5
NTHREADS = 16


@pytest.fixture(scope="module")
def fbp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_02174_gb300 import build
    build.build()
    import paper_2109_02174_gb300 as m
    return m


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _np(t):
    import torch
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def to_pairs(Q, pitch, dtype=np.float32):
    """Interpolation-ready rows: pair p = k + 1 holds ((Q[k]+Q[k+1])/2, Q[k+1]-Q[k]),
    k = -1 .. D-1, Q zero outside [0, D); the rest of the row is zero."""
    Q = np.asarray(Q, dtype=np.float64)
    A, D = Q.shape
    z = np.zeros((A, D + 2))
    z[:, 1:D + 1] = Q
    out = np.zeros((A, pitch), dtype=np.float64)
    out[:, 0:2 * (D + 1):2] = 0.5 * (z[:, :-1] + z[:, 1:])
    out[:, 1:2 * (D + 1):2] = z[:, 1:] - z[:, :-1]
    return out.astype(dtype)


def from_pairs(R, D):
    """Q[k] for k = 0 .. D-1: the left end, mid - slope/2, of the segment in pair k + 1."""
    R = np.asarray(R, dtype=np.float64)
    mid = R[:, 2:2 * (D + 1):2]
    slope = R[:, 3:2 * (D + 1):2]
    return mid - 0.5 * slope


def errors(got, ref):
    scale = float(np.abs(ref).max())
    return (float(np.abs(got - ref).max()) / scale,
            float(np.sqrt(np.mean((got - ref) ** 2))) / scale)


def assert_parity(got, ref, max_rel=MAX_REL, rmse_rel=RMSE_REL):
    e_max, e_rms = errors(got, ref)
    assert e_max <= max_rel and e_rms <= rmse_rel, f"max {e_max:.3e} rmse {e_rms:.3e}"


# ---------------------------------------------------------------- filter
PATHS = {"direct": 3, "fft": 2, "tc": 1}
# Filter bars, relative to max|Q|.  FP32 routes: rounding of an FP32 sum.  The
# 3xTF32 route also drops the lo*lo product and the hardware truncates the lo
# parts to tf32 (~2^-21 per product) and accumulates inside the tensor core:
# a few 1e-6 of max|Q| on random rows.
FILTER_ATOL = {"direct": 2e-6, "fft": 2e-6, "tc": 1e-5}


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("kind", [0, 1, 2])
def test_filter_matches_oracle(fbp, kind, path):
    A, D = 37, 211
    P = np.random.default_rng(20 + kind).standard_normal((A, D)).astype(np.float32)
    plan = fbp.Plan(150, A, D, filter=kind, filter_path=PATHS[path])
    assert plan.filter_path == PATHS[path]
    q = _np(plan.filter(_t(P)))
    assert q.shape == (A, plan.q_pitch) and plan.q_pitch % 8 == 0
    assert np.all(q[:, 2 * (D + 1):] == 0.0)
    ref = oracle.filter_rows(P.astype(np.float64), kind, 1.0)
    np.testing.assert_allclose(q, to_pairs(ref, plan.q_pitch, np.float64), rtol=0,
                               atol=FILTER_ATOL[path] * np.abs(ref).max())


@pytest.mark.parametrize("path", sorted(PATHS))
def test_filter_respects_row_stride(fbp, path):
    import torch
    A, D = 9, 50
    big = torch.randn(A, 64, device="cuda")
    plan = fbp.Plan(30, A, D, filter_path=PATHS[path])
    q = _np(plan.filter(big[:, :D]))
    ref = oracle.filter_rows(big[:, :D].double().cpu().numpy(), 0, 1.0)
    np.testing.assert_allclose(from_pairs(q, D), ref, rtol=0,
                               atol=FILTER_ATOL[path] * np.abs(ref).max())


@pytest.mark.parametrize("D,fft_len", [(2899, 0), (4096, 8192), (725, 4096), (1, 0), (2, 16)])
def test_fft_filter_lengths(fbp, D, fft_len):
    """FFT route at its size limits (N = 8192), an explicit longer N, and tiny rows."""
    A = 5
    P = np.random.default_rng(D).standard_normal((A, D)).astype(np.float32)
    plan = fbp.Plan(8, A, D, filter_path=2, fft_len=fft_len)
    assert plan.fft_len >= 2 * D - 1 and plan.fft_len & (plan.fft_len - 1) == 0
    q = _np(plan.filter(_t(P)))
    ref = oracle.filter_rows(P.astype(np.float64), 0, 1.0)
    np.testing.assert_allclose(q, to_pairs(ref, plan.q_pitch, np.float64), rtol=0,
                               atol=2e-6 * np.abs(ref).max())


@pytest.mark.parametrize("A,D", [(720, 725), (300, 2899), (129, 1), (1, 40), (257, 130)])
def test_tensor_core_filter_sizes(fbp, A, D):
    """Toeplitz route on the tensor cores (3xTF32): ragged M and N tiles, one-bin
    rows, a single row, the large detector."""
    P = np.random.default_rng(A + D).standard_normal((A, D)).astype(np.float32)
    plan = fbp.Plan(64, A, D, filter_path=1)
    assert plan.filter_path == 1
    q = _np(plan.filter(_t(P)))
    ref = oracle.filter_rows(P.astype(np.float64), 0, 1.0)
    np.testing.assert_allclose(q, to_pairs(ref, plan.q_pitch, np.float64), rtol=0,
                               atol=FILTER_ATOL["tc"] * np.abs(ref).max())
    plan.device_status()


# ---------------------------------------------------------------- backprojection
@pytest.mark.parametrize("n,A,D,tau", [
    (100, 37, 143, 1.0),     # 4x4 tiles with a ragged edge, 3 angle chunks (last partial)
    (64, 16, 91, 1.0),       # exact tiles, exactly one chunk
    (33, 50, 60, 0.8),       # one-pixel ragged tile, tau < 1
    (70, 21, 70, 1.6),       # tau > 1, detector narrower than the diagonal (zero extension)
])
def test_backproject_matches_oracle(fbp, n, A, D, tau):
    rng = np.random.default_rng(n * 7 + A)
    Q = rng.standard_normal((A, D)).astype(np.float32)
    th = oracle.default_angles(A)
    plan = fbp.Plan(n, A, D, det_spacing=tau)
    got = _np(plan.backproject(_t(to_pairs(Q, plan.q_pitch))))
    ref = oracle.backproject(Q.astype(np.float64), th, tau, n, nthreads=NTHREADS)
    assert_parity(got, ref)


@pytest.mark.parametrize("tile", [(32, 64), (32, 32), (8, 32)])
def test_backproject_tile_shapes(fbp, tile):
    """Every tile shape the plan can pick gives the same image within the bars."""
    n, A = 100, 37
    D = synthetic.det_for(n)
    Q = np.random.default_rng(3).standard_normal((A, D)).astype(np.float32)
    plan = fbp.Plan(n, A, D, tile_x=tile[0], tile_y=tile[1])
    got = _np(plan.backproject(_t(to_pairs(Q, plan.q_pitch))))
    ref = oracle.backproject(Q.astype(np.float64), oracle.default_angles(A), 1.0, n,
                             nthreads=NTHREADS)
    assert_parity(got, ref)


def test_backproject_arbitrary_angles(fbp):
    n, A = 48, 29
    D = synthetic.det_for(n)
    rng = np.random.default_rng(99)
    th = np.sort(rng.uniform(-3.0, 7.0, A))
    Q = rng.standard_normal((A, D)).astype(np.float32)
    plan = fbp.Plan(n, A, D, angles=th)
    got = _np(plan.backproject(_t(to_pairs(Q, plan.q_pitch))))
    ref = oracle.backproject(Q.astype(np.float64), th, 1.0, n, nthreads=NTHREADS)
    assert_parity(got, ref)


@pytest.mark.parametrize("n,A,D", [(1, 1, 1), (1, 3, 2), (2, 1, 4), (5, 3, 9), (8, 1, 3)])
def test_degenerate_sizes(fbp, n, A, D):
    rng = np.random.default_rng(n + 10 * A + 100 * D)
    P = rng.standard_normal((A, D)).astype(np.float32)
    th = oracle.default_angles(A)
    plan = fbp.Plan(n, A, D, filter=1)
    got = _np(plan.reconstruct(_t(P)))
    ref = oracle.fbp(P.astype(np.float64), th, 1.0, 1, n)
    if np.abs(ref).max() == 0:
        assert np.all(got == 0)
    else:
        assert_parity(got, ref)


def test_constant_rows_give_pi_c(fbp):
    n, A = 64, 45
    D = synthetic.det_for(n)
    plan = fbp.Plan(n, A, D)
    got = _np(plan.backproject(_t(to_pairs(np.full((A, D), 1.25), plan.q_pitch))))
    np.testing.assert_allclose(got, math.pi * 1.25, rtol=2e-6)


def test_deterministic_bits(fbp):
    spec = synthetic.SliceSpec(200, 150, synthetic.det_for(200), 8, seed=31)
    sino = _t(synthetic.sinogram(spec))
    plan = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det)
    a = _np(plan.reconstruct(sino))
    b = _np(plan.reconstruct(sino))
    c = _np(fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det).reconstruct(sino))
    assert np.array_equal(a, b) and np.array_equal(a, c)


# ---------------------------------------------------------------- whole FBP on the workloads
def _check_slice(fbp, spec, nthreads=NTHREADS, **opts):
    th = synthetic.default_angles(spec.n_angles)
    sino32 = synthetic.sinogram(spec, th).astype(np.float32)
    plan = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, filter=spec.filter,
                    det_spacing=spec.tau, **opts)
    got = _np(plan.reconstruct(_t(sino32)))
    plan.device_status()
    ref = oracle.fbp(sino32.astype(np.float64), th, spec.tau, spec.filter, spec.n_pix,
                     nthreads=nthreads)
    assert_parity(got, ref)
    return errors(got, ref)


@pytest.mark.parametrize("path", sorted(PATHS))
def test_plain_slice_256(fbp, path):
    """256x256, 180 angles, 363 bins, Ram-Lak (FFT length 1024), 10 ellipses (seed 1)."""
    _check_slice(fbp, synthetic.cfg_plain(), filter_path=PATHS[path], fft_len=1024)


@pytest.mark.parametrize("path", sorted(PATHS))
def test_float_slice_512_noisy(fbp, path):
    """512x512, 720 angles, 725 bins, Shepp-Logan, Poisson I0 = 1e5 (FP32 path)."""
    _check_slice(fbp, synthetic.cfg_float_double(), filter_path=PATHS[path])


def test_large_slice_2048_every_pixel(fbp, large_reference):
    """2048x2048, 2048 angles, 2899 bins (40 ellipses, seed 4), default plan:
    every pixel of the GPU image against the oracle's whole image."""
    spec, th, sino32, ref = large_reference
    plan = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, filter=spec.filter)
    got = _np(plan.reconstruct(_t(sino32)))
    plan.device_status()
    assert_parity(got, ref)


# ---------------------------------------------------------------- precision variants
def test_kahan_accumulation_meets_fp32_bars(fbp):
    """Kahan-compensated sum over angles (2048 x 2048-class angle count on a small image)."""
    spec = synthetic.SliceSpec(256, 2048, synthetic.det_for(256), 10, seed=41)
    e_max, e_rms = _check_slice(fbp, spec, accumulate=1)
    assert e_max <= MAX_REL and e_rms <= RMSE_REL


def test_fp16_pairs_error_is_stated(fbp):
    """FP16-stored (mid, slope) pairs: no bar from the spec; the error is reported.
    The bound below is a regression guard, about six times the measured error
    (max 7e-5, RMSE 1e-5): the storage rounding (2^-11 of each stored value) and
    the FP16 weight fed to the mixed-precision FMA, averaged over 180 angles."""
    import torch
    spec = synthetic.cfg_plain()
    th = synthetic.default_angles(spec.n_angles)
    sino32 = synthetic.sinogram(spec, th).astype(np.float32)
    plan = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, q_storage=2)
    q = plan.filter(_t(sino32))
    assert q.dtype == torch.float16
    got = _np(plan.backproject(q))
    ref = oracle.fbp(sino32.astype(np.float64), th, 1.0, 0, spec.n_pix, nthreads=NTHREADS)
    e_max, e_rms = errors(got, ref)
    print(f"fp16 pairs: max {e_max:.3e} rmse {e_rms:.3e} of max|f|")
    assert e_max < 5e-4 and e_rms < 1e-4


# ---------------------------------------------------------------- FP64 path
FP64_REL = 1e-10


def _fp64_slice(fbp, spec, filter_path=0):
    import torch
    th = synthetic.default_angles(spec.n_angles)
    sino = synthetic.sinogram(spec, th)
    plan = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, filter=spec.filter, dtype=1,
                    filter_path=filter_path)
    assert plan.dtype == torch.float64
    got = plan.reconstruct(torch.from_numpy(sino).cuda())
    torch.cuda.synchronize()
    plan.device_status()
    ref = oracle.fbp(sino, th, 1.0, spec.filter, spec.n_pix, nthreads=NTHREADS)
    return errors(got.cpu().numpy(), ref)


FP64_PATHS = {"fft": 2, "direct": 3}


@pytest.mark.parametrize("path", sorted(FP64_PATHS))
def test_fp64_float_double_slice_512(fbp, path):
    """The float-vs-double configuration on the FP64 GPU path, FFT and direct
    filter: <= 1e-10 of max|f|."""
    e_max, e_rms = _fp64_slice(fbp, synthetic.cfg_float_double(), FP64_PATHS[path])
    print(f"fp64 {path}: max {e_max:.3e} rmse {e_rms:.3e}")
    assert e_max <= FP64_REL


@pytest.mark.parametrize("path", sorted(FP64_PATHS))
@pytest.mark.parametrize("n,A,D", [(3, 2, 5), (33, 17, 40), (70, 21, 60), (65, 33, 93),
                                   (64, 9, 1500)])
def test_fp64_small_and_ragged(fbp, n, A, D, path):
    """Odd angle counts leave the last row of the FFT route's row pairs alone;
    FFT lengths 16, 128 (one radix-2 pass first), 256 and 4096 (the longest
    FP64 FFT, 128 KB of shared memory)."""
    spec = synthetic.SliceSpec(n, A, D, 4, seed=n + A, filter=0)
    e_max, _ = _fp64_slice(fbp, spec, FP64_PATHS[path])
    assert e_max <= FP64_REL


@pytest.mark.parametrize("path", sorted(FP64_PATHS))
@pytest.mark.parametrize("tau", [0.7, 1.6])
def test_fp64_given_angles_and_spacing(fbp, path, tau):
    """Unsorted caller-given angles over a full turn and a non-unit bin width
    (the fixed-point coordinate's table scales cos/tau and sin/tau; at tau =
    1.6 the detector is narrower than the image diagonal)."""
    import torch
    n, A, D = 80, 37, 75
    th = np.random.default_rng(int(10 * tau)).uniform(0.0, 2.0 * np.pi, A)
    P = np.random.default_rng(int(100 * tau)).normal(size=(A, D))
    plan = fbp.Plan(n, A, D, angles=th, det_spacing=tau, filter=1, dtype=1,
                    filter_path=FP64_PATHS[path])
    got = plan.reconstruct(torch.from_numpy(P).cuda())
    torch.cuda.synchronize()
    plan.device_status()
    ref = oracle.fbp(P, th, tau, 1, n, nthreads=NTHREADS)
    e_max, _ = errors(got.cpu().numpy(), ref)
    assert e_max <= FP64_REL


def test_fp64_fft_route_is_the_default_and_matches_direct(fbp):
    """AUTO resolves to the FP64 FFT when its length fits; the two FP64 routes
    give the same filtered pairs to rounding (linear convolution either way)."""
    import torch
    spec = synthetic.SliceSpec(150, 91, synthetic.det_for(150), 6, seed=77, filter=1)
    th = synthetic.default_angles(spec.n_angles)
    sino = torch.from_numpy(synthetic.sinogram(spec, th)).cuda()
    auto = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, filter=1, dtype=1)
    direct = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, filter=1, dtype=1, filter_path=3)
    assert auto.filter_path == 2 and auto.fft_len == 512
    qa, qd = auto.filter(sino), direct.filter(sino)
    torch.cuda.synchronize()
    qa, qd = qa.cpu().numpy(), qd.cpu().numpy()
    assert np.abs(qa - qd).max() <= 1e-12 * np.abs(qd).max()


def test_fp64_rejects_fp32_only_options(fbp):
    with pytest.raises(fbp.FbpError) as e:
        fbp.Plan(64, 10, 91, dtype=1, filter_path=1)
    assert e.value.status == fbp.FBP_ERR_UNSUPPORTED
    with pytest.raises(fbp.FbpError) as e:
        fbp.Plan(64, 10, 91, dtype=1, filter_path=2, fft_len=8192)
    assert e.value.status == fbp.FBP_ERR_UNSUPPORTED
    with pytest.raises(fbp.FbpError) as e:
        fbp.Plan(64, 10, 91, dtype=1, q_storage=2)
    assert e.value.status == fbp.FBP_ERR_UNSUPPORTED


# ---------------------------------------------------------------- Eq. 1 on load
@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("i0", [1e4, 5.0])
def test_intensity_input_matches_oracle(fbp, path, i0):
    """Photon counts in (plan option i0): each filter route converts them to
    line integrals -ln(max(I, 1)/i0) as it loads them; the image matches the
    oracle's conversion followed by its FBP.  At i0 = 5 many rays count zero
    photons, which exercises the one-count floor."""
    import torch
    spec = synthetic.SliceSpec(200, 180, synthetic.det_for(200), 8, seed=31, filter=1, i0=i0,
                               noise_seed=131)
    th = synthetic.default_angles(spec.n_angles)
    counts = synthetic.photon_counts(spec, th)
    if i0 < 100:
        assert (counts == 0).sum() > 200
    plan = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, filter=spec.filter,
                    filter_path=PATHS[path], i0=i0)
    img = plan.reconstruct(torch.from_numpy(counts.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    plan.device_status()
    ref = oracle.fbp(oracle.lambert_beer(counts, i0), th, 1.0, spec.filter, spec.n_pix,
                     nthreads=NTHREADS)
    assert_parity(img.cpu().numpy(), ref)


def test_intensity_input_fp64_path(fbp):
    import torch
    spec = synthetic.SliceSpec(96, 90, synthetic.det_for(96), 6, seed=32, filter=0, i0=50.0,
                               noise_seed=132)
    th = synthetic.default_angles(spec.n_angles)
    counts = synthetic.photon_counts(spec, th)
    plan = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, filter=0, dtype=1, i0=50.0)
    img = plan.reconstruct(torch.from_numpy(counts).cuda())
    torch.cuda.synchronize()
    ref = oracle.fbp(oracle.lambert_beer(counts, 50.0), th, 1.0, 0, spec.n_pix)
    got = img.cpu().numpy()
    assert np.abs(got - ref).max() <= FP64_REL * np.abs(ref).max()


def test_intensity_option_rejects_bad_i0(fbp):
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(fbp.FbpError) as e:
            fbp.Plan(32, 8, 46, i0=bad)
        assert e.value.status == fbp.FBP_ERR_INVALID_ARG


# ---------------------------------------------------------------- projector
def test_radon_forward_matches_oracle(fbp):
    n, A = 57, 33
    D = synthetic.det_for(n)
    th = oracle.default_angles(A)
    img = np.random.default_rng(5).random((n, n)).astype(np.float32)
    plan = fbp.Plan(n, A, D)
    got = _np(plan.radon_forward(_t(img)))
    ref = oracle.forward(img.astype(np.float64), th, D)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-5 * np.abs(ref).max())


def test_gpu_adjoint_pair(fbp):
    """<R x, y> = (A/pi) <x, B y> for radon_forward and the unfiltered backprojection."""
    n, A = 80, 40
    D = synthetic.det_for(n)
    rng = np.random.default_rng(6)
    x = rng.standard_normal((n, n)).astype(np.float32)
    y = rng.standard_normal((A, D)).astype(np.float32)
    plan = fbp.Plan(n, A, D, filter=2)
    Rx = _np(plan.radon_forward(_t(x)))
    By = _np(plan.backproject(_t(to_pairs(y, plan.q_pitch))))
    lhs = float(np.sum(Rx * y))
    rhs = (A / math.pi) * float(np.sum(x.astype(np.float64) * By))
    scale = float(np.sum(np.abs(Rx * y)))
    assert abs(lhs - rhs) <= 1e-5 * scale


# ---------------------------------------------------------------- errors
def test_misaligned_and_null_buffers_are_rejected(fbp):
    import torch
    plan = fbp.Plan(32, 8, 46)
    q = torch.zeros(8 * plan.q_pitch + 4, device="cuda")
    img = torch.zeros(32 * 32 + 4, device="cuda")
    with pytest.raises(fbp.FbpError) as e:
        fbp.fbp_backproject(plan.handle, q.data_ptr() + 4, img.data_ptr(), 0)
    assert e.value.status == fbp.FBP_ERR_ALIGNMENT
    with pytest.raises(fbp.FbpError) as e:
        fbp.fbp_backproject(plan.handle, 0, img.data_ptr(), 0)
    assert e.value.status == fbp.FBP_ERR_INVALID_ARG
    with pytest.raises(fbp.FbpError) as e:
        fbp.fbp_filter(plan.handle, q.data_ptr(), 10, img.data_ptr(), 0)
    assert e.value.status == fbp.FBP_ERR_INVALID_ARG
    plan.device_status()


def test_maximum_sizes_direct_route(fbp):
    """An 8192^2 image with 11587 bins: beyond the FFT route's reach (2 n_det - 1
    > 8192), so the plan takes the direct filter; sampled pixels (and a full
    row through the centre) against the oracle."""
    import torch
    n, A = 8192, 8
    D = synthetic.det_for(n)
    spec = synthetic.SliceSpec(n, A, D, 6, seed=81, filter=0)
    th = synthetic.default_angles(A)
    sino = synthetic.sinogram(spec, th).astype(np.float32)
    plan = fbp.Plan(n, A, D)
    assert plan.filter_path == fbp.FBP_PATH_DIRECT
    img = plan.reconstruct(torch.from_numpy(sino).cuda())
    torch.cuda.synchronize()
    plan.device_status()
    Q = oracle.filter_rows(sino.astype(np.float64), 0, 1.0, nthreads=NTHREADS)
    rng = np.random.default_rng(81)
    rows = np.concatenate([rng.integers(0, n, 400), np.full(512, n // 2)])
    cols = np.concatenate([rng.integers(0, n, 400), np.arange(0, n, 16)])
    ref = oracle.backproject_pixels(Q, th, 1.0, n, rows, cols)
    got = img[torch.from_numpy(rows).cuda(), torch.from_numpy(cols).cuda()].cpu().numpy()
    assert_parity(got.astype(np.float64), ref)


# ---------------------------------------------------------------- point-symmetric tile pairs
@pytest.mark.parametrize("geom", [
    dict(n=256, A=180, D=363, tile=(8, 32)),
    dict(n=128, A=90, D=183, tile=(32, 32)),
    dict(n=128, A=45, D=120, tau=1.6, tile=(32, 64)),
    dict(n=64, A=50, D=120, tau=0.8, tile=(32, 32)),
    dict(n=192, A=120, D=273, tile=(32, 32), q_storage=2),
    dict(n=128, A=360, D=183, tile=(32, 32), accumulate=1),
    dict(n=256, A=180, D=363, tile=(8, 32), accumulate=1),
])
def test_point_pairs_match_oracle(fbp, geom):
    """Plans whose work items are tile pairs mirrored through the image centre
    (one detector position per pixel and partner) meet the bars; their image
    differs from the unpaired plan's only by rounding."""
    g = dict(geom)
    n, A, D = g.pop("n"), g.pop("A"), g.pop("D")
    tau = g.pop("tau", 1.0)
    tx, ty = g.pop("tile")
    spec = synthetic.SliceSpec(n, A, D, 8, seed=77 + n + A, tau=tau)
    th = synthetic.default_angles(A)
    sino32 = synthetic.sinogram(spec, th).astype(np.float32)
    imgs = {}
    for pp in (1, -1):
        plan = fbp.Plan(n, A, D, det_spacing=tau, tile_x=tx, tile_y=ty, point_pairs=pp, **g)
        imgs[pp] = _np(plan.reconstruct(_t(sino32)))
        plan.device_status()
    assert not np.array_equal(imgs[1], imgs[-1])  # the paired path ran
    ref = oracle.fbp(sino32.astype(np.float64), th, tau, 0, n, nthreads=NTHREADS)
    if g.get("q_storage") == 2:
        e_max, e_rms = errors(imgs[1], ref)
        assert e_max < 5e-4 and e_rms < 1e-4
        e2 = errors(imgs[-1], ref)
        assert abs(e_max - e2[0]) < 0.5 * e2[0] + 1e-6
    else:
        assert_parity(imgs[1], ref)


def test_point_pairs_fall_back_where_the_tiling_is_not_symmetric(fbp):
    """n not a multiple of the tile, or a tile grid odd in both directions
    (96 x 96 in 32 x 32 tiles: the centre tile is its own partner): the plan
    keeps single-tile items, the same bits as with the option off."""
    for n, (tx, ty) in ((100, (32, 32)), (96, (32, 32))):
        A, D = 60, synthetic.det_for(n)
        sino = _t(synthetic.sinogram(synthetic.SliceSpec(n, A, D, 6, seed=n)))
        a = _np(fbp.Plan(n, A, D, tile_x=tx, tile_y=ty, point_pairs=1).reconstruct(sino))
        b = _np(fbp.Plan(n, A, D, tile_x=tx, tile_y=ty, point_pairs=-1).reconstruct(sino))
        assert np.array_equal(a, b), n
