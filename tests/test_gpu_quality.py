"""GPU: PSNR (Eq. 3) and SSIM (Eq. 4) on the device match the FP64 oracle's
on the same float32 images: reconstructions against the oracle's image, a
precision variant against the FP32 path, identical images, ragged shapes with
a row stride, images smaller than the SSIM window; the same bits every run."""
import math

import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu
# SSIM: FP64 local statistics on both sides; the device forms 1 - SSIM from the
# differences of the images, the oracle from two-pass variances, so 1 - SSIM
# must agree to 1e-3 of itself, also for near-identical images, plus an
# absolute floor: the oracle sums its n per-window values (each <= 1) in
# FP64, and each addition may round by half an ulp of the running sum, so its
# mean carries up to n * 2^-53 (2.8e-11 for the 502 x 502 windows of a 512^2
# image) -- more than 1 - SSIM itself when two images differ by FP32 rounding.
SSIM_REL_DIST = 1e-3
PSNR_RTOL = 1e-9   # squared differences formed exactly, summed in FP64


@pytest.fixture(scope="module")
def fbp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_02174_gb300 import build
    build.build()
    import paper_2109_02174_gb300 as m
    return m


def _check(fbp, x, y, rng=0.0):
    import torch
    got = fbp.quality(x, y, rng)
    xs = x.double().cpu().numpy()
    ys = y.double().cpu().numpy()
    want_psnr = oracle.psnr(xs, ys)[0]
    want_ssim = oracle.ssim(xs, ys, rng)
    if math.isinf(want_psnr):
        assert math.isinf(got[0])
    else:
        assert got[0] == pytest.approx(want_psnr, rel=PSNR_RTOL)
    if math.isnan(want_ssim):
        assert math.isnan(got[1])
    else:
        windows = (xs.shape[0] - 10) * (xs.shape[1] - 10)
        assert got[1] <= 1.0
        assert abs(got[1] - want_ssim) <= SSIM_REL_DIST * abs(1.0 - want_ssim) + \
            windows * 2.0 ** -53, (1.0 - got[1], 1.0 - want_ssim)
    return got


def test_reconstruction_against_oracle_image(fbp):
    import torch
    spec = synthetic.cfg_plain()
    th = synthetic.default_angles(spec.n_angles)
    sino = synthetic.sinogram(spec, th)
    plan = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, filter=spec.filter)
    img = plan.reconstruct(torch.from_numpy(sino.astype(np.float32)).cuda())
    ref = oracle.fbp(sino.astype(np.float32).astype(np.float64), th, 1.0, spec.filter, spec.n_pix)
    ref_t = torch.from_numpy(ref.astype(np.float32)).cuda()
    db, s = _check(fbp, img, ref_t)
    assert db > 80 and s > 0.9999  # FP32 path against the FP64 oracle


def test_near_identical_pair_distance_from_one_is_relative_accurate(fbp):
    """y = x + 3e-5 (3e-4) x max|x| x noise on a reconstruction: 1 - SSIM is
    about 6e-7 (6e-5), far above the oracle's summation floor (6.7e-12 for
    246 x 246 windows), and must agree to 1e-3 of itself."""
    import torch
    spec = synthetic.cfg_plain()
    x = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det).reconstruct(
        torch.from_numpy(synthetic.sinogram(spec).astype(np.float32)).cuda())
    g = torch.Generator(device="cuda").manual_seed(11)
    for amp in (3e-5, 3e-4):
        y = x + amp * x.abs().max() * torch.randn(x.shape, device="cuda", generator=g)
        db, s = _check(fbp, y, x)
        want = oracle.ssim(y.double().cpu().numpy(), x.double().cpu().numpy(), 0.0)
        assert 1e-9 < 1.0 - want < 1e-3
        floor = (x.shape[0] - 10) * (x.shape[1] - 10) * 2.0 ** -53
        assert abs((1.0 - s) - (1.0 - want)) <= SSIM_REL_DIST * (1.0 - want) + floor
        assert SSIM_REL_DIST * (1.0 - want) > 10 * floor  # the relative bar is what binds


def test_near_identical_pairs_keep_their_distance_from_one(fbp):
    """The FP32, Kahan and FP16-pair images of the float-vs-double slice against
    the FP64 path's image (the bench's quality table): 1 - SSIM (down to about
    1e-12) matches the oracle's within the bars of _check, and is never below
    0 (SSIM never above 1)."""
    import torch
    spec = synthetic.cfg_float_double()
    sino64 = torch.from_numpy(synthetic.sinogram(spec)).cuda()
    ref = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, filter=spec.filter,
                   dtype=1).reconstruct(sino64).float()
    s32 = sino64.float()
    for opt in ({}, {"accumulate": 1}, {"q_storage": 2}):
        img = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, filter=spec.filter,
                       **opt).reconstruct(s32)
        db, s = _check(fbp, img, ref)
        assert 0.0 < 1.0 - s < 1e-4, (opt, 1.0 - s)


def test_fp16_pairs_against_fp32(fbp):
    import torch
    spec = synthetic.cfg_float_double()
    sino = torch.from_numpy(synthetic.sinogram(spec).astype(np.float32)).cuda()
    a = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, filter=spec.filter).reconstruct(sino)
    b = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, filter=spec.filter,
                 q_storage=2).reconstruct(sino)
    _check(fbp, b, a)
    _check(fbp, b, a, rng=2.0)


def test_identical_ragged_small_and_deterministic(fbp):
    import torch
    g = torch.Generator(device="cuda").manual_seed(3)
    wide = torch.rand((37, 64), device="cuda", generator=g)
    x = wide[:, :53]                     # row stride 64 > 53 columns
    wide2 = wide + 0.05 * torch.rand((37, 64), device="cuda", generator=g)
    y = wide2[:, :53]
    db, s = _check(fbp, x, x)
    assert math.isinf(db) and s == 1.0
    first = _check(fbp, x, y)
    assert fbp.quality(x, y) == first  # same bits
    small = torch.rand((10, 40), device="cuda", generator=g)
    _check(fbp, small, small * 0.9)      # no window fits: SSIM NaN


def test_quality_argument_errors(fbp):
    import torch
    x = torch.zeros((16, 16), device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    lib = fbp.load_library()
    need = fbp.fbp_quality_scratch_bytes(16, 16)
    sc = torch.zeros(need, dtype=torch.uint8, device="cuda")
    s = int(torch.cuda.current_stream().cuda_stream)
    assert lib.fbp_quality(x.data_ptr(), x.data_ptr(), 16, 16, 16, 0.0, sc.data_ptr(), need - 1,
                           out.data_ptr(), s) == fbp.FBP_ERR_INVALID_ARG
    assert lib.fbp_quality(x.data_ptr(), x.data_ptr(), 16, 16, 8, 0.0, sc.data_ptr(), need,
                           out.data_ptr(), s) == fbp.FBP_ERR_INVALID_ARG
    assert lib.fbp_quality(x.data_ptr() + 4, x.data_ptr(), 16, 15, 16, 0.0, sc.data_ptr(), need,
                           out.data_ptr(), s) == fbp.FBP_ERR_ALIGNMENT
