"""GPU: the bounded device waits run out, report FBP_ERR_TIMEOUT, and leave the
device usable.

No fault is made on the GPU: with the test-only hook the first CTA of a
kernel withholds the arrival of one pipeline stage (and issues no copy for
it), so the waits on that stage run out after a short limit (5 ms here).
Each test then checks, through the C ABI:
  - the status word reports FBP_ERR_TIMEOUT;
  - the next normal launch of the same plan (or the same captured batch,
    whose work counter the timed-out launch left where it stopped) gives
    the bits it gave before the fault, over images first filled with NaN;
  - after a tensor-core filter timeout, the next tensor-core launch runs, so
    the timed-out CTA released its tensor memory.
The hook and the limit are restored even when a test fails.
"""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu

LIMIT_S = 0.005


@pytest.fixture(scope="module")
def fbp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_02174_gb300 import build
    build.build()
    import paper_2109_02174_gb300 as m
    yield m
    m.fbp_test_withhold_arrival(m.FBP_TEST_WITHHOLD_NONE)
    m.fbp_set_wait_limit(0.0)


@pytest.fixture
def hook(fbp):
    """Arm the withholding hook with a short wait limit; disarm afterwards."""
    import torch

    def arm(kernel, stage):
        torch.cuda.synchronize()
        fbp.fbp_set_wait_limit(LIMIT_S)
        fbp.fbp_test_withhold_arrival(kernel, stage)

    yield arm
    torch.cuda.synchronize()
    fbp.fbp_test_withhold_arrival(fbp.FBP_TEST_WITHHOLD_NONE)
    fbp.fbp_set_wait_limit(0.0)


def _sino(spec):
    import torch
    return torch.from_numpy(synthetic.sinogram(spec).astype(np.float32)).cuda()


def _expect_timeout(call):
    import paper_2109_02174_gb300 as fbp
    with pytest.raises(fbp.FbpError) as e:
        call()
    assert e.value.status == fbp.FBP_ERR_TIMEOUT, e.value
    assert "bounded device wait" in fbp.fbp_last_error()


def disarm(fbp):
    import torch
    torch.cuda.synchronize()
    fbp.fbp_test_withhold_arrival(fbp.FBP_TEST_WITHHOLD_NONE)
    fbp.fbp_set_wait_limit(0.0)


def test_single_slice_backprojection_times_out_and_recovers(fbp, hook):
    import torch
    spec = synthetic.SliceSpec(256, 180, 363, 10, seed=61)
    plan = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det)
    sino = _sino(spec)
    want = plan.reconstruct(sino).cpu().numpy()
    plan.device_status()
    for stage in (0, 1, 4):
        hook(fbp.FBP_TEST_WITHHOLD_BACKPROJECT, stage)
        out = torch.full((spec.n_pix, spec.n_pix), float("nan"), device="cuda")
        plan.reconstruct(sino, out=out)
        _expect_timeout(plan.device_status)
        # the first CTA's first tile stops at the withheld stage: never written
        assert np.isnan(out[:32, :8].cpu().numpy()).all()
        disarm(fbp)
        out.fill_(float("nan"))
        plan.reconstruct(sino, out=out)
        torch.cuda.synchronize()
        plan.device_status()
        assert np.array_equal(out.cpu().numpy(), want), stage


def test_batched_backprojection_times_out_and_resets_its_counter(fbp, hook):
    """A captured batch of eight slices of one plan: two-slice work items taken
    from the launch's counter.  After the timed-out launch the same graph is
    launched again and every tile is written."""
    import torch
    n, A = 384, 360
    D = synthetic.det_for(n)
    plan = fbp.Plan(n, A, D)
    sinos = [_sino(synthetic.SliceSpec(n, A, D, 8, seed=70 + i)) for i in range(8)]
    batch = fbp.Batch([plan] * 8, sinos)
    assert batch.kernel_count == 2
    batch.launch()
    torch.cuda.synchronize()
    batch.status()
    want = [im.cpu().numpy() for im in batch.images]
    for stage in (0, 3):
        hook(fbp.FBP_TEST_WITHHOLD_BACKPROJECT, stage)
        for im in batch.images:
            im.fill_(float("nan"))
        batch.launch()
        _expect_timeout(batch.status)
        assert any(np.isnan(im.cpu().numpy()).any() for im in batch.images)
        disarm(fbp)
        for im in batch.images:
            im.fill_(float("nan"))
        batch.launch()
        torch.cuda.synchronize()
        batch.status()
        for w, im in zip(want, batch.images):
            assert np.array_equal(im.cpu().numpy(), w), stage
    # and the batch still equals the slices alone
    assert np.array_equal(plan.reconstruct(sinos[5]).cpu().numpy(), want[5])


def test_tensor_core_filter_times_out_and_releases_tensor_memory(fbp, hook):
    """The loader warps of the first CTA withhold one K chunk's arrival: the
    MMA warp's wait runs out, the CTA waits for its committed MMAs and issued
    copies, frees its tensor memory and leaves.  The next tensor-core launches
    (which allocate all 512 columns of every SM they run on) complete."""
    import torch
    A, D = 300, 725
    plan = fbp.Plan(256, A, D, filter_path=fbp.FBP_PATH_TOEPLITZ_TC)
    assert plan.filter_path == fbp.FBP_PATH_TOEPLITZ_TC
    P = torch.from_numpy(np.random.default_rng(5).standard_normal((A, D)).astype(np.float32)).cuda()
    want = plan.filter(P).cpu().numpy()
    plan.device_status()
    for stage in (0, 2, 7):
        hook(fbp.FBP_TEST_WITHHOLD_FILTER_TC, stage)
        q = torch.full((A, plan.q_pitch), float("nan"), device="cuda")
        plan.filter(P, out=q)
        _expect_timeout(plan.device_status)
        disarm(fbp)
        for _ in range(2):
            q.fill_(float("nan"))
            plan.filter(P, out=q)
            torch.cuda.synchronize()
            plan.device_status()
            assert np.array_equal(q.cpu().numpy(), want), stage


def test_wait_limit_argument_checks(fbp):
    for bad in (-1.0, float("nan"), float("inf"), 1e-9, 1e5):
        with pytest.raises(fbp.FbpError) as e:
            fbp.fbp_set_wait_limit(bad)
        assert e.value.status == fbp.FBP_ERR_INVALID_ARG
    with pytest.raises(fbp.FbpError) as e:
        fbp.fbp_test_withhold_arrival(9, 0)
    assert e.value.status == fbp.FBP_ERR_INVALID_ARG
    with pytest.raises(fbp.FbpError) as e:
        fbp.fbp_test_withhold_arrival(fbp.FBP_TEST_WITHHOLD_BACKPROJECT, -2)
    assert e.value.status == fbp.FBP_ERR_INVALID_ARG
