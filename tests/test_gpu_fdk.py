"""GPU: FDK cone-beam reconstruction (the paper's future work) matches the
FP64 oracle within the FP32 bars: random projections, an ellipsoid phantom
under a moderate cone, ragged volume sizes with caller-given angles and
non-unit detector spacings; the same bits every run; bad geometries rejected
on the host."""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu
MAX_REL, RMSE_REL = 1e-4, 2e-5


@pytest.fixture(scope="module")
def fbp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_02174_gb300 import build
    build.build()
    import paper_2109_02174_gb300 as m
    return m


def _run(fbp, P, beta, R, du, dv, kind, nx, ny, nz, give_beta=True):
    import torch
    A, nv, nu = P.shape
    plan = fbp.FdkPlan(A, nv, nu, R, nx, ny, nz, du=du, dv=dv,
                       beta=beta if give_beta else None, filter=kind)
    vol = plan.reconstruct(torch.from_numpy(P.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    plan.device_status()
    ref = oracle.fdk(P.astype(np.float32).astype(np.float64), beta, R, du, dv, kind, nx, ny, nz,
                     nthreads=16)
    return vol.cpu().numpy().astype(np.float64), ref, plan


def _assert_bars(got, ref):
    scale = np.abs(ref).max()
    e_max = np.abs(got - ref).max() / scale
    e_rms = np.sqrt(np.mean((got - ref) ** 2)) / scale
    assert e_max <= MAX_REL and e_rms <= RMSE_REL, f"max {e_max:.3e} rmse {e_rms:.3e}"


def test_fdk_random_projections(fbp):
    P = np.random.default_rng(21).normal(size=(60, 20, 48))
    beta = synthetic.cone_beta(60)
    got, ref, _ = _run(fbp, P, beta, 60.0, 1.0, 1.0, 0, 32, 32, 16, give_beta=False)
    _assert_bars(got, ref)


def test_fdk_ellipsoid_phantom(fbp):
    n = 64
    beta = synthetic.cone_beta(180)
    ell = synthetic.random_ellipsoids(8, seed=22, n=n)
    P = synthetic.cone_projection(ell, beta, 150.0, 128, 96)
    got, ref, _ = _run(fbp, P, beta, 150.0, 1.0, 1.0, 1, n, n, n)
    _assert_bars(got, ref)


def test_fdk_ragged_sizes_given_angles_and_spacings(fbp):
    rng = np.random.default_rng(23)
    beta = np.sort(rng.uniform(0, 2 * np.pi, 73))
    P = synthetic.cone_projection(synthetic.random_ellipsoids(5, seed=24, n=32), beta, 90.0,
                                  70, 41, du=0.8, dv=1.2)
    got, ref, _ = _run(fbp, P, beta, 90.0, 0.8, 1.2, 1, 37, 29, 21)
    _assert_bars(got, ref)


def test_fdk_deterministic_and_rejects_bad_geometry(fbp):
    import torch
    P = torch.from_numpy(np.random.default_rng(25).normal(size=(40, 16, 40)).astype(np.float32)).cuda()
    plan = fbp.FdkPlan(40, 16, 40, 50.0, 24, 24, 16)
    a = plan.reconstruct(P).cpu().numpy()
    b = plan.reconstruct(P).cpu().numpy()
    assert np.array_equal(a, b)
    with pytest.raises(fbp.FbpError) as e:
        fbp.FdkPlan(40, 16, 40, 10.0, 32, 32, 16)  # the volume reaches the source circle
    assert e.value.status == fbp.FBP_ERR_INVALID_ARG


def test_fdk_bench_geometry_every_voxel(fbp):
    """The reconstruction bench.py times: 256^3 voxels from 360 projections of
    448 x 320 bins over a full turn, source radius 1024 (its largest windows
    and stage ring), seeded normal projections, Ram-Lak.  Every voxel against
    the oracle's volume."""
    A, nv, nu = 360, 320, 448
    P = np.random.default_rng(26).standard_normal((A, nv, nu)).astype(np.float32)
    beta = synthetic.cone_beta(A)
    got, ref, _ = _run(fbp, P, beta, 1024.0, 1.0, 1.0, 0, 256, 256, 256, give_beta=False)
    _assert_bars(got, ref)
