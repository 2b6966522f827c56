"""GPU: the launch configuration bench.py times, at its full size.  64 slices
of the float-vs-double workload (512 x 512, 720 angles, 725 bins, Shepp-Logan,
Poisson noise), one plan from the autotuner with a batch hint of 64 (so the
same filter route, tile and angle chunk as the bench), in one captured graph
(two slices per backprojection work item).  Every pixel of every slice
matches the FP64 oracle's image within the FP32 bars, and every slice equals
its alone result bit for bit."""
import os

import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu
MAX_REL, RMSE_REL = 1e-4, 2e-5
SLICES = 64


@pytest.fixture(scope="module")
def fbp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_02174_gb300 import build
    build.build()
    import paper_2109_02174_gb300 as m
    return m


def test_bench_batch_matches_oracle_and_alone(fbp):
    import torch
    specs = [synthetic.cfg_float_double_slice(i) for i in range(SLICES)]
    s0 = specs[0]
    th = synthetic.default_angles(s0.n_angles)
    plan = fbp.Plan(s0.n_pix, s0.n_angles, s0.n_det, filter=s0.filter, autotune=True,
                    batch_hint=SLICES)
    host = [synthetic.sinogram(s, th).astype(np.float32) for s in specs]
    sinos = [torch.from_numpy(h).cuda() for h in host]
    batch = fbp.Batch([plan] * SLICES, sinos)
    batch.launch()
    torch.cuda.synchronize()
    batch.status()
    worst = (0.0, 0.0)
    for i in range(SLICES):
        got = batch.images[i].cpu().numpy()
        alone = plan.reconstruct(sinos[i])
        torch.cuda.synchronize()
        assert np.array_equal(got, alone.cpu().numpy()), i
        ref = oracle.fbp(host[i].astype(np.float64), th, s0.tau, s0.filter, s0.n_pix,
                         nthreads=os.cpu_count() or 1)
        scale = np.abs(ref).max()
        err = got.astype(np.float64) - ref
        e_max = np.abs(err).max() / scale
        e_rms = np.sqrt(np.mean(err ** 2)) / scale
        assert e_max <= MAX_REL and e_rms <= RMSE_REL, (i, e_max, e_rms)
        worst = (max(worst[0], e_max), max(worst[1], e_rms))
    print(f"64 bench slices, every pixel: worst max {worst[0]:.3e}, worst rmse {worst[1]:.3e}")
