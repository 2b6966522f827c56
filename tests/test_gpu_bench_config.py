"""GPU: the launch configuration bench.py times, at its full size.  64 slices
of the float-vs-double workload (512 x 512, 720 angles, 725 bins, Shepp-Logan,
Poisson noise), one plan from the autotuner with a batch hint of 64 (so the
same filter route, tile and angle chunk as the bench), in one captured graph
(two slices per backprojection work item).  Sampled pixels of slices from
either end and the middle of the batch match the FP64 oracle within the FP32
bars, and those slices equal their alone results bit for bit."""
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
    rng = np.random.default_rng(64)
    for i in (0, 1, 31, 32, 62, 63):
        got = batch.images[i].cpu().numpy()
        alone = plan.reconstruct(sinos[i])
        torch.cuda.synchronize()
        assert np.array_equal(got, alone.cpu().numpy()), i
        Q = oracle.filter_rows(host[i].astype(np.float64), s0.filter, 1.0, nthreads=16)
        rows = np.concatenate([rng.integers(0, s0.n_pix, 500), np.full(64, 256)])
        cols = np.concatenate([rng.integers(0, s0.n_pix, 500), np.arange(0, 512, 8)])
        ref = oracle.backproject_pixels(Q, th, 1.0, s0.n_pix, rows, cols)
        scale = np.abs(ref).max()
        err = got[rows, cols].astype(np.float64) - ref
        assert np.abs(err).max() <= MAX_REL * scale, (i, np.abs(err).max() / scale)
        assert np.sqrt(np.mean(err ** 2)) <= RMSE_REL * scale, i
