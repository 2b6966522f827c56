"""GPU: the continuous-batching server.  Requests arriving on a Poisson clock
are admitted under an HBM budget and batched into overlapping waves; each
image must be bit-identical to the same slice reconstructed alone (and so
within the FP32 bars of the oracle, spot-checked here).  Failures are made on
the host: bad or oversized requests, cancellation, a wait that times out, a
producer thread that dies mid-stream."""
import math
import threading
import time

import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu

MAX_REL = 1e-4
RMSE_REL = 2e-5


@pytest.fixture(scope="module")
def fbp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_02174_gb300 import build
    build.build()
    import paper_2109_02174_gb300 as m
    return m


def _stream(count, seed, rate=2000.0):
    """Arrival times and small mixed geometries (n in {64,128,200}, A in {90,180,360})."""
    rng = synthetic.SplitMix64(seed)
    t, out = 0.0, []
    for r in range(count):
        t += -math.log(1.0 - rng.uniform()) / rate
        n = rng.choice((64, 128, 200))
        a = rng.choice((90, 180, 360))
        out.append((t, synthetic.SliceSpec(n, a, synthetic.det_for(n), 5, seed=7000 + r,
                                           i0=1e5, noise_seed=17000 + r)))
    return out


def _host(spec):
    import torch
    s = torch.from_numpy(synthetic.sinogram(spec).astype(np.float32)).pin_memory()
    img = torch.empty((spec.n_pix, spec.n_pix), dtype=torch.float32).pin_memory()
    return s, img


def _alone(fbp, spec, sino_host):
    import torch
    # the server's plans take the largest backprojection tile that fits
    plan = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, tile_x=-1, tile_y=-1)
    out = plan.reconstruct(sino_host.cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_results_in_the_mix_equal_alone(fbp):
    reqs = _stream(60, seed=61)
    bufs = [_host(s) for _, s in reqs]
    server = fbp.Server(hbm_budget_bytes=2 << 30, max_wave=16, n_streams=2)
    t0 = time.perf_counter()
    ids = []
    for (t, spec), (s, img) in zip(reqs, bufs):
        while time.perf_counter() - t0 < t:
            pass
        ids.append(server.submit(s, img, spec.n_pix))
    for rid in ids:
        server.wait(rid, 60.0)
    st = server.stats()
    assert st["completed"] == 60 and st["failed"] == 0
    assert st["waves"] >= 2
    for (_, spec), (s, img), rid in zip(reqs, bufs, ids):
        assert server.info(rid)[0] == fbp.Server.DONE
        assert np.array_equal(img.numpy(), _alone(fbp, spec, s)), spec
    # spot-check three requests against the FP64 oracle
    for k in (0, 29, 59):
        spec = reqs[k][1]
        ref = oracle.fbp(bufs[k][0].numpy().astype(np.float64),
                         synthetic.default_angles(spec.n_angles), 1.0, 0, spec.n_pix,
                         nthreads=16)
        got = bufs[k][1].numpy().astype(np.float64)
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= MAX_REL * scale
        assert np.sqrt(np.mean((got - ref) ** 2)) <= RMSE_REL * scale
    server.close()


def test_small_budget_stalls_admission_but_completes(fbp):
    """A budget that holds one of the largest requests: the rest wait for memory, in order."""
    reqs = _stream(12, seed=62)
    bufs = [_host(s) for _, s in reqs]
    biggest = max(4 * (s.n_angles * s.n_det + s.n_angles * (2 * s.n_det + 16) + s.n_pix ** 2)
                  for _, s in reqs)
    server = fbp.Server(hbm_budget_bytes=max(biggest + 4096, 1 << 20), max_wave=4, n_streams=2)
    ids = [server.submit(s, img, spec.n_pix) for (_, spec), (s, img) in zip(reqs, bufs)]
    server.drain(120.0)
    st = server.stats()
    assert st["completed"] == 12 and st["admission_stalls"] > 0
    assert st["peak_bytes"] <= st["budget_bytes"] and st["bytes_in_use"] == 0
    for (_, spec), (s, img), rid in zip(reqs, bufs, ids):
        assert np.array_equal(img.numpy(), _alone(fbp, spec, s))
    server.close()


def test_bad_and_oversized_requests_are_rejected_at_submit(fbp):
    import torch
    server = fbp.Server(hbm_budget_bytes=8 << 20, max_wave=4, n_streams=1)
    spec = synthetic.SliceSpec(64, 90, synthetic.det_for(64), 4, seed=3)
    s, img = _host(spec)
    with pytest.raises(fbp.FbpError) as e:
        server.submit(s, img, n_pix=0)  # corrupted geometry
    assert e.value.status == fbp.FBP_ERR_INVALID_ARG
    big = torch.zeros((1440, 1450), dtype=torch.float32).pin_memory()
    bimg = torch.zeros((1024, 1024), dtype=torch.float32).pin_memory()
    with pytest.raises(fbp.FbpError) as e:
        server.submit(big, bimg, n_pix=1024)  # ~29 MB > 8 MiB budget
    assert e.value.status == fbp.FBP_ERR_BUDGET
    rid = server.submit(s, img, spec.n_pix)  # the server still serves good requests
    server.wait(rid, 60.0)
    assert np.array_equal(img.numpy(), _alone(fbp, spec, s))
    st = server.stats()
    assert st["submitted"] == 1 and st["completed"] == 1
    server.close()


def test_cancel_queued_request_and_wait_timeout(fbp):
    """With room for one request at a time, later ones queue: one is cancelled
    while queued; a zero-length wait on a queued request reports a timeout."""
    specs = [synthetic.SliceSpec(200, 360, synthetic.det_for(200), 4, seed=80 + k)
             for k in range(4)]
    bufs = [_host(s) for s in specs]
    one = 4 * (360 * 284 + 360 * (2 * 284 + 16) + 200 * 200)
    server = fbp.Server(hbm_budget_bytes=one + (1 << 20), max_wave=1, n_streams=1)
    ids = [server.submit(s, img, sp.n_pix) for sp, (s, img) in zip(specs, bufs)]
    with pytest.raises(fbp.FbpError) as e:
        server.wait(ids[3], 0.0)
    assert e.value.status == fbp.FBP_ERR_TIMEOUT
    try:
        server.cancel(ids[3])
        cancelled = True
    except fbp.FbpError:
        cancelled = False  # it was admitted already: also a valid outcome
    server.drain(120.0)
    st = server.stats()
    assert st["completed"] == (3 if cancelled else 4)
    for sp, (s, img), rid in list(zip(specs, bufs, ids))[:3]:
        assert np.array_equal(img.numpy(), _alone(fbp, sp, s))
    if cancelled:
        assert server.info(ids[3])[0] == fbp.Server.CANCELLED
    server.close()


def test_producer_thread_that_dies_leaves_server_serving(fbp):
    reqs = _stream(20, seed=63)
    bufs = [_host(s) for _, s in reqs]
    server = fbp.Server(hbm_budget_bytes=1 << 30, max_wave=8, n_streams=2)
    submitted = []

    def producer(lo, hi, die_at=None):
        for k in range(lo, hi):
            if k == die_at:
                raise RuntimeError("producer crashed")
            spec = reqs[k][1]
            submitted.append((k, server.submit(bufs[k][0], bufs[k][1], spec.n_pix)))

    errors = []

    def guarded(*a):
        try:
            producer(*a)
        except RuntimeError as exc:
            errors.append(exc)

    t1 = threading.Thread(target=guarded, args=(0, 10, 6))
    t2 = threading.Thread(target=guarded, args=(10, 20))
    t1.start(); t2.start(); t1.join(); t2.join()
    assert len(errors) == 1 and len(submitted) == 16
    server.drain(120.0)
    assert server.stats()["completed"] == 16
    for k, rid in submitted:
        spec = reqs[k][1]
        assert np.array_equal(bufs[k][1].numpy(), _alone(fbp, spec, bufs[k][0]))
    server.close()
