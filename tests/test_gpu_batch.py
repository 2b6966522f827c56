"""GPU: batched reconstruction (one captured graph, one persistent launch per
kernel configuration) is bit-identical to each slice reconstructed alone, and
matches the FP64 oracle within the FP32 bars."""
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


def _sino(spec):
    import torch
    return torch.from_numpy(synthetic.sinogram(spec).astype(np.float32)).cuda()


def _alone(fbp, plan, sino):
    import torch
    img = plan.reconstruct(sino)
    torch.cuda.synchronize()
    return img.cpu().numpy()


def _parity(got, sino_t, spec):
    th = synthetic.default_angles(spec.n_angles)
    ref = oracle.fbp(sino_t.double().cpu().numpy(), th, spec.tau, spec.filter, spec.n_pix,
                     nthreads=NTHREADS)
    scale = np.abs(ref).max()
    e_max = np.abs(got - ref).max() / scale
    e_rms = np.sqrt(np.mean((got - ref) ** 2)) / scale
    assert e_max <= MAX_REL and e_rms <= RMSE_REL, f"max {e_max:.3e} rmse {e_rms:.3e}"


def small_uneven_specs(count=12, seed=33):
    rng = synthetic.SplitMix64(seed)
    out = []
    for s in range(count):
        n = rng.choice((64, 96, 128, 200))
        a = rng.choice((45, 90, 180, 360))
        out.append(synthetic.SliceSpec(n, a, synthetic.det_for(n), 6, seed=500 + s,
                                       filter=s % 2))
    return out


def test_batch_matches_alone_bitwise_and_oracle(fbp):
    import torch
    specs = small_uneven_specs()
    plans = [fbp.Plan(s.n_pix, s.n_angles, s.n_det, filter=s.filter) for s in specs]
    sinos = [_sino(s) for s in specs]
    batch = fbp.Batch(plans, sinos)
    batch.launch()
    torch.cuda.synchronize()
    batch.status()
    for spec, plan, sino, img in zip(specs, plans, sinos, batch.images):
        got = img.cpu().numpy()
        assert np.array_equal(got, _alone(fbp, plan, sino)), spec
        _parity(got.astype(np.float64), sino, spec)


def test_batch_relaunch_sees_new_data(fbp):
    import torch
    specs = small_uneven_specs(5, seed=34)
    plans = [fbp.Plan(s.n_pix, s.n_angles, s.n_det) for s in specs]
    sinos = [_sino(s) for s in specs]
    batch = fbp.Batch(plans, sinos)
    batch.launch()
    first = [im.clone() for im in batch.images]
    for s, t in zip(specs, sinos):
        s2 = synthetic.SliceSpec(s.n_pix, s.n_angles, s.n_det, 6, seed=s.seed + 77)
        t.copy_(_sino(s2))
    batch.launch()
    torch.cuda.synchronize()
    for plan, sino, im, f in zip(plans, sinos, batch.images, first):
        now = im.cpu().numpy()
        assert not np.array_equal(now, f.cpu().numpy())
        assert np.array_equal(now, _alone(fbp, plan, sino))


def test_dynamic_work_handout_recomputes_every_tile(fbp):
    """The batch's backprojection launches hand out work items from a counter
    that each launch must leave at zero: after the images are cleared, every
    relaunch (and a run through the host pipeline, whose chunks take the
    other counter set) writes every tile again, bit-identical to alone."""
    import torch
    specs = small_uneven_specs(9, seed=36)
    plans = [fbp.Plan(s.n_pix, s.n_angles, s.n_det, filter=s.filter) for s in specs]
    sinos = [_sino(s) for s in specs]
    want = [_alone(fbp, p, t) for p, t in zip(plans, sinos)]
    batch = fbp.Batch(plans, sinos)
    for _ in range(4):
        for im in batch.images:
            im.fill_(float("nan"))
        batch.launch()
        torch.cuda.synchronize()
        batch.status()
        for w, im in zip(want, batch.images):
            assert np.array_equal(im.cpu().numpy(), w)
    host_in = [t.cpu().contiguous().pin_memory() for t in sinos]
    for _ in range(2):
        host_out = [torch.full((s.n_pix, s.n_pix), float("nan")).pin_memory() for s in specs]
        batch.run_host(host_in, host_out)
        torch.cuda.synchronize()
        batch.status()
        for w, h in zip(want, host_out):
            assert np.array_equal(h.numpy(), w)
    for im in batch.images:
        im.fill_(float("nan"))
    batch.launch()
    torch.cuda.synchronize()
    for w, im in zip(want, batch.images):
        assert np.array_equal(im.cpu().numpy(), w)


def test_concurrent_batches_on_two_streams(fbp):
    """Two batches over the same plans (own buffers and work counters) launched
    on two streams without synchronising between them: their persistent
    launches share the GPU and hand out work independently, and every image
    is the one its slice gets alone."""
    import torch
    specs = small_uneven_specs(10, seed=37)
    plans = [fbp.Plan(s.n_pix, s.n_angles, s.n_det, filter=s.filter) for s in specs]
    sinos_a = [_sino(s) for s in specs]
    sinos_b = [(-0.5 * t).contiguous() for t in sinos_a]
    want_a = [_alone(fbp, p, t) for p, t in zip(plans, sinos_a)]
    want_b = [_alone(fbp, p, t) for p, t in zip(plans, sinos_b)]
    ba, bb = fbp.Batch(plans, sinos_a), fbp.Batch(plans, sinos_b)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    for _ in range(3):
        for im in ba.images + bb.images:
            im.fill_(float("nan"))
        torch.cuda.synchronize()
        ba.launch(sa)
        bb.launch(sb)
        ba.launch(sa)
        torch.cuda.synchronize()
        ba.status()
        bb.status()
        for w, im in zip(want_a, ba.images):
            assert np.array_equal(im.cpu().numpy(), w)
        for w, im in zip(want_b, bb.images):
            assert np.array_equal(im.cpu().numpy(), w)


def test_batch_mixes_kernel_configurations(fbp):
    """Slices whose plans pick different kernels (tile shape, FP16 pairs, Kahan)
    share one batch; each still equals its own alone result bit for bit."""
    import torch
    n, A = 96, 60
    D = synthetic.det_for(n)
    tc = fbp.Plan(n, A, D, filter_path=1)
    plans = [fbp.Plan(n, A, D), fbp.Plan(n, A, 2 * D, det_spacing=0.45),
             fbp.Plan(n, A, D, q_storage=2), fbp.Plan(n, A, D, accumulate=1),
             fbp.Plan(n, A, D, tile_x=8, tile_y=32), tc, tc, fbp.Plan(n, A, D, filter_path=3)]
    specs = [synthetic.SliceSpec(n, A, p.n_det, 5, seed=900 + i, tau=p.det_spacing)
             for i, p in enumerate(plans)]
    sinos = [_sino(s) for s in specs]
    batch = fbp.Batch(plans, sinos)
    batch.launch()
    torch.cuda.synchronize()
    for plan, sino, img in zip(plans, sinos, batch.images):
        assert np.array_equal(img.cpu().numpy(), _alone(fbp, plan, sino))


@pytest.mark.parametrize("q_storage", [0, 2])
def test_same_plan_slices_pair_up_bitwise(fbp, q_storage):
    """Slices sharing a plan go through two-slice work items (one index
    computation for both); an odd one out stays single.  Each image equals its
    alone result bit for bit."""
    import torch
    n, A = 150, 96
    D = synthetic.det_for(n)
    plan = fbp.Plan(n, A, D, q_storage=q_storage, angle_chunk=16)
    specs = [synthetic.SliceSpec(n, A, D, 6, seed=950 + i) for i in range(5)]
    sinos = [_sino(s) for s in specs]
    batch = fbp.Batch([plan] * 5, sinos)
    batch.launch()
    torch.cuda.synchronize()
    batch.status()
    for sino, img in zip(sinos, batch.images):
        assert np.array_equal(img.cpu().numpy(), _alone(fbp, plan, sino))


def test_batched_uneven_workload_64(fbp):
    """The batched configuration: 64 uneven slices (n in {256,384,512,768},
    A in {180,360,720,1440}) in one graph.  Every slice is bit-identical to its
    alone result, and every pixel of every slice is within the FP32 bars of the
    oracle's image."""
    import os

    import torch
    specs = synthetic.cfg_batch()
    plans = [fbp.Plan(s.n_pix, s.n_angles, s.n_det) for s in specs]
    sinos = [_sino(s) for s in specs]
    batch = fbp.Batch(plans, sinos)
    batch.launch()
    torch.cuda.synchronize()
    batch.status()
    imgs = [im.cpu().numpy() for im in batch.images]
    for plan, sino, img in zip(plans, sinos, imgs):
        assert np.array_equal(img, _alone(fbp, plan, sino))
    for i, s in enumerate(specs):
        th = synthetic.default_angles(s.n_angles)
        ref = oracle.fbp(sinos[i].double().cpu().numpy(), th, s.tau, s.filter, s.n_pix,
                         nthreads=os.cpu_count() or 1)
        scale = np.abs(ref).max()
        err = imgs[i].astype(np.float64) - ref
        assert np.abs(err).max() <= MAX_REL * scale, (i, np.abs(err).max() / scale)
        assert np.sqrt(np.mean(err ** 2)) <= RMSE_REL * scale, i


def test_batch_argument_errors(fbp):
    import torch
    plan = fbp.Plan(32, 8, 46)
    s = torch.zeros(8, 46, device="cuda")
    im = torch.zeros(32, 32, device="cuda")
    ws = plan.empty_workspace()
    good = fbp.fbp_batch_io(s.data_ptr(), 46, im.data_ptr(), ws.data_ptr())
    with pytest.raises(fbp.FbpError) as e:
        fbp.fbp_batch_build([], [])
    assert e.value.status == fbp.FBP_ERR_INVALID_ARG
    bad = fbp.fbp_batch_io(s.data_ptr() + 4, 46, im.data_ptr(), ws.data_ptr())
    with pytest.raises(fbp.FbpError) as e:
        fbp.fbp_batch_build([plan.handle], [bad])
    assert e.value.status == fbp.FBP_ERR_ALIGNMENT
    short = fbp.fbp_batch_io(s.data_ptr(), 40, im.data_ptr(), ws.data_ptr())
    with pytest.raises(fbp.FbpError) as e:
        fbp.fbp_batch_build([plan.handle], [short])
    assert e.value.status == fbp.FBP_ERR_INVALID_ARG
    h = fbp.fbp_batch_build([plan.handle], [good])
    fbp.fbp_batch_launch(h, 0)
    fbp.fbp_batch_status(h)
    fbp.fbp_batch_destroy(h)


def test_run_host_pipeline_equals_device_batch(fbp):
    """fbp_batch_run_host (six pipelined chunks: sinograms in on one stream,
    compute alternating between the caller's and a second stream, images out
    on a fourth) gives the device batch's
    bits; a second call with new host data returns the new images, so no copy
    of one call overtakes the compute of the other.  One slice's device
    sinogram has padded rows (ld_sino > n_det), which takes the 2-D copy."""
    import torch
    specs = small_uneven_specs(17, seed=35)
    plans = [fbp.Plan(s.n_pix, s.n_angles, s.n_det, filter=s.filter) for s in specs]
    sinos = [_sino(s) for s in specs]
    padded = torch.zeros((specs[3].n_angles, specs[3].n_det + 12), device="cuda")
    padded[:, :specs[3].n_det] = sinos[3]
    sinos[3] = padded[:, :specs[3].n_det]
    batch = fbp.Batch(plans, sinos)
    batch.launch()
    torch.cuda.synchronize()
    batch.status()
    want = [im.cpu().numpy() for im in batch.images]
    host_in = [s.cpu().contiguous().pin_memory() for s in sinos]
    host_out = [torch.full((s.n_pix, s.n_pix), float("nan")).pin_memory() for s in specs]
    for im in batch.images:
        im.zero_()
    batch.run_host(host_in, host_out)
    torch.cuda.synchronize()
    batch.status()
    for w, h in zip(want, host_out):
        assert np.array_equal(h.numpy(), w)
    # second call, new data: every image must follow its new sinogram
    new_in = [(2.0 * h).pin_memory() for h in host_in]
    batch.run_host(new_in, host_out)
    torch.cuda.synchronize()
    for plan, s_new, h in zip(plans, new_in, host_out):
        assert np.array_equal(h.numpy(), _alone(fbp, plan, s_new.cuda()))


def test_kernel_count_of_a_same_plan_batch(fbp):
    """Four slices of one FFT-route plan: one filter launch over all row pairs
    and one backprojection launch over all tiles (two slices per item)."""
    n, A = 96, 60
    D = synthetic.det_for(n)
    plan = fbp.Plan(n, A, D, filter_path=2)
    sinos = [_sino(synthetic.SliceSpec(n, A, D, 4, seed=990 + i)) for i in range(4)]
    batch = fbp.Batch([plan] * 4, sinos)
    assert batch.kernel_count == 2


def test_kahan_slices_pair_up_bitwise(fbp):
    """Kahan-compensated sums with FP32 pairs pair up into two-slice items as
    plain sums do (five slices of one plan: two pairs and one single, one
    backprojection launch); each image equals its alone result bit for bit and
    meets the bars.  With FP16 pairs a Kahan plan keeps one-slice items."""
    import torch
    n, A = 128, 360
    D = synthetic.det_for(n)
    specs = [synthetic.SliceSpec(n, A, D, 6, seed=1300 + i) for i in range(5)]
    sinos = [_sino(s) for s in specs]
    plan = fbp.Plan(n, A, D, filter_path=2, tile_x=32, tile_y=32, accumulate=1)
    batch = fbp.Batch([plan] * 5, sinos)
    assert batch.kernel_count == 2
    for im in batch.images:
        im.fill_(float("nan"))
    batch.launch()
    torch.cuda.synchronize()
    batch.status()
    for s, t, im in zip(specs, sinos, batch.images):
        got = im.cpu().numpy()
        assert np.array_equal(got, _alone(fbp, plan, t))
    _parity(batch.images[0].cpu().numpy().astype(np.float64), sinos[0], specs[0])
    p16 = fbp.Plan(n, A, D, filter_path=2, tile_x=32, tile_y=32, accumulate=1, q_storage=2)
    b16 = fbp.Batch([p16] * 3, sinos[:3])
    b16.launch()
    torch.cuda.synchronize()
    b16.status()
    for t, im in zip(sinos[:3], b16.images):
        assert np.array_equal(im.cpu().numpy(), _alone(fbp, p16, t))


@pytest.mark.parametrize("q_storage", [0, 2])
def test_odd_slices_ride_in_the_two_slice_launch(fbp, q_storage):
    """Five slices of one plan and one of another plan with the same kernel
    configuration: two pairs and two single slices, all in one two-slice
    backprojection launch (a single slice stages one row per angle).  One
    filter launch plus one backprojection launch; every image equals its
    alone result bit for bit, over images first filled with NaN (FP32 and
    FP16 pairs)."""
    import torch
    n, A = 96, 60
    D = synthetic.det_for(n)
    a = fbp.Plan(n, A, D, filter_path=2, tile_x=8, tile_y=32, q_storage=q_storage)
    b = fbp.Plan(128, 90, synthetic.det_for(128), filter_path=2, tile_x=8, tile_y=32,
                 q_storage=q_storage)
    plans = [a, a, b, a, a, a]
    specs = [synthetic.SliceSpec(p.n_pix, p.n_angles, p.n_det, 5, seed=1200 + i)
             for i, p in enumerate(plans)]
    sinos = [_sino(s) for s in specs]
    batch = fbp.Batch(plans, sinos)
    assert batch.kernel_count == 2
    for rep in range(2):
        for im in batch.images:
            im.fill_(float("nan"))
        batch.launch()
        torch.cuda.synchronize()
        batch.status()
        for p, s, im in zip(plans, sinos, batch.images):
            assert np.array_equal(im.cpu().numpy(), _alone(fbp, p, s)), rep


def test_point_pair_plans_in_batches_bitwise(fbp):
    """Slices of point-pair plans (a tile and its mirror image per work item;
    plain sums, FP16 pairs, Kahan sums) batched with other plans: each image
    equals its alone result bit for bit, and the batch launch takes the
    counter hand-out like the others."""
    import torch
    n, A = 128, 90
    D = synthetic.det_for(n)
    pp = fbp.Plan(n, A, D, tile_x=32, tile_y=32, point_pairs=1)
    pp16 = fbp.Plan(n, A, D, tile_x=32, tile_y=32, point_pairs=1, q_storage=2)
    ppk = fbp.Plan(n, A, D, tile_x=32, tile_y=32, point_pairs=1, accumulate=1)
    plain = fbp.Plan(n, A, D, tile_x=32, tile_y=32, point_pairs=-1)
    plans = [pp, pp, pp, plain, plain, pp16, ppk, ppk,
             fbp.Plan(256, 120, synthetic.det_for(256), tile_x=8, tile_y=32, point_pairs=1)]
    specs = [synthetic.SliceSpec(p.n_pix, p.n_angles, p.n_det, 6, seed=1200 + i)
             for i, p in enumerate(plans)]
    sinos = [_sino(s) for s in specs]
    batch = fbp.Batch(plans, sinos)
    for _ in range(2):
        for im in batch.images:
            im.fill_(float("nan"))
        batch.launch()
        torch.cuda.synchronize()
        batch.status()
        for plan, sino, img in zip(plans, sinos, batch.images):
            assert np.array_equal(img.cpu().numpy(), _alone(fbp, plan, sino))
