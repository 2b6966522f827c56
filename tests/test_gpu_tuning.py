"""GPU: the autotuner picks a valid filter route and backprojection shape per
geometry, caches it (in memory and in the FBP_TUNE_CACHE file), and plans made
from its choice meet the parity bars; the angle chunk never changes the bits."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fbp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_02174_gb300 import build
    build.build()
    import paper_2109_02174_gb300 as m
    return m


def test_autotune_choice_is_valid_and_cached(fbp):
    n, A = 128, 180
    D = synthetic.det_for(n)
    t1 = fbp.fbp_autotune(n, A, D, batch=4)
    assert (t1["tile_x"], t1["tile_y"]) in {(32, 64), (32, 32), (8, 32)}
    assert t1["angle_chunk"] in (8, 16, 32)
    assert t1["filter_path"] in (fbp.FBP_PATH_TOEPLITZ_TC, fbp.FBP_PATH_FFT, fbp.FBP_PATH_DIRECT)
    assert t1["filter_ms"] > 0 and t1["backproject_ms"] > 0
    t2 = fbp.fbp_autotune(n, A, D, batch=4)
    assert t2["from_cache"] == 1
    assert {k: t2[k] for k in ("tile_x", "tile_y", "angle_chunk", "filter_path")} == \
        {k: t1[k] for k in ("tile_x", "tile_y", "angle_chunk", "filter_path")}


def test_tuned_plan_meets_bars_and_batches_bitwise(fbp):
    import torch
    spec = synthetic.SliceSpec(160, 200, synthetic.det_for(160), 6, seed=71, filter=1)
    plan = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, filter=1, autotune=True, batch_hint=4)
    th = synthetic.default_angles(spec.n_angles)
    sino = torch.from_numpy(synthetic.sinogram(spec, th).astype(np.float32)).cuda()
    alone = plan.reconstruct(sino)
    batch = fbp.Batch([plan, plan], [sino, sino.clone()])
    batch.launch()
    torch.cuda.synchronize()
    got = alone.cpu().numpy()
    assert np.array_equal(got, batch.images[0].cpu().numpy())
    assert np.array_equal(got, batch.images[1].cpu().numpy())
    ref = oracle.fbp(sino.double().cpu().numpy(), th, 1.0, 1, spec.n_pix, nthreads=16)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-4 * scale
    assert np.sqrt(np.mean((got - ref) ** 2)) <= 2e-5 * scale


def test_angle_chunk_does_not_change_bits(fbp):
    import torch
    spec = synthetic.SliceSpec(96, 150, synthetic.det_for(96), 5, seed=72)
    sino = torch.from_numpy(synthetic.sinogram(spec).astype(np.float32)).cuda()
    imgs = []
    for ch in (8, 16, 32):
        plan = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, angle_chunk=ch)
        imgs.append(plan.reconstruct(sino).cpu().numpy())
    assert np.array_equal(imgs[0], imgs[1]) and np.array_equal(imgs[1], imgs[2])


def test_tuning_cache_file_survives_processes(fbp, tmp_path):
    cache = tmp_path / "tune.txt"
    code = ("import sys, json; sys.path.insert(0, %r); import paper_2109_02174_gb300 as f; "
            "print(json.dumps(f.fbp_autotune(64, 90, 92, batch=2)))" % ROOT)
    env = dict(os.environ, FBP_TUNE_CACHE=str(cache))
    out1 = json.loads(subprocess.check_output([sys.executable, "-c", code], env=env).decode()
                      .strip().splitlines()[-1])
    assert out1["from_cache"] == 0 and cache.exists()
    assert len(cache.read_text().strip().splitlines()) == 1
    out2 = json.loads(subprocess.check_output([sys.executable, "-c", code], env=env).decode()
                      .strip().splitlines()[-1])
    assert out2["from_cache"] == 1
    assert out2["tile_x"] == out1["tile_x"] and out2["filter_path"] == out1["filter_path"]


def test_autotune_keeps_fixed_route_tile_and_chunk(fbp):
    """A filter route, tile or angle chunk given in the base options is kept;
    only the rest is tuned (and cached under its own key)."""
    n, A = 128, 180
    D = synthetic.det_for(n)
    base = fbp.fbp_options_default()
    base.filter_path = fbp.FBP_PATH_FFT
    base.tile_x, base.tile_y = 8, 32
    t = fbp.fbp_autotune(n, A, D, base=base, batch=2)
    assert t["filter_path"] == fbp.FBP_PATH_FFT
    assert (t["tile_x"], t["tile_y"]) == (8, 32)
    assert t["angle_chunk"] in (8, 16, 32)
    base.angle_chunk = 32
    t2 = fbp.fbp_autotune(n, A, D, base=base, batch=2)
    assert (t2["tile_x"], t2["tile_y"], t2["angle_chunk"]) == (8, 32, 32)


def test_default_tile_rule(fbp):
    """An untuned plan takes the largest tile whose window fits and that cuts
    the image into at least one tile per two SMs; tile -1 takes the largest
    that fits.  The tile fixes the bits (the local coordinate's origin), so
    each choice is identified by matching an explicitly tiled plan."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    spec = synthetic.SliceSpec(256, 90, synthetic.det_for(256), 6, seed=71)
    sino = torch.from_numpy(synthetic.sinogram(spec).astype(np.float32)).cuda()

    def img(**opt):
        out = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, **opt).reconstruct(sino)
        torch.cuda.synchronize()
        return out.cpu().numpy()

    by_tile = {t: img(tile_x=t[0], tile_y=t[1]) for t in ((32, 64), (32, 32), (8, 32))}
    # 256^2: 32 tiles of 32x64, 64 of 32x32, 256 of 8x32
    expect = (32, 64) if 2 * 32 >= sms else (32, 32) if 2 * 64 >= sms else (8, 32)
    assert np.array_equal(img(), by_tile[expect])
    assert np.array_equal(img(tile_x=-1, tile_y=-1), by_tile[(32, 64)])
    assert not np.array_equal(by_tile[(32, 64)], by_tile[(8, 32)])



def test_default_plan_of_a_large_slice_takes_point_pairs(fbp):
    """From n_pix > 704 (on 152 SMs) the automatic tile is 32 x 32 with
    point-symmetric tile pairs (32 x 64 for FP16 pairs); a named tile keeps
    single-tile items unless point_pairs = 1 asks for them."""
    import torch
    n, A = 768, 90
    D = synthetic.det_for(n)
    sino = torch.from_numpy(
        synthetic.sinogram(synthetic.SliceSpec(n, A, D, 6, seed=7)).astype(np.float32)).cuda()

    def img(**opt):
        out = fbp.Plan(n, A, D, **opt).reconstruct(sino)
        torch.cuda.synchronize()
        return out.cpu().numpy()
    paired = img(tile_x=32, tile_y=32, point_pairs=1)
    single = img(tile_x=32, tile_y=32, point_pairs=-1)
    assert not np.array_equal(paired, single)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    if 4 * 24 * 12 >= 7 * sms:
        assert np.array_equal(img(), paired)
    assert np.array_equal(img(tile_x=32, tile_y=32), single)
    assert np.array_equal(img(point_pairs=-1), img(tile_x=32, tile_y=64, point_pairs=-1))
    # FP16 pairs keep the 32 x 64 tile under point pairs
    if 4 * 24 * 12 >= 7 * sms:
        assert np.array_equal(img(q_storage=2),
                              img(q_storage=2, tile_x=32, tile_y=64, point_pairs=1))
        assert not np.array_equal(img(q_storage=2),
                                  img(q_storage=2, tile_x=32, tile_y=32, point_pairs=1))
