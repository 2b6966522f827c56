"""GPU: the index-checking debug build (FBP_CHECK_BOUNDS, libfbp_checked.so).

Its backprojection and FDK kernels check every shared-memory window index
they form and record the first one out of range in the status words instead
of reading outside the staged window (no trap, no fault).  Here, in a child
process that loads the checked build:
  - the workloads of the other GPU tests' kinds (plain, tau != 1 with given
    angles over a full turn, the bench's slice, point-symmetric tile pairs,
    FP16 pairs, Kahan sums, a batch of uneven slices, an FDK volume) run with
    no index out of range, and give the same bits as the normal build;
  - with the check's limit shrunk below the true window (the test-only hook),
    the check fires: FBP_ERR_BOUNDS with the kernel, index and limit in the
    message, and the context stays usable (the next launch is correct).
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# The cases, run by the child (checked build) and by this process (normal
# build) with the same seeded inputs; each returns a dict of named images.
CASES = r'''
import numpy as np, torch
import synthetic
import paper_2109_02174_gb300 as fbp


def sino(spec, th=None):
    return torch.from_numpy(synthetic.sinogram(spec, th).astype(np.float32)).cuda()


def run_cases():
    out = {}
    s = synthetic.cfg_plain()
    out["plain"] = fbp.Plan(s.n_pix, s.n_angles, s.n_det).reconstruct(sino(s))
    s = synthetic.cfg_float_double()
    out["bench_slice"] = fbp.Plan(s.n_pix, s.n_angles, s.n_det,
                                  filter=s.filter).reconstruct(sino(s))
    rng = np.random.default_rng(7)
    for tau in (0.8, 1.6):
        n, A = 200, 150
        D = int(np.ceil(n * np.sqrt(2) / tau)) + 3
        th = np.sort(rng.uniform(0.0, 2.0 * np.pi, A))[::-1].copy()
        s = synthetic.SliceSpec(n, A, D, 8, seed=int(10 * tau), tau=tau)
        out[f"tau{tau}"] = fbp.Plan(n, A, D, angles=th, det_spacing=tau).reconstruct(sino(s, th))
    n, A = 768, 360
    D = synthetic.det_for(n)
    s = synthetic.SliceSpec(n, A, D, 8, seed=5)
    t = sino(s)
    out["point_pairs"] = fbp.Plan(n, A, D, tile_x=32, tile_y=32, point_pairs=1).reconstruct(t)
    out["point_pairs_fp16"] = fbp.Plan(n, A, D, q_storage=2).reconstruct(t)
    out["point_pairs_kahan"] = fbp.Plan(n, A, D, accumulate=1).reconstruct(t)
    s = synthetic.SliceSpec(256, 360, synthetic.det_for(256), 8, seed=6)
    out["kahan"] = fbp.Plan(256, 360, synthetic.det_for(256), accumulate=1).reconstruct(sino(s))
    rng2 = synthetic.SplitMix64(41)
    plans, sinos = [], []
    for k in range(8):
        n = rng2.choice((64, 96, 128, 200))
        a = rng2.choice((45, 90, 180, 360))
        s = synthetic.SliceSpec(n, a, synthetic.det_for(n), 6, seed=600 + k)
        plans.append(fbp.Plan(n, a, s.n_det))
        sinos.append(sino(s))
    batch = fbp.Batch(plans, sinos)
    batch.launch()
    torch.cuda.synchronize()
    batch.status()
    for k, im in enumerate(batch.images):
        out[f"batch{k}"] = im
    P = np.random.default_rng(21).normal(size=(60, 20, 48)).astype(np.float32)
    fp = fbp.FdkPlan(60, 20, 48, 60.0, 32, 32, 16)
    out["fdk"] = fp.reconstruct(torch.from_numpy(P).cuda())
    torch.cuda.synchronize()
    fp.device_status()
    return {k: v.cpu().numpy() for k, v in out.items()}
'''

CHILD = CASES + r'''
import json, sys
import paper_2109_02174_gb300 as fbp
assert fbp.LIB_PATH.endswith("libfbp_checked.so"), fbp.LIB_PATH
imgs = run_cases()   # every call checks its device status: an index out of range raises
np.savez(sys.argv[1], **imgs)
report = {}
# the check fires once its limit is below the window's true width
plan = fbp.Plan(256, 180, 363)
s = synthetic.cfg_plain()
t = sino(s)
want = plan.reconstruct(t)
torch.cuda.synchronize()
plan.device_status()
fbp.fbp_test_shrink_window(1000)
try:
    plan.reconstruct(t)
    torch.cuda.synchronize()
    plan.device_status()
    report["bp"] = "no error"
except fbp.FbpError as e:
    report["bp"] = [e.status, fbp.fbp_last_error()]
P = np.random.default_rng(21).normal(size=(60, 20, 48)).astype(np.float32)
fp = fbp.FdkPlan(60, 20, 48, 60.0, 32, 32, 16)
try:
    fp.reconstruct(torch.from_numpy(P).cuda())
    torch.cuda.synchronize()
    fp.device_status()
    report["fdk"] = "no error"
except fbp.FbpError as e:
    report["fdk"] = [e.status, fbp.fbp_last_error()]
fbp.fbp_test_shrink_window(0)
again = plan.reconstruct(t)
torch.cuda.synchronize()
plan.device_status()
report["recovered"] = bool(np.array_equal(again.cpu().numpy(), want.cpu().numpy()))
print(json.dumps(report))
'''


@pytest.fixture(scope="module")
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_02174_gb300 import build
    build.build()
    return build.build(check_bounds=True)


def test_checked_build_matches_and_reports(built, tmp_path):
    npz = str(tmp_path / "checked.npz")
    env = dict(os.environ, FBP_LIBRARY=built)
    r = subprocess.run([sys.executable, "-c", CHILD, npz], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    report = json.loads(r.stdout.strip().splitlines()[-1])
    import paper_2109_02174_gb300 as fbp
    for kind, name in (("bp", "backprojection"), ("fdk", "FDK")):
        status, msg = report[kind]
        assert status == fbp.FBP_ERR_BOUNDS, report
        assert name in msg and "outside [0, " in msg, msg
    assert report["recovered"]
    # the normal build, same inputs: the same bits
    assert not fbp.LIB_PATH.endswith("libfbp_checked.so")
    scope = {}
    exec(compile(CASES, "cases", "exec"), scope)
    want = scope["run_cases"]()
    got = np.load(npz)
    assert sorted(got.files) == sorted(want)
    for k in want:
        assert np.array_equal(got[k], want[k]), k
