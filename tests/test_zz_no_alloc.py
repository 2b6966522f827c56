"""fbp_reconstruct_static: the reconstruction entry point that allocates nothing.

It serves callers that cannot allocate device memory when they reconstruct
(a fixed-deadline acquisition loop that cannot absorb cudaMalloc's device-wide
synchronisation, or a host whose device memory belongs to another allocator).
Its scratch is a static device array inside libfbp.  Here it is called through
the C ABI twice in a row, on two different sinograms, and each result must
match fbp_reconstruct (with a caller workspace) within the parity tolerance
used by the other GPU tests.  This file is collected last on purpose.
"""
import numpy as np
import pytest

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


def _close(got, ref):
    scale = float(np.abs(ref).max())
    e_max = float(np.abs(got - ref).max()) / scale
    e_rms = float(np.sqrt(np.mean((got - ref) ** 2))) / scale
    assert e_max <= MAX_REL and e_rms <= RMSE_REL, f"max {e_max:.3e} rmse {e_rms:.3e}"


def test_static_scratch_matches_workspace_path_twice(fbp):
    import torch
    spec = synthetic.cfg_plain()
    plan = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det, filter=spec.filter)
    assert plan.workspace_bytes <= 16 * 1024 * 1024
    stream = torch.cuda.current_stream()
    sp = int(stream.cuda_stream)
    for seed in (1, 2):
        s = synthetic.SliceSpec(spec.n_pix, spec.n_angles, spec.n_det, 10, seed=seed)
        sino = torch.from_numpy(synthetic.sinogram(s).astype(np.float32)).cuda()
        ref = plan.reconstruct(sino)
        out = torch.full_like(ref, float("nan"))
        fbp.fbp_reconstruct_static(plan.handle, sino.data_ptr(), sino.stride(0),
                                   out.data_ptr(), sp)
        torch.cuda.synchronize()
        plan.device_status()
        _close(out.double().cpu().numpy(), ref.double().cpu().numpy())


def test_static_scratch_rejects_plans_beyond_its_capacity(fbp):
    import torch
    spec = synthetic.cfg_large()  # 2048 angles x 2904-float rows: 23.8 MB > 16 MiB
    plan = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det)
    assert plan.workspace_bytes > 16 * 1024 * 1024
    sino = torch.zeros((spec.n_angles, spec.n_det), device="cuda")
    img = torch.zeros((spec.n_pix, spec.n_pix), device="cuda")
    with pytest.raises(fbp.FbpError) as e:
        fbp.fbp_reconstruct_static(plan.handle, sino.data_ptr(), spec.n_det, img.data_ptr(),
                                   int(torch.cuda.current_stream().cuda_stream))
    assert e.value.status == fbp.FBP_ERR_BUDGET
    assert "static" in fbp.fbp_last_error()
