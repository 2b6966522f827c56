"""fbp_reconstruct_static: the reconstruction entry point that allocates nothing.

It serves callers that cannot allocate device memory when they reconstruct
(a fixed-deadline acquisition loop that cannot absorb cudaMalloc's device-wide
synchronisation, or a host whose device memory belongs to another allocator).
Its scratch is a static device array inside libfbp, whose address fbp_plan
looks up.  Here it is called through the C ABI:
  - first on an all-NaN sinogram, which leaves NaN throughout the shared
    array, so a later call that read anything it did not write would show it;
  - then twice in a row on two different sinograms, each result equal bit for
    bit to fbp_reconstruct with a caller workspace (same kernels, same bits)
    and within the parity tolerance of the other GPU tests;
  - with the device's free memory measured before the first of these calls
    and after the last: unchanged.
This file is collected last on purpose; it passes alone in a fresh process and
after the other tests.
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
    # every buffer and every reference result first: nothing below allocates
    poison = torch.full((spec.n_angles, spec.n_det), float("nan"), device="cuda")
    sinos, refs, outs = [], [], []
    for seed in (1, 2):
        s = synthetic.SliceSpec(spec.n_pix, spec.n_angles, spec.n_det, 10, seed=seed)
        sino = torch.from_numpy(synthetic.sinogram(s).astype(np.float32)).cuda()
        sinos.append(sino)
        refs.append(plan.reconstruct(sino))
        outs.append(torch.full_like(refs[-1], float("nan")))
    junk = torch.empty_like(refs[0])
    torch.cuda.synchronize()
    plan.device_status()
    free_before = torch.cuda.mem_get_info()[0]

    fbp.fbp_reconstruct_static(plan.handle, poison.data_ptr(), poison.stride(0),
                               junk.data_ptr(), sp)
    for sino, out in zip(sinos, outs):
        fbp.fbp_reconstruct_static(plan.handle, sino.data_ptr(), sino.stride(0),
                                   out.data_ptr(), sp)
    torch.cuda.synchronize()
    free_after = torch.cuda.mem_get_info()[0]
    plan.device_status()

    assert torch.isnan(junk).all()  # the poison went through the shared array
    for ref, out in zip(refs, outs):
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.array_equal(got, ref.cpu().numpy())
        _close(got.astype(np.float64), ref.double().cpu().numpy())
    assert free_after == free_before, f"device free memory moved by {free_before - free_after} B"


def test_static_scratch_rejects_plans_beyond_its_capacity(fbp):
    import torch
    spec = synthetic.cfg_large()  # 2048 angles x 5808-float rows: 47.6 MB > 16 MiB
    plan = fbp.Plan(spec.n_pix, spec.n_angles, spec.n_det)
    assert plan.workspace_bytes > 16 * 1024 * 1024
    sino = torch.zeros((spec.n_angles, spec.n_det), device="cuda")
    img = torch.zeros((spec.n_pix, spec.n_pix), device="cuda")
    with pytest.raises(fbp.FbpError) as e:
        fbp.fbp_reconstruct_static(plan.handle, sino.data_ptr(), spec.n_det, img.data_ptr(),
                                   int(torch.cuda.current_stream().cuda_stream))
    assert e.value.status == fbp.FBP_ERR_BUDGET
    assert "static" in fbp.fbp_last_error()
