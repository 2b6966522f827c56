"""GPU: a 3D volume from a stack of reconstructed slices (linear interpolation
along z) equals the FP64 oracle's on the same float32 slices, on uneven
spacing, for the vector path (n^2 a multiple of four) and the scalar one,
over more planes than one launch takes; bad arguments are rejected on the
host."""
import numpy as np
import pytest

import oracle
import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fbp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_02174_gb300 import build
    build.build()
    import paper_2109_02174_gb300 as m
    return m


def _compare(fbp, slices, z, zo):
    got = fbp.volume(slices, z, zo).cpu().numpy().astype(np.float64)
    want = oracle.volume(np.stack([s.cpu().numpy() for s in slices]).astype(np.float64), z, zo)
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 1e-6 * scale


@pytest.mark.parametrize("n", [64, 37])
def test_volume_matches_oracle(fbp, n):
    import torch
    g = torch.Generator(device="cuda").manual_seed(n)
    slices = [torch.randn((n, n), device="cuda", generator=g) for _ in range(7)]
    z = np.array([0.0, 1.0, 1.5, 3.0, 3.2, 5.0, 8.0])
    zo = np.linspace(0.0, 8.0, 300)  # two launches
    _compare(fbp, slices, z, zo)


def test_volume_of_a_reconstructed_batch(fbp):
    """The paper's use: the slices of a batch reconstruction, interpolated to
    four planes per slice gap."""
    import torch
    specs = [synthetic.SliceSpec(96, 90, synthetic.det_for(96), 6, seed=60 + k) for k in range(5)]
    plan = fbp.Plan(96, 90, synthetic.det_for(96))
    sinos = [torch.from_numpy(synthetic.sinogram(s).astype(np.float32)).cuda() for s in specs]
    batch = fbp.Batch([plan] * 5, sinos)
    batch.launch()
    torch.cuda.synchronize()
    z = np.arange(5) * 2.0
    _compare(fbp, batch.images, z, np.linspace(0.0, 8.0, 17))


def test_volume_argument_errors(fbp):
    import torch
    s = [torch.zeros((8, 8), device="cuda") for _ in range(3)]
    with pytest.raises(fbp.FbpError) as e:
        fbp.volume(s, [0.0, 1.0, 1.0], [0.5])
    assert e.value.status == fbp.FBP_ERR_INVALID_ARG
    with pytest.raises(fbp.FbpError) as e:
        fbp.volume(s, [0.0, 1.0, 2.0], [2.5])
    assert e.value.status == fbp.FBP_ERR_INVALID_ARG
