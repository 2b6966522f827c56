import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def large_reference():
    """The large slice (2048 x 2048, 2048 angles, 2899 bins, Ram-Lak, 40
    ellipses, seed 4): angles, its FP32-rounded sinogram and the FP64 oracle's
    whole image of that sinogram (all host cores), shared by the GPU tests that
    check every pixel of it."""
    import numpy as np

    import oracle
    import synthetic
    spec = synthetic.cfg_large()
    th = synthetic.default_angles(spec.n_angles)
    sino32 = synthetic.sinogram(spec, th).astype(np.float32)
    ref = oracle.fbp(sino32.astype(np.float64), th, spec.tau, spec.filter, spec.n_pix,
                     nthreads=os.cpu_count() or 1)
    return spec, th, sino32, ref
