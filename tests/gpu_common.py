"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest

import workloads as W

X = W.wavelength_grid()
T = W.hmi_filters(X)
LINE = W.FE6173


def f32(a):
    """Round to float32 and back: the oracle sees exactly the GPU's inputs."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.fixture(scope="session")
def vf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0901_2702_gb300 import build
    build.build()
    import paper_0901_2702_gb300 as v
    h = v.vfisv_create(0)
    yield v, h, torch
    h.close()
