import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libkf")


@pytest.fixture(scope="session")
def cuda_ctx_factory():
    """Builds libkf once per session and returns a Context factory."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1605_05508_gb300 import build as B
    B.build()
    from paper_1605_05508_gb300 import kf
    made = []

    def make(radii, **kw):
        c = kf.Context(radii, **kw)
        made.append(c)
        return c
    yield make
    for c in made:
        c.close()
