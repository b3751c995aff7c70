import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session", autouse=True)
def _built_libraries():
    """Build whatever native piece is missing or stale (the oracle, the CUDA
    library, the device input generator) before any test imports it."""
    import __graft_entry__
    import oracle
    import synth

    gbuild = __graft_entry__.builder()

    if not os.path.exists(oracle.LIB) or os.path.getmtime(oracle.LIB) < os.path.getmtime(oracle.SRC):
        oracle.build()
    if not gbuild.up_to_date():
        gbuild.build()
    src = os.path.join(os.path.dirname(synth.LIB_PATH), "synth.cu")
    if not os.path.exists(synth.LIB_PATH) or os.path.getmtime(synth.LIB_PATH) < os.path.getmtime(src):
        synth.build()
    yield
