import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    # test modules load libjx.so when they are collected: rebuild it first if
    # a source is newer (nvcc cross-compiles without a GPU)
    from paper_2605_19926_gb300 import build

    if build.needs_build():
        build.build()


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    oracle.lib()
    return oracle
