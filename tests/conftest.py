import functools
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@functools.lru_cache(maxsize=None)
def cached_system(cfg: int):
    from paper_2511_05222_gb300 import systems
    return systems.make_system(cfg)


@pytest.fixture(scope="session")
def sys0():
    return cached_system(0)


@pytest.fixture(scope="session")
def sys1():
    return cached_system(1)
