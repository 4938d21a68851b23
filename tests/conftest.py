import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


import pytest  # noqa: E402


@pytest.fixture(autouse=True)
def _fresh_tuning_cache():
    # the library keeps the autotuner's plans for the life of the process;
    # clear them before every test so that no test sees another's tuned plan
    from paper_2411_00991_gb300 import bdecon
    if bdecon._lib is not None:
        bdecon.set_tuning_cache(True)
    yield
