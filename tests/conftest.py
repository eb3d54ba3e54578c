import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    # pytest creates --basetemp itself but not its parent directory
    base = getattr(config.option, "basetemp", None)
    if base:
        os.makedirs(os.path.dirname(os.path.abspath(str(base))), exist_ok=True)
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")
