import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")
    # Modules that import the binding load libpnop.so at import time, during
    # collection: build it first (nvcc cross-compiles without a GPU; a no-op
    # when the library is up to date).
    from paper_2509_10103_gb300 import build
    build.build()
