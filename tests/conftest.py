import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: long CPU test")
    # The binding refuses to import without the compiled library, and the ABI
    # tests load it even without a GPU; a fresh checkout builds it here (nvcc
    # cross-compiles for sm_103a), once, before any test module is collected.
    from paper_2101_12408_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
