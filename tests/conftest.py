import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# cached fronts stay inside the repository unless HODLR_FRONT_CACHE says otherwise
os.environ.setdefault("HODLR_FRONT_CACHE", os.path.join(ROOT, ".front_cache"))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
