import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# A mutated copy of the oracle package (tests/test_oracle_mutants.py) is imported in place of the
# oracle's own when TSGM_ORACLE_ROOT names the folder that holds the copy.
if os.environ.get("TSGM_ORACLE_ROOT"):
    sys.path.insert(0, os.environ["TSGM_ORACLE_ROOT"])


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: full-size cases that take tens of seconds on the CPU")
