import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def madelung():
    """NaCl Madelung constant printed in Sec. 4.1, Eq. st1 (tests/golden/madelung_nacl.txt)."""
    path = os.path.join(ROOT, "tests", "golden", "madelung_nacl.txt")
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                return float(line)
    raise RuntimeError("no value in " + path)
