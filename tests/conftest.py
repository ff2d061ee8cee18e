import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU statistics")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_counts(d):
    """Exact c_n from tests/golden/saw_counts_d{d}.txt (index = n)."""
    vals = []
    with open(os.path.join(GOLDEN, "saw_counts_d%d.txt" % d)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            n, c = line.split()
            assert int(n) == len(vals)
            vals.append(int(c))
    return vals


@pytest.fixture(scope="session")
def exact_counts():
    return {2: load_counts(2), 3: load_counts(3)}
