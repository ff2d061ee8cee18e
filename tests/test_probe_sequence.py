"""The occupancy hash's probe sequence (host-side check of a property the kernel
relies on): probe i of a key looks at slot home + i(i+1)/2 mod 2^k, and the first
2^k probes visit every slot once, so an insertion into a table that is not full
always finds a free slot within the kernel's bound of 2^k probes."""
import numpy as np
import pytest


@pytest.mark.parametrize("log2h", list(range(1, 17)))
def test_triangular_probes_visit_every_slot(log2h):
    size = 1 << log2h
    i = np.arange(size, dtype=np.int64)
    for home in (0, 1, size // 3, size - 1):
        slots = (home + i * (i + 1) // 2) % size
        assert np.unique(slots).size == size


def test_triangular_probes_by_increments():
    # the kernel forms probe i + 1 from probe i by adding i + 1
    size = 1 << 10
    s, seen = 123, []
    for it in range(size):
        seen.append(s)
        s = (s + it + 1) & (size - 1)
    assert sorted(seen) == list(range(size))
