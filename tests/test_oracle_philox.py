"""Pin oracle.philox to numpy's independent Philox4x64-10 implementation."""
import numpy as np
import pytest

from oracle.philox import philox4x64_10, uniform53, draws

CASES = [((0, 0, 0, 0), (0, 0)), ((5, 0, 0, 0), (7, 9)),
         ((2**64 - 2, 3, 2**63, 11), (2**64 - 1, 12345)),
         ((123456789, 42, 0, 0), (20241202, 1023))]


@pytest.mark.parametrize("ctr,key", CASES)
def test_matches_numpy_philox(ctr, key):
    # numpy advances the counter by one before each block
    v = sum(int(w) << (64 * i) for i, w in enumerate(ctr))
    v = (v - 1) % 2**256
    c = [(v >> (64 * i)) & (2**64 - 1) for i in range(4)]
    bg = np.random.Philox(counter=np.array(c, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    want = [int(x) for x in bg.random_raw(4)]
    assert list(philox4x64_10(ctr, key)) == want


def test_uniform_range_and_resolution():
    assert uniform53(0) == 0.0
    assert uniform53(2**64 - 1) == 1.0 - 2.0**-53
    assert uniform53(1 << 11) == 2.0**-53


def test_stream_layout_distinct():
    a = draws(1, 2, 3, 4)
    assert a != draws(1, 2, 3, 5) and a != draws(1, 3, 3, 4) and a != draws(2, 2, 3, 4)
    assert all(0.0 <= u < 1.0 for u in a)
