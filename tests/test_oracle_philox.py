"""Pin the oracle's Philox4x64-10 to numpy's implementation of the same
published generator (numpy increments its 256-bit counter before each block,
so numpy's first block for counter c is Philox(c + 1))."""
import numpy as np
import pytest

from oracle.philox import philox4x64, philox4x64_np, uniform_from_word


@pytest.mark.parametrize("key", [(0, 0), (5, 7), (2**64 - 1, 12345), (0xDEADBEEF, 2**63)])
@pytest.mark.parametrize("ctr", [(0, 0, 0, 0), (41, 3, 9, 1), (2**64 - 2, 7, 2**64 - 1, 5)])
def test_matches_numpy(key, ctr):
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(ctr, dtype=np.uint64))
    ref = [int(v) for v in bg.random_raw(4)]
    nxt = list(ctr)
    nxt[0] = (nxt[0] + 1) % 2**64
    if nxt[0] == 0:
        nxt[1] = (nxt[1] + 1) % 2**64
    assert list(philox4x64(nxt, key)) == ref


def test_vectorised_equals_scalar():
    rng = np.random.default_rng(3)
    c = rng.integers(0, 2**63, size=(64, 4), dtype=np.int64).astype(np.uint64) * np.uint64(2)
    k0, k1 = 0x1234567890ABCDEF, 0xFEDCBA0987654321
    out = philox4x64_np(c[:, 0], c[:, 1], c[:, 2], c[:, 3], k0, k1)
    for i in range(64):
        assert tuple(int(w[i]) for w in out) == philox4x64(tuple(int(v) for v in c[i]), (k0, k1))


def test_uniform_range_and_resolution():
    u = uniform_from_word(np.array([0, 2**64 - 1, 2**11], dtype=np.uint64))
    assert u[0] == 0.0 and u[1] < 1.0 and u[1] == 1.0 - 2.0**-53 and u[2] == 2.0**-53
