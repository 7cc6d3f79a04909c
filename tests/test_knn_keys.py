"""The float32 kNN keeps its top-k list as 64-bit keys, (bits of d^2) << 32 |
index, and compares them as unsigned integers.  That is the (d^2, index)
order of the neighbour definition (ties broken by the smaller index) only
because a non-negative float32 orders like its bit pattern.  This checks
the premise in numpy on random, tied, tiny (subnormal and zero), huge and
infinite squared distances, and the two sentinel keys the kernel uses: 0
below every entry and the key of (+inf, INT_MAX) above every real one."""
import numpy as np


def _keys(d2, idx):
    bits = np.asarray(d2, np.float32).view(np.uint32).astype(np.uint64)
    return (bits << np.uint64(32)) | np.asarray(idx, np.uint32).astype(np.uint64)


def _lexsorted(d2, idx):
    return np.lexsort((np.asarray(idx, np.int64), np.asarray(d2, np.float64)))


def test_key_order_is_the_distance_index_order():
    rng = np.random.default_rng(0)
    tiny = np.float32(1e-45)  # the smallest subnormal
    pools = [
        rng.random(5000, dtype=np.float32) * np.float32(1e6),
        rng.integers(0, 20, 5000).astype(np.float32),            # many ties
        np.concatenate([np.zeros(50, np.float32), np.full(50, tiny),
                        rng.random(100, dtype=np.float32) * np.float32(1e-38)]),
        np.concatenate([rng.random(100, dtype=np.float32) * np.float32(3e38),
                        np.full(20, np.inf, np.float32)]),
    ]
    for d2 in pools:
        idx = rng.permutation(d2.size).astype(np.int64)
        idx[: d2.size // 3] = rng.integers(0, 2**31 - 1, d2.size // 3)  # large indices too
        order_keys = np.argsort(_keys(d2, idx), kind="stable")
        np.testing.assert_array_equal(d2[order_keys], d2[_lexsorted(d2, idx)])
        np.testing.assert_array_equal(idx[order_keys], idx[_lexsorted(d2, idx)])


def test_sentinel_keys_bound_every_real_key():
    rng = np.random.default_rng(1)
    d2 = np.concatenate([rng.random(1000, dtype=np.float32) * np.float32(1e30),
                         np.zeros(5, np.float32), np.full(5, np.inf, np.float32)])
    idx = rng.integers(0, 2**31 - 2, d2.size)
    keys = _keys(d2, idx)
    empty = np.uint64((0x7F800000 << 32) | 0x7FFFFFFF)
    assert (keys >= np.uint64(0)).all()           # the lower sentinel never moves up
    assert (keys < empty).all()                   # every real candidate beats an empty slot
    # a zero distance at index 0 equals the lower sentinel: it settles just
    # above it (the bubble stops on equality), which is still its place
    assert _keys([0.0], [0])[0] == np.uint64(0)


def test_key_halves_give_back_distance_and_index():
    rng = np.random.default_rng(2)
    d2 = rng.random(1000, dtype=np.float32) * np.float32(1e6)
    idx = rng.integers(0, 2**31 - 1, 1000)
    k = _keys(d2, idx)
    np.testing.assert_array_equal((k >> np.uint64(32)).astype(np.uint32).view(np.float32), d2)
    np.testing.assert_array_equal((k & np.uint64(0xFFFFFFFF)).astype(np.int64), idx)
