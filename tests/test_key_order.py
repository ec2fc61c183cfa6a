"""CPU checks of the closest-hit key encoding (a9, a11): key = FP32 bits of
t << 32 | triangle id, kept with a u64 minimum.

For t > 0, the IEEE-754 bit patterns of positive floats are ordered like the
floats, so the u64 minimum is the lexicographic minimum of (t, id): the
closest hit, with ties to the lower id.  The miss sentinel 0x7F800000FFFFFFFF
is above every key of a finite positive t and decodes to (+inf, 0xFFFFFFFF).
"""
import numpy as np

KEY_MISS = 0x7F800000FFFFFFFF
NO_HIT = 0xFFFFFFFF


def _keys(t, ids):
    bits = np.asarray(t, np.float32).view(np.uint32).astype(np.uint64)
    return (bits << np.uint64(32)) | np.asarray(ids, np.uint64)


def test_key_minimum_is_lexicographic_minimum():
    rng = np.random.default_rng(0)
    n = 200_000
    t = np.exp(rng.uniform(np.log(1e-30), np.log(1e30), n)).astype(np.float32)
    t[: n // 10] = rng.choice(t[: n // 100], n // 10)            # exact ties in t
    t[-1000:] = np.float32(1e-42) * rng.integers(1, 1000, 1000)   # subnormal distances
    ids = rng.integers(0, 2**32 - 1, n, dtype=np.uint64)
    k = _keys(t, ids)
    order_keys = np.argsort(k, kind="stable")
    order_lex = np.lexsort((ids, t.astype(np.float64)))
    assert np.array_equal(k[order_keys], k[order_lex])
    # groups of candidates for one ray: the key minimum picks the closest, lowest id on ties
    for _ in range(200):
        m = rng.integers(1, 40)
        sel = rng.choice(n, m, replace=False)
        kmin = k[sel].min()
        tb, ib = t[sel], ids[sel]
        best = np.lexsort((ib, tb.astype(np.float64)))[0]
        assert kmin == k[sel][best]


def test_miss_sentinel():
    tb = np.array([KEY_MISS >> 32], np.uint64).astype(np.uint32).view(np.float32)[0]
    assert np.isposinf(tb) and (KEY_MISS & 0xFFFFFFFF) == NO_HIT
    finite = _keys(np.array([np.finfo(np.float32).max, 1.0, 1e-45], np.float32), [NO_HIT, 0, 5])
    assert np.all(finite < np.uint64(KEY_MISS))
