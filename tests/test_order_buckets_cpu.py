"""The bound buckets that stand in for the paper's priority queues (Sec. 3,
query answering): survivors are counting-sorted by the top 12 bits of their
FP32 bound (8 exponent, 4 mantissa), and a refining thread stops at the first
survivor whose bucket floor exceeds the best-so-far threshold.  That is exact
only if the buckets are monotone in the bound and a bucket's floor never
exceeds a bound in it; restated here from the device functions and checked
over every exponent, subnormals, zero and infinity."""
import numpy as np


def order_bucket(lb: np.ndarray) -> np.ndarray:
    return (lb.astype(np.float32).view(np.uint32) & np.uint32(0x7FFFFFFF)) >> np.uint32(19)


def order_floor(b: np.ndarray) -> np.ndarray:
    return (b.astype(np.uint32) << np.uint32(19)).view(np.float32)


def bounds(rng, n=200_000):
    e = rng.integers(-149, 128, size=n).astype(np.float64)
    v = (rng.random(n) + 1.0) * np.exp2(e)
    v = np.concatenate([v[np.isfinite(v) & (v < 3.4e38)], [0.0, 1e-45, 2e-38, 1.0, 3.4e38, np.inf]])
    return np.sort(v.astype(np.float32))


def test_buckets_monotone_with_floor_below_every_member():
    v = bounds(np.random.default_rng(1))
    b = order_bucket(v)
    assert b.max() < 4096                              # kOrderBuckets
    assert np.all(np.diff(b.astype(np.int64)) >= 0)    # sorted bounds -> sorted buckets
    assert np.all(order_floor(b) <= v)
    nxt = order_floor(b + 1)                           # next bucket's floor lies above every member
    ok = (b + 1 < 4096) & np.isfinite(v)               # (past +inf the next pattern is a NaN)
    assert np.all(nxt[ok] > v[ok])


def test_bucket_spans_at_most_one_sixteenth():
    v = bounds(np.random.default_rng(2))
    v = v[(v >= np.float32(1.2e-38)) & np.isfinite(v)]    # normal numbers
    b = order_bucket(v)
    assert np.all(v.astype(np.float64) < order_floor(b).astype(np.float64) * (1.0 + 1.0 / 16.0) * (1 + 1e-12))


def test_stopping_at_the_first_floor_above_the_threshold_misses_nothing():
    # a thread walks survivors in bucket order (any order inside a bucket) and
    # stops at the first whose bucket floor exceeds thr: every survivor with
    # bound <= thr has been visited
    rng = np.random.default_rng(3)
    for _ in range(200):
        lb = (rng.random(500) * 10.0 ** rng.integers(-3, 4)).astype(np.float32)
        b = order_bucket(lb)
        perm = rng.permutation(lb.size)
        order = perm[np.argsort(b[perm], kind="stable")]          # bucket order, shuffled inside
        thr = np.float32(np.quantile(lb, rng.random()))
        seen = set()
        for i in order:
            if order_floor(np.array([b[i]]))[0] > thr:
                break
            seen.add(int(i))
        assert all(int(i) in seen for i in np.nonzero(lb <= thr)[0])
