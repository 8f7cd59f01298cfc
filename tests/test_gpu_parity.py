"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Integer results (iSAX words, leaf layout, returned ids) must be bit-exact;
distances within 1e-5 relative of the oracle's FP64 values (the tolerance
the method is held to).  Sizes span many scan tiles (1024 words) and leaves
and end in ragged tails.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
RTOL = 1e-5


@pytest.fixture(scope="module")
def m():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2110_07519_gb300 as mod

    return mod


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def check_knn(ids, dists, ref_ids, ref_d2):
    ids = ids.cpu().numpy() if hasattr(ids, "cpu") else ids
    dists = dists.cpu().numpy() if hasattr(dists, "cpu") else dists
    bad = np.argwhere(ids != ref_ids)
    assert bad.size == 0, f"id mismatch at {bad[:5].tolist()}: got {ids[tuple(bad[0])]} want {ref_ids[tuple(bad[0])]}"
    ref = np.sqrt(ref_d2)
    err = np.abs(dists.astype(np.float64) - ref) / np.maximum(ref, 1e-30)
    err[(ref == 0) & (dists == 0)] = 0
    assert err.max() <= RTOL, err.max()


# ---------------------------------------------------------------- summaries
@pytest.mark.parametrize("N,n,w,card", [(100_000, 256, 16, 256), (1, 256, 16, 256), (1037, 128, 16, 256),
                                        (5000, 128, 8, 16), (3001, 64, 16, 4), (700, 2048, 16, 256),
                                        (777, 1024, 4, 256), (999, 256, 16, 2)])
def test_summarize_bit_exact(m, N, n, w, card):
    x = synth.random_walks(N, n, seed=100 + N)
    got = m.messi_summarize(cuda(x), w, card).cpu().numpy()
    ref = oracle.summarize(x, w, card)
    assert np.array_equal(got[:, :w], ref)
    assert not got[:, w:].any()


def test_summarize_values_on_breakpoints(m):
    # rows whose PAA sits exactly on, just below and just above breakpoints:
    # the kernel must take the FP64 decision there and match the oracle
    beta = oracle.breakpoints(256)
    rows = []
    for b in beta[::7]:
        for v in (np.float32(b), np.nextafter(np.float32(b), np.float32(-9)),
                  np.nextafter(np.float32(b), np.float32(9))):
            rows.append(np.full(256, v, np.float32))
            r = np.full(256, v, np.float32)
            r[::2] += np.float32(0.25)
            r[1::2] -= np.float32(0.25)
            rows.append(r)
    x = np.stack(rows)
    got = m.messi_summarize(cuda(x), 16, 256).cpu().numpy()
    assert np.array_equal(got[:, :16], oracle.summarize(x, 16, 256))
    host = m.messi_summarize(x, 16, 256)               # host buffers, same kernel
    assert np.array_equal(host, got)


# ------------------------------------------------------------------ layout
@pytest.mark.parametrize("N,cap,card", [(20_000, 64, 256), (5000, 7, 16), (3000, 5000, 256)])
def test_leaf_layout_matches_oracle(m, N, cap, card):
    x = synth.random_walks(N, 128, seed=7 + N)
    x[100:160] = x[99]                                  # identical words -> one full-key leaf
    ix = m.messi_build(cuda(x), 16, card, leaf_capacity=cap)
    order, off, depth = m.messi_index_layout(ix)
    words = oracle.summarize(x, 16, card)
    r_order, r_off, r_depth = oracle.leaf_partition(words, card, cap)
    assert np.array_equal(order.astype(np.int64), r_order)        # Thm 1: a permutation, in key order
    assert np.array_equal(off.astype(np.int64), r_off)
    assert np.array_equal(depth.astype(np.int32), r_depth)
    info = m.messi_index_get_info(ix)
    assert info["n_leaves"] == len(r_depth)
    assert info["max_leaf_size"] == int(np.diff(r_off).max())


# ------------------------------------------------------------------- ED
@pytest.fixture(scope="module")
def c1(m):
    """100,000 random walks of length 256 (the small collection)."""
    x = synth.random_walks(100_000, 256, seed=synth.DATASET_SEED)
    ix = m.messi_build(cuda(x), 16, 256)
    return x, ix


def test_ed_1nn_fresh_queries(m, c1):
    x, ix = c1
    q = synth.random_walks(100, 256, seed=synth.QUERY_SEED)
    ids, d = m.messi_query(ix, cuda(q), k=1)
    m.messi_check(ix)
    r_ids, r_d2 = oracle.knn(x, q, 1)
    check_knn(ids, d, r_ids, r_d2)
    st = m.messi_query_stats(ix)
    assert st["queries"] == 100
    # words of leaves whose symbol box the bound prunes are never read
    assert 0 < st["lb_evaluated"] <= 100 * x.shape[0]
    assert st["lb_survivors"] < 100 * x.shape[0]


@pytest.mark.parametrize("k", [1, 10])
def test_ed_knn_query_mix(m, c1, k):
    x, ix = c1
    q = synth.query_mix(x, 60, seed=synth.QUERY_SEED + k)
    ids, d = m.messi_query(ix, cuda(q), k=k)
    m.messi_check(ix)
    check_knn(ids, d, *oracle.knn(x, q, k))


def test_host_buffers_same_as_device(m, c1):
    x, ix = c1
    q = synth.random_walks(8, 256, seed=31)
    ids_h, d_h = m.messi_query(ix, q, k=3)              # numpy in, numpy out
    ids_d, d_d = m.messi_query(ix, cuda(q), k=3)
    assert np.array_equal(ids_h, ids_d.cpu().numpy())
    assert np.array_equal(d_h, d_d.cpu().numpy())


def test_leaf_boxes_prune_and_stay_exact(m, c1):
    # fresh queries: most leaves' symbol boxes lie above the seed's bound, so
    # their words are never scanned, and the answer is still the oracle's
    x, ix = c1
    qq = synth.random_walks(12, 256, seed=synth.QUERY_SEED + 7)
    ids, d = m.messi_query(ix, cuda(qq), k=3)
    st = m.messi_query_stats(ix)
    info = m.messi_index_get_info(ix)
    m.messi_check(ix)
    check_knn(ids, d, *oracle.knn(x, qq, 3))
    assert 0 < st["leaves_live"] < len(qq) * info["n_leaves"]
    assert st["lb_evaluated"] < len(qq) * x.shape[0]


def test_ties_go_to_lowest_id(m):
    x = synth.random_walks(30_000, 256, seed=41)
    for dup in ((5, 29_000, 12_345), (77, 78, 20_000)):
        for j in dup[1:]:
            x[j] = x[dup[0]]
    ix = m.messi_build(cuda(x), 16, 256)
    q = np.concatenate([x[[29_000, 78, 77, 100]], synth.noisy_members(x, 6, 0.01, seed=3)[0]])
    for k in (1, 3, 5):
        ids, d = m.messi_query(ix, cuda(q), k=k)
        m.messi_check(ix)
        check_knn(ids, d, *oracle.knn(x, q, k))
    ids, d = m.messi_query(ix, cuda(q[:2]), k=3)
    assert ids.cpu().numpy()[0].tolist() == [5, 12_345, 29_000]
    assert d.cpu().numpy()[0].tolist() == [0.0, 0.0, 0.0]


def test_mass_ties_resolved_exactly(m):
    # 10,001 identical rows (more than one pass of the tie resolver holds) and
    # an all-zero query, against which every z-normalised row lies at nearly
    # the same distance: both resolve exactly, in every query form
    x = synth.random_walks(30_000, 128, seed=51)
    x[10_000:20_000] = x[123]
    ix = m.messi_build(cuda(x), 16, 256)
    q = np.stack([x[123], np.zeros(128, np.float32)])
    for k in (1, 7):
        ref = oracle.knn(x, q, k)
        ids, d = m.messi_query(ix, cuda(q), k=k)
        m.messi_check(ix)
        check_knn(ids, d, *ref)
        for mode in (m.MESSI_BATCH_LB_REFINE, m.MESSI_BATCH_TC_SCREEN):
            m.messi_set_batch_mode(ix, mode)
            ids, d = m.messi_query_batched(ix, cuda(q), k=k)
            m.messi_check(ix)
            check_knn(ids, d, *ref)
    ids, d = m.messi_query(ix, cuda(q[:1]), k=3)
    assert ids.cpu().numpy()[0].tolist() == [123, 10_000, 10_001]
    assert d.cpu().numpy()[0].tolist() == [0.0, 0.0, 0.0]


@pytest.mark.parametrize("N,k", [(1, 1), (2, 2), (50, 50), (1037, 7), (4099, 1024)])
def test_ed_edge_sizes(m, N, k):
    x = synth.random_walks(N, 64, seed=N)
    ix = m.messi_build(cuda(x), 16, 256, leaf_capacity=16)
    q = synth.random_walks(3, 64, seed=N + 1)
    ids, d = m.messi_query(ix, cuda(q), k=k)
    m.messi_check(ix)
    check_knn(ids, d, *oracle.knn(x, q, k))


def test_long_series_and_small_alphabet(m):
    x = synth.random_walks(3000, 1024, seed=51)
    ix = m.messi_build(cuda(x), 8, 16, leaf_capacity=100)
    q = synth.query_mix(x, 10, seed=52)
    ids, d = m.messi_query(ix, cuda(q), k=4)
    m.messi_check(ix)
    check_knn(ids, d, *oracle.knn(x, q, 4))


# ------------------------------------------------------------------- DTW
@pytest.fixture(scope="module")
def dtw_set(m):
    x = synth.random_walks(20_000, 256, seed=61)
    ix = m.messi_build(cuda(x), 16, 256)
    q = np.concatenate([synth.random_walks(6, 256, seed=62), synth.noisy_members(x, 6, 0.5, seed=63)[0]])
    return x, ix, q


@pytest.mark.parametrize("r,k", [(25, 1), (25, 5), (0, 1), (3, 2)])
def test_dtw_parity(m, dtw_set, r, k):
    x, ix, q = dtw_set
    ids, d = m.messi_query(ix, cuda(q), k=k, dist=m.MESSI_DTW, window=r)
    m.messi_check(ix)
    check_knn(ids, d, *oracle.knn(x, q, k, oracle.DTW, r))


def test_dtw_window_zero_equals_ed(m, dtw_set):
    x, ix, q = dtw_set
    a = m.messi_query(ix, cuda(q), k=3, dist=m.MESSI_DTW, window=0)
    b = m.messi_query(ix, cuda(q), k=3)
    assert np.array_equal(a[0].cpu().numpy(), b[0].cpu().numpy())


@pytest.mark.parametrize("n,r", [(128, 12), (128, 5), (128, 30), (64, 7), (64, 20), (256, 40)])
def test_dtw_window_shapes(m, n, r):
    # windows whose 2r+1 blocks do not divide the length (series ends)
    x = synth.random_walks(8000, n, seed=300 + n + r)
    ix = m.messi_build(cuda(x), 16, 256, leaf_capacity=300)
    q = np.concatenate([synth.random_walks(3, n, seed=301 + r), synth.noisy_members(x, 3, 1.0, seed=302 + r)[0]])
    for k in (1, 4):
        ids, d = m.messi_query(ix, cuda(q), k=k, dist=m.MESSI_DTW, window=r)
        m.messi_check(ix)
        check_knn(ids, d, *oracle.knn(x, q, k, oracle.DTW, r))


def test_dtw_many_logged_candidates(m):
    # fresh random-walk queries against 60K series: the first refinement wave
    # accepts tens of thousands of candidates against a loose seed threshold,
    # all of which the near-tie log must keep
    x = synth.random_walks(60000, 128, seed=310)
    ix = m.messi_build(cuda(x), 16, 256)
    q = synth.random_walks(6, 128, seed=311)
    for k in (1, 10):
        ids, d = m.messi_query(ix, cuda(q), k=k, dist=m.MESSI_DTW, window=12)
        m.messi_check(ix)
        check_knn(ids, d, *oracle.knn(x, q, k, oracle.DTW, 12))


def test_dtw_short_series_full_window(m):
    x = synth.random_walks(3000, 64, seed=71)
    ix = m.messi_build(cuda(x), 16, 256, leaf_capacity=50)
    q = synth.random_walks(4, 64, seed=72)
    for r in (6, 63):
        ids, d = m.messi_query(ix, cuda(q), k=2, dist=m.MESSI_DTW, window=r)
        m.messi_check(ix)
        check_knn(ids, d, *oracle.knn(x, q, 2, oracle.DTW, r))


# ------------------------------------------------------------ lower bounds
def test_lower_bounds_vs_oracle(m, c1):
    x, ix = c1
    sub = slice(0, 4000)
    beta = oracle.breakpoints(256)
    words = oracle.summarize(x[sub], 16, 256)
    for qi in synth.random_walks(3, 256, seed=81):
        lb = m.messi_lower_bounds(ix, cuda(qi)).cpu().numpy()[sub].astype(np.float64)
        pq = oracle.paa(qi, 16)
        ref = np.array([oracle.mindist_ed2(pq, w, 16, 256, beta) for w in words])
        ed = np.array([oracle.ed2(qi, row) for row in x[sub]])
        assert np.all(lb <= ref * (1 + 1e-12) + 1e-30)          # never above the exact bound
        assert np.all(lb >= ref * (1 - 2e-6) - 1e-6)            # and only rounding below it
        assert np.all(lb <= ed)                                  # Property 1
    qi = synth.random_walks(1, 256, seed=82)[0]
    lbd = m.messi_lower_bounds(ix, cuda(qi), m.MESSI_DTW, 25).cpu().numpy()[sub].astype(np.float64)
    pu, pl = oracle.envelope_paa(qi, 25, 16)
    U, L = oracle.envelope(qi, 25)
    refd = np.array([oracle.mindist_dtw2(pu, pl, w, 16, 256, beta) for w in words])
    assert np.all(lbd <= refd * (1 + 1e-12) + 1e-30)
    assert np.all(lbd >= refd * (1 - 2e-6) - 1e-6)
    lbk = np.array([oracle.lb_keogh2(U, L, row) for row in x[:300]])
    assert np.all(lbd[:300] <= lbk)


# ------------------------------------------------------------------ errors
def test_non_finite_query_reported(m, c1):
    x, ix = c1
    q = synth.random_walks(2, 256, seed=91)
    q[1, 17] = np.nan
    ids, d = m.messi_query(ix, cuda(q), k=2)
    with pytest.raises(m.MessiError) as e:
        m.messi_check(ix)
    assert e.value.status == 1
    ids = ids.cpu().numpy()
    assert (ids[1] == -1).all() and np.isnan(d.cpu().numpy()[1]).all()
    check_knn(ids[:1], d[:1], *oracle.knn(x, q[:1], 2))
    m.messi_check(ix)                                  # the status word was cleared


def test_non_finite_series_rejected(m):
    x = synth.random_walks(100, 64, seed=92)
    x[40, 3] = np.inf
    with pytest.raises(m.MessiError) as e:
        m.messi_build(cuda(x), 16, 256)
    assert e.value.status == 1
