"""The batched persistent fused form (many queries per launch) against the
FP64 oracle and against the per-query path: same ids, distances within
1e-5 relative of FP64, for several batch shapes including ragged tails."""
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


@pytest.fixture(scope="module")
def coll(m):
    x = synth.random_walks(100_000, 256, seed=synth.DATASET_SEED)
    ix = m.messi_build(torch.from_numpy(x).cuda(), 16, 256)
    q = synth.query_mix(x, 70, seed=synth.QUERY_SEED + 100)
    return x, ix, q


def check(ids, d, ref_ids, ref_d2):
    ids = ids.cpu().numpy() if hasattr(ids, "cpu") else ids
    d = d.cpu().numpy() if hasattr(d, "cpu") else d
    assert np.array_equal(ids, ref_ids), np.argwhere(ids != ref_ids)[:5]
    ref = np.sqrt(ref_d2)
    err = np.abs(d.astype(np.float64) - ref) / np.maximum(ref, 1e-30)
    err[(ref == 0) & (d == 0)] = 0
    assert err.max() <= RTOL


@pytest.mark.parametrize("mode", ["lb", "tc"])
@pytest.mark.parametrize("k", [1, 10])
@pytest.mark.parametrize("batch", [1, 16, 64, 0])
def test_batched_matches_oracle_and_plain(m, coll, k, batch, mode):
    x, ix, q = coll
    qd = torch.from_numpy(q).cuda()
    m.messi_set_batch_mode(ix, m.MESSI_BATCH_LB_REFINE if mode == "lb" else m.MESSI_BATCH_TC_SCREEN)
    try:
        ids, d = m.messi_query_batched(ix, qd, k=k, batch=batch)
    finally:
        m.messi_set_batch_mode(ix, m.MESSI_BATCH_TC_SCREEN)
    m.messi_check(ix)
    ref = oracle.knn(x, q, k)
    check(ids, d, *ref)
    pids, pd = m.messi_query(ix, qd, k=k)
    assert np.array_equal(ids.cpu().numpy(), pids.cpu().numpy())
    st = m.messi_query_stats(ix)
    assert st["queries"] == len(q)


def test_batched_host_buffers_and_ties(m):
    x = synth.random_walks(20_000, 128, seed=5)
    x[19_999] = x[3]
    x[10_000] = x[3]
    ix = m.messi_build(torch.from_numpy(x).cuda(), 16, 256, leaf_capacity=200)
    q = np.concatenate([x[[3, 10_000]], synth.query_mix(x, 9, seed=6)])
    ids, d = m.messi_query_batched(ix, q, k=3, batch=4)        # numpy in and out
    m.messi_check(ix)
    check(ids, d, *oracle.knn(x, q, 3))
    assert ids[0].tolist() == [3, 10_000, 19_999]


@pytest.mark.parametrize("nq,k,r", [(1, 1, 12), (6, 2, 12), (13, 5, 25), (13, 1, 0)])
def test_batched_dtw_overlapped_streams(m, coll, nq, k, r):
    """The batched DTW form (per-query kernel sequences on several streams,
    each with its own workspace): the FP64 oracle's ids and distances, equal
    to the per-query path's, for batches smaller and larger than the number
    of streams; the counters add up over the streams."""
    x, ix, q = coll
    sub = x[:20_000]
    iy = m.messi_build(torch.from_numpy(sub).cuda(), 16, 256)
    qd = torch.from_numpy(q[:nq].copy()).cuda()
    ids, d = m.messi_query_batched(iy, qd, k=k, dist=m.MESSI_DTW, window=r)
    m.messi_check(iy)
    st = m.messi_query_stats(iy)
    check(ids, d, *oracle.knn(sub, q[:nq], k, oracle.DTW, r))
    pids, pd = m.messi_query(iy, qd, k=k, dist=m.MESSI_DTW, window=r)
    m.messi_check(iy)
    sp = m.messi_query_stats(iy)
    assert np.array_equal(ids.cpu().numpy(), pids.cpu().numpy())
    assert np.array_equal(d.cpu().numpy(), pd.cpu().numpy())
    # the same work, counted over the streams
    assert st["queries"] == sp["queries"] == nq
    assert st["lb_evaluated"] == sp["lb_evaluated"]
    assert st["seeded"] == sp["seeded"]


def test_batched_dtw_host_buffers(m, coll):
    x, ix, q = coll
    sub = x[:20_000]
    iy = m.messi_build(torch.from_numpy(sub).cuda(), 16, 256)
    ids, d = m.messi_query_batched(iy, q[:9], k=3, dist=m.MESSI_DTW, window=12)   # numpy in and out
    m.messi_check(iy)
    check(ids, d, *oracle.knn(sub, q[:9], 3, oracle.DTW, 12))


def test_lb_form_graph_replay_matches_oracle(m, coll):
    # the lower-bound form replays one captured graph per full batch; two calls
    # with different query buffers reuse it with new argument tables
    x, ix, _ = coll
    m.messi_set_batch_mode(ix, m.MESSI_BATCH_LB_REFINE)
    try:
        for seed, nq in ((synth.QUERY_SEED + 300, 16 * 5 + 7), (synth.QUERY_SEED + 301, 16 * 3)):
            q = synth.query_mix(x, nq, seed=seed)
            ids, d = m.messi_query_batched(ix, torch.from_numpy(q).cuda(), k=3, batch=16)
            m.messi_check(ix)
            check(ids, d, *oracle.knn(x, q, 3))
            st = m.messi_query_stats(ix)
            assert st["queries"] == nq
            assert st["kernel_launches"] >= 7 * (nq // 16)
    finally:
        m.messi_set_batch_mode(ix, m.MESSI_BATCH_TC_SCREEN)


@pytest.mark.parametrize("mode", ["lb", "tc"])
def test_autotune_picks_a_valid_shape_and_stays_exact(m, coll, mode):
    x, ix, _ = coll
    m.messi_set_batch_mode(ix, m.MESSI_BATCH_LB_REFINE if mode == "lb" else m.MESSI_BATCH_TC_SCREEN)
    try:
        qt = synth.query_mix(x, 256, seed=synth.QUERY_SEED + 400)
        t = m.messi_autotune(ix, torch.from_numpy(qt).cuda(), k=1)
        assert t["batch"] in ((32, 64, 128, 256) if mode == "lb" else (128, 256))
        assert t["chunk_tiles"] in (16, 32, 64) and t["ctas_per_sm"] in (1, 2)
        assert t["ms_per_query"] > 0
        q = synth.query_mix(x, 40, seed=synth.QUERY_SEED + 401)
        ids, d = m.messi_query_batched(ix, torch.from_numpy(q).cuda(), k=2)   # batch 0: the tuned one
        m.messi_check(ix)
        check(ids, d, *oracle.knn(x, q, 2))
    finally:
        m.messi_set_batch_mode(ix, m.MESSI_BATCH_TC_SCREEN)
        m.messi_set_tuning(ix, 64, 32, 2)


def test_set_tuning_rejects_bad_shapes(m, coll):
    _, ix, _ = coll
    for bad in ((0, 32, 2), (64, 0, 2), (64, 32, 3)):
        with pytest.raises(m.MessiError):
            m.messi_set_tuning(ix, *bad)


@pytest.mark.parametrize("n,w", [(40, 10), (72, 9)])
def test_batched_lengths_outside_the_screen(m, n, w):
    # the tensor-core screen needs len % 16 == 0 (and len <= 2048); other lengths
    # take the lower-bound form in either batch mode and stay exact
    x = synth.random_walks(8_000, n, seed=60 + n)
    ix = m.messi_build(torch.from_numpy(x).cuda(), w, 256)
    q = synth.query_mix(x, 20, seed=61 + n)
    for mode in (m.MESSI_BATCH_TC_SCREEN, m.MESSI_BATCH_LB_REFINE):
        m.messi_set_batch_mode(ix, mode)
        ids, d = m.messi_query_batched(ix, torch.from_numpy(q).cuda(), k=4, batch=8)
        m.messi_check(ix)
        check(ids, d, *oracle.knn(x, q, 4))


@pytest.mark.parametrize("mode", ["lb", "tc"])
def test_batched_non_finite_query_isolated(m, coll, mode):
    # a query holding NaN / inf answers -1 / NaN and is reported; its batch
    # neighbours are unaffected
    x, ix, _ = coll
    q = synth.query_mix(x, 12, seed=synth.QUERY_SEED + 500)
    q[3, 40] = np.nan
    q[7, 0] = np.inf
    m.messi_set_batch_mode(ix, m.MESSI_BATCH_LB_REFINE if mode == "lb" else m.MESSI_BATCH_TC_SCREEN)
    try:
        ids, d = m.messi_query_batched(ix, torch.from_numpy(q).cuda(), k=3, batch=8)
        with pytest.raises(m.MessiError) as e:
            m.messi_check(ix)
        assert e.value.status == 1
    finally:
        m.messi_set_batch_mode(ix, m.MESSI_BATCH_TC_SCREEN)
    ids, d = ids.cpu().numpy(), d.cpu().numpy()
    bad = [3, 7]
    good = [i for i in range(12) if i not in bad]
    assert (ids[bad] == -1).all() and np.isnan(d[bad]).all()
    check(ids[good], d[good], *oracle.knn(x, q[good], 3))
    m.messi_check(ix)
