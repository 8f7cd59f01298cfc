"""Parity at full size, in the launch configuration the benchmark times.

The collections are drawn on the device exactly as bench.py draws them (10M
and 100M random walks of length 256); queries are the same class mix.  The
library answers whole batches (1024 queries per screened batch, as timed),
and a sample of the answers is checked against the FP64 oracle run over the
whole collection (rows copied to the host in chunks).  For DTW at 10M the
oracle checks each returned distance and that no row of a random 200K-row
sample beats the returned neighbour -- properties that hold at any size.
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


def oracle_over_device(data_t, queries, k, dist=oracle.ED, r=0, chunk=1 << 20):
    """FP64 brute force of `queries` over the device collection, chunk by chunk."""
    host = torch.empty((min(chunk, data_t.shape[0]), data_t.shape[1]), dtype=torch.float32, pin_memory=True)

    def blocks():
        for lo in range(0, data_t.shape[0], chunk):
            hi = min(data_t.shape[0], lo + chunk)
            host[: hi - lo].copy_(data_t[lo:hi])
            yield lo, host[: hi - lo].numpy()

    return oracle.knn_stream(blocks(), queries, k, dist, r)


def check_sample(ids, dists, sample, ref_ids, ref_d2):
    got_ids = ids.cpu().numpy()[sample]
    got_d = dists.cpu().numpy()[sample].astype(np.float64)
    assert np.array_equal(got_ids, ref_ids), (got_ids, ref_ids)
    ref = np.sqrt(ref_d2)
    assert np.all(np.abs(got_d - ref) <= RTOL * np.maximum(ref, 1e-30))


def mixed_queries(data, count, seed):
    q = synth.query_mix_torch(data, count, seed=seed)
    g = torch.Generator()
    g.manual_seed(seed)
    return q.index_select(0, torch.randperm(count, generator=g).to(q.device)).contiguous()


@pytest.mark.parametrize("n", [10_000_000, 100_000_000])
def test_ed_full_size_sampled(m, n):
    data = synth.random_walks_torch(n, 256, seed=synth.DATASET_SEED)
    ix = m.messi_build(data, 16, 256)
    q = mixed_queries(data, 1024, synth.QUERY_SEED + 17)
    # fresh, and one of each noise level (the mix is permuted: pick by class)
    sample = [0, 1, 700, 1500 % 1024, 1023]
    qs = q[sample].cpu().numpy()
    ref10 = oracle_over_device(data, qs, 10)
    ref1 = (ref10[0][:, :1], ref10[1][:, :1])     # (dist, id) order: the 1-NN heads the 10-NN
    del data
    torch.cuda.empty_cache()
    # screened batch, 1024 queries per launch as timed
    i1, d1 = m.messi_query_batched(ix, q, k=1, batch=1024)
    m.messi_check(ix)
    check_sample(i1, d1, sample, ref1[0], ref1[1])
    i10, d10 = m.messi_query_batched(ix, q, k=10, batch=1024)
    m.messi_check(ix)
    check_sample(i10, d10, sample, ref10[0], ref10[1])
    # plain path on the sampled queries
    p1, pd1 = m.messi_query(ix, q[sample], k=1)
    m.messi_check(ix)
    check_sample(p1, pd1, list(range(len(sample))), ref1[0], ref1[1])
    m.messi_free(ix)
    torch.cuda.empty_cache()


def test_dtw_10m_properties(m):
    n, r = 10_000_000, 25
    data = synth.random_walks_torch(n, 256, seed=synth.DATASET_SEED)
    ix = m.messi_build(data, 16, 256)
    q = torch.cat([synth.random_walks_torch(1, 256, seed=synth.QUERY_SEED + 3),
                   synth.noisy_members_torch(data, 1, 0.5, seed=synth.NOISE_SEED + 3)[0]]).contiguous()
    ids, d = m.messi_query(ix, q, k=1, dist=m.MESSI_DTW, window=r)
    m.messi_check(ix)
    ids, d = ids.cpu().numpy()[:, 0], d.cpu().numpy()[:, 0].astype(np.float64)
    qn = q.cpu().numpy()
    rng = np.random.default_rng(11)
    sample = np.sort(rng.choice(n, 200_000, replace=False))
    rows = data[torch.from_numpy(sample).cuda()].cpu().numpy()
    for j in range(len(qn)):
        own = data[int(ids[j])].cpu().numpy()
        exact = np.sqrt(oracle.dtw2(qn[j], own, r))
        assert abs(d[j] - exact) <= RTOL * max(exact, 1e-30)
        s_ids, s_d2 = oracle.knn(rows, qn[j:j + 1], 1, oracle.DTW, r)
        best_d, best_id = np.sqrt(s_d2[0, 0]), int(sample[s_ids[0, 0]])
        assert (best_d > exact) or (best_d == exact and best_id >= int(ids[j])) or best_id == int(ids[j])
    m.messi_free(ix)
    del data
    torch.cuda.empty_cache()
