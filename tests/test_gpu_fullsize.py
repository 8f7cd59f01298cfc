"""Parity at full size, in the launch configuration the benchmark times.

The collections are drawn on the device exactly as bench.py draws them (10M
and 100M random walks of length 256); queries are the same class mix.  The
library answers whole batches (1024 queries per screened batch, as timed),
and four queries of every class are checked against the FP64 oracle run over
the whole collection (rows copied to the host in chunks), for k = 1 and 10.
DTW at 10M with a 25-point window is checked against the oracle's brute
force over all 10M rows.
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


def classed_mix(data, count, seed, per_class):
    """The bench's query mix (half fresh walks, then noisy members with sigma
    0.1 / 0.5 / 1.0), permuted as one batch; returns the batch and, for each
    class, the batch positions of `per_class` of its queries."""
    q = synth.query_mix_torch(data, count, seed=seed)
    n_fresh = count // 2
    rest = count - n_fresh
    sizes = [n_fresh] + [rest // 3 + (1 if i < rest % 3 else 0) for i in range(3)]
    starts = np.cumsum([0] + sizes[:-1])
    g = torch.Generator()
    g.manual_seed(seed)
    perm = torch.randperm(count, generator=g)
    where = torch.empty_like(perm)
    where[perm] = torch.arange(count)          # batch position of original query i
    picks = [[int(where[int(a) + j]) for j in range(per_class)] for a in starts]
    return q.index_select(0, perm.to(q.device)).contiguous(), picks


@pytest.mark.parametrize("n", [10_000_000, 100_000_000])
def test_ed_full_size_sampled(m, n):
    data = synth.random_walks_torch(n, 256, seed=synth.DATASET_SEED)
    ix = m.messi_build(data, 16, 256)
    # 1024 mixed queries per screened batch, as timed; four queries of each
    # class (fresh walks, sigma 0.1 / 0.5 / 1.0 members) checked one by one
    q, picks = classed_mix(data, 1024, synth.QUERY_SEED + 17, 4)
    sample = [p for cls in picks for p in cls]
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
    # plain path on the sampled queries, k = 1 and 10
    p1, pd1 = m.messi_query(ix, q[sample], k=1)
    m.messi_check(ix)
    check_sample(p1, pd1, list(range(len(sample))), ref1[0], ref1[1])
    p10, pd10 = m.messi_query(ix, q[sample], k=10)
    m.messi_check(ix)
    check_sample(p10, pd10, list(range(len(sample))), ref10[0], ref10[1])
    m.messi_free(ix)
    torch.cuda.empty_cache()


def test_dtw_10m_full_oracle(m):
    """10M x 256 under DTW with a 25-point window: every returned id and
    distance against the FP64 brute force over the whole collection (the
    method's answer equals brute force, Theorem 2), for two fresh walks and
    two members with sigma 0.5 noise."""
    n, r = 10_000_000, 25
    data = synth.random_walks_torch(n, 256, seed=synth.DATASET_SEED)
    ix = m.messi_build(data, 16, 256)
    q = torch.cat([synth.random_walks_torch(2, 256, seed=synth.QUERY_SEED + 3),
                   synth.noisy_members_torch(data, 2, 0.5, seed=synth.NOISE_SEED + 3)[0]]).contiguous()
    ref_ids, ref_d2 = oracle_over_device(data, q.cpu().numpy(), 1, oracle.DTW, r)
    del data
    torch.cuda.empty_cache()
    ids, d = m.messi_query(ix, q, k=1, dist=m.MESSI_DTW, window=r)
    m.messi_check(ix)
    check_sample(ids, d, list(range(q.shape[0])), ref_ids, ref_d2)
    m.messi_free(ix)
    torch.cuda.empty_cache()
