"""Serving loop: requests submitted one at a time, the same requests
arriving as a Poisson stream, and the same requests as one burst released
at once (continuous batching, mixed ED / DTW and k) give identical results,
which also match the FP64 oracle; the burst shares batches and keeps several
requests in flight."""
import threading
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def m():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import paper_2110_07519_gb300 as mod

    return mod


def make_requests(x, count, seed):
    rng = np.random.default_rng(seed)
    qs = synth.query_mix(x, count, seed=seed)
    reqs = []
    for i in range(count):
        dtw = rng.random() < 0.2
        reqs.append((qs[i], int(rng.choice([1, 10])), 1 if dtw else 0, 12 if dtw else 0))
    return reqs


def test_alone_equals_in_the_mix_and_oracle(m):
    x = synth.random_walks(60_000, 128, seed=901)
    ix = m.messi_build(torch.from_numpy(x).cuda(), 16, 256)
    srv = m.messi_server_create(ix, max_batch=64, max_k=16, streams=2)
    reqs = make_requests(x, 120, seed=902)

    alone = []
    for q, k, dist, r in reqs:
        t = m.messi_server_submit(srv, q, k, dist, r)
        res = None
        while res is None:
            res = m.messi_server_poll(srv, t, k, wait_us=200_000)
        alone.append(res)

    # the same requests as a Poisson stream while results are collected
    rng = np.random.default_rng(903)
    order = rng.permutation(len(reqs))
    tickets = {}

    def producer():
        for i in order:
            q, k, dist, r = reqs[i]
            tickets[i] = m.messi_server_submit(srv, q, k, dist, r)
            time.sleep(rng.exponential(200e-6))

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    mixed = [None] * len(reqs)
    for i in order:
        k = reqs[i][1]
        while mixed[i] is None:
            mixed[i] = m.messi_server_poll(srv, tickets[i], k, wait_us=200_000)
    bad = [i for i in range(len(reqs))
           if not (np.array_equal(alone[i][0], mixed[i][0]) and np.array_equal(alone[i][1], mixed[i][1]))]
    if bad:
        lines = []
        for i in bad[:5]:
            q, k, dist, r = reqs[i]
            ref_ids, ref_d2 = oracle.knn(x, q, k, dist, r)
            lines.append(f"req {i}: dist={dist} k={k} r={r}\n alone {alone[i][0].tolist()} {alone[i][1].tolist()}"
                         f"\n mixed {mixed[i][0].tolist()} {mixed[i][1].tolist()}"
                         f"\n oracle {ref_ids[0].tolist()} {np.sqrt(ref_d2[0]).tolist()}")
        pytest.fail(f"{len(bad)} requests differ alone vs in the mix:\n" + "\n".join(lines))
    st = m.messi_server_get_stats(srv)
    assert st["completed"] == st["submitted"] == 2 * len(reqs)
    assert st["p99_ms"] >= st["p50_ms"] > 0

    # the same requests as one burst that arrives while admission is held:
    # on release the workers take them as shared batches, several requests in
    # flight at once, and every answer is unchanged
    m.messi_server_pause(srv)
    burst = {i: m.messi_server_submit(srv, *reqs[i]) for i in order}
    m.messi_server_pause(srv, False)
    together = [None] * len(reqs)
    for i in order:
        while together[i] is None:
            together[i] = m.messi_server_poll(srv, burst[i], reqs[i][1], wait_us=200_000)
    st2 = m.messi_server_get_stats(srv)
    assert st2["completed"] - st["completed"] == len(reqs)
    assert st2["batches"] - st["batches"] < len(reqs)     # requests shared batches
    assert st2["inflight_peak"] > 1
    for i in range(len(reqs)):
        assert np.array_equal(together[i][0], alone[i][0]) and np.array_equal(together[i][1], alone[i][1]), i

    # exactness of every answer against the oracle: one brute-force pass per
    # distance at the largest k (a k-NN answer is the prefix of the 10-NN)
    for dist, r in ((0, 0), (1, 12)):
        sel = [j for j in range(len(reqs)) if reqs[j][2] == dist]
        ref_ids, ref_d2 = oracle.knn(x, np.stack([reqs[j][0] for j in sel]), 10, dist, r)
        for row, i in enumerate(sel):
            k = reqs[i][1]
            assert np.array_equal(mixed[i][0], ref_ids[row, :k]), i
            ref = np.sqrt(ref_d2[row, :k])
            rel = np.abs(mixed[i][1] - ref) / np.maximum(ref, 1e-30)
            assert rel.max() <= 1e-5, i
    m.messi_server_destroy(srv)
    m.messi_check(ix)


def test_server_rejects_bad_requests(m):
    x = synth.random_walks(2000, 64, seed=904)
    ix = m.messi_build(torch.from_numpy(x).cuda(), 16, 256)
    srv = m.messi_server_create(ix, max_batch=8, max_k=4, streams=1, max_queued=1000)
    with pytest.raises(m.MessiError):
        m.messi_server_submit(srv, x[0], k=5)                 # above max_k
    with pytest.raises(m.MessiError):
        m.messi_server_submit(srv, x[0], k=1, dist=1, window=64)
    with pytest.raises(m.MessiError):
        m.messi_server_poll(srv, 12345, 1)                    # unknown ticket
    t = m.messi_server_submit(srv, x[7], k=2)
    res = None
    while res is None:
        res = m.messi_server_poll(srv, t, 2, wait_us=100_000)
    assert res[0][0] == 7 and res[1][0] == 0.0
    m.messi_server_destroy(srv)
