"""Failure paths that fault nothing: each error is made on the host or by a
bounded device wait that runs out, and the library reports it as a status.

* A k > 1 query whose result-array lock is held (test hook) gives up after
  its spin limit: messi_check reports MESSI_ETIMEOUT, and the next query,
  with the hook off, is exact again.
* A build larger than the device's free memory returns MESSI_ENOMEM before
  anything is allocated or read.
* A full arrival queue makes messi_server_submit return MESSI_EBUSY.
* A memory budget smaller than two requests holds admission back: requests
  run one at a time and still get exact answers.
"""
import ctypes

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


def exact(ids, dists, ref_ids, ref_d2):
    ref = np.sqrt(ref_d2)
    return np.array_equal(ids, ref_ids) and np.all(np.abs(dists.astype(np.float64) - ref)
                                                   <= RTOL * np.maximum(ref, 1e-30))


def test_held_result_lock_times_out_then_recovers(m):
    x = synth.random_walks(20_000, 64, seed=71)
    q = synth.query_mix(x, 4, seed=72)
    ix = m.messi_build(torch.from_numpy(x).cuda(), 16, 256)
    m.messi_debug_set_lock_fault(ix, spin_limit=0, hold_lock=True)
    m.messi_query(ix, torch.from_numpy(q).cuda(), k=10)
    with pytest.raises(m.MessiError) as e:
        m.messi_check(ix)
    assert e.value.status == 4                     # MESSI_ETIMEOUT
    m.messi_check(ix)                              # reported once, then cleared
    m.messi_debug_set_lock_fault(ix)               # defaults
    ids, d = m.messi_query(ix, torch.from_numpy(q).cuda(), k=10)
    m.messi_check(ix)
    r_ids, r_d2 = oracle.knn(x, q, 10)
    assert exact(ids.cpu().numpy(), d.cpu().numpy(), r_ids, r_d2)


def test_build_larger_than_device_is_enomem(m):
    lib = m._lib
    small = np.zeros((4, 4096), dtype=np.float32)   # host buffer; never read
    out = ctypes.c_void_p()
    n = (1 << 31)                                   # 2^31 x 4096 floats: 32 TiB
    st = lib.messi_build(ctypes.c_void_p(small.ctypes.data), n, 4096, 16, 256, None, ctypes.c_void_p(0),
                         ctypes.byref(out))
    assert st == 2, m.messi_last_error()            # MESSI_ENOMEM
    assert not out.value
    # the library stays usable
    x = synth.random_walks(3000, 64, seed=73)
    ix = m.messi_build(torch.from_numpy(x).cuda(), 16, 256)
    ids, _ = m.messi_query(ix, torch.from_numpy(x[5:6].copy()).cuda())
    assert int(ids[0, 0]) == 5


def test_full_arrival_queue_is_ebusy(m):
    x = synth.random_walks(10_000, 64, seed=74)
    ix = m.messi_build(torch.from_numpy(x).cuda(), 16, 256)
    srv = m.messi_server_create(ix, max_batch=8, max_k=4, streams=1, max_queued=1)
    m.messi_server_pause(srv)                      # the queue keeps what arrives
    t = m.messi_server_submit(srv, x[11], k=2)
    with pytest.raises(m.MessiError) as e:
        m.messi_server_submit(srv, x[12], k=2)
    assert e.value.status == 5                     # MESSI_EBUSY
    assert m.messi_server_poll(srv, t, 2) is None  # held, not answered yet
    m.messi_server_pause(srv, False)
    res = None
    while res is None:
        res = m.messi_server_poll(srv, t, 2, wait_us=200_000)
    assert res[0][0] == 11 and res[1][0] == 0.0
    st = m.messi_server_get_stats(srv)
    assert st["rejected"] == 1 and st["submitted"] == 1 and st["completed"] == 1
    m.messi_server_destroy(srv)


def test_small_memory_budget_holds_admission_back(m):
    x = synth.random_walks(30_000, 64, seed=75)
    ix = m.messi_build(torch.from_numpy(x).cuda(), 16, 256)
    # a budget below one request's cost: a request is admitted only when
    # nothing else is in flight, whatever the number of streams
    srv = m.messi_server_create(ix, max_batch=64, max_k=4, streams=2, mem_budget=1)
    qs = synth.query_mix(x, 24, seed=76)
    m.messi_server_pause(srv)
    tickets = [m.messi_server_submit(srv, q, k=3) for q in qs]
    m.messi_server_pause(srv, False)
    got = []
    for t in tickets:
        res = None
        while res is None:
            res = m.messi_server_poll(srv, t, 3, wait_us=200_000)
        got.append(res)
    st = m.messi_server_get_stats(srv)
    assert st["completed"] == len(qs)
    assert st["inflight_peak"] == 1                # never two requests at once
    assert st["batches"] == len(qs)
    assert st["budget_waits"] >= 1                 # a worker found the budget full
    m.messi_server_destroy(srv)
    r_ids, r_d2 = oracle.knn(x, qs, 3)
    for i, (ids, d, _) in enumerate(got):
        assert exact(ids, d, r_ids[i], r_d2[i]), i
