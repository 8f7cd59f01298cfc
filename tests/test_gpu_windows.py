"""Sliding-window subsequences (Sec. 2 and Sec. 6): the device windows are
bit-identical to the oracle's, and exact k-NN over an index of the windows of
one long series matches the FP64 oracle over the same windows."""
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


def long_series(length, seed):
    x = synth.random_walks(1, length, seed=seed, znorm=False)[0]
    x[5000:5300] = 3.0                      # constant windows (var = 0)
    x[9000:9100] *= 1000.0                  # a stretch of large magnitude
    return x


@pytest.mark.parametrize("n,stride,znorm", [(64, 1, True), (256, 1, True), (256, 3, True), (64, 5, False),
                                            (16, 2, True)])
def test_windows_bit_identical_to_oracle(m, n, stride, znorm):
    x = long_series(200_003, seed=41)
    got = m.messi_windows(torch.from_numpy(x).cuda(), n, stride, znorm)
    torch.cuda.synchronize()
    ref = oracle.windows(x, n, stride, znorm)
    g = got.cpu().numpy()
    assert g.shape == ref.shape == ((x.size - n) // stride + 1, n)
    assert np.array_equal(g.view(np.uint32), ref.view(np.uint32))


def test_windows_reject_bad_arguments(m):
    x = torch.zeros(100, device="cuda")
    out = torch.empty((37, 64), device="cuda")
    host = np.zeros(100, dtype=np.float32)
    lib = m._lib
    cnt = ctypes.c_uint64(0)
    ptr = ctypes.c_void_p
    EINVAL = 1
    assert lib.messi_windows(ptr(host.ctypes.data), 100, 64, 1, 1, ptr(out.data_ptr()), ctypes.byref(cnt), None) == EINVAL
    assert lib.messi_windows(ptr(x.data_ptr()), 100, 0, 1, 1, ptr(out.data_ptr()), ctypes.byref(cnt), None) == EINVAL
    assert lib.messi_windows(ptr(x.data_ptr()), 100, 64, 0, 1, ptr(out.data_ptr()), ctypes.byref(cnt), None) == EINVAL
    assert lib.messi_windows(ptr(x.data_ptr()), 50, 64, 1, 1, ptr(out.data_ptr()), ctypes.byref(cnt), None) == EINVAL
    assert lib.messi_windows(ptr(x.data_ptr()), 100, 64, 1, 1, ptr(out.data_ptr()), ctypes.byref(cnt), None) == 0
    assert cnt.value == 37
    with pytest.raises(ValueError):
        m.messi_windows(torch.from_numpy(host), 64)


def test_subsequence_knn_matches_oracle(m):
    x = long_series(300_255, seed=42)
    n = 256
    ix = m.messi_build_windows(torch.from_numpy(x).cuda(), n, stride=1, znorm=True)
    win = oracle.windows(x, n, 1, True)
    assert m.messi_index_get_info(ix)["n_series"] == win.shape[0]
    rng = np.random.default_rng(43)
    pick = rng.choice(win.shape[0], 12, replace=False)
    fresh = oracle.windows(synth.random_walks(1, 20_000, seed=44, znorm=False)[0], n, 997, True)[:12]
    noisy = (win[pick[:6]] + rng.normal(0.0, 0.1, size=(6, n))).astype(np.float32)
    q = np.concatenate([win[pick[6:]], noisy, fresh]).astype(np.float32)
    for k in (1, 5):
        ref_ids, ref_d2 = oracle.knn(win, q, k)
        for fn in (m.messi_query, m.messi_query_batched):
            ids, d = fn(ix, torch.from_numpy(q).cuda(), k=k)
            m.messi_check(ix)
            ids, d = ids.cpu().numpy(), d.cpu().numpy().astype(np.float64)
            assert np.array_equal(ids, ref_ids), (fn.__name__, k, np.argwhere(ids != ref_ids)[:5])
            ref = np.sqrt(ref_d2)
            err = np.abs(d - ref) / np.maximum(ref, 1e-30)
            err[(ref == 0) & (d == 0)] = 0
            assert err.max() <= RTOL
    # an exact copy of a window finds itself at distance 0
    ids, d = m.messi_query(ix, torch.from_numpy(win[pick[6:7]]).cuda(), k=1)
    assert int(ids[0, 0]) == int(pick[6]) and float(d[0, 0]) == 0.0
    m.messi_free(ix)
