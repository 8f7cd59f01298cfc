"""Tensor-core screening: the tcgen05 operand layout (one GEMM tile against
numpy) and the screened batched query path against the FP64 oracle."""
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


def tile_layout(mat16: np.ndarray) -> np.ndarray:
    """R x K f16 matrix -> the 8-row x 16-byte core-matrix layout (as uint16):
    core matrix (row group g, k-chunk j) at g*(K/8)*64 + j*64 halves, row r of
    it at r*8 halves."""
    R, K = mat16.shape
    out = np.zeros(R * K, dtype=np.uint16)
    bits = mat16.view(np.uint16)
    for r in range(R):
        for k in range(K):
            off = (r // 8) * (K // 8) * 64 + (k // 8) * 64 + (r % 8) * 8 + (k % 8)
            out[off] = bits[r, k]
    return out


@pytest.mark.parametrize("K,N", [(256, 128), (128, 128), (64, 256), (16, 32)])
def test_tc_gemm_tile_matches_numpy(m, K, N):
    rng = np.random.default_rng(K + N)
    A = rng.normal(size=(128, K)).astype(np.float16)
    B = rng.normal(size=(N, K)).astype(np.float16)
    D = m.messi_debug_tc_gemm(tile_layout(A), tile_layout(B), K, N, 128, (K // 8) * 128)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64)).T
    assert np.all(np.abs(D - ref) <= 1e-5 * scale + 1e-6)


@pytest.fixture(scope="module")
def coll(m):
    x = synth.random_walks(100_000, 256, seed=synth.DATASET_SEED)
    ix = m.messi_build(torch.from_numpy(x).cuda(), 16, 256)
    m.messi_set_batch_mode(ix, m.MESSI_BATCH_TC_SCREEN)
    return x, ix


def check(ids, d, ref_ids, ref_d2):
    ids = ids.cpu().numpy() if hasattr(ids, "cpu") else ids
    d = d.cpu().numpy() if hasattr(d, "cpu") else d
    assert np.array_equal(ids, ref_ids), np.argwhere(ids != ref_ids)[:5]
    ref = np.sqrt(ref_d2)
    err = np.abs(d.astype(np.float64) - ref) / np.maximum(ref, 1e-30)
    err[(ref == 0) & (d == 0)] = 0
    assert err.max() <= RTOL


@pytest.mark.parametrize("k,batch,nq", [(1, 0, 70), (1, 128, 300), (10, 64, 90), (3, 7, 20)])
def test_screened_batches_match_oracle(m, coll, k, batch, nq):
    x, ix = coll
    q = synth.query_mix(x, nq, seed=synth.QUERY_SEED + 7 * k + nq)
    ids, d = m.messi_query_batched(ix, torch.from_numpy(q).cuda(), k=k, batch=batch)
    m.messi_check(ix)
    check(ids, d, *oracle.knn(x, q, k))
    st = m.messi_query_stats(ix)
    assert st["queries"] == nq


def test_screened_ties_and_members(m):
    x = synth.random_walks(30_000, 128, seed=77)
    x[29_999] = x[11]
    x[200] = x[11]
    ix = m.messi_build(torch.from_numpy(x).cuda(), 16, 256, leaf_capacity=300)
    m.messi_set_batch_mode(ix, m.MESSI_BATCH_TC_SCREEN)
    q = np.concatenate([x[[11, 200, 5]], synth.noisy_members(x, 20, 1.0, seed=78)[0],
                        synth.random_walks(10, 128, seed=79)])
    for k in (1, 4):
        ids, d = m.messi_query_batched(ix, q, k=k, batch=16)
        m.messi_check(ix)
        check(ids, d, *oracle.knn(x, q, k))
    ids, d = m.messi_query_batched(ix, q[:1], k=3)
    assert ids[0].tolist() == [11, 200, 29_999]


def test_screen_length_512_streamed_query_tiles(m):
    # at len 512 two query tiles (256 KB of f16) no longer fit in shared
    # memory: they are streamed chunk by chunk with the series chunks, two per
    # CTA; three query tiles here make groups of two and of one
    x = synth.random_walks(40_000, 512, seed=85)
    ix = m.messi_build(torch.from_numpy(x).cuda(), 16, 256)
    m.messi_set_batch_mode(ix, m.MESSI_BATCH_TC_SCREEN)
    q = synth.query_mix(x, 300, seed=86)
    m.messi_set_profiling(ix, True)
    for k in (1, 5):
        ids, d = m.messi_query_batched(ix, torch.from_numpy(q).cuda(), k=k, batch=300)
        m.messi_check(ix)
        assert m.messi_query_stats(ix)["screened_queries"] >= 300      # the screen ran
        check(ids, d, *oracle.knn(x, q, k))
    m.messi_set_profiling(ix, False)


@pytest.mark.parametrize("n,N,nq", [(1024, 20_000, 300), (2048, 8_000, 130)])
def test_screen_streamed_query_chunks(m, n, N, nq):
    # beyond 512 points the query tiles are streamed chunk by chunk with the
    # series chunks; 300 queries make query-tile groups of two and of one
    x = synth.random_walks(N, n, seed=87 + n)
    ix = m.messi_build(torch.from_numpy(x).cuda(), 16, 256)
    m.messi_set_batch_mode(ix, m.MESSI_BATCH_TC_SCREEN)
    q = synth.query_mix(x, nq, seed=88 + n)
    m.messi_set_profiling(ix, True)
    for k in (1, 5):
        ids, d = m.messi_query_batched(ix, torch.from_numpy(q).cuda(), k=k, batch=nq)
        m.messi_check(ix)
        assert m.messi_query_stats(ix)["screened_queries"] >= nq      # the screen ran
        check(ids, d, *oracle.knn(x, q, k))
    m.messi_set_profiling(ix, False)


def test_screen_falls_back_outside_f16_range(m):
    x = synth.random_walks(5000, 64, seed=80) * 1e5        # beyond f16: no screen copy
    ix = m.messi_build(torch.from_numpy(x.astype(np.float32)).cuda(), 16, 256)
    m.messi_set_batch_mode(ix, m.MESSI_BATCH_TC_SCREEN)
    q = (synth.random_walks(6, 64, seed=81) * 1e5).astype(np.float32)
    ids, d = m.messi_query_batched(ix, q, k=2)
    m.messi_check(ix)
    check(ids, d, *oracle.knn(x.astype(np.float32), q, 2))


def test_overflowing_queries_screened_again_in_gathered_tiles(m):
    """Queries whose candidate lists overflow a pass are screened again on
    their own, gathered into the first query tile, and still answered exactly.

    For each special query q: 1500 rows q + p with p summing to zero over every
    pair of points (same PAA, so same iSAX word, at squared distance ~100)
    fill the seed leaf, so the first pass starts from a loose bound; k = 256
    lies beyond the top-k tightening, so 18000 rows spread over squared
    distances 10..90 all pass and overflow the 16384-entry candidate list.
    The second pass starts from the exact bound of the rechecked candidates."""
    rng = np.random.default_rng(90)
    L, k = 256, 256
    base = synth.random_walks(30_000, L, seed=91)
    special = synth.random_walks(2, L, seed=92)
    rows = [base]
    for j in range(2):
        a = rng.normal(0.0, 0.625, size=(1500, L // 2))
        rows.append(special[j] + np.stack([a, -a], axis=2).reshape(1500, L))
        u = rng.uniform(10.0, 90.0, size=18000)
        rows.append(special[j] + rng.normal(size=(18000, L)) * np.sqrt(u / L)[:, None])
    x = np.concatenate(rows).astype(np.float32)
    ix = m.messi_build(torch.from_numpy(x).cuda(), 16, 256, leaf_capacity=128)
    m.messi_set_batch_mode(ix, m.MESSI_BATCH_TC_SCREEN)
    q = synth.query_mix(base, 300, seed=93)
    q[5], q[250] = special[0], special[1]        # tile 0 row 5, tile 1 row 122
    m.messi_set_profiling(ix, True)
    ids, d = m.messi_query_batched(ix, torch.from_numpy(q).cuda(), k=k, batch=300)
    m.messi_check(ix)
    st = m.messi_query_stats(ix)
    m.messi_set_profiling(ix, False)
    assert st["scan_launches"] >= 2              # a second pass ran
    check(ids, d, *oracle.knn(x, q, k))
