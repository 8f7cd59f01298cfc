"""Pins for the FP64 oracle: what the paper and the mathematics fix.

Each test ties an oracle routine to something other than itself -- a closed
form, a textbook value, a hand-worked case, a library routine that computes
the same quantity by another route, an invariant the paper proves, or brute
force over every possibility on a tiny input -- so a dropped term, a wrong
sign or index or a transposed operand in the oracle fails one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------- breakpoints
def test_breakpoints_textbook_quartiles():
    # c = 4: the textbook N(0,1) quartiles -0.67449, 0, +0.67449.
    b = oracle.breakpoints(4)
    assert b.shape == (3,)
    assert b[1] == 0.0
    assert abs(b[2] - 0.6744897501960817) < 1e-15
    assert abs(b[0] + 0.6744897501960817) < 1e-15


def test_breakpoints_textbook_octiles():
    b = oracle.breakpoints(8)
    assert abs(b[6] - 1.1503493803760079) < 1e-14     # PhiInv(7/8)
    assert abs(b[4] - 0.31863936396437514) < 1e-15    # PhiInv(5/8)


@pytest.mark.parametrize("card", [2, 4, 8, 16, 32, 64, 128, 256])
def test_breakpoints_vs_scipy_symmetry_monotone(card):
    sp = pytest.importorskip("scipy.special")
    b = oracle.breakpoints(card)
    ref = sp.ndtri(np.arange(1, card) / card)
    assert np.all(np.abs(b - ref) <= 4 * np.spacing(np.abs(ref)) + 1e-300)
    assert np.all(np.diff(b) > 0)
    assert np.all(np.abs(b + b[::-1]) <= 4 * np.spacing(np.abs(b)))
    assert b[card // 2 - 1] == 0.0
    # the regions are equiprobable: Phi(beta_j) = j / c (scipy's ndtr)
    assert np.allclose(sp.ndtr(b), np.arange(1, card) / card, rtol=0, atol=1e-15)


@pytest.mark.parametrize("card", [2, 4, 8, 16, 32, 64, 128, 256])
def test_breakpoints_are_the_nearest_doubles(card):
    # beta_j is the double nearest the real quantile PhiInv(j/c): checked
    # against a 300-bit evaluation (mpmath's erfinv), 0 ulps
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 300
    b = oracle.breakpoints(card)
    for j in range(1, card):
        exact = mpmath.sqrt(2) * mpmath.erfinv(2 * mpmath.mpf(j) / card - 1)
        gap = abs(mpmath.mpf(b[j - 1]) - exact)
        for nb in (np.nextafter(b[j - 1], -np.inf), np.nextafter(b[j - 1], np.inf)):
            assert gap < abs(mpmath.mpf(nb) - exact), (card, j)


def test_breakpoint_examples_to_the_last_bit():
    # the nearest doubles of three textbook quantiles (their decimal forms
    # pin the value to the bit): PhiInv(1/4), PhiInv(7/8), PhiInv(1/256)
    assert oracle.breakpoints(4)[0] == -0.6744897501960817
    assert oracle.breakpoints(8)[6] == 1.150349380376008
    assert oracle.breakpoints(256)[0] == -2.6600674686174597


# ------------------------------------------------------------------- PAA
def test_paa_constant_and_ramp():
    n, w = 256, 16
    m = n // w
    assert np.all(oracle.paa(np.full(n, 3.25, np.float32), w) == 3.25)
    ramp = np.arange(n, dtype=np.float32)
    # mean of s*m .. s*m+m-1 is s*m + (m-1)/2
    assert np.array_equal(oracle.paa(ramp, w), np.arange(w) * m + (m - 1) / 2)


def test_paa_vs_numpy_mean():
    x = synth.random_walks(50, 128, seed=7)
    for row in x:
        ref = row.astype(np.float64).reshape(8, 16).mean(axis=1)
        assert np.allclose(oracle.paa(row, 8), ref, rtol=0, atol=1e-14)


# ------------------------------------------------------------------- SAX
def test_sax_word_paper_example():
    spec = {}
    for line in open(os.path.join(GOLDEN, "isax_word_example.txt")):
        if line.strip() and not line.startswith("#"):
            k, *v = line.split()
            spec[k] = v
    w, card = int(spec["segments"][0]), int(spec["cardinality"][0])
    word = [int(s, 2) for s in spec["word"]]            # 10 00 11 -> 2 0 3
    beta = oracle.breakpoints(card)
    # PAA values inside regions 2, 0, 3: (0, 0.674), (-inf, -0.674), (0.674, inf)
    p = np.array([0.3, -1.0, 1.2])
    sym = oracle.sax(p, card, beta)
    assert list(sym) == word
    assert "".join(format(int(s), "02b") for s in sym) == "".join(spec["word"])
    assert w == len(sym)


def test_sax_boundaries_upper_region():
    card = 4
    beta = oracle.breakpoints(card)
    # a value equal to a breakpoint goes to the upper region
    assert list(oracle.sax(beta, card, beta)) == [1, 2, 3]
    below = np.nextafter(beta, -np.inf)
    assert list(oracle.sax(below, card, beta)) == [0, 1, 2]
    assert list(oracle.sax([-1e300, 1e300], card, beta)) == [0, 3]


@pytest.mark.parametrize("card", [2, 16, 256])
def test_sax_vs_searchsorted(card):
    beta = oracle.breakpoints(card)
    rng = np.random.default_rng(3)
    p = np.concatenate([rng.normal(size=500), beta, np.nextafter(beta, np.inf),
                        np.nextafter(beta, -np.inf)])
    assert np.array_equal(oracle.sax(p, card, beta),
                          np.searchsorted(beta, p, side="right").astype(np.uint8))


def test_summarize_matches_rowwise():
    x = synth.random_walks(64, 256, seed=11)
    words = oracle.summarize(x, 16, 256)
    beta = oracle.breakpoints(256)
    for i in range(64):
        assert np.array_equal(words[i], oracle.sax(oracle.paa(x[i], 16), 256, beta))


# ------------------------------------------------------------ iSAX key
def test_isax_key_hand_worked():
    # w = 2, c = 4: symbols 2 = 10b and 1 = 01b.  Bit planes from the MSB:
    # plane 0 = (1, 0), plane 1 = (0, 1) -> key bits 1,0,0,1 then zeros.
    assert oracle.isax_key([2, 1], 4) == 0b1001 << 124
    # w = 16, c = 256: symbol 0x80 in segment 0 only -> the single top bit
    s = np.zeros(16, np.uint8)
    s[0] = 0x80
    assert oracle.isax_key(s, 256) == 1 << 127
    s[:] = 0
    s[15] = 1                              # last bit plane, last segment
    assert oracle.isax_key(s, 256) == 1


def test_isax_key_prefix_is_node_word():
    # The first d*w bits of the key are the first d bits of every symbol
    # (the node word at cardinality 2^d per segment, Sec. 2.2).
    rng = np.random.default_rng(5)
    for _ in range(50):
        sym = rng.integers(0, 256, 16).astype(np.uint8)
        key = oracle.isax_key(sym, 256)
        for d in range(1, 9):
            prefix = key >> (128 - 16 * d)
            expect = 0
            for j in range(d):
                for s in range(16):
                    expect = (expect << 1) | ((int(sym[s]) >> (7 - j)) & 1)
            assert prefix == expect


# ------------------------------------------------------------------ ED
def test_ed2_closed_form():
    assert oracle.ed2(np.zeros(256), np.ones(256)) == 256.0
    q = np.arange(8, dtype=np.float32)
    assert oracle.ed2(q, q) == 0.0
    assert oracle.ed2(q, q + 2) == 32.0


# ----------------------------------------------------------- mindist ED
def test_mindist_ed_closed_form():
    card, m = 4, 16
    beta = oracle.breakpoints(card)
    # one segment, candidate in region 3 = [0.674, inf), query PAA -1
    d = beta[2] + 1.0
    assert oracle.mindist_ed2([-1.0], [3], m, card, beta) == pytest.approx(m * d * d, rel=1e-15)
    # candidate in region 0 = (-inf, -0.674], query PAA 2 -> distance 2 + 0.674
    d = 2.0 - beta[0]
    assert oracle.mindist_ed2([2.0], [0], m, card, beta) == pytest.approx(m * d * d, rel=1e-15)
    # two segments add
    both = oracle.mindist_ed2([-1.0, 2.0], [3, 0], m, card, beta)
    assert both == pytest.approx(m * ((beta[2] + 1) ** 2 + (2 - beta[0]) ** 2), rel=1e-15)


def test_mindist_zero_inside_own_box():
    x = synth.random_walks(100, 256, seed=13)
    beta = oracle.breakpoints(256)
    for row in x:
        p = oracle.paa(row, 16)
        assert oracle.mindist_ed2(p, oracle.sax(p, 256, beta), 16, 256, beta) == 0.0


@pytest.mark.parametrize("card,w", [(256, 16), (16, 16), (4, 8)])
def test_mindist_lower_bounds_ed_all_pairs(card, w):
    # Property 1 (Sec. 4): mindist(PAA(Q), iSAX(C)) <= ED(Q, C) for every pair.
    n = 128
    x = synth.random_walks(150, n, seed=17)
    q = np.concatenate([synth.random_walks(10, n, seed=19), synth.noisy_members(x, 10, 0.1)[0]])
    beta = oracle.breakpoints(card)
    words = oracle.summarize(x, w, card)
    tight = 0
    for qi in q:
        pq = oracle.paa(qi, w)
        for i in range(x.shape[0]):
            lb = oracle.mindist_ed2(pq, words[i], n // w, card, beta)
            ed = oracle.ed2(qi, x[i])
            assert lb <= ed * (1 + 1e-12)
            tight += lb > 0.2 * ed
    assert tight > 0            # the bound is not trivially zero


# -------------------------------------------------------------- envelope
def test_envelope_hand_worked():
    U, L = oracle.envelope([1, 3, 2, 5, 4], 1)
    assert list(U) == [3, 3, 5, 5, 5]
    assert list(L) == [1, 1, 2, 2, 4]
    U, L = oracle.envelope([1, 3, 2, 5, 4], 0)
    assert list(U) == [1, 3, 2, 5, 4] and list(L) == [1, 3, 2, 5, 4]
    U, L = oracle.envelope([1, 3, 2, 5, 4], 10)       # window covers everything
    assert list(U) == [5] * 5 and list(L) == [1] * 5


def test_lb_keogh_hand_worked_and_r0_is_ed():
    assert oracle.lb_keogh2([3, 3, 5], [1, 1, 2], np.array([4, 0, 3], np.float32)) == 2.0
    x = synth.random_walks(20, 64, seed=23)
    q = synth.random_walks(1, 64, seed=29)[0]
    U, L = oracle.envelope(q, 0)
    for row in x:
        assert oracle.lb_keogh2(U, L, row) == oracle.ed2(q, row)


# ------------------------------------------------------------------ DTW
def test_dtw_hand_worked():
    q = np.array([0, 1, 2], np.float32)
    x = np.array([0, 0, 1], np.float32)
    # worked by hand: full window and r = 1 both give 1; ED^2 is 2
    assert oracle.dtw2(q, x, 2) == 1.0
    assert oracle.dtw2(q, x, 1) == 1.0
    assert oracle.dtw2(q, x, 0) == 2.0
    assert oracle.ed2(q, x) == 2.0
    # warping helps only with the window: q = (0, 1), x = (1, 1)
    assert oracle.dtw2([0, 1, 1], [0, 0, 1], 1) == 0.0


def _paths(n, r):
    """All warping paths from (0,0) to (n-1,n-1) inside the window."""
    out = []

    def go(i, j, acc):
        if (i, j) == (n - 1, n - 1):
            out.append(acc)
            return
        for di, dj in ((1, 0), (0, 1), (1, 1)):
            a, b = i + di, j + dj
            if a < n and b < n and abs(a - b) <= r:
                go(a, b, acc + [(a, b)])

    go(0, 0, [(0, 0)])
    return out


@pytest.mark.parametrize("r", [0, 1, 2, 4])
def test_dtw_vs_all_warping_paths(r):
    # DTW = minimum over every warping path of the summed squared costs.
    rng = np.random.default_rng(31 + r)
    n = 5
    for _ in range(20):
        q = rng.normal(size=n).astype(np.float32)
        x = rng.normal(size=n).astype(np.float32)
        best = min(sum((float(q[i]) - float(x[j])) ** 2 for i, j in p) for p in _paths(n, r))
        assert oracle.dtw2(q, x, r) == pytest.approx(best, rel=1e-13)


def test_lb_improved_hand_worked():
    # q = (0, 0, 0), x = (3, 0, -3), r = 1: the envelope of q is 0 everywhere,
    # so LB_Keogh = 9 + 0 + 9 and h = (0, 0, 0); q sits inside h's envelope,
    # so the second term is 0.  The r = 1 DTW is 18 too (every path pays both
    # ends), so the bound is tight here.
    q = np.zeros(3, dtype=np.float32)
    x = np.array([3.0, 0.0, -3.0], dtype=np.float32)
    assert oracle.lb_improved2(q, x, 1) == 18.0
    assert oracle.dtw2(q, x, 1) == 18.0
    # q = (0, 5, 0), x = (0, 0, 0), r = 0: U = L = q, h = q, second term 0:
    # the bound is LB_Keogh = ED = 25
    q2 = np.array([0.0, 5.0, 0.0], dtype=np.float32)
    assert oracle.lb_improved2(q2, np.zeros(3, np.float32), 0) == 25.0
    # q = (0, 4, 0, 0), x = (0, 0, 0, 4), r = 1: U = (4, 4, 4, 0),
    # L = (0, 0, 0, 0); x_3 = 4 > U_3 = 0 costs 16, h = (0, 0, 0, 0), whose
    # envelope is 0, and q_1 = 4 above it costs 16: bound 32
    q3 = np.array([0.0, 4.0, 0.0, 0.0], dtype=np.float32)
    x3 = np.array([0.0, 0.0, 0.0, 4.0], dtype=np.float32)
    assert oracle.lb_improved2(q3, x3, 1) == 32.0
    assert oracle.dtw2(q3, x3, 1) >= 32.0


@pytest.mark.parametrize("n,r", [(16, 0), (16, 1), (16, 3), (32, 5), (64, 6), (64, 63), (37, 4)])
def test_lb_keogh_le_lb_improved_le_dtw(n, r):
    rng = np.random.default_rng(40 + n + r)
    for t in range(60):
        q = rng.standard_normal(n).astype(np.float32)
        # smooth, noisy and shifted candidates
        if t % 3 == 0:
            x = np.cumsum(rng.standard_normal(n)).astype(np.float32)
        elif t % 3 == 1:
            x = (q + rng.normal(0, 1.0, n)).astype(np.float32)
        else:
            x = np.roll(q, rng.integers(-r - 1, r + 2)).astype(np.float32)
        U, L = oracle.envelope(q, r)
        lk = oracle.lb_keogh2(U, L, x)
        li = oracle.lb_improved2(q, x, r)
        d = oracle.dtw2(q, x, r)
        assert lk <= li * (1 + 1e-12) + 1e-12
        assert li <= d * (1 + 1e-12) + 1e-9


def test_dtw_invariants():
    n = 128
    x = synth.random_walks(40, n, seed=37)
    q = synth.random_walks(3, n, seed=41)
    beta = oracle.breakpoints(256)
    words = oracle.summarize(x, 16, 256)
    for qi in q:
        for r in (0, 3, 12, 30, n - 1):
            U, L = oracle.envelope(qi, r)
            pu = np.array([U[s * 8:(s + 1) * 8].mean() for s in range(16)])
            pl = np.array([L[s * 8:(s + 1) * 8].mean() for s in range(16)])
            for i, row in enumerate(x):
                dtw = oracle.dtw2(qi, row, r)
                lbk = oracle.lb_keogh2(U, L, row)
                lbi = oracle.mindist_dtw2(pu, pl, words[i], 8, 256, beta)
                assert lbi <= lbk * (1 + 1e-12) + 1e-12      # iSAX-envelope LB <= LB_Keogh
                assert lbk <= dtw * (1 + 1e-12)              # LB_Keogh <= DTW
                assert dtw <= oracle.ed2(qi, row)            # DTW <= ED
                if r == 0:
                    assert dtw == oracle.ed2(qi, row)
                    assert lbi == oracle.mindist_ed2(oracle.paa(qi, 16), words[i], 8, 256, beta)
        # wider window never increases DTW
        row = x[0]
        vals = [oracle.dtw2(qi, row, r) for r in range(0, 20)]
        assert all(a >= b for a, b in zip(vals, vals[1:]))


def test_envelope_paa_matches_means():
    q = synth.random_walks(1, 256, seed=43)[0]
    pu, pl = oracle.envelope_paa(q, 25, 16)
    U, L = oracle.envelope(q, 25)
    assert np.allclose(pu, U.reshape(16, 16).mean(1), atol=1e-14)
    assert np.allclose(pl, L.reshape(16, 16).mean(1), atol=1e-14)
    assert np.all(pu >= oracle.paa(q, 16)) and np.all(pl <= oracle.paa(q, 16))


# ------------------------------------------------------------------ k-NN
def _numpy_knn(x, q, k, fn):
    ids, ds = [], []
    for qi in q:
        d = np.array([fn(qi, row) for row in x])
        order = np.lexsort((np.arange(len(x)), d))[:k]    # by d, then id
        ids.append(order)
        ds.append(d[order])
    return np.array(ids), np.array(ds)


@pytest.mark.parametrize("k", [1, 5])
def test_knn_ed_vs_lexsort_with_ties(k):
    x = synth.random_walks(400, 64, seed=47)
    x[300] = x[17]            # exact duplicates: ties go to the lowest id
    x[301] = x[17]
    x[5] = x[250]
    q = np.concatenate([x[[17, 250, 3]], synth.random_walks(5, 64, seed=53)])
    ids, d2 = oracle.knn(x, q, k, oracle.ED, threads=3)
    rid, rd = _numpy_knn(x, q, k, lambda a, b: float(((a.astype(np.float64) - b) ** 2).sum()))
    assert np.array_equal(ids, rid)
    assert np.allclose(d2, rd, rtol=1e-12, atol=0)
    assert ids[0, 0] == 17 and ids[1, 0] == 5
    if k >= 3:
        assert list(ids[0, :3]) == [17, 300, 301]


def test_knn_dtw_vs_pairwise():
    x = synth.random_walks(120, 32, seed=59)
    q = synth.random_walks(4, 32, seed=61)
    ids, d2 = oracle.knn(x, q, 3, oracle.DTW, r=3, threads=2)
    rid, rd = _numpy_knn(x, q, 3, lambda a, b: oracle.dtw2(a, b, 3))
    assert np.array_equal(ids, rid) and np.array_equal(d2, rd)


def test_knn_stream_equals_whole():
    x = synth.random_walks(1000, 64, seed=67)
    q = synth.random_walks(6, 64, seed=71)
    whole = oracle.knn(x, q, 4)
    blocks = [(lo, x[lo:lo + 137]) for lo in range(0, 1000, 137)]
    part = oracle.knn_stream(blocks, q, 4)
    assert np.array_equal(whole[0], part[0]) and np.array_equal(whole[1], part[1])


# ------------------------------------------------------- leaf grouping
@pytest.mark.parametrize("N,cap,card", [(3000, 50, 256), (2000, 7, 16), (500, 1000, 256)])
def test_leaf_partition_properties(N, cap, card):
    w = 16
    x = synth.random_walks(N, 128, seed=73)
    x[10:40] = x[9]                      # 31 identical series -> identical keys
    words = oracle.summarize(x, w, card)
    order, off, depth = oracle.leaf_partition(words, card, cap)
    total = w * (card.bit_length() - 1)
    keys = oracle.isax_keys(words, card)
    assert sorted(order.tolist()) == list(range(N))           # Thm 1: each series once
    sk = [(keys[i], int(i)) for i in order]
    assert sk == sorted(sk)
    assert off[0] == 0 and off[-1] == N and np.all(np.diff(off) > 0)
    for li in range(len(depth)):
        lo, hi, d = off[li], off[li + 1], int(depth[li])
        assert w <= d <= total
        pre = {keys[i] >> (128 - d) for i in order[lo:hi]}
        assert len(pre) == 1                                   # one trie node
        p = pre.pop()
        members = sum(1 for kk in keys if kk >> (128 - d) == p)
        assert members == hi - lo                              # the whole node
        if hi - lo > cap:
            assert d == total                                  # only full-key duplicates overflow
        if d > w:                                              # its parent had to split
            parent = p >> 1
            assert sum(1 for kk in keys if kk >> (128 - d + 1) == parent) > cap


# ------------------------------------------------------ sliding windows
@pytest.mark.parametrize("length,n,stride", [(1000, 64, 1), (1003, 64, 3), (257, 256, 1), (300, 16, 7)])
def test_windows_plain_are_slices(length, n, stride):
    # Sec. 2 / Sec. 6: window i is series[i*stride .. i*stride + n); the
    # number of windows is the number of starts that leave n points
    x = np.random.default_rng(length + n).normal(size=length).astype(np.float32)
    w = oracle.windows(x, n, stride, znorm=False)
    ref = np.lib.stride_tricks.sliding_window_view(x, n)[::stride]
    assert w.shape == ref.shape == ((length - n) // stride + 1, n)
    assert np.array_equal(w, ref)


def test_windows_znorm_matches_numpy_population_moments():
    # z-normalisation (Sec. 2: mean 0, standard deviation 1) against numpy's
    # mean and population std in float64, a different summation order: equal
    # to within float32 rounding, and a sample std (n - 1) would be 0.2% off
    x = np.cumsum(np.random.default_rng(5).normal(size=5000)).astype(np.float32)
    n = 256
    w = oracle.windows(x, n, 5, znorm=True)
    raw = np.lib.stride_tricks.sliding_window_view(x, n)[::5].astype(np.float64)
    ref = (raw - raw.mean(axis=1, keepdims=True)) / raw.std(axis=1, keepdims=True)
    assert np.max(np.abs(w - ref)) < 2e-6
    assert np.max(np.abs(w.astype(np.float64).mean(axis=1))) < 1e-6
    assert np.max(np.abs(w.astype(np.float64).std(axis=1) - 1.0)) < 1e-6


def test_windows_constant_window_becomes_zeros():
    x = np.random.default_rng(6).normal(size=400).astype(np.float32)
    x[100:200] = 2.5
    w = oracle.windows(x, 64, 1, znorm=True)
    assert np.all(w[100:137] == 0.0)            # windows entirely inside the constant stretch
    assert np.any(w[99] != 0.0)                  # starts on a random point
