"""The register-band DTW walk of the refinement kernel, modelled on the CPU.

The kernel walks the candidate's columns: it keeps one column of the
Sakoe-Chiba band in 2R + 1 registers (band slot b of column j is the query
point i = j - R + b; slots outside the reach r or the matrix are +inf), reads
the previous column's slot b as the diagonal, slot b + 1 as the cell of the
previous column in the same row, and the new slot b - 1 as the cell below in
the same column.  The query values of a column come from four copies of the
query in shared memory, shifted by 0..3 points and padded with +inf, read
four at a time from 16-byte-aligned positions; a slot off the ends of the
query meets +inf and so stays +inf without a test, and only a window below
the reach (r < R) forces the slots farther than r to +inf.  Restated step by step in FP64, with the
kernel's index arithmetic for the copies, the walk must reproduce the
oracle's banded DTW (the textbook full-table recurrence, row by row over the
query) bit for bit: the arithmetic is the same, only the storage and the
order of the walk differ, so any indexing slip shows as a different value.
The band minimum of every column must also stay at or below the final
distance (the kernel abandons on it, every fourth column)."""
import math

import numpy as np
import pytest

import oracle

PAD = 36      # kDtwPad


def shifted_copies(q):
    n = q.size
    S = (n + 2 * PAD + 3) & ~3      # dtw_qstride: every copy 16-byte aligned
    Qs = np.zeros(4 * S)
    for e in range(4 * S):
        sh, t = divmod(e, S)
        m = t + sh - PAD
        Qs[e] = float(q[m]) if 0 <= m < n else math.inf
    return Qs, S


def band_walk(q, x, R, r):
    n, W = q.size, 2 * R + 1
    INF = math.inf
    Qs, S = shifted_copies(q)
    D = [0.0 if b == R else INF for b in range(W)]
    cmins = []
    for j in range(n):
        xj = float(x[j])
        t0 = j - R + PAD
        sh = t0 & 3
        base = sh * S + (t0 - sh)
        assert base % 4 == 0 and base >= 0                     # an aligned 16-byte load
        nv = (W + 3) // 4
        assert base + 4 * nv <= 4 * S                          # inside the four copies
        left = INF
        for b in range(W):
            i = j - R + b
            qv = Qs[base + b]
            assert qv == (float(q[i]) if 0 <= i < n else INF)
            up = D[b + 1] if b + 1 < W else INF
            best = min(D[b], up, left)
            d = xj - qv
            v = d * d + best
            if r != R and not (b - R <= r and R - b <= r):
                v = INF
            D[b] = v
            left = v
        cmins.append(min(D))
    return D[R], cmins


@pytest.mark.parametrize("n,R,r", [(8, 0, 0), (8, 2, 2), (16, 4, 1), (33, 6, 6), (64, 12, 8), (128, 12, 12),
                                   (100, 25, 25), (20, 25, 19), (4, 2, 2), (16, 32, 32), (64, 32, 20),
                                   (48, 16, 16)])
def test_band_walk_equals_the_oracle_dtw(n, R, r):
    rng = np.random.default_rng(n * 7 + R + r)
    for trial in range(10):
        q = np.cumsum(rng.normal(size=n)).astype(np.float32)
        x = (q + rng.normal(0.0, 0.7, size=n)).astype(np.float32) if trial % 2 else \
            np.cumsum(rng.normal(size=n)).astype(np.float32)
        d, cmins = band_walk(q, x, R, r)
        assert d == oracle.dtw2(q, x, r), (n, R, r, trial)
        assert all(c <= d for c in cmins), (n, R, r, trial)
