"""The register-band DTW walk of the refinement kernel, modelled on the CPU.

The kernel keeps one row of the Sakoe-Chiba band in 2R + 1 registers (band
slot b of row i is column i - R + b, slots outside the reach r or the row are
+inf), reads the previous row's slot b as the diagonal and slot b + 1 as the
cell above, and slides the candidate window by one point per row.  Restated
step by step in FP64, the walk must reproduce the oracle's banded DTW (the
textbook full-table recurrence) bit for bit: the arithmetic is the same, only
the storage differs, so any indexing slip shows as a different value."""
import math

import numpy as np
import pytest

import oracle


def band_walk(q, x, R, r):
    n, W = q.size, 2 * R + 1
    INF = math.inf
    D = [0.0 if b == R else INF for b in range(W)]
    xw = [float(x[b - R]) if 0 <= b - R < n else 0.0 for b in range(W)]
    for i in range(n):
        qi = float(q[i])
        left = INF
        for b in range(W):
            j = i - R + b
            up = D[b + 1] if b + 1 < W else INF
            best = min(min(D[b], up), left)
            d = qi - xw[b]
            inside = 0 <= j < n and (b - R <= r) and (R - b <= r)
            v = d * d + best if inside else INF
            D[b] = v
            left = v
        xw = xw[1:] + [float(x[i + 1 + R]) if i + 1 + R < n else 0.0]
    return D[R]


@pytest.mark.parametrize("n,R,r", [(8, 0, 0), (8, 2, 2), (16, 4, 1), (33, 6, 6), (64, 12, 8), (128, 12, 12),
                                   (100, 25, 25), (20, 25, 19)])
def test_band_walk_equals_the_oracle_dtw(n, R, r):
    rng = np.random.default_rng(n * 7 + R + r)
    for trial in range(10):
        q = np.cumsum(rng.normal(size=n)).astype(np.float32)
        x = (q + rng.normal(0.0, 0.7, size=n)).astype(np.float32) if trial % 2 else \
            np.cumsum(rng.normal(size=n)).astype(np.float32)
        assert band_walk(q, x, R, r) == oracle.dtw2(q, x, r), (n, R, r, trial)
