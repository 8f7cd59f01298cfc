"""The near-tie band, checked on the CPU against models of the FP32 distance
arithmetic.

Candidates are compared by FP32 squared distances, and every candidate within
a factor F = (1 + gamma)^2 of the k-th best is re-ranked in FP64 at the end.
That is exact only if each FP32 squared distance is within a relative gamma of
the exact one: ED gamma = (len/16 + 32) u, DTW gamma = (2 len + 32) u,
u = 2^-24.  Here the ED sum is modelled in the order the warp kernels use
(each of 32 lanes takes every 32nd group of 4 points, groups of 64 float4 at a
time, fused multiply-adds; then an xor-butterfly over the lanes), and the
banded DTW recurrence cell by cell in float32 (with and without the product
contracted into the add), against FP64 -- on random walks, near-identical
rows (small distances) and rows with all differences equal (every rounding
error of one size), for lengths up to 2048."""
import math

import numpy as np
import pytest

import oracle

U = 2.0 ** -24


def fmaf(a, b, c):
    return np.float32(float(a) * float(b) + float(c))


def warp_ed2_model(q, x):
    n4 = q.size // 4
    acc = [np.float32(0.0)] * 32
    for base in range(0, n4, 64):
        for t in range(2):
            for lane in range(32):
                i = base + lane + 32 * t
                if i < n4:
                    for e in range(4):
                        d = np.float32(q[4 * i + e] - x[4 * i + e])
                        acc[lane] = fmaf(d, d, acc[lane])
    for off in (16, 8, 4, 2, 1):                       # v += shfl_xor(v, off), read by lane 0
        acc = [np.float32(acc[l] + acc[l ^ off]) for l in range(32)]
    return float(acc[0])


def dtw2_model(q, x, r, fused):
    n = q.size
    INF = np.float32(np.inf)
    prev = [INF] * n
    for i in range(n):
        cur = [INF] * n
        for j in range(max(0, i - r), min(n, i + r + 1)):
            if i == 0 and j == 0:
                best = np.float32(0.0)
            else:
                best = min(prev[j], cur[j - 1] if j > 0 else INF, prev[j - 1] if j > 0 else INF)
            d = np.float32(q[i] - x[j])
            cur[j] = fmaf(d, d, best) if fused else np.float32(np.float32(d * d) + best)
        prev = cur
    return float(prev[n - 1])


def pair(kind, n, rng):
    q = np.cumsum(rng.normal(size=n))
    q = (q - q.mean()) / q.std()
    if kind == "walk":
        x = np.cumsum(rng.normal(size=n))
        x = (x - x.mean()) / x.std()
    elif kind == "near":
        x = q + rng.normal(0.0, 1e-3, size=n)
    else:                                               # every difference the same size
        x = q + 0.3 * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    return q.astype(np.float32), x.astype(np.float32)


@pytest.mark.parametrize("n", [16, 256, 1024, 2048])
@pytest.mark.parametrize("kind", ["walk", "near", "equal"])
def test_ed_fp32_within_band(n, kind):
    rng = np.random.default_rng(n + len(kind))
    q, x = pair(kind, n, rng)
    exact = float(np.sum((q.astype(np.float64) - x.astype(np.float64)) ** 2))
    got = warp_ed2_model(q, x)
    gamma = (n / 16.0 + 32.0) * U
    assert abs(got - exact) <= gamma * exact, (n, kind, abs(got - exact) / exact / U)


@pytest.mark.parametrize("n,r", [(16, 2), (128, 12), (256, 25)])
@pytest.mark.parametrize("kind", ["walk", "near", "equal"])
@pytest.mark.parametrize("fused", [True, False])
def test_dtw_fp32_within_band(n, r, kind, fused):
    rng = np.random.default_rng(3 * n + r + len(kind))
    q, x = pair(kind, n, rng)
    exact = oracle.dtw2(q, x, r)
    got = dtw2_model(q, x, r, fused)
    gamma = (2.0 * n + 32.0) * U
    assert abs(got - exact) <= gamma * exact, (n, r, kind, fused, abs(got - exact) / exact / U)
