"""The screen's error bound, checked on the CPU against models of its
arithmetic.

The tensor-core screen estimates q.x from f16 copies of both vectors with
FP32 accumulation and widens the estimate c by
    |q.x - c| <= 1.002 (2^-10 + (len + 16) 2^-23) |q||x| + 1.002 2^-24 sqrt(len) (|q| + |x|)
(f16 rounding of both operands, subnormals included, and FP32 accumulation in
any order with up to 2 ulp per addition).  Here the f16 rounding is numpy's
(round to nearest even) and the accumulation is modelled three ways --
sequential and pairwise round-to-nearest, and sequential round-toward-zero
(a pessimistic model of an adder that truncates) -- on random walks, on
all-positive rows (no cancellation: the largest accumulated error), on rows
whose f16 rounding errors all share one sign (the worst case of the f16
term), on rows near the f16 subnormal range and near its maximum, for every
length the screen takes (16 .. 2048)."""
import math

import numpy as np
import pytest

U = 2.0 ** -24


def bound(n, qn, xn):
    return 1.002 * (2.0 ** -10 + (n + 16) * 2.0 ** -23) * qn * xn + 1.002 * U * math.sqrt(n) * (qn + xn)


def f32_add_rz(a, b):
    """float32 a + b rounded toward zero (the float64 sum of two float32
    values whose exponents differ by < 29 is exact; otherwise it is already
    correctly rounded and the step below keeps it on the zero side)."""
    s = float(np.float64(a) + np.float64(b))
    r = np.float32(s)
    if abs(float(r)) > abs(s):
        r = np.nextafter(r, np.float32(0.0))
    return r


def accumulate(p, mode):
    if mode == "seq":
        acc = np.float32(0.0)
        for v in p:
            acc = np.float32(acc + v)
        return float(acc)
    if mode == "pairwise":
        v = list(p)
        while len(v) > 1:
            v = [np.float32(v[i] + v[i + 1]) if i + 1 < len(v) else v[i] for i in range(0, len(v), 2)]
        return float(v[0])
    acc = np.float32(0.0)
    for v in p:
        acc = f32_add_rz(acc, v)
    return float(acc)


def rows(kind, n, rng):
    if kind == "walk":
        x = np.cumsum(rng.normal(size=(2, n)), axis=1)
        x = (x - x.mean(1, keepdims=True)) / np.maximum(x.std(1, keepdims=True), 1e-12)
    elif kind == "positive":
        x = rng.uniform(0.5, 1.5, size=(2, n))
    elif kind == "aligned":
        # every element just below the midpoint 1 + 2^-11 (times a power of two):
        # f16 rounds each one down by almost half an ulp, so the rounding errors
        # of both operands add up with one sign -- the worst case of the f16 term
        scale = 2.0 ** rng.integers(-1, 3, size=(2, n))
        x = scale * (1.0 + 2.0 ** -11 - 2.0 ** -20)
    elif kind == "tiny":
        x = rng.normal(size=(2, n)) * 2.0 ** -16          # f16 subnormal territory
    else:
        x = rng.uniform(30000.0, 65000.0, size=(2, n))     # near the largest screened values
    return x.astype(np.float32)


@pytest.mark.parametrize("n", [16, 64, 256, 512, 1024, 2048])
@pytest.mark.parametrize("kind", ["walk", "positive", "aligned", "tiny", "large"])
def test_screen_dot_product_bound_holds(n, kind):
    rng = np.random.default_rng(n * 7 + len(kind))
    q, x = rows(kind, n, rng)
    exact = float(np.dot(q.astype(np.float64), x.astype(np.float64)))
    qn = math.sqrt(float(np.dot(q.astype(np.float64), q.astype(np.float64))))
    xn = math.sqrt(float(np.dot(x.astype(np.float64), x.astype(np.float64))))
    p = q.astype(np.float16).astype(np.float32) * x.astype(np.float16).astype(np.float32)   # exact products
    b = bound(n, qn, xn)
    for mode in ("seq", "pairwise", "rz"):
        c = accumulate(p, mode)
        assert abs(exact - c) <= b, (n, kind, mode, abs(exact - c), b)


def test_bound_is_tight_for_aligned_rounding():
    # the aligned case uses nearly all of the f16 term: a bound with half the
    # f16 coefficient would fail it
    rng = np.random.default_rng(3)
    q, x = rows("aligned", 64, rng)
    exact = float(np.dot(q.astype(np.float64), x.astype(np.float64)))
    qn = math.sqrt(float(np.dot(q.astype(np.float64), q.astype(np.float64))))
    xn = math.sqrt(float(np.dot(x.astype(np.float64), x.astype(np.float64))))
    p = q.astype(np.float16).astype(np.float32) * x.astype(np.float16).astype(np.float32)
    err = abs(exact - accumulate(p, "seq"))
    assert err > 0.5 * bound(64, qn, xn)


def test_bound_is_not_vacuous():
    # the f16 term dominates: for unit-norm rows the bound is about 1e-3 of
    # |q||x| at len 256, so it still separates near from far neighbours
    assert bound(256, 16.0, 16.0) / 256.0 < 1.3e-3
    assert bound(2048, 45.0, 45.0) / 2025.0 < 1.3e-3
