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
from fractions import Fraction

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


# ------------------------------------------------ the candidate test itself
# The epilogue's test, restated with the kernel's constants and rounding
# directions in float32 (each operation below names the rounding the kernel
# asks for), to check the claim it rests on: a pair whose true squared
# distance is at most U is always a candidate -- both under the CTA-wide test
# and under the rare path's re-test with the query's own slack.
KP = float(np.float32(7.2e-7))


def rn(v):
    return float(np.float32(v))


def ru(v):
    r = np.float32(v)
    return float(r) if float(r) >= v else float(np.nextafter(r, np.float32(np.inf)))


def rd(v):
    r = np.float32(v)
    return float(r) if float(r) <= v else float(np.nextafter(r, np.float32(-np.inf)))


def rd_exact(v):
    # a rational rounded down to float32 (the fma's single rounding)
    r = np.float32(float(v))
    while Fraction(float(r)) > v:
        r = np.nextafter(r, np.float32(-np.inf))
    while Fraction(float(np.nextafter(r, np.float32(np.inf)))) <= v:
        r = np.nextafter(r, np.float32(np.inf))
    return float(r)


def norms(v):
    ss = 0.0
    for t in v.astype(np.float64):
        ss += t * t
    return rn(ss), ru(math.sqrt(ss * (1.0 + 1e-12)))      # |v|^2 to nearest, |v| rounded up


def query_constants(n, qn, qnorm):
    f = np.float32
    coef = f(1.002) * (f(9.765625e-4) + f(n + 16) * f(1.1920929e-7))
    beta = f(5.9604645e-8) * f(math.sqrt(n)) * f(1.002)
    alpha = (f(qnorm) * (f(2) * coef + f(2) * f(KP)) + beta) * (f(1) + f(1e-6))
    gamma = (beta * f(qnorm) + f(KP) * f(qn)) * (f(1) + f(1e-6))
    return float(alpha), float(gamma)


@pytest.mark.parametrize("n", [16, 128, 256, 1024, 2048])
@pytest.mark.parametrize("scale", [1.0, 100.0])
def test_candidate_test_has_no_false_negatives(n, scale):
    rng = np.random.default_rng(n + int(scale))
    q = np.cumsum(rng.normal(size=n))
    q = ((q - q.mean()) / q.std() * scale).astype(np.float32)
    qn, qnorm = norms(q)
    alpha, gamma = query_constants(n, qn, qnorm)
    omk = rn(1.0 - KP)
    for sigma in (0.0, 1e-4, 1e-3, 1e-2, 0.1, 1.0, None):
        if sigma is None:
            x = np.cumsum(rng.normal(size=n))
            x = ((x - x.mean()) / x.std() * scale).astype(np.float32)
        else:
            x = (q + rng.normal(0.0, sigma * scale, size=n)).astype(np.float32)
        xn, xnrm = norms(x)
        d2 = float(np.sum((q.astype(np.float64) - x.astype(np.float64)) ** 2))
        U = ru(d2)                                       # the tightest float32 bound of d^2
        p = q.astype(np.float16).astype(np.float32) * x.astype(np.float16).astype(np.float32)
        for mode in ("seq", "rz"):
            c = accumulate(p, mode)
            E = rd(rd(qn - gamma) - U)                               # __fsub_rd twice
            r = ru(xnrm * alpha + ru(-xn * omk))                     # __fmaf_ru(xnrm, amax, __fmul_ru(..))
            assert ru(2.0 * c + r) >= E, (n, scale, sigma, mode)     # __fmaf_ru(2, acc, r) >= E
            # the warp's first test: E - 2 acc by a packed FMA rounded down, its
            # minimum over the queries against r
            assert rd_exact(Fraction(E) - 2 * Fraction(c)) <= r, (n, scale, sigma, mode)
            lhs = rn(xnrm * alpha + rn(2.0 * c + rn(-xn * omk)))     # fmaf(xnrm, alpha, fmaf(2, acc, -xn omk))
            assert lhs >= E, (n, scale, sigma, mode)


@pytest.mark.parametrize("n", [16, 128, 256, 1024, 2048])
@pytest.mark.parametrize("scale", [1.0, 100.0])
def test_upper_end_bounds_the_true_distance(n, scale):
    # the rare path lowers U_q with up = (s + eps) rounded up; the k-th
    # smallest of these bounds the k-th distance only if every up >= d^2
    rng = np.random.default_rng(10 * n + int(scale))
    q = np.cumsum(rng.normal(size=n))
    q = ((q - q.mean()) / q.std() * scale).astype(np.float32)
    qn, qnorm = norms(q)
    alpha, gamma = query_constants(n, qn, qnorm)
    for sigma in (0.0, 1e-4, 1e-3, 1e-2, 0.1, 1.0, None):
        if sigma is None:
            x = np.cumsum(rng.normal(size=n))
            x = ((x - x.mean()) / x.std() * scale).astype(np.float32)
        else:
            x = (q + rng.normal(0.0, sigma * scale, size=n)).astype(np.float32)
        xn, xnrm = norms(x)
        d2 = float(np.sum((q.astype(np.float64) - x.astype(np.float64)) ** 2))
        p = q.astype(np.float16).astype(np.float32) * x.astype(np.float16).astype(np.float32)
        for mode in ("seq", "pairwise", "rz"):
            c = accumulate(p, mode)
            shat = rn(-2.0 * c + rn(xn + qn))                        # fmaf(-2, acc, xn + qn)
            eps = rn(xnrm * alpha + rn(gamma + rn(KP * xn)))         # fmaf(xnrm, alpha, gamma + kappa' xn)
            up = max(ru(ru(shat + eps) * float(np.float32(1.0000003))), 0.0)
            assert up >= d2, (n, scale, sigma, mode, up, d2)
