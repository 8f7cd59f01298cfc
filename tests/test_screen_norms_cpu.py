"""CPU model of the row norms of the tensor-core screen's f16 copy
(k_make_screen_copy, csrc/screen.cu).

The kernel sums x_i^2 in FP32 arithmetic as an unevaluated pair hi + lo:
each product is split exactly into p + e (p = x*x rounded, e = fma(x, x, -p)),
p enters hi through an exact two-sum whose error goes to lo, e is added to
lo; the row's lanes are ck / 4 for the tile's K chunk ck (64, 32 or 16), and
lane j takes the four values 4 j .. 4 j + 3 of every chunk in order; the
lanes then combine their pairs by an xor butterfly (offsets ck / 8 .. 1) and
the first rounds hi + lo once: to nearest for |x|^2, and upward, widened
by 2^-20 and square-rooted upward for |x|, all in FP32.  Restated here in
float32 (numpy float32 operations round to nearest like the kernel's; the
exact product error of a float32 square is exact in float64 and fits a
float32; the directed roundings by exact rational comparison), the pair
must lie within 1e-9 of the exact squared norm -- the slack the screen's
error bound keeps for the norms beyond their final FP32 rounding -- the
nearest-rounded |x|^2 must equal the exact pair rounded once, and the upper
norm must not fall below the exact norm, for every length the screen takes,
on random walks, constant rows, rows of one large and many tiny values, and
rows near the f16 range limit."""
from fractions import Fraction

import numpy as np
import pytest

F32 = np.float32


def two_sum_pair(hi, lo, b):
    s = F32(hi + b)
    bb = F32(s - hi)
    err = F32(F32(hi - F32(s - bb)) + F32(b - bb))
    return s, F32(lo + err)


def chunk_k(n):
    return 64 if n % 64 == 0 else 32 if n % 32 == 0 else 16


def kernel_norm(x):
    x = x.astype(F32)
    n = len(x)
    ck = chunk_k(n)
    lpr = ck // 4                      # lanes per row, one float4 of each chunk
    lanes = []
    for j in range(lpr):
        hi, lo = F32(0), F32(0)
        for c in range(n // ck):
            for e in range(4):
                v = x[c * ck + 4 * j + e]
                p = F32(v * v)
                err = F32(float(v) * float(v) - float(p))    # fma(v, v, -p): exact
                hi, lo = two_sum_pair(hi, lo, p)
                lo = F32(lo + err)
        lanes.append((hi, lo))
    off = lpr // 2
    while off >= 1:
        new = []
        for j in range(lpr):
            a = lanes[j]
            b = lanes[j ^ off]
            hi, lo = two_sum_pair(a[0], a[1], b[0])
            new.append((hi, F32(lo + b[1])))
        lanes = new
        off //= 2
    hi, lo = lanes[0]
    return hi, lo


def f32_round(fr: Fraction, up: bool) -> float:
    # a rational rounded to float32, toward +inf (up) or -inf
    r = np.float32(float(fr))
    while (Fraction(float(r)) < fr) if up else (Fraction(float(r)) > fr):
        r = np.nextafter(r, np.float32(np.inf if up else -np.inf))
    return float(r)


def upper_norm(hi, lo):
    # __fsqrt_ru(__fmul_ru(__fadd_ru(hi, lo), 1 + 2^-20))
    s = f32_round(Fraction(float(hi)) + Fraction(float(lo)), True)
    s = f32_round(Fraction(s) * Fraction(1 + 2 ** -20), True)
    r = np.float32(np.sqrt(s))
    while Fraction(float(r)) ** 2 < Fraction(s):
        r = np.nextafter(r, np.float32(np.inf))
    while Fraction(float(np.nextafter(r, np.float32(-np.inf)))) ** 2 >= Fraction(s):
        r = np.nextafter(r, np.float32(-np.inf))
    return float(r)


def rows(rng, n):
    walk = np.cumsum(rng.standard_normal(n))
    walk = (walk - walk.mean()) / walk.std()
    spike = np.full(n, 1e-3)
    spike[rng.integers(n)] = 300.0
    return {
        "walk": walk,
        "constant": np.full(n, 0.7),
        "spike": spike,
        "f16_edge": rng.uniform(60000, 65000, n) * rng.choice([-1, 1], n),
        "tiny": rng.standard_normal(n) * 1e-6,
    }


@pytest.mark.parametrize("n", [16, 32, 48, 64, 96, 128, 256, 512, 1024, 2048])
def test_compensated_norm_within_slack(n):
    rng = np.random.default_rng(n)
    for name, x in rows(rng, n).items():
        x = x.astype(F32)
        exact = sum(Fraction(float(v)) ** 2 for v in x)
        hi, lo = kernel_norm(x)
        sd = Fraction(float(hi)) + Fraction(float(lo))
        assert abs(sd - exact) <= Fraction(1, 10 ** 9) * exact, (n, name)
        # |x|^2 to nearest: one float32 addition of the pair, correctly rounded
        assert float(np.float32(hi) + np.float32(lo)) == float(np.float32(float(sd)))
        up = upper_norm(hi, lo)
        assert Fraction(up) ** 2 >= exact, (n, name)
