"""CPU model of the row norms of the tensor-core screen's f16 copy
(k_make_screen_copy, csrc/screen.cu).

The kernel sums x_i^2 in FP32 arithmetic as an unevaluated pair hi + lo:
each product is split exactly into p + e (p = x*x rounded, e = fma(x, x, -p)),
p enters hi through an exact two-sum whose error goes to lo, e is added to
lo; lane l takes the values k0 .. k0+7 for k0 = 8 l, 8 l + 256, ...; the 32
lanes then combine their pairs by an xor butterfly (offsets 16, 8, 4, 2, 1)
and lane 0 forms hi + lo in FP64.  Restated here in float32 (numpy float32
operations round to nearest like the kernel's; the exact product error of
a float32 square is exact in float64 and fits a float32), the result must
lie within 1e-9 of the exact squared norm -- the slack the screen's error
bound keeps for the norms beyond their final FP32 rounding -- and the upper
norm sqrt(sd (1 + 1e-9)) must not fall below the exact norm, for every
length the screen takes, on random walks, constant rows, rows of one large
and many tiny values, and rows near the f16 range limit."""
from fractions import Fraction

import numpy as np
import pytest

F32 = np.float32


def two_sum_pair(hi, lo, b):
    s = F32(hi + b)
    bb = F32(s - hi)
    err = F32(F32(hi - F32(s - bb)) + F32(b - bb))
    return s, F32(lo + err)


def kernel_norm(x):
    x = x.astype(F32)
    n = len(x)
    lanes = []
    for lane in range(32):
        hi, lo = F32(0), F32(0)
        for k0 in range(lane * 8, n, 256):
            for i in range(8):
                v = x[k0 + i]
                p = F32(v * v)
                e = F32(float(v) * float(v) - float(p))      # fma(v, v, -p): exact
                hi, lo = two_sum_pair(hi, lo, p)
                lo = F32(lo + e)
        lanes.append((hi, lo))
    for off in (16, 8, 4, 2, 1):
        new = []
        for lane in range(32):
            a = lanes[lane]
            b = lanes[lane ^ off]
            hi, lo = two_sum_pair(a[0], a[1], b[0])
            new.append((hi, F32(lo + b[1])))
        lanes = new
    hi, lo = lanes[0]
    return float(hi) + float(lo)


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


@pytest.mark.parametrize("n", [16, 64, 128, 256, 512, 1024, 2048])
def test_compensated_norm_within_slack(n):
    rng = np.random.default_rng(n)
    for name, x in rows(rng, n).items():
        x = x.astype(F32)
        exact = sum(Fraction(float(v)) ** 2 for v in x)
        sd = kernel_norm(x)
        assert abs(Fraction(sd) - exact) <= Fraction(1, 10 ** 9) * exact, (n, name)
        up = np.sqrt(sd * (1.0 + 1e-9))
        assert Fraction(up) ** 2 >= exact, (n, name)
