"""The summarisation's FP32 shortcut, checked on the CPU against a model of
its arithmetic.

Each segment mean is summed in FP32 (pairs within a float4, then an
xor-butterfly over the lanes that hold the segment; longer segments add per
lane first) and its symbol is taken by comparing against FP32 copies of the
breakpoints.  That symbol is kept only if the mean lies farther than
1.01 u (A + 2|p| + 2) from both edges of its region (A = the FP32 sum of
|x| over the segment); otherwise the segment is re-summed in FP64 in index
order.  The claim: a kept symbol always equals the symbol of the FP64
sequential mean (the oracle's definition).  Segments here are drawn with
their exact mean a few ulps from a breakpoint, where a wrong margin would
show."""
import numpy as np
import pytest

import oracle

U = 2.0 ** -24


def f32(v):
    return np.float32(v)


def segment_sum_model(x, m):
    """FP32 sum and abs-sum of one segment of m points (m a power of two >= 4)
    in the kernel's order."""
    g = x.reshape(-1, 4)
    v = [f32(f32(a + b) + f32(c + d)) for a, b, c, d in g]
    a = [f32(f32(abs(p) + abs(q)) + f32(abs(r) + abs(s))) for p, q, r, s in g]
    M4 = m // 4
    if M4 <= 32:
        off = M4 // 2
        while off >= 1:
            v = [f32(v[i] + v[i ^ off]) for i in range(M4)]
            a = [f32(a[i] + a[i ^ off]) for i in range(M4)]
            off //= 2
        return v[0], a[0]
    # longer segments: lane l adds its groups l, l + 32, ... then a 32-lane butterfly
    acc = [f32(0.0)] * 32
    aac = [f32(0.0)] * 32
    for i in range(M4):
        acc[i % 32] = f32(acc[i % 32] + v[i])
        aac[i % 32] = f32(aac[i % 32] + a[i])
    for off in (16, 8, 4, 2, 1):
        acc = [f32(acc[l] + acc[l ^ off]) for l in range(32)]
        aac = [f32(aac[l] + aac[l ^ off]) for l in range(32)]
    return acc[0], aac[0]


def kernel_symbol(x, m, b32):
    S, A = segment_sum_model(x, m)
    p = f32(S / f32(m))
    sym = int(np.sum(b32 <= p))
    marg = f32(f32(1.01) * f32(U) * f32(A + f32(2.0) * abs(p) + f32(2.0))) + f32(1e-30)
    ok = True
    if sym > 0:
        ok = ok and f32(p - b32[sym - 1]) > marg
    if sym < b32.size:
        ok = ok and f32(b32[sym] - p) > marg
    return sym, ok


@pytest.mark.parametrize("m", [4, 16, 64, 128, 256])
@pytest.mark.parametrize("card", [4, 256])
def test_kept_fp32_symbol_equals_fp64_symbol(m, card):
    rng = np.random.default_rng(m * card)
    b64 = oracle.breakpoints(card)
    b32 = b64.astype(np.float32)
    kept = 0
    for trial in range(300):
        beta = b64[rng.integers(0, b64.size)]
        spread = 10.0 ** rng.uniform(-6, 0)
        x = (beta + spread * rng.normal(size=m)).astype(np.float32)
        # shift so the FP64 mean sits a few ulps (of beta) from the breakpoint
        mean64 = sum(float(t) for t in x) / m
        target = beta + rng.integers(-8, 9) * np.spacing(np.float32(max(abs(beta), 1e-3)))
        x = (x.astype(np.float64) + (target - mean64)).astype(np.float32)
        s64 = 0.0
        for t in x:
            s64 += float(t)
        sym64 = int(np.sum(b64 <= s64 / m))
        sym, ok = kernel_symbol(x, m, b32)
        if ok:
            kept += 1
            assert sym == sym64, (m, card, trial)
    assert kept < 300            # the adversarial segments do exercise the fallback


def test_random_rows_mostly_take_the_fp32_shortcut():
    # away from the breakpoints the shortcut is the common case
    b32 = oracle.breakpoints(256).astype(np.float32)
    rng = np.random.default_rng(5)
    kept = sum(kernel_symbol(rng.normal(size=16).astype(np.float32), 16, b32)[1] for _ in range(500))
    assert kept > 450
