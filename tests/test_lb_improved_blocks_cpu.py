"""The LB_Improved walks of the DTW filter, modelled on the CPU.

When the window reach equals the kernel's template reach, the second
LB_Improved term takes each point's envelope of h (the candidate clamped into
the query's envelope, a window of W = 2R + 1 points) from blocks of B = W + 1
points: a window ending at block slot k <= B - 3 is the previous block's
suffix from slot k + 2 and the current block's prefix to k; at k = B - 2 the
prefix alone; at k = B - 1 the current block's own suffix from slot 1.  The
row and the envelope are read 4 points per load when B is a multiple of 4,
else 2, from positions that are multiples of that width.  Below the template
reach, the register-window walk reads the newest 2r + 1 of 2R + 1 slots.  This restates both walks step by step (float32 values,
sums rounded toward -inf) and checks that (a) every envelope it forms equals
the window max/min of h taken directly, clipped at the ends, and (b) the
bound never exceeds the oracle's FP64 LB_Improved."""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle


def rd32(fr: Fr) -> float:
    f = float(np.float32(float(fr)))
    if Fr(f) > fr:
        f = float(np.nextafter(np.float32(f), np.float32(-np.inf)))
    return f


def blocked_model(q, U, L, x, R):
    n, W = q.size, 2 * R + 1
    B = W + 1
    VW = 4 if B % 4 == 0 else 2
    assert n % 4 == 0                      # series lengths are multiples of 4
    hlast = float(min(max(x[0], L[0]), U[0]))
    smx, smn = [hlast] * B, [hlast] * B
    acc1 = acc2 = 0.0
    env = {}
    for j0 in range(0, n + R, B):
        pmx = pmn = 0.0
        cv = uv = lv = None
        for k in range(B):
            j = j0 + k
            if k % VW == 0 and j < n:
                assert j % VW == 0 and j + VW <= n             # an aligned vector load inside the row
                cv, uv, lv = x[j:j + VW], U[j:j + VW], L[j:j + VW]
            h = hlast
            if j < n:
                c, u, l = float(cv[k % VW]), float(uv[k % VW]), float(lv[k % VW])
                assert (c, u, l) == (float(x[j]), float(U[j]), float(L[j]))
                d = max(rd32(Fr(c) - Fr(u)), rd32(Fr(l) - Fr(c)), 0.0)     # the kernel's branch-free form
                acc1 = rd32(Fr(acc1) + Fr(rd32(Fr(d) * Fr(d))))
                h = min(max(c, l), u)
                hlast = h
            pmx = h if k == 0 else max(pmx, h)
            pmn = h if k == 0 else min(pmn, h)
            mx, mn = pmx, pmn
            if k + 2 < B:
                mx, mn = max(smx[k + 2], pmx), min(smn[k + 2], pmn)
            smx[k] = h
            smn[k] = h
            if k + 1 == B:
                for kk in range(B - 2, -1, -1):
                    smx[kk] = max(smx[kk], smx[kk + 1])
                    smn[kk] = min(smn[kk], smn[kk + 1])
                mx, mn = smx[1], smn[1]
            p = j - R
            if 0 <= p < n:
                env[p] = (mx, mn)
                qv = float(q[p])
                d = max(rd32(Fr(qv) - Fr(mx)), rd32(Fr(mn) - Fr(qv)), 0.0)
                acc2 = rd32(Fr(acc2) + Fr(rd32(Fr(d) * Fr(d))))
    return rd32(Fr(acc1) + Fr(acc2)), env


@pytest.mark.parametrize("n,R", [(16, 1), (16, 4), (36, 2), (100, 6), (128, 12), (256, 25), (40, 13),
                                 (8, 0), (64, 32), (256, 20), (12, 8)])
def test_blocked_envelopes_and_bound(n, R):
    rng = np.random.default_rng(n * 31 + R)
    for trial in range(20):
        q = np.cumsum(rng.normal(size=n)).astype(np.float32)
        x = (q + rng.normal(0.0, 0.5 + trial % 3, size=n)).astype(np.float32) if trial % 2 else \
            np.cumsum(rng.normal(size=n)).astype(np.float32)
        U64, L64 = oracle.envelope(q, R)
        U, L = U64.astype(np.float32), L64.astype(np.float32)        # max/min of floats: exact
        lb, env = blocked_model(q, U, L, x, R)
        h = np.minimum(np.maximum(x, L), U)
        for p in range(n):
            lo, hi = max(0, p - R), min(n - 1, p + R)
            assert env[p] == (float(h[lo:hi + 1].max()), float(h[lo:hi + 1].min())), (n, R, trial, p)
        assert lb <= oracle.lb_improved2(q, x, R), (n, R, trial)


def thread_model(q, U, L, x, R, r):
    """The register-window variant (template reach R, window r <= R)."""
    n, W = q.size, 2 * R + 1
    h0 = float(min(max(x[0], L[0]), U[0]))
    hw = [h0] * W
    lo_b = 2 * (R - r)
    acc1 = acc2 = 0.0
    env = {}
    for i in range(n + r):
        h = hw[W - 1]
        if i < n:
            c, u, l = float(x[i]), float(U[i]), float(L[i])
            d = 0.0
            if c > u:
                d = rd32(Fr(c) - Fr(u))
            elif c < l:
                d = rd32(Fr(l) - Fr(c))
            acc1 = rd32(Fr(acc1) + Fr(rd32(Fr(d) * Fr(d))))
            h = min(max(c, l), u)
        hw = hw[1:] + [h]
        p = i - r
        if p >= 0:
            vals = [hw[b] if b >= lo_b else h for b in range(W - 1)] + [h]
            mx, mn = max(vals), min(vals)
            env[p] = (mx, mn)
            qv = float(q[p])
            d = 0.0
            if qv > mx:
                d = rd32(Fr(qv) - Fr(mx))
            elif qv < mn:
                d = rd32(Fr(mn) - Fr(qv))
            acc2 = rd32(Fr(acc2) + Fr(rd32(Fr(d) * Fr(d))))
    return rd32(Fr(acc1) + Fr(acc2)), env


@pytest.mark.parametrize("n,R,r", [(16, 4, 1), (33, 4, 3), (100, 8, 6), (128, 16, 12), (256, 32, 25), (40, 6, 6)])
def test_register_window_envelopes_and_bound(n, R, r):
    rng = np.random.default_rng(n * 17 + R + r)
    for trial in range(20):
        q = np.cumsum(rng.normal(size=n)).astype(np.float32)
        x = (q + rng.normal(0.0, 0.5 + trial % 3, size=n)).astype(np.float32) if trial % 2 else \
            np.cumsum(rng.normal(size=n)).astype(np.float32)
        U64, L64 = oracle.envelope(q, r)
        U, L = U64.astype(np.float32), L64.astype(np.float32)
        lb, env = thread_model(q, U, L, x, R, r)
        h = np.minimum(np.maximum(x, L), U)
        for p in range(n):
            lo, hi = max(0, p - r), min(n - 1, p + r)
            assert env[p] == (float(h[lo:hi + 1].max()), float(h[lo:hi + 1].min())), (n, R, r, trial, p)
        assert lb <= oracle.lb_improved2(q, x, r), (n, R, r, trial)
