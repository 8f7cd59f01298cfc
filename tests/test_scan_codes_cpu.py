"""CPU model of the scan's 16-bit table (k_lb_scan, csrc/query.cu).

The scan replaces each FP32 table entry T (already rounded down) by
code = min(65535, floor(T / D)) with D a power of two: the smallest one
>= R / 4096 (R = the pruning threshold, or 16 x the largest entry when no
threshold exists), never below the smallest normal float.  A word survives
when its code sum is at most floor(threshold / D), and its stored bound is
(code sum) * D.  This file restates those steps in float32 exactly as the
kernel takes them and checks, on random tables and thresholds including the
edge cases (threshold 0, infinite, tiny, huge), that:
  * code * D never exceeds its entry, so a stored bound never exceeds the
    sum of the FP32 entries (and so never the exact bound);
  * a word the codes prune has an FP32 entry sum above the threshold (no
    false prune), whatever the order of the integer additions;
  * without a capped code, the codes lose less than 16 D <= R / 128
    against the FP32 sum;
  * a capped code alone exceeds the threshold.
"""
import numpy as np
import pytest

F32 = np.float32
TINY = F32(1.17549435e-38)


def scan_codes(lut, thrp):
    lut = lut.astype(F32)
    if np.isfinite(thrp):
        R = F32(thrp)
    else:
        R = F32(16) * lut.max()
    m, e = np.frexp(F32(R * F32(1.0 / 4096.0)))
    D = F32(np.ldexp(F32(1), int(e))) if (R > 0 and m > 0) else TINY
    D = max(D, TINY)
    c = lut / D                                    # exact: D is a power of two
    codes = np.where(c >= F32(65535), 65535, np.floor(c)).astype(np.uint32)
    if np.isfinite(thrp):
        q = F32(thrp) / D
        limit = 0xFFFFFFFF if q >= F32(4294967040.0) else int(q)
    else:
        limit = 0xFFFFFFFF
    return codes, D, limit


def tables(rng, scale):
    # a query table: 16 segments x 256 symbols, zero at the query's symbol and
    # growing away from it (the shape of m * d^2), rounded down to float32
    q = rng.integers(0, 256, 16)
    v = np.arange(256)
    lut = np.zeros((16, 256), dtype=np.float64)
    for s in range(16):
        d = np.abs(v - q[s]) * rng.uniform(0.005, 0.05)
        lut[s] = 16.0 * d * d * scale
    return np.nextafter(lut.astype(F32), F32(0)).clip(0).astype(F32)


@pytest.mark.parametrize("scale", [1e-6, 1.0, 37.5, 1e6])
@pytest.mark.parametrize("thr_kind", ["typical", "zero", "inf", "tiny", "huge"])
def test_codes_never_overprune(scale, thr_kind):
    from fractions import Fraction

    rng = np.random.default_rng(int(scale * 7) % 1000 + len(thr_kind))
    lut = tables(rng, scale)
    thrp = {"typical": F32(lut.mean() * 16), "zero": F32(0), "inf": F32(np.inf),
            "tiny": F32(1e-30), "huge": F32(3e38)}[thr_kind]
    codes, D, limit = scan_codes(lut.reshape(-1), thrp)
    codes = codes.reshape(16, 256)
    Dq = Fraction(float(D))
    # every code times D stays at or below its entry
    assert np.all(codes.astype(np.float64) * float(D) <= lut.astype(np.float64))
    R = Fraction(float(thrp)) if np.isfinite(thrp) else 16 * Fraction(float(lut.max()))
    if R > 0:
        assert Dq * 4096 >= R and (Dq * 2048 < R or D == TINY)
    words = rng.integers(0, 256, size=(3000, 16))
    # words near the query's symbols too, so some survive
    words[:1000] = np.clip(np.argmin(lut, axis=1)[None, :] + rng.integers(-3, 4, size=(1000, 16)), 0, 255)
    for w in words:
        ent = lut[np.arange(16), w]
        cs = codes[np.arange(16), w]
        total = int(cs.sum())
        half = int(cs[:8].sum())
        exact = sum(Fraction(float(x)) for x in ent)
        # stored bound below the FP32 entry sum
        assert Fraction(total) * Dq <= exact
        # lost at most 16 D (a capped code loses more, but prunes the word)
        if not (cs == 65535).any():
            assert exact - Fraction(total) * Dq < 16 * Dq
        if np.isfinite(thrp):
            pruned = half > limit or total > limit
            if pruned:
                assert exact > Fraction(float(thrp))
        # a capped code alone exceeds any finite threshold
        if np.isfinite(thrp) and (cs == 65535).any():
            assert Fraction(65535) * Dq > Fraction(float(thrp))
