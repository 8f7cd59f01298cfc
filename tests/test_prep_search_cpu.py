"""CPU models of three steps of the query preparation (k_prep,
csrc/query.cu), checked against their plain definitions.

* Seed leaf (approxSearch, Sec. 3.1): the count of leaves whose first key is
  <= the query key.  The kernel finds it with a (B+1)-way search: each round
  the B threads of the block test evenly spaced pivots of the open range
  [lo, hi], and the count of true answers (__syncthreads_count) narrows it;
  the last <= B positions are tested one per thread.  The definition is
  bisect_right over the ascending keys.
* Query key (Sec. 2.2, the iSAX key of the index's sort): for each bit plane
  j, most significant first, the j-th bit of every segment's symbol, segment
  0 first.  The kernel collects each plane with one warp ballot (lane s holds
  segment s) and bit-reverses it; the definition is the bit-by-bit
  interleaving.
* Segment means (Sec. 2.2, PAA): the FP64 sum of a segment's floats divided
  by m, a power of two; the kernel multiplies by 1/m built from its exponent
  bits, which must give the same bits as the division.
"""
import bisect
import random

import pytest


def kary_count(keys, q, nb):
    """The kernel's search, step for step: returns (count, rounds)."""
    lo, hi = 0, len(keys)
    rounds = 0
    while hi - lo > nb:
        step = (hi - lo + nb) // (nb + 1)
        c = sum(1 for t in range(nb)
                if lo + (t + 1) * step - 1 < hi and keys[lo + (t + 1) * step - 1] <= q)
        nlo = lo + c * step
        if c < nb:
            hi = min(hi, lo + (c + 1) * step - 1)
        lo = nlo
        rounds += 1
        assert lo <= hi
    lo += sum(1 for t in range(nb) if lo + t < hi and keys[lo + t] <= q)
    return lo, rounds


@pytest.mark.parametrize("nb", [1, 2, 3, 7, 32, 256])
@pytest.mark.parametrize("seed", range(6))
def test_kary_search_equals_bisect(nb, seed):
    rng = random.Random(seed * 101 + nb)
    for _ in range(40):
        n = rng.choice([0, 1, 2, nb - 1, nb, nb + 1, 2 * nb + 3, 1000, 65_537])
        n = max(n, 0)
        span = rng.choice([3, 50, 1 << 40])   # many duplicates, few, none
        keys = sorted(rng.randrange(span) for _ in range(n))
        probes = [-1, span, rng.randrange(span)] + ([keys[0], keys[-1], keys[n // 2]] if n else [])
        for q in probes:
            got, _ = kary_count(keys, q, nb)
            assert got == bisect.bisect_right(keys, q), (n, q, nb)


def test_kary_search_rounds_at_index_sizes():
    # 100M series in leaves of ~2,000: ~50K leaves; 256 threads need 2 rounds
    # (the binary search took 16 dependent loads)
    keys = list(range(0, 2 * 50_000, 2))
    for q in (-5, 0, 1, 33_333, 99_998, 10**9):
        got, rounds = kary_count(keys, q, 256)
        assert got == bisect.bisect_right(keys, q)
        assert rounds <= 2


def interleave_bitwise(sym, w, bits):
    """Bit-by-bit definition: plane j (MSB first), segment 0 first."""
    key = 0
    for j in range(bits):
        for s in range(w):
            key = (key << 1) | ((sym[s] >> (bits - 1 - j)) & 1)
    return key << (128 - w * bits)


def brev32(x):
    return int(f"{x:032b}"[::-1], 2)


def interleave_ballot(sym, w, bits):
    """The kernel's form: one ballot per plane, bit-reversed into a w-bit field,
    shifted into a 128-bit (hi, lo) pair, then aligned to the top."""
    M = (1 << 64) - 1
    khi = klo = 0
    for j in range(bits):
        mask = sum(1 << s for s in range(32) if s < w and (sym[s] >> (bits - 1 - j)) & 1)
        field = brev32(mask) >> (32 - w)
        khi = ((khi << w) | (klo >> (64 - w))) & M
        klo = ((klo << w) | field) & M
    used = w * bits
    if used < 128:
        sh = 128 - used
        if sh >= 64:
            khi, klo = (klo << (sh - 64)) & M, 0
        else:
            khi, klo = ((khi << sh) | (klo >> (64 - sh))) & M, (klo << sh) & M
    return (khi << 64) | klo


@pytest.mark.parametrize("w", [1, 2, 3, 4, 8, 15, 16])
@pytest.mark.parametrize("bits", [1, 2, 4, 8])
def test_ballot_key_equals_bitwise_interleaving(w, bits):
    rng = random.Random(w * 17 + bits)
    for _ in range(50):
        sym = [rng.randrange(1 << bits) for _ in range(w)] + [0] * (32 - w)
        assert interleave_ballot(sym, w, bits) == interleave_bitwise(sym, w, bits)


def test_ballot_key_model_catches_a_missing_bit_reversal():
    # without the reversal segment 0 lands in the lowest bit of each plane
    sym = [1, 0, 0, 0] + [0] * 28
    w, bits = 4, 1
    assert interleave_ballot(sym, w, bits) == 1 << 127
    unreversed = 1 << (128 - w)               # the raw ballot, shifted to the top
    assert unreversed != interleave_bitwise(sym, w, bits)


def pow2_recip_bits(m):
    """The kernel's 1/m for m = 2^e: exponent field 1023 - e, mantissa 0."""
    import struct
    e = m.bit_length() - 1
    return struct.unpack("<d", struct.pack("<q", (1023 - e) << 52))[0]


@pytest.mark.parametrize("m", [4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096])
def test_segment_mean_by_reciprocal_equals_division(m):
    # the PAA of a segment is (sequential FP64 sum of its floats) / m; the
    # kernel multiplies by the exact 1/m instead, which must give the same bits
    import numpy as np
    assert pow2_recip_bits(m) == 1.0 / m
    rng = np.random.default_rng(m)
    tiny = np.float32(1.4e-45)                 # the smallest subnormal float
    cases = [rng.standard_normal(m).astype(np.float32) * s for s in (1e-38, 1e-3, 1.0, 1e30)]
    cases.append(np.full(m, np.finfo(np.float32).max, dtype=np.float32))
    cases.append(np.full(m, -np.finfo(np.float32).max, dtype=np.float32))
    cases.append(np.array([tiny] + [0.0] * (m - 1), dtype=np.float32))
    cases.append(np.array([tiny, -tiny] * (m // 2), dtype=np.float32))
    for x in cases:
        s = 0.0
        for v in x:
            s += float(v)
        assert s * pow2_recip_bits(m) == s / m
        assert np.float64(s * pow2_recip_bits(m)).tobytes() == np.float64(s / m).tobytes()
