"""The lower-bound table, modelled exactly on the CPU.

Per query segment s and symbol v the table holds m * d^2, d the distance from
the query's FP64 PAA to the region of v (Property 1), every operation rounded
toward -inf (and d shrunk by 2^-40 (|edge| + |p| + 1) for the FP64 rounding of
the PAA values), and a word's bound is the FP32 sum of its entries rounded
toward -inf.  The regions come from the library's own breakpoints, which may
differ from the oracle's in the last bit.  Modelled here with exact rational
arithmetic and explicit rounding, the bound must never exceed the oracle's
FP64 mindist -- on random words and on queries whose PAA sits within a few
ulps of a breakpoint, where the one-bit breakpoint differences matter."""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle


def rd64(fr: Fr) -> float:
    f = float(fr)
    return f if Fr(f) <= fr else math.nextafter(f, -math.inf)


def rd32(fr: Fr) -> float:
    f = float(np.float32(float(fr)))
    if Fr(f) > fr:
        f = float(np.nextafter(np.float32(f), np.float32(-np.inf)))
    return f


def gap_rd(edge: float, p: float) -> float:
    d = rd64(Fr(edge) - Fr(p))
    slack = 9.094947017729282e-13 * (abs(edge) + abs(p) + 1.0)      # FP64, to nearest
    d = rd64(Fr(d) - Fr(slack))
    return d if d > 0.0 else 0.0


def entry(p: float, v: int, beta: np.ndarray, m: int) -> float:
    lo = -math.inf if v == 0 else float(beta[v - 1])
    hi = math.inf if v == beta.size else float(beta[v])
    d = 0.0
    if p < lo:
        d = gap_rd(lo, p)
    elif p > hi:
        d = gap_rd(p, hi)
    return rd32(Fr(rd64(Fr(rd64(Fr(d) * Fr(d))) * m)))


def word_bound(paa_q, word, beta, m):
    lb = 0.0
    for s, v in enumerate(word):
        lb = rd32(Fr(lb) + Fr(entry(float(paa_q[s]), int(v), beta, m)))   # __fadd_rd
    return lb


@pytest.mark.parametrize("card,w,m", [(4, 4, 16), (256, 16, 16), (256, 8, 32)])
def test_table_bound_never_exceeds_the_oracle_mindist(card, w, m):
    import paper_2110_07519_gb300 as lib

    beta_lib = lib.messi_breakpoints(card)
    beta_orc = oracle.breakpoints(card)
    rng = np.random.default_rng(card + w)
    for trial in range(300):
        if trial % 2:
            # PAA values a few ulps from (library) breakpoints
            idx = rng.integers(0, beta_lib.size, size=w)
            paa_q = beta_lib[idx] + rng.integers(-4, 5, size=w) * np.spacing(np.abs(beta_lib[idx]) + 1e-3)
        else:
            paa_q = rng.normal(size=w)
        word = rng.integers(0, card, size=w)
        lb = word_bound(paa_q, word, beta_lib, m)
        exact = oracle.mindist_ed2(paa_q, word.astype(np.uint8), m, card, beta_orc)
        assert lb <= exact, (card, w, m, trial, lb, exact)


def entry_dtw(pu: float, pl: float, v: int, beta: np.ndarray, m: int) -> float:
    lo = -math.inf if v == 0 else float(beta[v - 1])
    hi = math.inf if v == beta.size else float(beta[v])
    d = 0.0
    if pu < lo:
        d = gap_rd(lo, pu)             # ABOVE: the upper envelope's PAA below the region
    elif pl > hi:
        d = gap_rd(pl, hi)             # BELOW
    return rd32(Fr(rd64(Fr(rd64(Fr(d) * Fr(d))) * m)))


@pytest.mark.parametrize("card,w,m", [(4, 4, 16), (256, 16, 16)])
def test_dtw_table_bound_never_exceeds_the_oracle_mindist(card, w, m):
    import paper_2110_07519_gb300 as lib

    beta_lib = lib.messi_breakpoints(card)
    beta_orc = oracle.breakpoints(card)
    rng = np.random.default_rng(7 * card + w)
    for trial in range(300):
        idx = rng.integers(0, beta_lib.size, size=w)
        near = beta_lib[idx] + rng.integers(-4, 5, size=w) * np.spacing(np.abs(beta_lib[idx]) + 1e-3)
        centre = near if trial % 2 else rng.normal(size=w)
        half = np.abs(rng.normal(size=w)) * (0.0 if trial % 3 == 0 else 0.3)
        pu, pl = centre + half, centre - half            # envelope PAAs, upper >= lower
        word = rng.integers(0, card, size=w)
        lb = 0.0
        for s in range(w):
            lb = rd32(Fr(lb) + Fr(entry_dtw(float(pu[s]), float(pl[s]), int(word[s]), beta_lib, m)))
        exact = oracle.mindist_dtw2(pu, pl, word.astype(np.uint8), m, card, beta_orc)
        assert lb <= exact, (card, w, m, trial, lb, exact)
