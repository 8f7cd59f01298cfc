"""Survivor enumeration after the scan, modelled on the CPU.

The lower-bound scan leaves each of its G regions with a count of survivors;
the ordering and refinement kernels enumerate them as 32-entry chunks
numbered across all regions (an exclusive prefix of ceil(count / 32)), find
a chunk's region by binary search (the last region whose prefix is <= the
chunk), and give lane l the entry (chunk - prefix) * 32 + l when it is below
the region's count.  Restated here, that must visit every survivor of every
region exactly once, with empty regions anywhere (the search must skip them)."""
import numpy as np


def chunk_prefix(counts):
    prefix = np.zeros(len(counts) + 1, dtype=np.int64)
    prefix[1:] = np.cumsum([(c + 31) >> 5 for c in counts])
    return prefix


def region_of(ch, prefix, G):
    lo, hi = 0, G
    while hi - lo > 1:
        mid = (lo + hi) >> 1
        if prefix[mid] <= ch:
            lo = mid
        else:
            hi = mid
    return lo


def test_every_survivor_visited_once():
    rng = np.random.default_rng(4)
    for trial in range(300):
        G = int(rng.integers(1, 200))
        counts = rng.integers(0, 100, size=G)
        counts[rng.random(G) < 0.4] = 0                     # many empty regions
        if trial % 7 == 0:
            counts[:] = 0
            counts[rng.integers(0, G)] = int(rng.integers(1, 70))
        prefix = chunk_prefix(counts)
        seen = []
        for ch in range(int(prefix[G])):
            rg = region_of(ch, prefix, G)
            for lane in range(32):
                within = (ch - prefix[rg]) * 32 + lane
                if within < counts[rg]:
                    seen.append((rg, int(within)))
        expect = [(g, i) for g in range(G) for i in range(int(counts[g]))]
        assert sorted(seen) == expect, trial
        assert len(seen) == len(set(seen))
