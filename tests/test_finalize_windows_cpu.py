"""The final step's windowed ranking of near-tied candidates, modelled on the
CPU.

When more candidates lie in the near-tie band than one pass holds, the log is
taken window by window: a window's in-band entries are ranked by (FP64
distance, id), its best k distinct rows are kept (the log may hold a row
twice, even under two FP32 keys: screened batches re-offer rows, and rows
are told apart by id), and they are merged with the running top-k, again
keeping distinct rows.  Restated here with small windows, that
must equal ranking every distinct in-band row at once -- with duplicates
placed anywhere, mass ties in the FP64 distance, and k from 1 to beyond a
window."""
import numpy as np
import pytest


def windowed(log, band, d64, k, W):
    running = []                                     # list of (d64, id, P)
    for w0 in range(0, len(log), W):
        win = [P for P in log[w0:w0 + W] if P[0] <= band]
        win.sort(key=lambda P: (d64[P[1]], P[1]))
        best = []
        for P in win:
            if len(best) == k:
                break
            if best and P[1] == best[-1][1]:      # the same row (its id), whatever its FP32 key
                continue
            best.append(P)
        merged = sorted(best + running, key=lambda P: (d64[P[1]], P[1]))
        running = []
        for i, P in enumerate(merged):
            if len(running) == k:
                break
            if i > 0 and P[1] == merged[i - 1][1]:
                continue
            running.append(P)
    return [P[1] for P in running]


def reference(log, band, d64, k):
    ids = sorted({P[1] for P in log if P[0] <= band}, key=lambda i: (d64[i], i))
    return ids[:k]


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8, 20])
@pytest.mark.parametrize("W", [4, 7, 16])
def test_windowed_ranking_equals_global_ranking(k, W):
    rng = np.random.default_rng(100 * k + W)
    for trial in range(200):
        n = int(rng.integers(1, 60))
        ids = rng.choice(1000, size=n, replace=False)
        # FP64 distances with many exact ties; the FP32 key is a rounding of it
        d64 = {int(i): float(rng.integers(0, 6)) + (0.0 if trial % 2 else float(rng.random())) for i in ids}
        rows = [(np.float32(d64[int(i)]).item(), int(i)) for i in ids]
        log = rows + [rows[j] for j in rng.integers(0, n, size=int(rng.integers(0, 2 * n)))]   # duplicates
        # the same row logged again under a different FP32 key (one ulp off),
        # as a differently ordered FP32 evaluation could give
        for j in rng.integers(0, n, size=int(rng.integers(0, n // 2 + 1))):
            key, rid = rows[j]
            log.append((float(np.nextafter(np.float32(key), np.float32(np.inf))), rid))
        order = rng.permutation(len(log))
        log = [log[j] for j in order]
        band = float(rng.uniform(0, 6))
        assert windowed(log, band, d64, k, W) == reference(log, band, d64, k), (k, W, trial)
