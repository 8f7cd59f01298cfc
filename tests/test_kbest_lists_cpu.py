"""CPU model of the screen's k-best lists (k_tc_screen, csrc/screen.cu).

For k > 1 each query keeps one list in global memory of the k smallest
upper ends s + eps met so far, starting from the seed leaf's k best; its
k-th entry bounds the query's true k-th squared distance from above, and the
screen tests every pair against it.  That holds because every entry is the
upper end of a different row: the screen meets each (query, row) pair once,
skips the seed leaf's rows (already in the list), and a later pass (for
queries whose candidate lists overflowed) meets the rows again, so it adds
nothing.  The model draws true distances and upper ends, inserts them in a
random order from many CTAs, and checks the bound after every insertion;
letting a later pass insert again, or the seed rows enter twice, breaks it.
"""
import random

import pytest


def insert(lst, k, up):
    # the kernel's insertion under the list lock: keep the k smallest, sorted
    if up < lst[k - 1]:
        j = k - 1
        while j > 0 and lst[j - 1] > up:
            lst[j] = lst[j - 1]
            j -= 1
        lst[j] = up
    return lst[k - 1]


def run(k, seed, second_pass_inserts=False, seed_rows_again=False):
    rng = random.Random(seed)
    n = 600
    d2 = [rng.uniform(0.0, 100.0) for _ in range(n)]
    eps = [rng.uniform(0.0, 0.02) for _ in range(n)]
    ups = [d2[i] + eps[i] for i in range(n)]        # every upper end >= its row's distance
    seed_rows = list(range(40))                      # the seed leaf
    true_kth = sorted(d2)[k - 1]
    lst = sorted(ups[i] for i in seed_rows)[:k] + [float("inf")] * max(0, k - len(seed_rows))
    violated = False
    passes = 2 if second_pass_inserts else 1
    for _ in range(passes):
        order = [i for i in range(n) if i not in seed_rows or seed_rows_again]
        rng.shuffle(order)                           # CTAs meet rows in any order
        for i in order:
            bound = insert(lst, k, ups[i])
            if bound < true_kth:
                violated = True
    return violated


@pytest.mark.parametrize("k", [2, 5, 10, 16])
@pytest.mark.parametrize("seed", range(10))
def test_kth_upper_end_bounds_the_true_kth_distance(k, seed):
    assert not run(k, seed)


@pytest.mark.parametrize("k", [2, 10, 16])
def test_inserting_rows_twice_breaks_the_bound(k):
    # the reasons a later pass adds nothing and the screen skips the seed rows
    assert any(run(k, s, second_pass_inserts=True) for s in range(10))
    assert any(run(k, s, seed_rows_again=True) for s in range(10))
