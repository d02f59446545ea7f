"""The batch's split of a kernel group's CTAs between its streams: host logic
of the C ABI (prost_batch_split), checked without a GPU against its stated
rule and invariants."""

import math

import numpy as np
import pytest

import paper_1302_2073_gb300 as pg


def _rule(budget, w, cap):
    """The documented rule, step by step: floor of the proportional share
    clamped to [1, cap], leftovers one at a time to the largest remaining
    fraction under its cap, and any excess from the one-CTA minimum taken one
    at a time from the largest count (lowest index on a tie, both)."""
    ws = sum(w)
    share = [budget * x / ws for x in w]
    c = [min(max(int(math.floor(s)), 1), cp) for s, cp in zip(share, cap)]
    frac = [s - math.floor(s) for s in share]
    while sum(c) < budget:
        open_ = [i for i in range(len(w)) if c[i] < cap[i]]
        if not open_:
            break
        best = max(open_, key=lambda i: (frac[i], -i))
        c[best] += 1
        frac[best] -= 1.0
    while sum(c) > budget:             # the minimum of one CTA each overshot
        big = max(range(len(c)), key=lambda i: (c[i], -i))
        c[big] -= 1
    return c


def test_hand_cases():
    # equal weights: even split
    assert pg.prost_batch_split(152, [1.0, 1.0], [1000, 1000]) == [76, 76]
    # 1 : 3 of 8 -> 2, 6
    assert pg.prost_batch_split(8, [1.0, 3.0], [100, 100]) == [2, 6]
    # 10 CTAs over thirds: 3.33 each, the tie goes to the lowest index
    assert pg.prost_batch_split(10, [1.0, 1.0, 1.0], [9, 9, 9]) == [4, 3, 3]
    # a capped stream gives its share away
    assert pg.prost_batch_split(152, [1.0, 1.0], [5, 1000]) == [5, 147]
    # every stream capped below the budget: the CTAs the caps allow
    assert pg.prost_batch_split(152, [1.0, 2.0], [3, 4]) == [3, 4]
    # a tiny weight still gets one CTA
    assert pg.prost_batch_split(16, [1e-9, 1.0], [100, 100]) == [1, 15]
    # two tiny weights lifted to one CTA each: the largest gives one back
    assert pg.prost_batch_split(10, [1e-9, 1e-9, 1.0], [100, 100, 100]) == [1, 1, 8]
    # one stream takes the whole budget up to its cap
    assert pg.prost_batch_split(152, [7.0], [1000]) == [152]


@pytest.mark.parametrize("seed", range(40))
def test_random_groups_follow_the_rule_and_its_invariants(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 40))
    budget = int(rng.integers(n, 4 * 152 + 1))
    # sizes from a few pixels to 1080p RGB, so some shares fall below one CTA
    rows = np.exp(rng.uniform(0.0, np.log(3 * 1920 * 1080), size=n))
    alpha = float(rng.choice([0.5, 0.75, 1.0]))
    w = list(rows ** alpha)
    cap = [int(x) for x in rng.integers(1, 400, size=n)]
    got = pg.prost_batch_split(budget, w, cap)
    assert got == _rule(budget, w, cap)
    assert all(1 <= g <= c for g, c in zip(got, cap))
    assert sum(got) == min(budget, sum(cap))
    # monotone in the weight among uncapped streams, up to the one CTA that a
    # tie broken by index in the give-back step can cost
    free = [i for i in range(n) if got[i] < cap[i]]
    for i in free:
        for j in free:
            if w[i] > w[j]:
                assert got[i] >= got[j] - 1
    # each stream within one CTA of its proportional share, when no cap binds
    # and every share is at least one CTA
    share = [budget * x / sum(w) for x in w]
    if len(free) == n and min(share) >= 1.0:
        assert all(abs(g - s) < 1.0 for g, s in zip(got, share))


@pytest.mark.parametrize("budget,w,cap", [
    (1, [1.0, 1.0], [5, 5]),          # fewer CTAs than streams
    (8, [], []),                      # no stream
    (8, [0.0, 1.0], [5, 5]),          # non-positive weight
    (8, [float("nan"), 1.0], [5, 5]),
    (8, [float("inf"), 1.0], [5, 5]),
    (8, [1.0, 1.0], [0, 5]),          # cap below one
])
def test_invalid_arguments(budget, w, cap):
    with pytest.raises(pg.ProstError):
        pg.prost_batch_split(budget, w, cap)


@pytest.mark.parametrize("seed", range(20))
def test_uncapped_shares_round_to_within_one_cta(seed):
    # 640x480 to 1080p RGB streams on one to four CTAs per SM: every share is
    # above one CTA and no cap binds, so each stream is within one CTA of its
    # proportional share and the budget is used exactly
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 25))
    budget = 152 * int(rng.integers(1, 5))
    w = list(rng.uniform(3 * 640 * 480, 3 * 1920 * 1080, size=n) ** 0.75)
    got = pg.prost_batch_split(budget, w, [10 ** 6] * n)
    share = [budget * x / sum(w) for x in w]
    assert sum(got) == budget
    assert all(abs(g - s) < 1.0 for g, s in zip(got, share))
    assert got == _rule(budget, w, [10 ** 6] * n)
