"""Pins of the reference block-step scheduler (oracle/sorting_list.py) to things other than
itself: exact rational next times (Fractions), the structural facts the paper's sorting list
relies on (Sec. 3.3.1: the active particles form a prefix of the step-sorted list, and a
block step moves the clock by the smallest step), the synchronisation invariant of
hierarchical steps, and hand-worked small cases of the block rule."""
from fractions import Fraction

import numpy as np

import workloads as W
from oracle.sorting_list import SortingList


def test_two_levels_by_hand():
    s = SortingList(np.array([3, 4, 4, 3, 5]), level_min=0, level_max=10, tick_level=10)
    # steps 1/8, 1/16, 1/16, 1/8, 1/32: the list is level 5, then 4, 4, then 3, 3
    assert list(s.order) == [4, 1, 2, 0, 3]
    T, act = s.next()
    assert T == 2 ** 10 // 32 and list(act) == [4]
    s.update([5])
    T, act = s.next()
    assert T == 2 ** 10 // 16 and sorted(act) == [1, 2, 4]
    s.update([5, 4, 4])  # list order: 4, 1, 2
    T, act = s.next()
    assert T == 3 * 2 ** 10 // 32 and list(act) == [4]
    s.update([5])
    T, act = s.next()
    assert T == 2 ** 10 // 8 and sorted(act) == [0, 1, 2, 3, 4]


def test_block_rule_cases():
    s = SortingList(np.array([4, 4, 4, 4]), level_min=2, level_max=6, tick_level=8)
    T, act = s.next()  # T = 1/16: a doubling to 1/8 is not commensurate
    w = s.update([3, 1, 9, 4])
    assert list(w) == [4, 4, 6, 4]
    s2 = SortingList(np.array([4, 4]), level_min=3, level_max=6, tick_level=8)
    s2.next(); s2.update([4, 4])
    T, _ = s2.next()  # T = 1/8: doubling to 1/8 is commensurate; -2 is cut to one doubling
    assert T == 2 ** 8 // 8
    assert list(s2.update([2, 3])) == [3, 3]
    s3 = SortingList(np.array([3]), level_min=3, level_max=6, tick_level=8)
    s3.next()
    assert list(s3.update([1])) == [3]  # level_min clamps


def test_random_run_against_exact_rational_times():
    """300 block steps of 2000 particles with seeded level requests: at every step the active
    set equals the brute-force minimum of exact rational next times, it is the prefix of the
    list, the list is sorted by step, the clock moves by the smallest step, and every
    particle's last time is a multiple of its step."""
    cl = W.plummer(2000, 91)
    lv = W.step_levels(W.block_steps(cl, seed=91, dt_min=0.5 ** 14, dt_max=0.5 ** 3))
    s = SortingList(lv, level_min=3, level_max=14, tick_level=20)
    tl = [Fraction(0)] * 2000
    for k in range(300):
        T, act = s.next()
        nxt = [tl[i] + Fraction(1, 2 ** int(s.level[i])) for i in range(2000)]
        tmin = min(nxt)
        assert Fraction(T, 2 ** 20) == tmin
        assert set(act) == {i for i in range(2000) if nxt[i] == tmin}
        assert set(s.order[:act.size]) == set(act)
        assert T - s.T == 2 ** 20 // 2 ** int(s.level.max())
        want = W.level_requests(s.level[s.order[:act.size]], seed=1000 + k)
        s.update(want)
        for i in act:
            tl[i] = tmin
        lev = s.level[s.order]
        assert np.all(lev[:-1] >= lev[1:])
        assert all((tl[i] / Fraction(1, 2 ** int(s.level[i]))).denominator == 1 for i in range(0, 2000, 7))
    assert s.T > 0 and s.level.min() >= 3 and s.level.max() <= 14


def test_list_is_stable_within_a_level():
    lv = np.array([5, 5, 4, 5, 4, 5])
    s = SortingList(lv, level_min=0, level_max=8, tick_level=8)
    assert list(s.order) == [0, 1, 3, 5, 2, 4]
    s.next()
    s.update([6, 5, 6, 5])  # particles 0, 1, 3, 5 in list order
    assert list(s.order) == [0, 3, 1, 5, 2, 4]
