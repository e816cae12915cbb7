"""The work lists of the persistent tensor-core launches (sht_work_lists), on
the host: every item is run exactly once, each list keeps the serving order,
lists differ in total cost by at most one item's cost, and ties go to the
lowest list -- checked on hand-worked cases and on costs shaped like the
(m, ring block) items of an lmax 2048 plan."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def sht():
    from paper_1010_1260_gb300 import build, sht as s
    build.build()
    s.lib()
    return s


def _lists(off, items):
    return [items[off[b]:off[b + 1]].tolist() for b in range(len(off) - 1)]


def _check_partition(costs, nlists, off, items):
    n = len(costs)
    assert off[0] == 0 and off[-1] == n and np.all(np.diff(off) >= 0)
    assert sorted(items.tolist()) == list(range(n))  # every item exactly once
    totals = []
    for lst in _lists(off, items):
        assert lst == sorted(lst)                      # serving order kept
        totals.append(int(np.sum(np.asarray(costs, dtype=np.int64)[lst])) if lst else 0)
    if n:
        assert max(totals) - min(totals) <= max(costs)
    return totals


def test_equal_costs_deal_round_robin(sht):
    off, items = sht.work_lists([1] * 10, 4)
    assert _lists(off, items) == [[0, 4, 8], [1, 5, 9], [2, 6], [3, 7]]


def test_worked_example_least_loaded_first(sht):
    # 5 goes to list 0; the five 1s all go to list 1, which stays below 5
    # until the last of them
    off, items = sht.work_lists([5, 1, 1, 1, 1, 1], 2)
    assert _lists(off, items) == [[0], [1, 2, 3, 4, 5]]
    # ties between equal totals go to the lower list
    off, items = sht.work_lists([2, 2, 1, 1, 3], 2)
    # 0 -> L0 (2), 1 -> L1 (2), 2 -> L0 (3, tie at 2), 3 -> L1 (3), 4 -> L0 (6, tie at 3)
    assert _lists(off, items) == [[0, 2, 4], [1, 3]]


def test_more_lists_than_items_and_empty(sht):
    off, items = sht.work_lists([7, 3, 9], 5)
    assert off.tolist() == [0, 1, 2, 3, 3, 3] and items.tolist() == [0, 1, 2]
    off, items = sht.work_lists([], 3)
    assert off.tolist() == [0, 0, 0, 0] and items.size == 0


def test_random_costs_balance(sht):
    rng = np.random.default_rng(11)
    for nlists in (1, 7, 152):
        costs = rng.integers(0, 1000, size=3000)
        off, items = sht.work_lists(costs, nlists)
        _check_partition(costs.tolist(), nlists, off, items)


def test_plan_shaped_costs(sht):
    """(m, ring block) items of an lmax 2048 plan with 16 ring blocks, m-major:
    the degrees left after a skip that grows toward the polar blocks and large
    m, plus the per-item share; 152 lists end within one item of each other,
    under 2 % of the mean."""
    L, nrb = 2048, 16
    rng = np.random.default_rng(5)
    costs = []
    for m in range(L + 1):
        ng = (L - m + 1 + 63) // 64
        for rb in range(nrb):
            polar = 1.0 - rb / (nrb - 1)
            g0 = min(ng - 1, int(ng * polar * m / (L + 1) * rng.uniform(0.8, 1.0)))
            costs.append(L - m + 1 - 64 * g0 + 48)
    off, items = sht.work_lists(costs, 152)
    totals = _check_partition(costs, 152, off, items)
    mean = sum(costs) / 152
    assert (max(totals) - min(totals)) / mean < 0.02
    # the round robin the lists replace gives CTA b only ring blocks b and b + 8 mod 16
    rr = [sum(costs[j] for j in range(b, len(costs), 152)) for b in range(152)]
    assert (max(rr) - min(rr)) / mean > 0.1


def test_bad_arguments(sht):
    L = sht.lib()
    c = (ctypes.c_longlong * 2)(1, -1)
    off = (ctypes.c_int * 3)()
    it = (ctypes.c_int * 2)()
    assert L.sht_work_lists(2, c, 2, off, it) == sht.SHT_EINVAL
    assert b"negative" in L.sht_last_error()
    c2 = (ctypes.c_longlong * 2)(1, 1)
    assert L.sht_work_lists(2, c2, 0, off, it) == sht.SHT_EINVAL
    assert L.sht_work_lists(-1, c2, 2, off, it) == sht.SHT_EINVAL
    assert L.sht_work_lists(2, None, 2, off, it) == sht.SHT_EINVAL
    assert L.sht_work_lists(2, c2, 2, off, it) == sht.SHT_OK
