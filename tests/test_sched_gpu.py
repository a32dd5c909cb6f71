"""The device block-step scheduler (nb_sched, Sec. 3.3.1) against the reference scheduler of
oracle/sorting_list.py, step by step: block time, number of active particles, granted
levels, per-level counts and the whole list must be identical (integer work: bit-exact).
Both sides get the same requested levels, generated from the oracle's own state."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle.sorting_list import SortingList

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def run_both(levels, lmin, lmax, steps, seed0, device_want=False):
    from paper_1504_03687_gb300 import Scheduler
    ref = SortingList(levels, level_min=lmin, level_max=lmax, tick_level=48)
    gpu = Scheduler(levels, lmin, lmax)
    lst, lev, t0 = gpu.get()
    np.testing.assert_array_equal(lst, ref.order)
    sizes = []
    for k in range(steps):
        T, act = ref.next()
        t, na = gpu.next()
        assert t == T * 2.0 ** -48 and na == act.size, (k, t, T, na, act.size)
        assert set(gpu.active().cpu().numpy()) == set(act)
        want = W.level_requests(ref.level[ref.order[:act.size]], seed=seed0 + k)
        g_ref = ref.update(want)
        g = gpu.update(torch.as_tensor(want, device=DEV) if device_want else want)
        g = g.cpu().numpy() if torch.is_tensor(g) else g
        np.testing.assert_array_equal(g, g_ref)
        sizes.append(na)
    lst, lev, t_now = gpu.get()
    np.testing.assert_array_equal(lst, ref.order)
    np.testing.assert_array_equal(lev, ref.level)
    assert t_now == ref.T * 2.0 ** -48
    np.testing.assert_array_equal(gpu.counts(), np.bincount(ref.level, minlength=64))
    gpu.close()
    return sizes


def test_scheduler_matches_reference_plummer_50k():
    """400 block steps, levels 3..14 from the local dynamical time; every list compared at the
    end (and the active sets at every step); blocks from one particle to the whole set."""
    cl = W.plummer(50000, 92)
    lv = W.step_levels(W.block_steps(cl, seed=92, dt_min=0.5 ** 14, dt_max=0.5 ** 3))
    sizes = run_both(lv, 3, 14, 400, 5000)
    assert min(sizes) < 100 and max(sizes) > min(sizes)


def test_scheduler_full_size_two_levels():
    """2^20 particles on levels 3 and 4 (every step re-sorts half or all of the list through
    the multi-CTA path), device-side requests."""
    rng = np.random.default_rng(93)
    lv = rng.integers(3, 5, 1 << 20).astype(np.int32)
    sizes = run_both(lv, 2, 6, 6, 6000, device_want=True)
    assert max(sizes) == 1 << 20


def test_scheduler_list_serves_as_active_index(gpu_lib):
    """The zero-copy view of the active particles drives nb_regular_force directly."""
    from paper_1504_03687_gb300 import Context, Scheduler
    cl, rs2 = W.plummer_1k_equal()
    lv = W.step_levels(W.block_steps(cl, seed=0, dt_min=0.5 ** 10))
    sch = Scheduler(lv, 3, 10)
    ctx = Context(cl.n, precision="fp64", nb_cap=64)
    ctx.set_predicted(torch.as_tensor(cl.x, device=DEV), torch.as_tensor(cl.v, device=DEV),
                      torch.as_tensor(cl.m, device=DEV))
    t, na = sch.next()
    idx = sch.active()
    assert idx.dtype == torch.int32 and idx.shape[0] == na
    r1 = ctx.regular_force(idx, rs2)
    ctx.sync()
    r2 = ctx.regular_force(idx.cpu().numpy(), rs2)
    np.testing.assert_array_equal(r1.acc.cpu().numpy(), r2.acc)
    sch.update(np.full(na, 10, np.int32))
    sch.close()
    ctx.close()


def test_scheduler_degenerate_cases_and_errors():
    from paper_1504_03687_gb300 import NBError, Scheduler
    from paper_1504_03687_gb300.api import NB_ERR_ARG, NB_ERR_STATE
    run_both(np.array([7], np.int32), 7, 7, 5, 7000)       # one particle, one level
    run_both(np.full(3000, 9, np.int32), 4, 12, 40, 7100)  # all synchronised at first
    with pytest.raises(NBError) as e:
        Scheduler(np.array([3, 20], np.int32), 3, 12)
    assert e.value.status == NB_ERR_ARG
    with pytest.raises(NBError) as e:  # device levels are checked by the initial sort
        Scheduler(torch.tensor([3, 70, 5], dtype=torch.int32, device=DEV), 3, 12)
    assert e.value.status == NB_ERR_ARG
    s = Scheduler(np.array([5, 6, 6], np.int32), 3, 12)
    with pytest.raises(NBError) as e:
        s.update(np.array([6], np.int32))
    assert e.value.status == NB_ERR_STATE
    s.next()
    with pytest.raises(NBError) as e:
        s.next()
    assert e.value.status == NB_ERR_STATE
    s.close()
