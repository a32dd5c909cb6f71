"""Checks of the seeded workload generators against the models' own mathematics."""
import math

import numpy as np

import oracle
import workloads as W


def test_plummer_half_mass_radius_and_virial():
    cl = W.plummer(1 << 18, 5)
    r = np.sqrt((cl.x ** 2).sum(1))
    # r_h = a / sqrt(2^(2/3) - 1) for the Plummer model; a = 3π/16 -> 0.7686
    rh = W.PLUMMER_A_NBODY / math.sqrt(2 ** (2 / 3) - 1)
    assert abs(np.median(r) - rh) < 0.01
    assert abs((cl.m * (cl.v ** 2).sum(1)).sum() - 0.5) < 0.005  # 2K = -W = 1/2
    assert np.abs((cl.m[:, None] * cl.x).sum(0)).max() < 1e-12


def test_kroupa_mean_mass_closed_form():
    (m0, m1, m2), (a1, a2) = W.KROUPA_BREAKS, W.KROUPA_SLOPES
    c2 = m1 ** (a2 - a1)
    num = (m1 ** (2 - a1) - m0 ** (2 - a1)) / (2 - a1) + c2 * (m2 ** (2 - a2) - m1 ** (2 - a2)) / (2 - a2)
    den = (m1 ** (1 - a1) - m0 ** (1 - a1)) / (1 - a1) + c2 * (m2 ** (1 - a2) - m1 ** (1 - a2)) / (1 - a2)
    m = W.kroupa_masses(2_000_000, np.random.default_rng(0))
    assert m.min() >= m0 and m.max() <= m2
    assert abs(m.mean() / (num / den) - 1) < 0.01
    # fraction below the break
    assert abs((m < m1).mean() - W.kroupa_segment_weights()[0]) < 0.002


def test_king_w0_6_concentration_and_tidal_boundary():
    km = W.king_model(6.0)
    # King (1966): W0 = 6 has concentration c = log10(r_t / r_0) ~ 1.26
    assert 1.23 < km.concentration < 1.29
    assert km.W[-1] < 1e-6 and abs(km.M[-1] - 1) < 1e-12
    # grid refinement leaves the solution unchanged
    km2 = W.king_model(6.0, n_grid=8000)
    assert abs(km2.potential_energy / km.potential_energy - 1) < 1e-4


def test_king_sample_is_virialised():
    cl = W.king(1 << 14, 7, masses="kroupa")
    K, Wp = oracle.energy(cl.m, cl.x, cl.v)
    assert abs(Wp + 0.5) < 0.03
    assert abs(2 * K / -Wp - 1) < 0.06


def test_king_binaries_are_centre_of_mass_particles():
    cl = W.king(1 << 14, 8, binary_fraction=0.05)
    nb = cl.extra["binary_index"].size
    assert nb == round(0.05 * cl.n)
    assert abs(cl.m.sum() - 1) < 1e-12
    a = cl.extra["binary_a_au"]
    assert a.min() >= 0.005 and a.max() <= 50


def test_active_blocks_follow_sorted_step_list():
    cl = W.plummer(4096, 1)
    steps = W.block_steps(cl, seed=1)
    lv = np.log2(steps)
    assert np.all(lv == np.round(lv)) and steps.max() <= 0.125 and steps.min() >= 0.5 ** 22
    blk = W.active_block(steps, 100)
    assert blk.dtype == np.int32 and len(set(blk.tolist())) == 100
    # every particle outside the block has a step >= the largest inside it
    assert steps[np.setdiff1d(np.arange(cl.n), blk)].min() >= steps[blk].max()
    # the small-step particles sit in the core
    r = np.sqrt((cl.x ** 2).sum(1))
    assert np.median(r[blk]) < np.median(r)


def test_neighbour_radius_gives_target_median():
    from scipy.spatial import cKDTree
    cl = W.plummer(1 << 14, 9, masses="kroupa")
    rs2 = W.neighbour_radius2(cl.x, 80)
    counts = np.array([len(c) - 1 for c in cKDTree(cl.x).query_ball_point(cl.x, math.sqrt(rs2))])
    assert 75 <= np.median(counts) <= 85


def test_generators_are_seeded():
    a = W.plummer(1000, 3, masses="kroupa")
    b = W.plummer(1000, 3, masses="kroupa")
    c = W.plummer(1000, 4, masses="kroupa")
    assert np.array_equal(a.x, b.x) and np.array_equal(a.m, b.m)
    assert not np.array_equal(a.x, c.x)


def test_ensemble_layout():
    e = W.ensemble(n_clusters=6, seed=4)
    assert e.cluster_off[-1] == e.m.shape[0] == e.x.shape[0]
    for c in range(6):
        lo, hi = e.cluster_off[c], e.cluster_off[c + 1]
        act = e.idx[e.active_off[c]:e.active_off[c + 1]]
        assert act.min() >= lo and act.max() < hi
        assert 256 <= hi - lo <= 32768
