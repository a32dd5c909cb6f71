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


def _ks(sample, cdf):
    s = np.sort(sample)
    n = s.size
    f = cdf(s)
    return max(np.max(np.arange(1, n + 1) / n - f), np.max(f - np.arange(n) / n))


def test_plummer_sampler_follows_its_distribution_function():
    """Raw Plummer samples (before the centre-of-mass shift): radii against the truncated
    cumulative mass M(r)/x_max (Kolmogorov-Smirnov at the 99.9 % level), every speed below the
    local escape speed, q = v/v_esc against the normalised isotropic distribution
    q^2 (1 - q^2)^(7/2), and isotropic directions of positions and velocities."""
    n, a, x_max = 200000, W.PLUMMER_A_NBODY, 0.999
    pos, vel = W.plummer_positions_velocities(n, np.random.default_rng(12), a=a, x_max=x_max)
    r = np.sqrt((pos ** 2).sum(1))
    crit = 1.95 / math.sqrt(n)
    assert _ks(r, lambda s: W.plummer_enclosed_mass(s, a) / x_max) < crit
    v = np.sqrt((vel ** 2).sum(1))
    v_esc = math.sqrt(2.0) * (1.0 + r * r / (a * a)) ** (-0.25) / math.sqrt(a)
    q = v / v_esc
    assert q.max() < 1.0 and q.min() >= 0.0
    grid = np.linspace(0.0, 1.0, 20001)
    dens = grid ** 2 * (1.0 - grid ** 2) ** 3.5
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (dens[1:] + dens[:-1]) * np.diff(grid))])
    cum /= cum[-1]
    assert _ks(q, lambda s: np.interp(s, grid, cum)) < crit
    for u in (pos / r[:, None], vel / v[:, None]):
        assert np.abs(u.mean(0)).max() < 5.0 / math.sqrt(n)
        assert np.abs((u ** 2).mean(0) - 1.0 / 3.0).max() < 5.0 / math.sqrt(n)
