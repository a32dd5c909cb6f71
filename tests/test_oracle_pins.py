"""Pins of the FP64 CPU oracle to things other than itself.

Each test ties one oracle function to a closed form, an invariant, a textbook
special case or brute force, chosen so that a plausible mistake (a dropped or
mis-signed term, a wrong power of r, an i/j swap, a transposed operand) fails at
least one of them:

  force/jerk/pot : Newton's third law (sum m a = 0, sum m jerk = 0); jerk as the
                   time derivative of acc along straight-line motion; acc as
                   minus the gradient of the potential energy built from pot;
                   the Plummer potential energy -3π/(32a); two-body Kepler orbit
  neighbours     : brute-force k-d tree ball query (scipy)
  predictor      : exact rational evaluation of constant-jerk motion
  Hermite        : Kepler orbit (Kepler's equation) with 4th-order convergence,
                   energy conservation on the 1024-body Plummer sphere
  adjoint        : central finite differences of the forward, and autograd of an
                   independently written dense PyTorch formula
  AC integrator  : reduces bit for bit to the plain Hermite run when every particle
                   is a neighbour; energy conservation and its convergence with the
                   regular step parameter on the 1024-body Plummer sphere
  irregular force: lists plus the rest of the particles add up to the all-j sums
                   (with neighbour-only prediction against the all-particle
                   predictor); Newton's third law and the pair energy inside an
                   isolated group; jerk as d acc/dt along the prediction
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W


def _all_idx(n):
    return np.arange(n, dtype=np.int32)


# ---------------------------------------------------------------- force/jerk/pot
def test_newton_third_law_unequal_masses():
    cl = W.plummer(1024, 11, masses="kroupa")
    a, j, p, _, _ = oracle.regular_force(cl.x, cl.v, cl.m, _all_idx(cl.n), 0.0, lists=False)
    ma, mj = cl.m[:, None] * a, cl.m[:, None] * j
    assert np.abs(ma.sum(0)).max() <= 1e-13 * np.abs(ma).sum()
    assert np.abs(mj.sum(0)).max() <= 1e-13 * np.abs(mj).sum()
    # a plausible slip, m_i instead of m_j, breaks the law by O(1)
    assert np.abs(ma.sum(0)).max() < 1e-9


def test_jerk_is_time_derivative_of_acc():
    """jerk_i = d acc_i/dt along x(t) = x + v t (exact identity for the direct sum)."""
    cl = W.plummer(1024, 12, masses="kroupa")
    idx = _all_idx(cl.n)
    _, j, _, _, _ = oracle.regular_force(cl.x, cl.v, cl.m, idx, 0.0, lists=False)

    def acc_at(h):
        return oracle.regular_force(cl.x + h * cl.v, cl.v, cl.m, idx, 0.0, lists=False)[0]
    h = 1e-4
    d1 = (acc_at(h) - acc_at(-h)) / (2 * h)
    d2 = (acc_at(h / 2) - acc_at(-h / 2)) / h
    rich = (4 * d2 - d1) / 3  # Richardson: O(h^4)
    e = np.linalg.norm(rich - j, axis=1) / np.linalg.norm(j, axis=1)
    assert np.median(e) < 1e-8
    assert e.max() < 1e-6


def test_acc_is_minus_gradient_of_potential_energy():
    """m_i acc_i = -dW/dx_i with W = 1/2 sum m_i pot_i (links pot's form to acc's)."""
    cl = W.plummer(64, 13, masses="kroupa")
    idx = _all_idx(cl.n)
    a, _, _, _, _ = oracle.regular_force(cl.x, cl.v, cl.m, idx, 0.0, lists=False)

    def Wtot(x):
        _, _, p, _, _ = oracle.regular_force(x, cl.v, cl.m, idx, 0.0, lists=False)
        return 0.5 * np.dot(cl.m, p)
    h = 1e-5
    rng = np.random.default_rng(0)
    for i in rng.choice(cl.n, 8, replace=False):
        for c in range(3):
            xp, xm = cl.x.copy(), cl.x.copy()
            xp[i, c] += h
            xm[i, c] -= h
            g = (Wtot(xp) - Wtot(xm)) / (2 * h)
            assert abs(-g - cl.m[i] * a[i, c]) <= 1e-6 * (abs(cl.m[i] * a[i, c]) + 1e-3 * cl.m[i])


def test_plummer_potential_energy():
    """W of untruncated Plummer samples -> -3π/(32a) (times 1 - 1/N for N bodies of mass 1/N).

    With a = 3π/16 this is -1/2, so the virial total energy is -3π/(64a) = -1/4.
    """
    n, seeds = 16384, range(100, 106)
    ws, ks = [], []
    for s in seeds:
        cl = W.plummer(n, s, x_max=1.0)
        K, Wp = oracle.energy(cl.m, cl.x, cl.v)
        ws.append(Wp)
        ks.append(K)
    ws = np.array(ws)
    expect = -3 * math.pi / (32 * W.PLUMMER_A_NBODY) * (1 - 1 / n)
    assert abs(expect + 0.5 * (1 - 1 / n)) < 1e-15
    sem = ws.std(ddof=1) / math.sqrt(len(ws))
    assert abs(ws.mean() - expect) < 5 * sem + 2e-4
    # total energy of the (virial) samples is W/2 = -3π/(64 a) = -1/4
    E = ws + np.array(ks)
    assert abs(E.mean() + 3 * math.pi / (64 * W.PLUMMER_A_NBODY)) < 3e-3


def test_pot_half_sum_equals_pair_energy():
    """W from pot (1/2 sum m pot) equals the i<j pair sum of orc_energy."""
    cl = W.plummer(512, 14, masses="kroupa")
    _, _, p, _, _ = oracle.regular_force(cl.x, cl.v, cl.m, _all_idx(cl.n), 0.0, lists=False)
    _, Wp = oracle.energy(cl.m, cl.x, cl.v)
    assert abs(0.5 * np.dot(cl.m, p) - Wp) <= 1e-13 * abs(Wp)


def test_two_body_closed_form():
    """N = 2: acc_1 = m_2 r/r^3, pot_1 = -m_2/r, jerk_1 = m_2 (w/r^3 - 3 (r.w) r/r^5)."""
    x = np.array([[0.1, -0.2, 0.3], [0.4, 0.5, -0.7]])
    v = np.array([[0.3, 0.1, -0.2], [-0.1, 0.2, 0.4]])
    m = np.array([0.25, 0.75])
    a, j, p, _, _ = oracle.regular_force(x, v, m, _all_idx(2), 0.0, lists=False)
    r = x[1] - x[0]
    w = v[1] - v[0]
    d = np.linalg.norm(r)
    np.testing.assert_allclose(a[0], m[1] * r / d ** 3, rtol=1e-14)
    np.testing.assert_allclose(a[1], -m[0] * r / d ** 3, rtol=1e-14)
    np.testing.assert_allclose(j[0], m[1] * (w / d ** 3 - 3 * np.dot(r, w) * r / d ** 5), rtol=1e-13)
    np.testing.assert_allclose(p, [-m[1] / d, -m[0] / d], rtol=1e-14)


def test_tiny_n_against_exact_rational_sums():
    """Brute force on N = 6 with every sum formed in exact rational arithmetic.

    Only 1/|r| is irrational; it is taken from math.sqrt in double and the rest
    is exact, so the oracle's FP64 ascending-j sum must agree to ~1e-14.
    """
    rng = np.random.default_rng(5)
    n = 6
    x = rng.standard_normal((n, 3))
    v = rng.standard_normal((n, 3))
    m = rng.random(n) + 0.1
    idx = np.array([4, 0, 2], dtype=np.int32)
    a, j, p, _, _ = oracle.regular_force(x, v, m, idx, 0.0, lists=False)
    for k, i in enumerate(idx):
        A = [Fraction(0)] * 3
        J = [Fraction(0)] * 3
        P = Fraction(0)
        for jj in range(n):
            if jj == i:
                continue
            r = [Fraction(x[jj, c]) - Fraction(x[i, c]) for c in range(3)]
            w = [Fraction(v[jj, c]) - Fraction(v[i, c]) for c in range(3)]
            r2 = sum(q * q for q in r)
            rinv = Fraction(1.0 / math.sqrt(float(r2)))
            mj = Fraction(m[jj])
            rw = sum(r[c] * w[c] for c in range(3))
            for c in range(3):
                A[c] += mj * rinv ** 3 * r[c]
                J[c] += mj * rinv ** 3 * (w[c] - 3 * rw * rinv ** 2 * r[c])
            P -= mj * rinv
        np.testing.assert_allclose(a[k], [float(q) for q in A], rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(j[k], [float(q) for q in J], rtol=1e-12, atol=1e-14)
        assert abs(p[k] - float(P)) <= 1e-14 * abs(float(P))


# ---------------------------------------------------------------- neighbours
def test_neighbour_sets_match_kdtree():
    from scipy.spatial import cKDTree
    cl, rs2 = W.plummer_1k_equal()
    idx = _all_idx(cl.n)
    _, _, _, cnt, lists = oracle.regular_force(cl.x, cl.v, cl.m, idx, rs2, cap=1024)
    tree = cKDTree(cl.x)
    rs = math.sqrt(rs2)
    counts = []
    for i in range(cl.n):
        ref = set(tree.query_ball_point(cl.x[i], rs * (1 + 1e-6))) - {i}
        inner = set(tree.query_ball_point(cl.x[i], rs * (1 - 1e-6))) - {i}
        got = set(lists[i].tolist())
        assert inner <= got <= ref, i
        assert list(lists[i]) == sorted(lists[i])
        counts.append(len(got))
    assert 40 <= np.median(counts) <= 60  # r_s was chosen for a median of ~50
    assert np.array_equal(np.array(counts), cnt)


def test_neighbour_cap_keeps_first_in_ascending_order():
    cl, rs2 = W.plummer_1k_equal()
    idx = _all_idx(cl.n)[::7]
    _, _, _, cnt_full, full = oracle.regular_force(cl.x, cl.v, cl.m, idx, rs2, cap=1024)
    _, _, _, cnt, cut = oracle.regular_force(cl.x, cl.v, cl.m, idx, rs2, cap=16)
    assert np.array_equal(cnt, cnt_full)
    assert (cnt > 16).any()
    for a, b in zip(full, cut):
        assert np.array_equal(a[:16], b)


def test_per_particle_rs2_and_self_exclusion():
    cl, rs2 = W.plummer_1k_equal()
    idx = np.array([3, 900, 17], dtype=np.int32)
    rs2v = np.array([rs2, 0.0, 4 * rs2])
    _, _, _, cnt, lists = oracle.regular_force(cl.x, cl.v, cl.m, idx, rs2v, cap=1024)
    assert cnt[1] == 0
    for k, i in enumerate(idx):
        d2 = ((cl.x - cl.x[i]) ** 2).sum(1)
        d2[i] = np.inf
        assert set(lists[k]) == set(np.nonzero(d2 < rs2v[k])[0])


# ---------------------------------------------------------------- predictor
def test_predictor_exact_for_constant_jerk_motion():
    rng = np.random.default_rng(3)
    n = 16
    # dyadic inputs so the exact rational answer is known
    q = lambda s: np.round(rng.standard_normal(s) * 256) / 256
    x, v, a, j = q((n, 3)), q((n, 3)), q((n, 3)), q((n, 3))
    t_last = np.round(rng.random(n) * 64) / 64
    t = 1.25
    xp, vp = oracle.predict(t, x, v, a, j, t_last)
    for i in range(n):
        dt = Fraction(t) - Fraction(t_last[i])
        for c in range(3):
            X = Fraction(x[i, c]) + Fraction(v[i, c]) * dt + Fraction(a[i, c]) * dt ** 2 / 2 \
                + Fraction(j[i, c]) * dt ** 3 / 6
            V = Fraction(v[i, c]) + Fraction(a[i, c]) * dt + Fraction(j[i, c]) * dt ** 2 / 2
            assert abs(xp[i, c] - float(X)) <= 4e-16 * (abs(float(X)) + 1)
            assert abs(vp[i, c] - float(V)) <= 4e-16 * (abs(float(V)) + 1)


# ---------------------------------------------------------------- Hermite integrator
def _kepler_relative(t, a=1.0, e=0.5, M=1.0):
    """Relative position of a bound two-body orbit started at pericentre on +x."""
    nmean = math.sqrt(M / a ** 3)
    Mt = nmean * t
    E = Mt
    for _ in range(60):
        E -= (E - e * math.sin(E) - Mt) / (1 - e * math.cos(E))
    return np.array([a * (math.cos(E) - e), a * math.sqrt(1 - e * e) * math.sin(E), 0.0])


def _kepler_ics(a=1.0, e=0.5):
    rp = a * (1 - e)
    vp = math.sqrt((1 + e) / (a * (1 - e)))  # G M = 1
    m = np.array([0.5, 0.5])
    x = np.array([[-0.5 * rp, 0, 0], [0.5 * rp, 0, 0]])
    v = np.array([[0, -0.5 * vp, 0], [0, 0.5 * vp, 0]])
    return m, x, v


def test_hermite_kepler_fourth_order():
    m, x, v = _kepler_ics()
    errs = []
    for k in (6, 7, 8):
        xe, ve, _ = oracle.hermite_run(m, x, v, 4.0, dt_fixed=0.5 ** k)
        rel = xe[1] - xe[0]
        errs.append(np.linalg.norm(rel - _kepler_relative(4.0)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 12 < r1 < 20 and 12 < r2 < 20, errs
    assert errs[-1] < 1e-7


def test_hermite_kepler_block_steps_conserve_energy():
    m, x, v = _kepler_ics()
    K0, W0 = oracle.energy(m, x, v)
    xe, ve, st = oracle.hermite_run(m, x, v, 8.0, eta=0.01, dt_max=0.125)
    K1, W1 = oracle.energy(m, xe, ve)
    assert abs((K1 + W1) - (K0 + W0)) < 2e-6 * abs(K0 + W0)
    assert np.linalg.norm(xe[1] - xe[0] - _kepler_relative(8.0)) < 1e-4


def test_energy_drift_plummer_1k():
    """|dE/E| <= 1e-6 over one N-body time unit, eta = 0.02, power-of-two steps."""
    cl, _ = W.plummer_1k_equal()
    K0, W0 = oracle.energy(cl.m, cl.x, cl.v)
    xe, ve, st = oracle.hermite_run(cl.m, cl.x, cl.v, 1.0, eta=0.02)
    K1, W1 = oracle.energy(cl.m, xe, ve)
    assert abs((K1 + W1) / (K0 + W0) - 1) <= 1e-6
    assert st[0] > 100  # many distinct blocks: hierarchical steps were exercised


# ---------------------------------------------------------------- adjoint
def _loss_forward(x, v, m, idx, ga, gj, gp):
    a, j, p, _, _ = oracle.regular_force(x, v, m, idx, 0.0, lists=False)
    return (ga * a).sum() + (gj * j).sum() + (gp * p).sum()


def test_adjoint_against_central_differences():
    cl = W.plummer(96, 21, masses="kroupa")
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(cl.n, 40, replace=False)).astype(np.int32)[::-1].copy()
    ga, gj = rng.standard_normal((40, 3)), rng.standard_normal((40, 3))
    gp = rng.standard_normal(40)
    gx, gv, gm = oracle.regular_force_vjp(cl.x, cl.v, cl.m, idx, ga, gj, gp)
    h = 1e-6
    for _ in range(24):
        which = rng.integers(0, 3)
        p = int(rng.integers(0, cl.n))
        c = int(rng.integers(0, 3))
        args = [cl.x.copy(), cl.v.copy(), cl.m.copy()]
        base = args[which]
        if which == 2:
            step = h * base[p]
            base[p] += step
            fp = _loss_forward(*args, idx, ga, gj, gp)
            base[p] -= 2 * step
            fm = _loss_forward(*args, idx, ga, gj, gp)
            fd, an = (fp - fm) / (2 * step), gm[p]
        else:
            base[p, c] += h
            fp = _loss_forward(*args, idx, ga, gj, gp)
            base[p, c] -= 2 * h
            fm = _loss_forward(*args, idx, ga, gj, gp)
            fd, an = (fp - fm) / (2 * h), (gx if which == 0 else gv)[p, c]
        assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-2 * np.abs([gx, gv][min(which, 1)]).max()), (which, p, c, fd, an)


def test_adjoint_against_dense_autograd():
    torch = pytest.importorskip("torch")
    cl = W.plummer(200, 22, masses="kroupa")
    rng = np.random.default_rng(2)
    idx = rng.permutation(cl.n)[:77].astype(np.int32)
    ga, gj, gp = rng.standard_normal((77, 3)), rng.standard_normal((77, 3)), rng.standard_normal(77)
    X = torch.tensor(cl.x, dtype=torch.float64, requires_grad=True)
    V = torch.tensor(cl.v, dtype=torch.float64, requires_grad=True)
    M = torch.tensor(cl.m, dtype=torch.float64, requires_grad=True)
    I = torch.tensor(idx, dtype=torch.long)
    # dense formulation: all pairs at once, self pairs removed by a mask
    R = X[None, :, :] - X[I][:, None, :]
    Wv = V[None, :, :] - V[I][:, None, :]
    mask = torch.ones(len(idx), cl.n, dtype=torch.float64)
    mask[torch.arange(len(idx)), I] = 0.0
    d = torch.sqrt((R * R).sum(-1) + (1 - mask))
    inv3 = mask / d ** 3
    acc = (M[None, :, None] * inv3[..., None] * R).sum(1)
    rw = (R * Wv).sum(-1)
    jerk = (M[None, :, None] * (inv3[..., None] * Wv - 3 * (rw * mask / d ** 5)[..., None] * R)).sum(1)
    pot = -(M[None, :] * mask / d).sum(1)
    L = (torch.tensor(ga) * acc).sum() + (torch.tensor(gj) * jerk).sum() + (torch.tensor(gp) * pot).sum()
    L.backward()
    gx, gv, gm = oracle.regular_force_vjp(cl.x, cl.v, cl.m, idx, ga, gj, gp)
    np.testing.assert_allclose(gx, X.grad.numpy(), rtol=1e-10, atol=1e-10 * np.abs(gx).max())
    np.testing.assert_allclose(gv, V.grad.numpy(), rtol=1e-10, atol=1e-10 * np.abs(gv).max())
    np.testing.assert_allclose(gm, M.grad.numpy(), rtol=1e-10, atol=1e-10 * np.abs(gm).max())


def test_oracle_reproduces_stored_fixture():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "oracle_n8.json")) as f:
        g = json.load(f)
    xp, vp = oracle.predict(g["t"], g["x"], g["v"], g["a"], g["jerk0"], g["t_last"])
    np.testing.assert_array_equal(xp, g["xp"])
    acc, jerk, pot, cnt, lists = oracle.regular_force(xp, vp, g["m"], g["idx"], g["rs2"], cap=8)
    np.testing.assert_allclose(acc, g["acc"], rtol=1e-15)
    np.testing.assert_allclose(jerk, g["jerk"], rtol=1e-15)
    np.testing.assert_allclose(pot, g["pot"], rtol=1e-15)
    assert cnt.tolist() == g["nb_count"] and [l.tolist() for l in lists] == g["nb_lists"]


def test_schedule_record_and_replay_reproduce_the_run():
    """A recorded block-step schedule replayed from the start reproduces the run bit for bit."""
    cl = W.plummer(128, 31)
    xr, vr, st = oracle.hermite_run(cl.m, cl.x, cl.v, 0.25, eta=0.02)
    x1, v1, sched = oracle.hermite_record(cl.m, cl.x, cl.v, 0.25, eta=0.02)
    np.testing.assert_array_equal(x1, xr)
    np.testing.assert_array_equal(v1, vr)
    assert len(sched) == st[0] and sum(len(a) for _, a in sched) == st[1]
    assert all(sched[b][0] < sched[b + 1][0] for b in range(len(sched) - 1))
    x2, v2 = oracle.hermite_replay(cl.m, cl.x, cl.v, sched)
    np.testing.assert_array_equal(x2, xr)
    np.testing.assert_array_equal(v2, vr)


def test_pair_sums_restrict_the_definition():
    """Sums over all sources equal regular_force; sums over disjoint source sets add up."""
    cl = W.plummer(300, 41, masses="kroupa")
    idx = np.arange(0, 300, 7, dtype=np.int32)
    a, j, p, _, _ = oracle.regular_force(cl.x, cl.v, cl.m, idx, 0.0, lists=False)
    all_j = np.arange(300, dtype=np.int32)
    a2, j2, p2 = oracle.pair_sums(cl.x, cl.v, cl.m, idx, all_j)
    np.testing.assert_array_equal(a, a2)
    np.testing.assert_array_equal(p, p2)
    a3, j3, p3 = oracle.pair_sums(cl.x, cl.v, cl.m, idx, all_j[:100])
    a4, j4, p4 = oracle.pair_sums(cl.x, cl.v, cl.m, idx, all_j[100:])
    np.testing.assert_allclose(a3 + a4, a, rtol=1e-12, atol=1e-12 * np.abs(a).max())
    np.testing.assert_allclose(j3 + j4, j, rtol=1e-12, atol=1e-12 * np.abs(j).max())


def test_local_finite_difference_matches_adjoint():
    cl = W.plummer(400, 42, masses="kroupa")
    rng = np.random.default_rng(9)
    idx = rng.permutation(400)[:150].astype(np.int32)
    ga, gj, gp = rng.standard_normal((150, 3)), rng.standard_normal((150, 3)), rng.standard_normal(150)
    gx, gv, gm = oracle.regular_force_vjp(cl.x, cl.v, cl.m, idx, ga, gj, gp)
    for p in (int(idx[3]), int(np.setdiff1d(np.arange(400), idx)[5])):
        for which, ref in (("x", gx[p, 1]), ("v", gv[p, 2]), ("m", gm[p])):
            c = 1 if which == "x" else 2
            fd = oracle.loss_fd(cl.x, cl.v, cl.m, idx, ga, gj, gp, which, p, c, h=1e-5 if which != "m" else 1e-9)
            assert abs(fd - ref) <= 1e-6 * abs(ref) + 1e-9, (which, p, fd, ref)


# ---------------------------------------------------------------- irregular force
def _csr(lists):
    off = np.zeros(len(lists) + 1, np.int64)
    off[1:] = np.cumsum([len(l) for l in lists])
    flat = np.concatenate(lists).astype(np.int32) if lists else np.zeros(0, np.int32)
    return off, flat


def test_irregular_plus_outside_equals_all_sources():
    """With a and jerk nonzero and t != t_last: the irregular sums over each row's neighbour
    list (neighbour-only prediction) plus the sums over the rest of the particles (after
    predicting all particles) give the all-j regular force of the predicted state.  Pins
    the list restriction and shows that predicting only the neighbours reproduces the
    all-particle prediction."""
    cl = W.plummer(1024, 43, masses="kroupa")
    rng = np.random.default_rng(43)
    a0, j0 = rng.standard_normal((1024, 3)), 10 * rng.standard_normal((1024, 3))
    tl = -rng.integers(0, 4, 1024) * 2.0 ** -10
    t = 2.0 ** -11
    xp, vp = oracle.predict(t, cl.x, cl.v, a0, j0, tl)
    rs2 = W.neighbour_radius2(xp, 40, seed=43)
    idx = rng.permutation(1024)[:64].astype(np.int32)
    a_all, j_all, p_all, cnt, lists = oracle.regular_force(xp, vp, cl.m, idx, rs2, cap=1024)
    assert (cnt > 0).mean() > 0.5
    off, flat = _csr(lists)
    ai, ji, pi = oracle.irregular_force(t, cl.x, cl.v, a0, j0, tl, cl.m, idx, off, flat)
    for k in range(idx.size):
        rest = np.setdiff1d(np.arange(1024, dtype=np.int32), lists[k])
        ao, jo, po = oracle.pair_sums(xp, vp, cl.m, idx[k:k + 1], rest)
        np.testing.assert_allclose(ai[k] + ao[0], a_all[k], rtol=1e-12, atol=1e-12 * np.abs(a_all[k]).max())
        np.testing.assert_allclose(ji[k] + jo[0], j_all[k], rtol=1e-11, atol=1e-11 * np.abs(j_all[k]).max())
        assert abs(pi[k] + po[0] - p_all[k]) <= 1e-12 * abs(p_all[k])
    # the irregular part is the close, dominant part of the force for these rows
    assert np.median(np.linalg.norm(ai[cnt > 0], axis=1) / np.linalg.norm(a_all[cnt > 0], axis=1)) > 0.05


def test_irregular_force_of_an_isolated_group_obeys_newton():
    """Six particles in a tight group far from 300 others, r_s around the group: each member's
    list is the other five, the irregular forces are the group's own mutual forces, and
    sum m acc = sum m jerk = 0 over the group."""
    rng = np.random.default_rng(44)
    far = W.plummer(300, 44)
    xg = 0.01 * rng.standard_normal((6, 3)) + np.array([30.0, 0.0, 0.0])
    vg = 0.3 * rng.standard_normal((6, 3))
    mg = rng.uniform(0.5, 2.0, 6) / 300
    x = np.concatenate([far.x, xg]); v = np.concatenate([far.v, vg]); m = np.concatenate([far.m, mg])
    z = np.zeros_like(x)
    tl = np.zeros(306)
    idx = np.arange(300, 306, dtype=np.int32)
    _, _, _, cnt, lists = oracle.regular_force(x, v, m, idx, 1.0, cap=16)
    assert list(cnt) == [5] * 6 and all(set(l) == set(range(300, 306)) - {i} for l, i in zip(lists, idx))
    off, flat = _csr(lists)
    a, j, p = oracle.irregular_force(0.0, x, v, z, z, tl, m, idx, off, flat)
    ma, mj = mg[:, None] * a, mg[:, None] * j
    assert np.abs(ma.sum(0)).max() <= 1e-13 * np.abs(ma).sum()
    assert np.abs(mj.sum(0)).max() <= 1e-13 * np.abs(mj).sum()
    # the group's potential energy from the irregular potentials is the pair sum
    W_pairs = -sum(mg[a_] * mg[b_] / np.linalg.norm(xg[a_] - xg[b_]) for a_ in range(6) for b_ in range(a_ + 1, 6))
    assert abs(0.5 * (mg * p).sum() - W_pairs) <= 1e-13 * abs(W_pairs)


def test_irregular_jerk_is_time_derivative_along_prediction():
    """With a = jerk = 0 the prediction is straight-line motion, so for fixed lists the
    irregular jerk is d/dt of the irregular acceleration (Richardson central differences)."""
    cl = W.plummer(2000, 45, masses="kroupa")
    rs2 = W.neighbour_radius2(cl.x, 50, seed=45)
    idx = np.arange(0, 2000, 13, dtype=np.int32)
    _, _, _, _, lists = oracle.regular_force(cl.x, cl.v, cl.m, idx, rs2, cap=2000)
    off, flat = _csr(lists)
    z, tl = np.zeros_like(cl.x), np.zeros(2000)

    def acc_at(t):
        return oracle.irregular_force(t, cl.x, cl.v, z, z, tl, cl.m, idx, off, flat)[0]
    _, j, _ = oracle.irregular_force(0.0, cl.x, cl.v, z, z, tl, cl.m, idx, off, flat)
    h = 1e-5
    d1 = (acc_at(h) - acc_at(-h)) / (2 * h)
    d2 = (acc_at(h / 2) - acc_at(-h / 2)) / h
    rich = (4 * d2 - d1) / 3
    has = off[1:] > off[:-1]
    assert has.mean() > 0.5 and not rich[~has].any() and not j[~has].any()
    e = np.linalg.norm(rich[has] - j[has], axis=1) / np.linalg.norm(j[has], axis=1)
    assert np.median(e) < 1e-7 and e.max() < 1e-5


def test_irregular_force_edge_cases():
    cl = W.plummer(50, 46)
    z, tl = np.zeros_like(cl.x), np.zeros(50)
    idx = np.array([3, 7], np.int32)
    # empty lists give zeros; i itself in its own list is skipped
    a, j, p = oracle.irregular_force(0.0, cl.x, cl.v, z, z, tl, cl.m, idx, np.array([0, 0, 2]), np.array([7, 9], np.int32))
    assert not a[0].any() and not p[0]
    a2, _, p2 = oracle.irregular_force(0.0, cl.x, cl.v, z, z, tl, cl.m, idx[1:], np.array([0, 1]), np.array([9], np.int32))
    np.testing.assert_array_equal(a[1], a2[0])
    assert p[1] == p2[0]
    with pytest.raises(IndexError):
        oracle.irregular_force(0.0, cl.x, cl.v, z, z, tl, cl.m, idx, np.array([0, 1, 2]), np.array([1, 50], np.int32))
    with pytest.raises(IndexError):
        oracle.irregular_force(0.0, cl.x, cl.v, z, z, tl, cl.m, idx, np.array([0, 2, 1]), np.array([1, 2], np.int32))


# ---------------------------------------------------------------- Ahmad-Cohen integrator
def test_ac_reduces_to_hermite_when_every_particle_is_a_neighbour():
    """With r_s covering the whole system and a fixed r_s, the regular force is exactly zero
    and the AC run must equal the plain block-step Hermite run (pinned above by the Kepler
    orbit and energy conservation) bit for bit."""
    import ctypes
    cl = W.plummer(256, 101)
    xh, vh = cl.x.copy(), cl.v.copy()
    st = np.zeros(4)
    lib = oracle._load()
    rc = lib.orc_hermite_run(256, cl.m.ctypes.data, xh.ctypes.data, vh.ctypes.data, ctypes.c_double(0.25),
                             ctypes.c_double(0.02), ctypes.c_double(0.01), ctypes.c_double(0.125),
                             ctypes.c_double(0.0), ctypes.c_int64(0), st.ctypes.data)
    assert rc == 0
    x, v, _, info = oracle.ac_run(cl.m, cl.x, cl.v, 1e300, 0.25, eta_irr=0.02, eta_reg=0.03, eta_s=0.01,
                                  cap=256, nb_opt=0)
    assert info["rc"] == 0 and info["blocks"] == int(st[0]) and info["irregular_steps"] == int(st[1])
    np.testing.assert_array_equal(x, xh)
    np.testing.assert_array_equal(v, vh)


def test_ac_energy_conservation_and_regular_step_convergence():
    """Plummer 1024, r_s adapted towards 50 neighbours: |dE/E| at t = 1 below 1e-5, and ten
    times smaller regular-step accuracy parameter cuts it at least fourfold (the regular
    force's extrapolation is the scheme's leading error); every particle ends at t = 1; far
    fewer regular (all-j) steps than irregular ones; the lists sit at the target size."""
    cl, rs2 = W.plummer_1k_equal()
    E0 = sum(oracle.energy(cl.m, cl.x, cl.v))
    errs = []
    for eta_reg in (0.03, 0.003):
        x, v, r2, info = oracle.ac_run(cl.m, cl.x, cl.v, rs2, 1.0, eta_irr=0.02, eta_reg=eta_reg, eta_s=0.01,
                                       cap=256, nb_opt=50)
        assert info["rc"] == 0 and np.all(info["t"] == 1.0) and np.all(info["dt"] <= info["DT"])
        errs.append(abs(sum(oracle.energy(cl.m, x, v)) - E0) / abs(E0))
        if eta_reg == 0.03:
            assert info["regular_steps"] < 0.25 * info["irregular_steps"]
            assert 40 <= np.median(info["nb_count"]) <= 62
    assert errs[0] < 1e-5 and errs[1] < errs[0] / 4, errs


def _two_circular_binaries(d=1.0, a=0.1):
    """Two equal-mass circular binaries (total mass 1/2 each, separation a) on a circular
    mutual orbit of separation d, with inclined orbital planes: each member's only neighbour
    is its partner, and the regular force on it (from the other binary) is smooth in time."""
    def rot(axis, ang):
        u = np.asarray(axis, float) / np.linalg.norm(axis)
        K = np.array([[0, -u[2], u[1]], [u[2], 0, -u[0]], [-u[1], u[0], 0]])
        return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K

    def binary(R):
        w = np.sqrt(0.5 / a)
        return (np.array([[a / 2, 0, 0], [-a / 2, 0, 0]]) @ R.T,
                np.array([[0, w / 2, 0], [0, -w / 2, 0]]) @ R.T)
    xa, va = binary(rot([1, 0.3, 0.2], 0.4))
    xb, vb = binary(rot([0.2, 1, 0.5], 1.1))
    w = np.sqrt(1.0 / d)
    x = np.concatenate([xa + [d / 2, 0, 0], xb - [d / 2, 0, 0]])
    v = np.concatenate([va + [0, w / 2, 0], vb - [0, w / 2, 0]])
    return np.full(4, 0.25), x, v


def test_ac_regular_force_extrapolation_order():
    """Between regular steps the integrator extrapolates the regular force to third order in
    tau = t - T_i from its value, derivative and the second and third derivatives of the last
    Hermite interpolation (the Ahmad-Cohen scheme, Sec. 2).  Its error is therefore O(DT^4) in
    the force and O(DT^3) in the jerk when tau is a fixed fraction of the regular step DT.
    Measured directly: the regular step is forced to DT = 2^-k (dt_max, infinite eta_reg),
    the irregular steps are much smaller, and the run ends at t = 1/2 + DT/2, half a regular
    step after the last regular time 1/2; the total force and jerk the integrator holds there
    are compared with the all-j sums over the very predicted state they were evaluated on (the
    list part is exact, so the difference is the extrapolation error alone).  Halving DT must
    cut the force error 16-fold and the jerk error 8-fold: a dropped or mis-scaled third-
    derivative term leaves 8 and 4, a wrong second-derivative term 4 and 2."""
    m, x, v = _two_circular_binaries()
    idx = np.arange(4, dtype=np.int32)
    eF, eJ = [], []
    for k in range(6, 10):
        H = 2.0 ** -k
        _, _, _, info = oracle.ac_run(m, x, v, 0.3 ** 2, 0.5 + H / 2, eta_irr=2.5e-4, eta_reg=1e30, eta_s=1e-3,
                                      dt_max=H, cap=8, nb_opt=0)
        assert info["rc"] == 0 and list(info["nb_count"]) == [1, 1, 1, 1]
        assert np.all(info["t"] == 0.5 + H / 2) and np.all(info["T"] == 0.5) and np.all(info["DT"] == H)
        assert np.all(info["dt"] <= H / 4)
        a, j, _, _, _ = oracle.regular_force(info["xp"], info["vp"], m, idx, 0.3 ** 2, cap=8)
        eF.append(np.abs(info["acc"] - a).max() / np.abs(a).max())
        eJ.append(np.abs(info["jerk"] - j).max() / np.abs(j).max())
    rF = [eF[q] / eF[q + 1] for q in range(3)]
    rJ = [eJ[q] / eJ[q + 1] for q in range(3)]
    assert all(13.0 < r < 20.0 for r in rF), (eF, rF)
    assert all(6.5 < r < 10.0 for r in rJ), (eJ, rJ)
    assert 1e-9 < eF[0] < 1e-5 and 1e-8 < eJ[0] < 1e-4, (eF, eJ)
