"""Irregular force of the Ahmad-Cohen scheme (nb_irregular_force) against the FP64 oracle.

Inputs: the Hermite state (x, v, a, jerk at t_last) of the 131072-body Plummer cluster at a
late block time (t = 1), active blocks from the sorted step list, and the oracle's own
neighbour lists (cap 512) of the predicted state — never lists from the CUDA path.

Bars: FP64 e_i <= 1e-12 per row (vector 2-norm), or |delta| <= 1e-12 * sum over the list of
|term| (summation order differs); mixed median e_i <= 2e-6 and max e_i <= 1e-4 over the rows
with a non-empty list; rows with an empty list are exactly zero in both precisions.  The
regular/irregular split (all-j sums minus the list sums) must equal that difference bit for
bit, and the oracle's difference within 1e-11 (FP64) or 2e-4 (mixed) of the larger of the
all-j sum and the list's term sum (the errors of the two parts add)."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def csr(lists):
    off = np.zeros(len(lists) + 1, np.int64)
    off[1:] = np.cumsum([len(l) for l in lists])
    flat = np.concatenate(lists).astype(np.int32) if len(lists) and off[-1] else np.zeros(0, np.int32)
    return off, flat


def list_term_sums(xp, vp, m, idx, lists):
    """sum over each row's list of |acc term|, |jerk term|, |pot term| (tolerance normaliser)."""
    out = np.zeros((len(idx), 3))
    for k, (i, l) in enumerate(zip(idx, lists)):
        l = l[l != i]
        if not l.size:
            continue
        r = xp[l] - xp[i]
        w = vp[l] - vp[i]
        d = np.sqrt((r * r).sum(1))
        out[k] = [(m[l] / d ** 2).sum(),
                  (m[l] * (np.linalg.norm(w, axis=1) / d ** 3 + 3 * np.abs((r * w).sum(1)) / d ** 4)).sum(),
                  (m[l] / d).sum()]
    return out


def rows_err(got, ref):
    if got.ndim == 2:
        return np.linalg.norm(got - ref, axis=1), np.linalg.norm(ref, axis=1)
    return np.abs(got - ref), np.abs(ref)


def check(prec, got, ref, ts, nonempty):
    for q in range(3):
        g = got[q].cpu().numpy() if torch.is_tensor(got[q]) else got[q]
        d, s = rows_err(g, ref[q])
        assert not g[~nonempty].any() and not ref[q][~nonempty].any()
        d, s = d[nonempty], s[nonempty]
        if prec == "fp64":
            assert np.all((d <= 1e-12 * s) | (d <= 1e-12 * ts[nonempty, q])), (q, float((d / s).max()))
        else:
            e = d / s
            assert np.median(e) <= 2e-6 and e.max() <= 1e-4, (q, float(np.median(e)), float(e.max()))


@pytest.fixture(scope="module")
def setup():
    cl, rs2 = W.plummer_128k_kroupa()
    steps = W.block_steps(cl, seed=1)
    a0, j0, tl = W.hermite_state(cl, seed=5, t_block=1.0, steps=steps)
    t = 1.0
    xp, vp = oracle.predict(t, cl.x, cl.v, a0, j0, tl)
    return cl, rs2, steps, a0, j0, tl, t, xp, vp


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n_i", [1, 100, 4096, 16384])
def test_irregular_force_matches_oracle(gpu_lib, setup, prec, n_i):
    from paper_1504_03687_gb300 import Context
    cl, rs2, steps, a0, j0, tl, t, xp, vp = setup
    idx = W.active_block(steps, n_i)
    _, _, _, cnt, lists = oracle.regular_force(xp, vp, cl.m, idx, rs2, cap=512)
    off, flat = csr(lists)
    ref = oracle.irregular_force(t, cl.x, cl.v, a0, j0, tl, cl.m, idx, off, flat)
    ctx = Context(cl.n, precision=prec, nb_cap=512)
    ctx.set_particles(*[T(q) for q in (cl.x, cl.v, a0, j0, cl.m, tl)])
    got = ctx.irregular_force(t, T(idx), T(off), T(flat) if flat.size else T(np.zeros(1, np.int32)))
    ctx.sync()
    check(prec, got, ref, list_term_sums(xp, vp, cl.m, idx, lists), cnt > 0)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_split_host_buffers_and_state_refresh(gpu_lib, prec):
    """Host-buffer calls; the regular/irregular split of a regular-force result; a second
    nb_set_particles with another state rebuilds the state records."""
    from paper_1504_03687_gb300 import Context
    cl = W.plummer(6000, 81, masses="kroupa")
    steps = W.block_steps(cl, seed=81)
    idx = W.active_block(steps, 700)
    ctx = Context(6000, precision=prec, nb_cap=256)
    for seed, t in ((3, 0.5), (4, 2.0)):
        a0, j0, tl = W.hermite_state(cl, seed=seed, t_block=t, steps=steps)
        xp, vp = oracle.predict(t, cl.x, cl.v, a0, j0, tl)
        rs2 = float(W.neighbour_radius2(xp, 60, seed=seed))
        all_ref = oracle.regular_force(xp, vp, cl.m, idx, rs2, cap=6000)
        lists = all_ref[4]
        off, flat = csr(lists)
        irr_ref = oracle.irregular_force(t, cl.x, cl.v, a0, j0, tl, cl.m, idx, off, flat)
        ts = list_term_sums(xp, vp, cl.m, idx, lists)
        ctx.set_particles(cl.x, cl.v, a0, j0, cl.m, tl)
        ctx.predict(t)
        res = ctx.regular_force(idx, rs2, nb_capacity=700 * 256)
        all_got = [res.acc.copy(), res.jerk.copy(), res.pot.copy()]
        irr = ctx.irregular_force(t, idx, off, flat, regular=res)
        check(prec, irr, irr_ref, ts, all_ref[3] > 0)
        # the split: res now holds the all-j result minus the list sums
        for q, (reg, a_got) in enumerate(zip((res.acc, res.jerk, res.pot), all_got)):
            np.testing.assert_array_equal(reg, a_got - irr[q])
            outside_ref = all_ref[q] - irr_ref[q]
            d, _ = rows_err(reg, outside_ref)
            _, s_all = rows_err(all_ref[q], all_ref[q])
            bar = 1e-11 if prec == "fp64" else 2e-4  # the all-j error and the list error add
            assert np.all(d <= bar * np.maximum(s_all, ts[:, q])), (prec, q, float((d / s_all).max()))
    ctx.close()


def test_irregular_force_degenerate_inputs(gpu_lib):
    from paper_1504_03687_gb300 import Context, NBError
    from paper_1504_03687_gb300.api import NB_ERR_ARG, NB_ERR_STATE
    cl = W.plummer(3000, 82)
    z, tl = np.zeros_like(cl.x), np.zeros(3000)
    ctx = Context(3000, precision="fp64", nb_cap=64)
    ctx.set_particles(cl.x, cl.v, z, z, cl.m, tl)
    idx = np.array([5, 9, 11], np.int32)
    # empty lists give zeros; the row's own index in its list is skipped
    a, j, p = ctx.irregular_force(0.0, idx, np.array([0, 0, 2, 2]), np.array([9, 20], np.int32))
    assert not a[0].any() and not a[2].any() and not p[2]
    a2, _, p2 = ctx.irregular_force(0.0, idx[1:2], np.array([0, 1]), np.array([20], np.int32))
    np.testing.assert_array_equal(a[1], a2[0])
    # n_i = 0 is a no-op
    ctx.irregular_force(0.0, idx[:0], np.zeros(1, np.int64), np.zeros(0, np.int32))
    # host mode rejects bad indices and decreasing offsets before any GPU work
    for off, nb in ((np.array([0, 1, 1, 1]), np.array([3000], np.int32)),
                    (np.array([0, 2, 1, 2]), np.array([1, 2], np.int32))):
        with pytest.raises(NBError) as e:
            ctx.irregular_force(0.0, idx, off, nb)
        assert e.value.status == NB_ERR_ARG
    # device mode: a bad neighbour index is skipped and reported by the deferred status
    a_d, _, _ = ctx.irregular_force(0.0, T(idx[1:2]), T(np.array([0, 2])), T(np.array([20, 4000], np.int32)))
    with pytest.raises(NBError):
        ctx.sync()
    np.testing.assert_array_equal(a_d.cpu().numpy()[0], a2[0])
    # needs the Hermite state, not only a predicted one
    ctx2 = Context(3000, precision="mixed", nb_cap=64)
    ctx2.set_predicted(cl.x, cl.v, cl.m)
    with pytest.raises(NBError) as e:
        ctx2.irregular_force(0.0, idx, np.array([0, 0, 0, 0]), np.zeros(1, np.int32))
    assert e.value.status == NB_ERR_STATE
    ctx.close()
    ctx2.close()


def test_fp64_forms_agree_bit_for_bit(gpu_lib, setup):
    """The same rows in one call (all particles predicted once: N_i >= N/128 for FP64, N/8
    for mixed) and in calls of 32 rows (neighbour-only prediction): FP64 results identical,
    mixed within the mixed bars of each other."""
    from paper_1504_03687_gb300 import Context
    cl, rs2, steps, a0, j0, tl, t, xp, vp = setup
    idx = W.active_block(steps, 16384)
    _, _, _, cnt, lists = oracle.regular_force(xp, vp, cl.m, idx, rs2, cap=512)
    off, flat = csr(lists)
    for prec in ("fp64", "mixed"):
        ctx = Context(cl.n, precision=prec, nb_cap=512)
        ctx.set_particles(*[T(q) for q in (cl.x, cl.v, a0, j0, cl.m, tl)])
        big = [q.cpu().numpy() for q in ctx.irregular_force(t, T(idx), T(off), T(flat))]
        parts = []
        for k0 in range(0, 16384, 32):
            o = off[k0:k0 + 33] - off[k0]
            nbs = flat[off[k0]:off[k0 + 32]]
            nbs = nbs if nbs.size else np.zeros(1, np.int32)
            parts.append([q.cpu().numpy() for q in ctx.irregular_force(t, T(idx[k0:k0 + 32]), T(o), T(nbs))])
        ctx.sync()
        small = [np.concatenate([p_[q] for p_ in parts]) for q in range(3)]
        for q in range(3):
            if prec == "fp64":
                np.testing.assert_array_equal(big[q], small[q])
            else:
                d, sref = rows_err(big[q][cnt > 0], small[q][cnt > 0])
                e = d / sref
                assert np.median(e) <= 2e-6 and e.max() <= 1e-4
        ctx.close()


@pytest.mark.parametrize("n_i", [64, 4096])
def test_mixed_late_time_far_from_the_origin(gpu_lib, n_i):
    """Mixed irregular force of a cluster translated by (1e4, -2e4, 3e3) at block time
    t = 4096 + 37/2^14 with steps of 2^-12 .. 2^-16: both the base differences of the positions
    and t - t_last (formed from hi/lo halves of both times) would lose most of their digits in
    single precision; in double-single the rows stay within the mixed bars. Both forms: the
    neighbour-only one (64 rows) and predict-all (4096 rows: 4096 x 8 >= N)."""
    from paper_1504_03687_gb300 import Context
    n = 6000
    cl = W.plummer(n, 91, masses="kroupa")
    x = cl.x + np.array([1.0e4, -2.0e4, 3.0e3])
    rng = np.random.default_rng(91)
    t = 4096.0 + 37.0 / 2 ** 14
    dt = 2.0 ** -rng.integers(12, 17, n)
    tl = t - dt * rng.integers(0, 2, n)
    a0 = rng.standard_normal((n, 3))
    j0 = 10.0 * rng.standard_normal((n, 3))
    xp, vp = oracle.predict(t, x, cl.v, a0, j0, tl)
    rs2 = float(W.neighbour_radius2(xp, 50, seed=91))
    idx = np.sort(rng.choice(n, n_i, replace=False)).astype(np.int32)
    _, _, _, cnt, lists = oracle.regular_force(xp, vp, cl.m, idx, rs2, cap=256)
    off, flat = csr(lists)
    ref = oracle.irregular_force(t, x, cl.v, a0, j0, tl, cl.m, idx, off, flat)
    ctx = Context(n, precision="mixed", nb_cap=256)
    ctx.set_particles(*[T(q) for q in (x, cl.v, a0, j0, cl.m, tl)])
    got = ctx.irregular_force(t, T(idx), T(off), T(flat) if flat.size else T(np.zeros(1, np.int32)))
    ctx.sync()
    check("mixed", got, ref, list_term_sums(xp, vp, cl.m, idx, lists), cnt > 0)
    ctx.close()
