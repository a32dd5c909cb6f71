"""GPU adjoint (VJP) of the regular-force step, its autograd binding and the chained
Hermite integrator, against the FP64 oracle.

Bars: the FP64 GPU VJP matches the oracle VJP to 1e-10 relative per particle (or
1e-10 of the largest row, for rows whose sum cancels); the mixed VJP to 2e-5 median
and 1e-3 max (same normalisation); both match O(N) central finite differences of the
oracle's forward at sampled coordinates to 1e-5 (FP64) / 1e-3 (mixed) relative; the
chained K-step gradient of the final kinetic energy matches finite differences of the
oracle's replay of the same frozen schedule to 1e-5 relative.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def row_err(got, ref):
    g, r = np.atleast_2d(got.T).T, np.atleast_2d(ref.T).T
    d = np.linalg.norm((g - r).reshape(len(g), -1), axis=1)
    s = np.linalg.norm(r.reshape(len(r), -1), axis=1)
    return d / np.maximum(s, 1e-3 * s.max())


def make_ctx(n, prec):
    from paper_1504_03687_gb300 import Context
    return Context(n, precision=prec, nb_cap=64)


def gpu_vjp(ctx, cl, idx, ga, gj, gp):
    ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
    gx, gv, gm = ctx.regular_force_backward(T(idx), T(ga), T(gj), T(gp))
    ctx.sync()
    return gx.cpu().numpy(), gv.cpu().numpy(), gm.cpu().numpy()


def test_mixed_fused_backward_with_close_pairs(gpu_lib):
    """Dense block (the fused pass, anchored separations) on a Plummer sphere with a tight pair
    planted next to every 40th particle, 1e-6 to 1e-3 apart, the cluster far from the origin:
    the pairs too close for the anchored separation are masked and replayed in double-single
    form, so the mixed bars against the oracle VJP hold."""
    cl = W.plummer(4000, 79, masses="kroupa")
    rng = np.random.default_rng(79)
    near = np.arange(0, 4000, 40)
    d = rng.standard_normal((near.size, 3))
    d *= (10.0 ** rng.uniform(-6, -3, near.size) / np.linalg.norm(d, axis=1))[:, None]

    class C:
        pass
    c = C()
    c.x = np.concatenate([cl.x, cl.x[near] + d]) + np.array([300.0, -200.0, 50.0])
    c.v = np.concatenate([cl.v, cl.v[near] + 0.1 * rng.standard_normal((near.size, 3))])
    c.m = np.concatenate([cl.m, cl.m[near]])
    n = c.x.shape[0]
    idx = rng.permutation(n).astype(np.int32)
    ga, gj, gp = rng.standard_normal((n, 3)), rng.standard_normal((n, 3)), rng.standard_normal(n)
    ref = oracle.regular_force_vjp(c.x, c.v, c.m, idx, ga, gj, gp)
    ctx = make_ctx(n, "mixed")
    got = gpu_vjp(ctx, c, idx, ga, gj, gp)
    ctx.close()
    for q in range(3):
        e = row_err(got[q], ref[q])
        assert np.median(e) <= 2e-5 and e.max() <= 1e-3, (q, float(np.median(e)), float(e.max()))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n,n_i", [(1000, 900), (1000, 137)])  # the fused pass and the two passes
def test_backward_rejects_duplicate_indices_and_is_reproducible(gpu_lib, prec, n, n_i):
    """Each active row writes its cotangents into its particle's record, so an index named
    twice is an argument error (reported, never summed in a racing order); with unique
    indices two calls give bit-identical gradients."""
    from paper_1504_03687_gb300 import api
    cl = W.plummer(n, 60, masses="kroupa")
    rng = np.random.default_rng(n_i)
    idx = rng.permutation(n)[:n_i].astype(np.int32)
    ga, gj, gp = rng.standard_normal((n_i, 3)), rng.standard_normal((n_i, 3)), rng.standard_normal(n_i)
    ctx = make_ctx(n, prec)
    a = gpu_vjp(ctx, cl, idx, ga, gj, gp)
    b = gpu_vjp(ctx, cl, idx, ga, gj, gp)
    for q in range(3):
        assert np.array_equal(a[q], b[q])
    dup = idx.copy()
    dup[n_i // 2] = dup[1]
    with pytest.raises(api.NBError, match="more than once"):
        gpu_vjp(ctx, cl, dup, ga, gj, gp)
    # the context stays usable and the next call is correct again
    c = gpu_vjp(ctx, cl, idx, ga, gj, gp)
    for q in range(3):
        assert np.array_equal(a[q], c[q])
    ctx.close()


@pytest.mark.parametrize("n,n_i", [(512, 512), (1000, 137), (3000, 1), (3000, 33), (4099, 2050), (2048, 1800),
                                   (3001, 3001)])
def test_backward_matches_oracle_vjp(gpu_lib, n, n_i):
    cl = W.plummer(n, 50 + n_i, masses="kroupa")
    rng = np.random.default_rng(n_i)
    idx = rng.permutation(n)[:n_i].astype(np.int32)
    ga, gj, gp = rng.standard_normal((n_i, 3)), rng.standard_normal((n_i, 3)), rng.standard_normal(n_i)
    ref = oracle.regular_force_vjp(cl.x, cl.v, cl.m, idx, ga, gj, gp)
    for prec, med, mx in (("fp64", 1e-10, 1e-10), ("mixed", 2e-5, 1e-3)):
        ctx = make_ctx(n, prec)
        got = gpu_vjp(ctx, cl, idx, ga, gj, gp)
        for q in range(3):
            e = row_err(got[q], ref[q])
            assert np.median(e) <= med and e.max() <= mx, (prec, q, float(np.median(e)), float(e.max()))
        ctx.close()


def test_backward_host_buffers(gpu_lib):
    cl = W.plummer(700, 61, masses="kroupa")
    rng = np.random.default_rng(3)
    idx = rng.permutation(700)[:300].astype(np.int32)
    ga, gj, gp = rng.standard_normal((300, 3)), rng.standard_normal((300, 3)), rng.standard_normal(300)
    ctx = make_ctx(700, "fp64")
    dev = gpu_vjp(ctx, cl, idx, ga, gj, gp)
    ctx.set_predicted(cl.x, cl.v, cl.m)
    gx, gv, gm = np.empty((700, 3)), np.empty((700, 3)), np.empty(700)
    s = ctx.lib.nb_regular_force_backward(ctx.h, 300, idx.ctypes.data, ga.ctypes.data, gj.ctypes.data,
                                          gp.ctypes.data, gx.ctypes.data, gv.ctypes.data, gm.ctypes.data, 0)
    assert s == 0
    np.testing.assert_array_equal(gx, dev[0])
    np.testing.assert_array_equal(gm, dev[2])


def test_autograd_function_against_dense_torch(gpu_lib):
    from paper_1504_03687_gb300.autograd import regular_force
    cl = W.plummer(256, 62, masses="kroupa")
    rng = np.random.default_rng(4)
    idx = rng.permutation(256)[:90].astype(np.int32)
    wa, wj, wp = (torch.tensor(rng.standard_normal(s), dtype=torch.float64, device=DEV)
                  for s in ((90, 3), (90, 3), (90,)))
    ctx = make_ctx(256, "fp64")
    X = T(cl.x).requires_grad_(True)
    V = T(cl.v).requires_grad_(True)
    M = T(cl.m).requires_grad_(True)
    a, j, p = regular_force(X, V, M, T(idx), ctx)
    ((wa * a).sum() + (wj * j).sum() + (wp * p).sum()).backward()
    # dense FP64 formula, autograd
    X2 = T(cl.x).requires_grad_(True)
    V2 = T(cl.v).requires_grad_(True)
    M2 = T(cl.m).requires_grad_(True)
    I = T(idx).long()
    R = X2[None] - X2[I][:, None]
    Wv = V2[None] - V2[I][:, None]
    mask = torch.ones(90, 256, dtype=torch.float64, device=DEV)
    mask[torch.arange(90), I] = 0
    d = torch.sqrt((R * R).sum(-1) + (1 - mask))
    acc = (M2[None, :, None] * (mask / d ** 3)[..., None] * R).sum(1)
    rw = (R * Wv).sum(-1)
    jerk = (M2[None, :, None] * ((mask / d ** 3)[..., None] * Wv - 3 * (rw * mask / d ** 5)[..., None] * R)).sum(1)
    pot = -(M2[None] * mask / d).sum(1)
    ((wa * acc).sum() + (wj * jerk).sum() + (wp * pot).sum()).backward()
    torch.testing.assert_close(a, acc, rtol=1e-12, atol=1e-12)
    for g1, g2 in ((X.grad, X2.grad), (V.grad, V2.grad), (M.grad, M2.grad)):
        torch.testing.assert_close(g1, g2, rtol=1e-10, atol=1e-10 * float(g2.abs().max()))


@pytest.mark.slow
def test_full_block_65536_against_local_finite_differences(gpu_lib):
    """Adjoint at N = 65536 (Plummer, Kroupa), full active block, checked by central FD on
    64 random coordinates across x, v and m."""
    cl, _ = W.plummer_64k_kroupa()
    n = cl.n
    rng = np.random.default_rng(11)
    idx = np.arange(n, dtype=np.int32)
    ga, gj = rng.standard_normal((n, 3)), rng.standard_normal((n, 3))
    gp = np.ones(n)
    picks = [(["x", "v", "m"][q % 3], int(rng.integers(0, n)), int(rng.integers(0, 3))) for q in range(64)]
    fd = []
    for which, p, c in picks:
        h = 1e-6 if which != "m" else 1e-6 * cl.m[p]
        fd.append(oracle.loss_fd(cl.x, cl.v, cl.m, idx, ga, gj, gp, which, p, c, h=h))
    fd = np.array(fd)
    for prec, tol in (("fp64", 1e-5), ("mixed", 1e-3)):
        ctx = make_ctx(n, prec)
        gx, gv, gm = gpu_vjp(ctx, cl, idx, ga, gj, gp)
        got = np.array([gx[p, c] if w == "x" else gv[p, c] if w == "v" else gm[p] for w, p, c in picks])
        scale = np.array([np.abs(gx).max() if w == "x" else np.abs(gv).max() if w == "v" else np.abs(gm).max()
                          for w, _, _ in picks])
        err = np.abs(got - fd) / np.maximum(np.abs(fd), 1e-4 * scale)
        assert err.max() <= tol, (prec, float(err.max()), float(np.median(err)))
        ctx.close()


def test_hermite_chain_gradient_matches_oracle_replay(gpu_lib):
    """d(final kinetic energy)/d(initial conditions) through K block steps of a frozen
    schedule, with checkpoint-and-recompute every 8 steps, vs FD of the oracle's replay."""
    from paper_1504_03687_gb300.autograd import hermite_chain
    n, K = 2048, 24
    cl = W.plummer(n, 63, masses="kroupa")
    _, _, sched = oracle.hermite_record(cl.m, cl.x, cl.v, 1.0, eta=0.02, max_blocks=K)
    assert len(sched) == K
    ctx = make_ctx(n, "fp64")
    x0 = T(cl.x).requires_grad_(True)
    v0 = T(cl.v).requires_grad_(True)
    m = T(cl.m)
    schedule = [(t, T(a)) for t, a in sched]
    xf, vf = hermite_chain(x0, v0, m, schedule, ctx, checkpoint_every=8)
    ke = 0.5 * (m[:, None] * vf * vf).sum()
    ke.backward()
    # forward equals the oracle replay
    xr, vr = oracle.hermite_replay(cl.m, cl.x, cl.v, sched)
    np.testing.assert_allclose(xf.detach().cpu().numpy(), xr, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(vf.detach().cpu().numpy(), vr, rtol=1e-9, atol=1e-11)

    def ke_of(x, v):
        _, vv = oracle.hermite_replay(cl.m, x, v, sched)
        return 0.5 * (cl.m[:, None] * vv * vv).sum()
    rng = np.random.default_rng(5)
    gx, gv = x0.grad.cpu().numpy(), v0.grad.cpu().numpy()
    # coordinates of particles the schedule moves (their gradients are not at the FD noise floor)
    moved = np.unique(np.concatenate([a for _, a in sched]))
    ke0 = 0.5 * (cl.m[:, None] * cl.v * cl.v).sum()
    h = 1e-5
    floor = 50 * np.finfo(float).eps * ke0 / h  # rounding noise of the central difference
    for _ in range(6):
        p, c = int(rng.choice(moved)), int(rng.integers(0, 3))
        for which, g in (("x", gx), ("v", gv)):
            def shifted(d):
                x, v = cl.x.copy(), cl.v.copy()
                (x if which == "x" else v)[p, c] += d
                return ke_of(x, v)
            d1 = (shifted(h) - shifted(-h)) / (2 * h)
            d2 = (shifted(h / 2) - shifted(-h / 2)) / h
            fd = (4 * d2 - d1) / 3
            assert abs(fd - g[p, c]) <= 1e-5 * abs(fd) + floor, (which, p, c, fd, g[p, c])
    ctx.close()
