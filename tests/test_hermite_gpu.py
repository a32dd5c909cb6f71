"""The Hermite predictor and corrector over caller arrays and their VJP kernels (through the
C ABI), the O(N) steps of the differentiable block-step chain.

Bars: the array predictor is bit-identical to nb_predict (the same function) and within 4 ulp
of the term magnitudes of the oracle's term-by-term Taylor sum; the corrector is bit-identical
to its definition evaluated in the same operation order in FP64 without FMA (numpy); each VJP
passes the dot-product test against its own forward kernel (both maps are linear in the
differentiated inputs for fixed times), <g, L d> = <L^T g, d>, to 1e-13 relative."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def make_ctx(n, prec="fp64"):
    from paper_1504_03687_gb300 import Context
    return Context(n, precision=prec, nb_cap=16)


@pytest.fixture(scope="module")
def state():
    cl, _ = W.plummer_1k_equal()
    steps = W.block_steps(cl, seed=0)
    a0, j0, tl = W.hermite_state(cl, seed=1, t_block=0.5, steps=steps)
    return cl, a0, j0, tl


def test_array_predictor_equals_nb_predict_and_the_oracle(gpu_lib, state):
    cl, a0, j0, tl = state
    ctx = make_ctx(cl.n)
    ctx.set_particles(T(cl.x), T(cl.v), T(a0), T(j0), T(cl.m), T(tl))
    ctx.predict(0.5)
    xp_ctx, vp_ctx = ctx.get_predicted()
    xp, vp = ctx.hermite_predict(0.5, T(cl.x), T(cl.v), T(a0), T(j0), T(tl))
    torch.cuda.synchronize()
    assert torch.equal(xp, xp_ctx) and torch.equal(vp, vp_ctx)
    rx, rv = oracle.predict(0.5, cl.x, cl.v, a0, j0, tl)
    dt = (0.5 - tl)[:, None]
    eps = np.finfo(float).eps
    bx = np.abs(cl.x) + np.abs(cl.v * dt) + np.abs(a0 * dt ** 2 / 2) + np.abs(j0 * dt ** 3 / 6)
    bv = np.abs(cl.v) + np.abs(a0 * dt) + np.abs(j0 * dt ** 2 / 2)
    assert np.all(np.abs(xp.cpu().numpy() - rx) <= 4 * eps * bx)
    assert np.all(np.abs(vp.cpu().numpy() - rv) <= 4 * eps * bv)
    ctx.close()


def test_corrector_is_its_definition(gpu_lib):
    rng = np.random.default_rng(3)
    n = 5000
    xp, vp, a0, j0, a1, j1 = (rng.standard_normal((n, 3)) for _ in range(6))
    t = 0.75
    tl = t - 2.0 ** -rng.integers(3, 20, n).astype(np.float64)
    ctx = make_ctx(16)
    x1, v1 = ctx.hermite_correct(t, T(tl), T(xp), T(vp), T(a0), T(j0), T(a1), T(j1))
    torch.cuda.synchronize()
    h = (t - tl)[:, None]
    da = a0 - a1
    a2 = (-6.0 * da - h * (4.0 * j0 + 2.0 * j1)) / (h * h)
    a3 = (12.0 * da + 6.0 * h * (j0 + j1)) / (h * h * h)
    rx = xp + h * h * h * h / 24.0 * a2 + h * h * h * h * h / 120.0 * a3
    rv = vp + h * h * h / 6.0 * a2 + h * h * h * h / 24.0 * a3
    np.testing.assert_array_equal(x1.cpu().numpy(), rx)
    np.testing.assert_array_equal(v1.cpu().numpy(), rv)
    ctx.close()


def _dot(us, vs):
    return sum(float((u * v).sum()) for u, v in zip(us, vs))


def test_predictor_vjp_dot_product(gpu_lib):
    rng = np.random.default_rng(4)
    n = 3000
    t = 1.25
    tl = T(t - rng.uniform(0, 0.25, n))
    d = [T(rng.standard_normal((n, 3))) for _ in range(4)]  # directions in (x, v, a, jerk)
    g = [T(rng.standard_normal((n, 3))) for _ in range(2)]  # cotangents of (xp, vp)
    ctx = make_ctx(16)
    Ld = ctx.hermite_predict(t, *d, tl)
    LTg = ctx.hermite_predict_backward(t, tl, *g)
    torch.cuda.synchronize()
    lhs, rhs = _dot(g, Ld), _dot(LTg, d)
    scale = sum(float((u.abs() * v.abs()).sum()) for u, v in zip(g, Ld))
    assert abs(lhs - rhs) <= 1e-13 * scale, (lhs, rhs)
    ctx.close()


def test_corrector_vjp_dot_product(gpu_lib):
    rng = np.random.default_rng(5)
    n = 3000
    t = 0.5
    tl = T(t - 2.0 ** -rng.integers(2, 16, n).astype(np.float64))
    d = [T(rng.standard_normal((n, 3))) for _ in range(6)]  # directions in (xp, vp, a0, j0, a1, j1)
    g = [T(rng.standard_normal((n, 3))) for _ in range(2)]  # cotangents of (x1, v1)
    ctx = make_ctx(16)
    Ld = ctx.hermite_correct(t, tl, *d)
    LTg = ctx.hermite_correct_backward(t, tl, *g)
    torch.cuda.synchronize()
    lhs, rhs = _dot(g, Ld), _dot(LTg, d)
    scale = sum(float((u.abs() * v.abs()).sum()) for u, v in zip(LTg, d))
    assert abs(lhs - rhs) <= 1e-13 * scale, (lhs, rhs)
    ctx.close()


def test_hermite_calls_reject_bad_arguments(gpu_lib):
    from paper_1504_03687_gb300 import api
    ctx = make_ctx(16)
    lib = ctx.lib
    assert lib.nb_hermite_predict(ctx.h, -1, 0.0, None, None, None, None, None, None, None) == api.NB_ERR_ARG
    assert lib.nb_hermite_correct(ctx.h, 4, 0.0, None, None, None, None, None, None, None, None, None) == api.NB_ERR_ARG
    assert lib.nb_hermite_predict_backward(ctx.h, 0, 0.0, None, None, None, None, None, None, None) == api.NB_OK
    ctx.close()
