"""The spatial row order of the anchored mixed force kernel (nb_row_order), and the anchored
kernel itself on blocks that take each form of the ordering.

Bars: the device permutation is bit-identical to a numpy restatement of its definition (Morton
keys of the records' FP32 hi parts, 8 bits per coordinate over the block's bounding box, a stable
sort); the anchored kernel meets the mixed bars against the FP64 oracle, and its neighbour lists
are bit-identical to the double-single packed kernel's (the same r^2 decides them)."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def hi_part(x):
    """FP32 hi part of the mixed j-record: x with its 29 low mantissa bits cleared."""
    return (np.ascontiguousarray(x).view(np.int64) & ~np.int64((1 << 29) - 1)).view(np.float64).astype(np.float32)


def spread8(a):
    a = a.astype(np.uint32) & 0xFF
    a = (a | (a << 8)) & 0x00F00F
    a = (a | (a << 4)) & 0x0C30C3
    a = (a | (a << 2)) & 0x249249
    return a


def expected_order(x, idx, n):
    ok = (idx >= 0) & (idx < n)
    h = hi_part(x[np.where(ok, idx, 0)])
    keys = np.full(idx.size, 0xFFFFFF, np.uint32)
    if ok.any():
        lo, hi = h[ok].min(0), h[ok].max(0)
        ext = (hi - lo).astype(np.float32)
        with np.errstate(divide="ignore"):
            inv = np.where(ext > 0, np.float32(256) / ext, np.float32(0)).astype(np.float32)
        t = ((h - lo).astype(np.float32) * inv).astype(np.float32)
        q = np.clip(np.trunc(t), 0, 255).astype(np.int64)
        k = spread8(q[:, 0]) | (spread8(q[:, 1]) << 1) | (spread8(q[:, 2]) << 2)
        keys[ok] = k[ok]
    return np.argsort(keys, kind="stable").astype(np.int32)


@pytest.fixture(scope="module")
def p128k():
    cl, rs2 = W.plummer_128k_kroupa()
    return cl, rs2, W.block_steps(cl, seed=1)


@pytest.mark.parametrize("n_i", [1, 700, 4096, 4097, 20000, 131072])
def test_row_order_matches_its_definition(gpu_lib, p128k, n_i):
    from paper_1504_03687_gb300 import Context
    cl, _, steps = p128k
    idx = W.active_block(steps, n_i)
    ctx = Context(cl.n, precision="mixed", nb_cap=64)
    ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
    perm = ctx.row_order(T(idx)).cpu().numpy()
    again = ctx.row_order(T(idx)).cpu().numpy()
    ctx.close()
    np.testing.assert_array_equal(perm, expected_order(cl.x, idx, cl.n))
    np.testing.assert_array_equal(perm, again)


def test_row_order_puts_bad_rows_last(gpu_lib, p128k):
    from paper_1504_03687_gb300 import Context
    cl, _, steps = p128k
    idx = W.active_block(steps, 5000).copy()
    idx[[3, 1000, 4999]] = [-1, cl.n, -7]
    ctx = Context(cl.n, precision="mixed", nb_cap=64)
    ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
    perm = ctx.row_order(T(idx)).cpu().numpy()
    ctx.close()
    np.testing.assert_array_equal(perm, expected_order(cl.x, idx, cl.n))
    assert list(perm[-3:]) == [3, 1000, 4999]


@pytest.mark.parametrize("variant", [10, 11, 12, 13, 14, 15, 16, 17, 18, 19])
def test_anchored_kernel_on_a_large_block(gpu_lib, p128k, variant):
    """20000 rows (the many-CTA ordering), forced anchored variant against the oracle on
    sampled rows; all lists bit-identical to the double-single packed kernel's."""
    from paper_1504_03687_gb300 import Context
    cl, rs2, steps = p128k
    idx = W.active_block(steps, 20000)
    ctx = Context(cl.n, precision="mixed", nb_cap=512)
    ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
    ctx.set_plan_override(1, variant, 0)
    res = ctx.regular_force(T(idx), rs2)
    ctx.sync()
    ctx.set_plan_override(1, 4, 0)
    base = ctx.regular_force(T(idx), rs2)
    ctx.sync()
    assert torch.equal(base.nb_off, res.nb_off) and torch.equal(base.nb_count, res.nb_count)
    tot = int(base.nb_off[-1])
    assert torch.equal(base.nb_idx[:tot], res.nb_idx[:tot])
    sel = np.sort(np.random.default_rng(variant).choice(idx.size, 256, replace=False))
    ref = oracle.regular_force(cl.x, cl.v, cl.m, idx[sel], rs2, cap=512, lists=False)
    for name, g, r in (("acc", res.acc, ref[0]), ("jerk", res.jerk, ref[1]), ("pot", res.pot, ref[2])):
        g = g[sel].cpu().numpy()
        e = (np.linalg.norm(g - r, axis=1) / np.linalg.norm(r, axis=1)) if g.ndim == 2 else np.abs(g - r) / np.abs(r)
        assert np.median(e) <= 2e-6 and e.max() <= 1e-4, (name, float(np.median(e)), float(e.max()))
    # the same call twice: bit for bit (the order and the anchors are deterministic)
    ctx.set_plan_override(1, variant, 0)
    again = ctx.regular_force(T(idx), rs2)
    ctx.sync()
    assert torch.equal(again.acc, res.acc) and torch.equal(again.jerk, res.jerk) and torch.equal(again.pot, res.pot)
    ctx.close()


def test_anchored_kernel_with_close_pairs(gpu_lib):
    """Pairs far closer than the rows' distance to their anchor (the masked pairs that the
    replay adds in double-single form): a Plummer sphere with a tight pair planted next to
    every 50th particle, 1e-7 to 1e-4 apart, and a cluster far from the origin."""
    from paper_1504_03687_gb300 import Context
    cl = W.plummer(8192, 78, masses="kroupa")
    rng = np.random.default_rng(78)
    x, v, m = cl.x.copy(), cl.v.copy(), cl.m.copy()
    near = np.arange(0, 8192, 50)
    d = rng.standard_normal((near.size, 3))
    d *= (10.0 ** rng.uniform(-7, -4, near.size) / np.linalg.norm(d, axis=1))[:, None]
    x = np.concatenate([x, x[near] + d]) + np.array([300.0, -200.0, 50.0])
    v = np.concatenate([v, v[near] + 0.1 * rng.standard_normal((near.size, 3))])
    m = np.concatenate([m, m[near]])
    n = x.shape[0]
    rs2 = float(W.neighbour_radius2(x, 50, seed=78))
    idx = np.random.default_rng(1).permutation(n).astype(np.int32)
    ref = oracle.regular_force(x, v, m, idx, rs2, cap=512)
    ctx = Context(n, precision="mixed", nb_cap=512)
    ctx.set_predicted(T(x), T(v), T(m))
    for variant in (10, 11, 12, 13, 14, 15, 16, 17, 18, 19):
        ctx.set_plan_override(1, variant, 0)
        res = ctx.regular_force(T(idx), rs2)
        ctx.sync()
        for name, g, r in (("acc", res.acc, ref[0]), ("jerk", res.jerk, ref[1]), ("pot", res.pot, ref[2])):
            g = g.cpu().numpy()
            e = (np.linalg.norm(g - r, axis=1) / np.linalg.norm(r, axis=1)) if g.ndim == 2 else np.abs(g - r) / np.abs(r)
            assert np.median(e) <= 2e-6 and e.max() <= 1e-4, (variant, name, float(np.median(e)), float(e.max()))
        got = res.neighbour_lists()
        cnt = res.nb_count.cpu().numpy()
        rs = np.sqrt(rs2)
        for k, i in enumerate(idx):
            a, b = set(got[k].tolist()), set(ref[4][k].tolist())
            if a != b:
                dd = np.sqrt(((x[list(a ^ b)] - x[i]) ** 2).sum(1))
                assert np.all(np.abs(dd - rs) <= 1e-6 * rs), (variant, k)
            assert abs(int(cnt[k]) - int(ref[3][k])) <= len(a ^ b)
    ctx.close()
