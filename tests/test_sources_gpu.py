"""Source-range restriction (nb_set_source_range) and the split of the particle set between
the GPUs of one node (Sec. 3.4), emulated on one GPU: every shard's call sums over its own
source range, and merging the shards in range order gives the unrestricted result.

Bars: neighbour lists and true counts bit-identical to the unrestricted call; FP64 sums equal
up to the order of the additions (1e-12 relative per row, or 1e-12 of the largest row);
mixed sums within the mixed bars (2e-6 median, 1e-4 max relative) of the unrestricted mixed
call (a shard may run another kernel variant, which rounds its FP32 tile sums differently)
and of the FP64 oracle on sampled rows."""
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
    return d / np.maximum(s, 1e-12 * s.max())


@pytest.fixture(scope="module")
def cluster():
    cl, rs2 = W.plummer_128k_kroupa()
    steps = W.block_steps(cl, seed=1)
    return cl, rs2, steps


def combine_shards(parts, cap):
    """Single-process stand-in for the source-sharded exchange: the shards' sums and counts
    added in shard order (what the ranks' all-reduce computes), the lists merged by the
    library's merge."""
    from paper_1504_03687_gb300.dist import merge_source_lists
    acc, jerk, pot, count = (sum(p[q] for p in parts) for q in (0, 1, 2, 5))
    off, idx = merge_source_lists([p[3] for p in parts], [p[4] for p in parts], cap)
    return acc, jerk, pot, off, idx, count


def run_sharded(ctx, idx_d, rs2, shards, cap):
    parts = []
    for lo, hi in shards:
        if lo == hi:
            continue
        ctx.set_source_range(lo, hi)
        r = ctx.regular_force(idx_d, rs2, nb_capacity=int(idx_d.shape[0]) * cap)
        parts.append((r.acc, r.jerk, r.pot, r.nb_off, r.nb_idx, r.nb_count))
    ctx.set_source_range(0, 0)
    ctx.sync()
    return combine_shards(parts, cap)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n_i", [1, 37, 1024, 16384])
@pytest.mark.parametrize("world", [2, 3, 8])
def test_sharded_sources_reproduce_full_call(gpu_lib, cluster, prec, n_i, world):
    from paper_1504_03687_gb300 import Context
    from paper_1504_03687_gb300.dist import shard_sources
    cl, rs2, steps = cluster
    cap = 64  # below the typical count: many lists are cut inside one shard or across shards
    idx = W.active_block(steps, n_i)
    ctx = Context(cl.n, precision=prec, nb_cap=cap)
    ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
    idx_d = T(idx)
    full = ctx.regular_force(idx_d, rs2, nb_capacity=n_i * cap)
    ctx.sync()
    got = run_sharded(ctx, idx_d, rs2, [shard_sources(cl.n, world, r) for r in range(world)], cap)
    off = full.nb_off.cpu().numpy()
    np.testing.assert_array_equal(got[3].cpu().numpy(), off)
    np.testing.assert_array_equal(got[4].cpu().numpy()[:off[-1]], full.nb_idx.cpu().numpy()[:off[-1]])
    np.testing.assert_array_equal(got[5].cpu().numpy(), full.nb_count.cpu().numpy())
    med, mx = (1e-12, 1e-12) if prec == "fp64" else (2e-6, 1e-4)
    for g, f in ((got[0], full.acc), (got[1], full.jerk), (got[2], full.pot)):
        e = row_err(g.cpu().numpy(), f.cpu().numpy())
        assert np.median(e) <= med and e.max() <= mx, (prec, float(np.median(e)), float(e.max()))
    if prec == "mixed":
        sel = np.arange(0, n_i, max(1, n_i // 48))
        ref = oracle.regular_force(cl.x, cl.v, cl.m, idx[sel], rs2, cap=cap, lists=False)
        for q in range(3):
            e = row_err(got[q].cpu().numpy()[sel], ref[q])
            assert np.median(e) <= 2e-6 and e.max() <= 1e-4, (q, float(np.median(e)), float(e.max()))
    ctx.close()


def test_source_range_ragged_tail_and_host_buffers(gpu_lib):
    """A particle count that is not a multiple of the range alignment, ranges that end at
    n, host-buffer calls; and the restricted call against the oracle's restricted sums."""
    from paper_1504_03687_gb300 import Context
    cl = W.plummer(5000, 71, masses="kroupa")
    rs2 = float(W.neighbour_radius2(cl.x, 40, seed=71))
    idx = np.random.default_rng(71).permutation(5000)[:777].astype(np.int32)
    for prec in ("fp64", "mixed"):
        ctx = Context(5000, precision=prec, nb_cap=128)
        ctx.set_predicted(cl.x, cl.v, cl.m)
        for lo, hi in ((0, 256), (256, 4096), (4096, 5000), (768, 5000)):
            ctx.set_source_range(lo, hi)
            r = ctx.regular_force(idx, rs2)
            a, j, p = oracle.pair_sums(cl.x, cl.v, cl.m, idx, np.arange(lo, hi, dtype=np.int32))
            tol = 1e-12 if prec == "fp64" else 1e-4
            for g, ref in ((r.acc, a), (r.jerk, j), (r.pot, p)):
                e = row_err(g, ref)
                assert e.max() <= tol, (prec, lo, hi, float(e.max()))
            _, _, _, cnt, lists = oracle.regular_force(cl.x, cl.v, cl.m, idx, rs2, cap=5000)
            inside = [l[(l >= lo) & (l < hi)] for l in lists]
            assert [len(l) for l in inside] == list(r.nb_count)
            for k, l in enumerate(r.neighbour_lists()):
                np.testing.assert_array_equal(l, inside[k][:128])
        ctx.set_source_range(0, 0)
        full = ctx.regular_force(idx, rs2)
        a, j, p, cnt, _ = oracle.regular_force(cl.x, cl.v, cl.m, idx, rs2, cap=128)
        assert row_err(full.acc, a).max() <= (1e-12 if prec == "fp64" else 1e-4)
        ctx.close()


def test_source_range_errors(gpu_lib):
    from paper_1504_03687_gb300 import Context, NBError
    from paper_1504_03687_gb300.api import NB_ERR_ARG, NB_ERR_STATE
    cl = W.plummer(3000, 72)
    ctx = Context(4096, precision="fp64", nb_cap=32)
    ctx.set_predicted(T(cl.x), T(cl.v), T(cl.m))
    idx = T(np.arange(10, dtype=np.int32))
    for lo, hi in ((1, 300), (256, 256), (512, 256), (-256, 10), (0, 4097)):
        with pytest.raises(NBError) as e:
            ctx.set_source_range(lo, hi)
        assert e.value.status == NB_ERR_ARG
    ctx.set_source_range(0, 3500)  # fits n_max but not the 3000 loaded particles
    with pytest.raises(NBError) as e:
        ctx.regular_force(idx, 0.01)
    assert e.value.status == NB_ERR_STATE
    ctx.set_source_range(0, 1000)  # ends neither at n nor on the alignment
    with pytest.raises(NBError) as e:
        ctx.regular_force(idx, 0.01)
    assert e.value.status == NB_ERR_STATE
    ctx.set_source_range(0, 1024)
    g = torch.zeros((10, 3), dtype=torch.float64, device=DEV)
    with pytest.raises(NBError) as e:
        ctx.regular_force_backward(idx, g, g, torch.zeros(10, dtype=torch.float64, device=DEV))
    assert e.value.status == NB_ERR_STATE
    ctx.set_source_range(0, 0)
    ctx.regular_force(idx, 0.01)
    ctx.sync()
    ctx.close()
