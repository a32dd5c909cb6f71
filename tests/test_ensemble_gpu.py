"""Batched ensemble form: many independent clusters of uneven N in one persistent launch.

Each cluster is compared with the FP64 oracle run on that cluster alone (the mixed bar:
median <= 2e-6, max <= 1e-4 relative per particle; neighbour sets outside the 1e-6 band),
every batch tile variant gives the same neighbour lists, a captured CUDA graph replays to
bitwise-identical results, and an active index outside its own cluster is reported.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


@pytest.fixture(scope="module")
def small_ensemble():
    return W.ensemble(n_clusters=24, seed=5, n_lo=64, n_hi=4096)


def run_batched(e, variant=-1, graph=False):
    from paper_1504_03687_gb300 import Context
    ctx = Context(e.cluster_off[-1], precision="mixed", nb_cap=256)
    ctx.set_predicted(T(e.x), T(e.v), T(e.m))
    ctx.batch_plan(e.cluster_off, e.active_off, variant)
    idx, rs2 = T(e.idx), T(e.rs2)
    out = ctx.regular_force_batched(idx, rs2)
    ctx.sync()
    if graph:
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                ctx.regular_force_batched(idx, rs2, out=out)
        return ctx, out, g
    return ctx, out


def test_batched_matches_oracle_per_cluster(gpu_lib, small_ensemble):
    e = small_ensemble
    ctx, out = run_batched(e)
    acc, jerk, pot = out.acc.cpu().numpy(), out.jerk.cpu().numpy(), out.pot.cpu().numpy()
    lists = out.neighbour_lists()
    errs = []
    for c in range(len(e.sizes)):
        lo, hi = e.cluster_off[c], e.cluster_off[c + 1]
        r0, r1 = e.active_off[c], e.active_off[c + 1]
        loc = (e.idx[r0:r1] - lo).astype(np.int32)
        ref = oracle.regular_force(e.x[lo:hi], e.v[lo:hi], e.m[lo:hi], loc, e.rs2[c], cap=256)
        errs.append(np.linalg.norm(acc[r0:r1] - ref[0], axis=1) / np.linalg.norm(ref[0], axis=1))
        ej = np.linalg.norm(jerk[r0:r1] - ref[1], axis=1) / np.linalg.norm(ref[1], axis=1)
        ep = np.abs(pot[r0:r1] - ref[2]) / np.abs(ref[2])
        assert ej.max() <= 1e-4 and ep.max() <= 1e-4, c
        rs = math.sqrt(e.rs2[c])
        for q in range(r1 - r0):
            got = set((lists[r0 + q] - lo).tolist())
            want = set(ref[4][q].tolist())
            if got != want:
                d = np.sqrt(((e.x[lo:hi][list(got ^ want)] - e.x[lo + loc[q]]) ** 2).sum(1))
                assert np.all(np.abs(d - rs) <= 1e-6 * rs), (c, q)
    errs = np.concatenate(errs)
    assert np.median(errs) <= 2e-6 and errs.max() <= 1e-4
    ctx.close()


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_every_batch_tile_gives_the_same_lists(gpu_lib, small_ensemble, variant):
    ctx0, ref = run_batched(small_ensemble, 0)
    ctx, out = run_batched(small_ensemble, variant)
    assert torch.equal(out.nb_off, ref.nb_off)
    tot = int(ref.nb_off[-1])
    assert torch.equal(out.nb_idx[:tot], ref.nb_idx[:tot])
    torch.testing.assert_close(out.acc, ref.acc, rtol=1e-6, atol=0)
    ctx.close()
    ctx0.close()


def test_graph_replay_is_bitwise_identical(gpu_lib, small_ensemble):
    ctx, out, g = run_batched(small_ensemble, graph=True)
    first = (out.acc.clone(), out.jerk.clone(), out.pot.clone(), out.nb_off.clone())
    for _ in range(3):
        out.acc.zero_()
        g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out.acc, first[0]) and torch.equal(out.jerk, first[1])
    assert torch.equal(out.pot, first[2]) and torch.equal(out.nb_off, first[3])
    ctx.close()


def test_index_outside_its_cluster_is_reported(gpu_lib, small_ensemble):
    from paper_1504_03687_gb300 import Context, api
    e = small_ensemble
    ctx = Context(e.cluster_off[-1], precision="mixed", nb_cap=256)
    ctx.set_predicted(T(e.x), T(e.v), T(e.m))
    ctx.batch_plan(e.cluster_off, e.active_off)
    idx = e.idx.copy()
    idx[0] = e.cluster_off[-1] - 1  # row 0 belongs to cluster 0 but names the last particle
    ctx.regular_force_batched(T(idx), T(e.rs2))
    with pytest.raises(api.NBError) as err:
        ctx.sync()
    assert err.value.status == api.NB_ERR_ARG
    ctx.close()
