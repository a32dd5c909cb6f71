"""Multi-rank host logic on CPU (gloo, world sizes 2 and 3): the copy-algorithm row sharding and the
result exchange reproduce the single-rank result exactly.  Each rank computes its share of
the active rows with the FP64 oracle (the GPU path is exercised on one GPU elsewhere)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import workloads as W
from paper_1504_03687_gb300.dist import allgather_rows, shard_rows


def test_shard_rows_partitions_exactly():
    for n_i in (0, 1, 5, 1000, 1 << 20):
        for world in (1, 2, 3, 8):
            parts = [shard_rows(n_i, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n_i
            assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cl, rs2 = W.plummer_1k_equal()
        idx = W.active_block(W.block_steps(cl, seed=0), 301)
        lo, hi = shard_rows(idx.size, world, rank)
        a, j, p, cnt, lists = oracle.regular_force(cl.x, cl.v, cl.m, idx[lo:hi], rs2, cap=64)
        off = np.zeros(hi - lo + 1, np.int64)
        off[1:] = np.cumsum([len(l) for l in lists])
        flat = np.concatenate(lists).astype(np.int32) if lists else np.zeros(0, np.int32)
        res = allgather_rows(torch.from_numpy(a), torch.from_numpy(j), torch.from_numpy(p),
                             torch.from_numpy(off), torch.from_numpy(flat))
        if rank == 0:
            out.put([t.numpy() for t in res])
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_copy_algorithm_exchange_matches_single_rank(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    cl, rs2 = W.plummer_1k_equal()
    idx = W.active_block(W.block_steps(cl, seed=0), 301)
    a, j, p, cnt, lists = oracle.regular_force(cl.x, cl.v, cl.m, idx, rs2, cap=64)
    np.testing.assert_array_equal(got[0], a)
    np.testing.assert_array_equal(got[1], j)
    np.testing.assert_array_equal(got[2], p)
    off = np.zeros(idx.size + 1, np.int64)
    off[1:] = np.cumsum([len(l) for l in lists])
    np.testing.assert_array_equal(got[3], off)
    np.testing.assert_array_equal(got[4], np.concatenate(lists))


# ------------------------------------------------------------------ source sharding

def test_shard_sources_partitions_on_aligned_starts():
    from paper_1504_03687_gb300.dist import shard_sources
    for n in (1, 255, 256, 1000, 4099, 1 << 20):
        for world in (1, 2, 3, 8):
            parts = [shard_sources(n, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[r][1] == parts[r + 1][0] for r in range(world - 1))
            assert all(lo % 256 == 0 for lo, _ in parts)
            assert all(abs((b - a) - n / world) < 256 for a, b in parts)


def _range_result(cl, idx, lo, hi, cap):
    """Oracle result of the rows idx summed over the sources [lo, hi) only: the restricted
    pair sums, and the full neighbour sets restricted to the range (first cap kept)."""
    a, j, p = oracle.pair_sums(cl.x, cl.v, cl.m, idx, np.arange(lo, hi, dtype=np.int32))
    _, _, _, _, lists = oracle.regular_force(cl.x, cl.v, cl.m, idx, _range_result.rs2, cap=cl.n)
    inside = [l[(l >= lo) & (l < hi)] for l in lists]
    cnt = np.array([len(l) for l in inside], np.int32)
    kept = [l[:cap] for l in inside]
    off = np.zeros(len(idx) + 1, np.int64)
    off[1:] = np.cumsum([len(l) for l in kept])
    flat = np.concatenate(kept).astype(np.int32) if kept else np.zeros(0, np.int32)
    return [torch.from_numpy(q) for q in (a, j, p, off, flat, cnt)]


def _check_against_full(got, cl, idx, rs2, cap):
    a, j, p, cnt, lists = oracle.regular_force(cl.x, cl.v, cl.m, idx, rs2, cap=cap)
    for g, r in ((got[0], a), (got[1], j), (got[2], p)):
        np.testing.assert_allclose(g.numpy(), r, rtol=1e-12, atol=1e-13 * np.abs(r).max())
    off = np.zeros(idx.size + 1, np.int64)
    off[1:] = np.cumsum([len(l) for l in lists])
    np.testing.assert_array_equal(got[3].numpy(), off)
    np.testing.assert_array_equal(got[4].numpy()[:off[-1]], np.concatenate(lists))
    np.testing.assert_array_equal(got[5].numpy(), cnt)


def combine_shards(parts, cap):
    """Single-process stand-in for the exchange: the shards' sums and counts added in shard
    order (what the all-reduce computes), their lists merged by the library's merge."""
    from paper_1504_03687_gb300.dist import merge_source_lists
    acc, jerk, pot, count = (sum(p[q] for p in parts) for q in (0, 1, 2, 5))
    off, idx = merge_source_lists([p[3] for p in parts], [p[4] for p in parts], cap)
    return acc, jerk, pot, off, idx, count


def test_merged_source_shards_match_full_set():
    """Three unequal source ranges, cap 16 (most lists are cut, some inside the first
    range, some across ranges): sums up to reassociation, lists and counts exact."""
    from paper_1504_03687_gb300.dist import shard_sources
    cl, rs2 = W.plummer_1k_equal()
    _range_result.rs2 = rs2
    idx = W.active_block(W.block_steps(cl, seed=0), 301)
    cap = 16
    parts = [_range_result(cl, idx, *shard_sources(cl.n, 3, r), cap) for r in range(3)]
    _check_against_full(combine_shards(parts, cap), cl, idx, rs2, cap)


def _source_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1504_03687_gb300.dist import reduce_sources, shard_sources
        cl, rs2 = W.plummer_1k_equal()
        _range_result.rs2 = rs2
        idx = W.active_block(W.block_steps(cl, seed=0), 301)
        lo, hi = shard_sources(cl.n, world, rank)
        part = _range_result(cl, idx, lo, hi, 24)
        res = reduce_sources(*part, nb_cap=24)
        if rank == 0:
            out.put([t.numpy() for t in res])
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])  # 3 ranks: source shards of 256, 256 and 512 particles
def test_source_sharded_exchange_matches_single_rank(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_source_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    cl, rs2 = W.plummer_1k_equal()
    idx = W.active_block(W.block_steps(cl, seed=0), 301)
    _check_against_full([torch.from_numpy(g) for g in got], cl, idx, rs2, 24)


# ------------------------------------------------------------------ failure detection
def _leave(out):
    out.close()
    out.join_thread()  # flush this process's messages before the hard exit
    os._exit(0)


def _dropout_worker(rank, world, port, out):
    from datetime import timedelta
    from paper_1504_03687_gb300.dist import Heartbeat, PeerLost
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0, timeout=timedelta(seconds=30))
    dist.init_process_group("gloo", store=store, rank=rank, world_size=world, timeout=timedelta(seconds=20))
    hb = Heartbeat(store, rank, world, timeout_s=3.0)
    t = torch.full((4,), float(rank))
    for step in range(3):
        if rank == 1 and step == 1:
            out.put(("left", rank, step))
            _leave(out)  # leaves between steps: no collective is in flight, no heartbeat posted
        hb.beat(step)
        try:
            hb.wait(step)
        except PeerLost as e:
            out.put(("lost", rank, step, str(e)))
            _leave(out)
        bufs = [torch.zeros(4) for _ in range(world)]
        dist.all_gather(bufs, t)
        out.put(("step", rank, step, [float(b[0]) for b in bufs]))
    out.put(("done", rank))
    _leave(out)


def test_rank_leaving_between_steps_is_detected_by_heartbeat():
    """Rank 1 leaves between steps 0 and 1 without posting its step-1 heartbeat; rank 0 must
    report the loss at its step-1 check (a bounded store wait) and never enter the step-1
    collective."""
    import time
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dropout_worker, args=(r, 2, port, q)) for r in range(2)]
    t0 = time.time()
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(timeout=90)
        assert pr.exitcode == 0
    msgs = []
    while True:
        try:
            msgs.append(q.get(timeout=2))
        except Exception:
            break
    assert time.time() - t0 < 80
    assert ("step", 0, 0, [0.0, 1.0]) in msgs and ("step", 1, 0, [0.0, 1.0]) in msgs
    assert ("left", 1, 1) in msgs
    lost = [m for m in msgs if m[0] == "lost"]
    assert len(lost) == 1 and lost[0][1] == 0 and lost[0][2] == 1
    assert not any(m[0] == "step" and m[2] >= 1 for m in msgs)

def _bench_worker(rank, world, port, out):
    """The benchmark's copy-algorithm step on gloo ranks, the oracle standing in for the
    device call: every rank computes its share of the rows of three blocks and the results
    are all-gathered."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        blocks, force = _bench_problem()
        res = bench.copy_algorithm_step(blocks, [force] * len(blocks), world, rank)
        if rank == 0:
            out.put([[t.numpy() for t in r] for r in res])
    finally:
        dist.destroy_process_group()


def _bench_problem():
    cl, rs2 = W.plummer_1k_equal()
    order = W.sorted_step_list(W.block_steps(cl, seed=0)).astype(np.int32)
    blocks = [order[:b] for b in (1, 37, 300)]

    def force(rows):
        a, j, p, cnt, lists = oracle.regular_force(cl.x, cl.v, cl.m, np.asarray(rows), rs2, cap=64)
        off = np.zeros(len(rows) + 1, np.int64)
        off[1:] = np.cumsum([len(l) for l in lists])
        flat = np.concatenate(lists).astype(np.int32) if len(lists) else np.zeros(0, np.int32)
        return tuple(torch.from_numpy(np.ascontiguousarray(t)) for t in (a, j, p, off, flat))
    return blocks, force


@pytest.mark.parametrize("world", [2, 3])
def test_bench_copy_algorithm_step_matches_one_rank(world):
    """bench.py's timed step under torchrun (row-sharded copy algorithm, all-gather of the row
    results) gives every block exactly as one rank computing all rows does."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    blocks, force = _bench_problem()
    one = bench.copy_algorithm_step(blocks, [force] * len(blocks), 1, 0)
    assert len(got) == len(one) == 3
    for g, o in zip(got, one):
        for a, b in zip(g, o):
            np.testing.assert_array_equal(a, b.numpy())
