"""Multi-rank host logic on CPU (gloo, world size 2): the copy-algorithm row sharding and the
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


def test_copy_algorithm_exchange_matches_single_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
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
