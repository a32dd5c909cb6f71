"""Splitting the regular-force step across ranks, in the two ways the paper uses.

Row sharding (the copy algorithm of Sec. 3.1): every rank holds all N particles and
computes the regular force of a contiguous, balanced share of the active rows; the per-row
results are then exchanged so that every rank has the whole block (the O(N_i) "Comm.R."
exchange of Table 1 / Table 2).  The CSR neighbour lists are exchanged as counts plus
concatenated indices and re-offset.

Source sharding (the GPUs of one node, Sec. 3.4): every rank sums over its own contiguous
share of the source particles (nb_set_source_range) for all active rows; the partial sums
and the true counts are added by the backend's all-reduce, the neighbour lists concatenated
in rank order (which keeps them in ascending j) and cut at nb_cap.

Any torch.distributed backend works (NCCL between GPUs, gloo on the host).
"""
from __future__ import annotations

import torch


def shard_rows(n_i: int, world: int, rank: int) -> tuple[int, int]:
    """Balanced contiguous share [lo, hi) of n_i active rows for `rank` of `world`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n_i, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def allgather_rows(acc, jerk, pot, nb_off=None, nb_idx=None, group=None):
    """Gather every rank's row block (acc (k,3), jerk (k,3), pot (k)) and, optionally, its
    CSR lists (nb_off (k+1) int64, nb_idx) into the full block in rank order."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    k = torch.tensor([acc.shape[0]], dtype=torch.int64, device=acc.device)
    ks = [torch.zeros_like(k) for _ in range(world)]
    dist.all_gather(ks, k, group=group)
    ks = [int(q.item()) for q in ks]
    kmax = max(ks) if ks else 0

    def gather_padded(t):
        # all_gather needs equal shapes: pad every rank's block to the largest one
        pad = torch.zeros((kmax,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
        pad[:t.shape[0]] = t
        bufs = [torch.zeros_like(pad) for _ in range(world)]
        dist.all_gather(bufs, pad, group=group)
        return torch.cat([b[:ks[r]] for r, b in enumerate(bufs)], 0)

    acc_all = gather_padded(acc)
    jerk_all = gather_padded(jerk)
    pot_all = gather_padded(pot)
    if nb_off is None:
        return acc_all, jerk_all, pot_all, None, None
    cnt = (nb_off[1:] - nb_off[:-1]).to(torch.int64)
    cnt_all = gather_padded(cnt)
    used = int(nb_off[-1].item())
    lens = torch.tensor([used], dtype=torch.int64, device=acc.device)
    lens_all = [torch.zeros_like(lens) for _ in range(world)]
    dist.all_gather(lens_all, lens, group=group)
    lens_all = [int(q.item()) for q in lens_all]
    lmax = max(lens_all) if lens_all else 0
    padded = torch.zeros(max(lmax, 1), dtype=nb_idx.dtype, device=nb_idx.device)
    padded[:used] = nb_idx[:used]
    bufs = [torch.zeros_like(padded) for _ in range(world)]
    dist.all_gather(bufs, padded, group=group)
    idx_all = torch.cat([b[:lens_all[r]] for r, b in enumerate(bufs)], 0)
    off_all = torch.zeros(cnt_all.shape[0] + 1, dtype=torch.int64, device=acc.device)
    off_all[1:] = torch.cumsum(cnt_all, 0)
    return acc_all, jerk_all, pot_all, off_all, idx_all


SOURCE_ALIGN = 256  # nb_set_source_range wants range starts on this multiple


def shard_sources(n: int, world: int, rank: int, align: int = SOURCE_ALIGN) -> tuple[int, int]:
    """Contiguous share [lo, hi) of the n source particles for `rank` of `world`: the even
    split points r*n/world rounded down to multiples of `align` (so every share is within
    `align` of n/world and starts on a multiple of `align`), the last share ending at n.
    Empty shares (lo == hi) are possible when n < world * align."""
    if world < 1 or not 0 <= rank < world or align < 1:
        raise ValueError("bad rank/world/align")

    def cut(r):
        return n if r == world else (r * n // world) // align * align
    return cut(rank), cut(rank + 1)


def merge_source_lists(offs, idxs, nb_cap: int):
    """Neighbour lists of the source shards, merged: every row's lists concatenated in shard
    order (which keeps them in ascending j, the shards being ascending source ranges) and cut
    at nb_cap.  offs[r] (n_i + 1) int64 and idxs[r] are shard r's CSR lists, all on one
    device, each complete up to nb_cap (no CSR overflow).  Returns (nb_off, nb_idx)."""
    dev = offs[0].device
    n_i = offs[0].shape[0] - 1
    kept = [(o[1:] - o[:-1]).to(torch.int64) for o in offs]
    total = torch.stack(kept).sum(0) if kept else torch.zeros(n_i, dtype=torch.int64, device=dev)
    merged = torch.clamp(total, max=nb_cap)
    off = torch.zeros(n_i + 1, dtype=torch.int64, device=dev)
    off[1:] = torch.cumsum(merged, 0)
    out = torch.empty(max(int(off[-1].item()), 1), dtype=torch.int32, device=dev)
    before = torch.zeros(n_i, dtype=torch.int64, device=dev)  # entries of earlier shards per row
    rows_all = torch.arange(n_i, device=dev)
    for o, ix, k in zip(offs, idxs, kept):
        used = int(o[-1].item())
        if used:
            row = torch.repeat_interleave(rows_all, k)
            local = torch.arange(used, device=dev) - o[:-1][row]
            dest = before[row] + local
            keep = dest < nb_cap
            out[(off[:-1][row] + dest)[keep]] = ix[:used][keep]
        before += k
    return off, out


def reduce_sources(acc, jerk, pot, nb_off=None, nb_idx=None, nb_count=None, nb_cap: int = 512, group=None):
    """Source-sharded exchange on every rank: the partial sums and the true neighbour counts
    are reduced by the backend (an all-reduce sum: NCCL between GPUs, gloo on the host; the
    order of its additions is the backend's, fixed for a given backend and rank count), and
    the neighbour lists are gathered and merged in rank order (merge_source_lists).  Returns
    (acc, jerk, pot, nb_off, nb_idx, nb_count) of the full source set."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    acc, jerk, pot = acc.clone(), jerk.clone(), pot.clone()
    for t in (acc, jerk, pot):
        dist.all_reduce(t, group=group)
    if nb_off is None:
        return acc, jerk, pot, None, None, None
    count = nb_count.clone()
    dist.all_reduce(count, group=group)

    def gather_same(t):
        bufs = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(bufs, t.contiguous(), group=group)
        return bufs

    offs = gather_same(nb_off)
    used = int(nb_off[-1].item())
    lens = gather_same(torch.tensor([used], dtype=torch.int64, device=acc.device))
    lmax = max(int(q.item()) for q in lens)
    padded = torch.zeros(max(lmax, 1), dtype=nb_idx.dtype, device=nb_idx.device)
    padded[:used] = nb_idx[:used]
    off, idx = merge_source_lists(offs, gather_same(padded), nb_cap)
    return acc, jerk, pot, off, idx, count


class PeerLost(RuntimeError):
    """A rank did not report between two steps within the heartbeat's limit."""


class Heartbeat:
    """Host-side liveness check between steps.  Every rank posts one key per step to the
    store of its process group and, before it launches the next step's collectives, waits a
    bounded time for the keys of all other ranks; a rank that has left is then noticed
    between steps (PeerLost) rather than inside a collective, and no rank's GPU work is left
    waiting on it."""

    def __init__(self, store, rank: int, world: int, timeout_s: float = 10.0, prefix: str = "nbgpu/alive"):
        self.store, self.rank, self.world = store, rank, world
        self.timeout_s, self.prefix = timeout_s, prefix

    def beat(self, step: int) -> None:
        self.store.set(f"{self.prefix}/{step}/{self.rank}", "1")

    def wait(self, step: int) -> None:
        from datetime import timedelta
        keys = [f"{self.prefix}/{step}/{r}" for r in range(self.world) if r != self.rank]
        try:
            self.store.wait(keys, timedelta(seconds=self.timeout_s))
        except Exception as e:  # timeout, or the store's host rank has gone
            raise PeerLost(f"step {step}: a rank did not report within {self.timeout_s} s") from e
