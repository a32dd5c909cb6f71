"""Splitting the regular-force step across ranks, in the two ways the paper uses.

Row sharding (the copy algorithm of Sec. 3.1): every rank holds all N particles and
computes the regular force of a contiguous, balanced share of the active rows; the per-row
results are then exchanged so that every rank has the whole block (the O(N_i) "Comm.R."
exchange of Table 1 / Table 2).  The CSR neighbour lists are exchanged as counts plus
concatenated indices and re-offset.

Source sharding (the GPUs of one node, Sec. 3.4): every rank sums over its own contiguous
share of the source particles (nb_set_source_range) for all active rows; the partial sums
are added in rank order, the neighbour lists concatenated in rank order (which keeps them
in ascending j) and cut at nb_cap, and the true counts added.

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


def combine_source_shards(parts, nb_cap: int):
    """Merge per-source-range results into the full-set result.

    parts: [(acc, jerk, pot, nb_off, nb_idx, nb_count), ...] in ascending range order, all
    torch tensors on one device, for the same active rows; nb_off / nb_idx / nb_count may be
    None throughout.  Each part's lists must be complete up to nb_cap (no CSR overflow).
    Returns (acc, jerk, pot, nb_off, nb_idx, nb_count): sums added in part order, lists
    concatenated in part order and cut at nb_cap, counts added."""
    acc, jerk, pot = (p.clone() for p in parts[0][:3])
    for p in parts[1:]:
        acc += p[0]
        jerk += p[1]
        pot += p[2]
    if parts[0][3] is None:
        return acc, jerk, pot, None, None, None
    dev = acc.device
    n_i = acc.shape[0]
    kept = [(p[3][1:] - p[3][:-1]).to(torch.int64) for p in parts]
    total = torch.stack(kept).sum(0) if kept else torch.zeros(n_i, dtype=torch.int64, device=dev)
    merged = torch.clamp(total, max=nb_cap)
    off = torch.zeros(n_i + 1, dtype=torch.int64, device=dev)
    off[1:] = torch.cumsum(merged, 0)
    out = torch.empty(max(int(off[-1].item()), 1), dtype=torch.int32, device=dev)
    before = torch.zeros(n_i, dtype=torch.int64, device=dev)  # entries of earlier parts per row
    rows_all = torch.arange(n_i, device=dev)
    for p, k in zip(parts, kept):
        used = int(p[3][-1].item())
        if used:
            row = torch.repeat_interleave(rows_all, k)
            local = torch.arange(used, device=dev) - p[3][:-1][row]
            dest = before[row] + local
            keep = dest < nb_cap
            out[(off[:-1][row] + dest)[keep]] = p[4][:used][keep]
        before += k
    count = parts[0][5].clone()
    for p in parts[1:]:
        count += p[5]
    return acc, jerk, pot, off, out, count


def reduce_sources(acc, jerk, pot, nb_off=None, nb_idx=None, nb_count=None, nb_cap: int = 512, group=None):
    """Source-sharded exchange: gather every rank's partial result for the same active rows
    and merge them in rank order (combine_source_shards) on every rank, so that the sums
    are added in a fixed order whatever the backend."""
    import torch.distributed as dist
    world = dist.get_world_size(group)

    def gather_same(t):
        bufs = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(bufs, t.contiguous(), group=group)
        return bufs

    accs, jerks, pots = gather_same(acc), gather_same(jerk), gather_same(pot)
    if nb_off is None:
        parts = [(a, j, p, None, None, None) for a, j, p in zip(accs, jerks, pots)]
        return combine_source_shards(parts, nb_cap)
    offs, counts = gather_same(nb_off), gather_same(nb_count)
    used = int(nb_off[-1].item())
    lens = gather_same(torch.tensor([used], dtype=torch.int64, device=acc.device))
    lmax = max(int(q.item()) for q in lens)
    padded = torch.zeros(max(lmax, 1), dtype=nb_idx.dtype, device=nb_idx.device)
    padded[:used] = nb_idx[:used]
    idxs = gather_same(padded)
    parts = list(zip(accs, jerks, pots, offs, idxs, counts))
    return combine_source_shards(parts, nb_cap)


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
