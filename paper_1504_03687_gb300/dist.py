"""Row sharding of the regular-force step across ranks (the copy algorithm of Sec. 3.1).

Every rank holds all N particles and computes the regular force of a contiguous, balanced
share of the active rows; the per-row results are then exchanged so that every rank has
the whole block (the O(N_i) "Comm.R." exchange of Table 1 / Table 2).  The CSR neighbour
lists are exchanged as counts plus concatenated indices and re-offset.  Any
torch.distributed backend works (NCCL between GPUs, gloo on the host).
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
