"""torch.autograd binding of the regular-force step and its hand-written adjoint.

RegularForce.apply(xp, vp, m, idx, rs2, ctx) -> (acc, jerk, pot): the forward runs
nb_set_predicted + nb_regular_force (no neighbour lists); the backward runs
nb_set_predicted on the saved state + nb_regular_force_backward, the CUDA VJP
kernels.  Gradients flow to xp, vp and m (all particles).

hermite_chain(...) composes the fourth-order Hermite predictor/corrector (plain
torch FP64 tensor ops, O(N) per step) with RegularForce over K block steps of a
frozen schedule, with torch.utils.checkpoint segments, to differentiate a final-
state observable with respect to the initial conditions.
"""
from __future__ import annotations

import torch


class RegularForce(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xp, vp, m, idx, rs2, nbctx):
        nbctx.set_predicted(xp.detach().contiguous(), vp.detach().contiguous(), m.detach().contiguous())
        res = nbctx.regular_force(idx, rs2, neighbours=False)
        ctx.save_for_backward(xp, vp, m, idx)
        ctx.nbctx = nbctx
        return res.acc, res.jerk, res.pot

    @staticmethod
    def backward(ctx, g_acc, g_jerk, g_pot):
        xp, vp, m, idx = ctx.saved_tensors
        nb = ctx.nbctx
        nb.set_predicted(xp.detach().contiguous(), vp.detach().contiguous(), m.detach().contiguous())
        zeros = lambda t, shape: torch.zeros(shape, dtype=torch.float64, device=idx.device) if t is None \
            else t.contiguous()
        n_i = idx.shape[0]
        gx, gv, gm = nb.regular_force_backward(idx, zeros(g_acc, (n_i, 3)), zeros(g_jerk, (n_i, 3)),
                                               zeros(g_pot, (n_i,)))
        return gx, gv, gm, None, None, None


def regular_force(xp, vp, m, idx, nbctx, rs2=0.0):
    """Differentiable (acc, jerk, pot) of the active block idx."""
    return RegularForce.apply(xp, vp, m, idx, rs2, nbctx)


# ------------------------------------------------------------------------------------------
def predict(x, v, a, j, dt):
    """Hermite predictor to the block time (Taylor series to the jerk term)."""
    dt = dt[:, None]
    xp = x + v * dt + a * dt * dt / 2 + j * dt * dt * dt / 6
    vp = v + a * dt + j * dt * dt / 2
    return xp, vp


def correct(xp, vp, a0, j0, a1, j1, h):
    """Fourth-order Hermite corrector for a step of length h (per row)."""
    h = h[:, None]
    da = a0 - a1
    a2 = (-6 * da - h * (4 * j0 + 2 * j1)) / (h * h)
    a3 = (12 * da + 6 * h * (j0 + j1)) / (h * h * h)
    x1 = xp + h ** 4 / 24 * a2 + h ** 5 / 120 * a3
    v1 = vp + h ** 3 / 6 * a2 + h ** 4 / 24 * a3
    return x1, v1


def block_step(state, m, active, t_next, nbctx):
    """One block step of a frozen schedule: predict all, force on the active set, correct it.

    state = (x, v, a, j, t_last); t_last (FP64, not differentiated) gives each active
    particle's step h = t_next - t_last.
    """
    x, v, a, j, t_last = state
    xp, vp = predict(x, v, a, j, t_next - t_last)
    a1, j1, _ = regular_force(xp, vp, m, active, nbctx)
    act = active.long()
    h = t_next - t_last[act]
    x1, v1 = correct(xp[act], vp[act], a[act], j[act], a1, j1, h)
    x = x.index_copy(0, act, x1)
    v = v.index_copy(0, act, v1)
    a = a.index_copy(0, act, a1)
    j = j.index_copy(0, act, j1)
    t_last = t_last.index_fill(0, act, t_next)
    return x, v, a, j, t_last


def hermite_chain(x0, v0, m, schedule, nbctx, checkpoint_every: int = 8):
    """Differentiable block-step Hermite integration along a frozen schedule.

    schedule: list of (t_next, active_idx int32 device tensor), as recorded by a forward
    run with step control; the step selection itself is not differentiated.  The start
    force and jerk of all particles are computed from (x0, v0).  Every
    `checkpoint_every` block steps form one torch.utils.checkpoint segment (activations
    recomputed in the backward pass).  Returns the final (x, v).
    """
    from torch.utils.checkpoint import checkpoint
    n = x0.shape[0]
    all_idx = torch.arange(n, dtype=torch.int32, device=x0.device)
    a0, j0, _ = regular_force(x0, v0, m, all_idx, nbctx)
    t_last = torch.zeros(n, dtype=torch.float64, device=x0.device)
    state = (x0, v0, a0, j0, t_last)

    def segment(seg, *st):
        for t_next, act in seg:
            st = block_step(st, m, act, t_next, nbctx)
        return st

    for k in range(0, len(schedule), checkpoint_every):
        state = checkpoint(segment, schedule[k:k + checkpoint_every], *state, use_reentrant=False)
    return state[0], state[1]
