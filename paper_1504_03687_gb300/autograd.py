"""torch.autograd binding of the regular-force step, the Hermite predictor and corrector, and
their hand-written adjoints.

RegularForce.apply(xp, vp, m, idx, rs2, ctx) -> (acc, jerk, pot): the forward runs
nb_set_predicted + nb_regular_force (no neighbour lists); the backward runs
nb_set_predicted on the saved state + nb_regular_force_backward, the CUDA VJP
kernels.  Gradients flow to xp, vp and m (all particles).

Predict / Correct: nb_hermite_predict and nb_hermite_correct forward, their VJP kernels
(nb_hermite_predict_backward, nb_hermite_correct_backward) backward.

hermite_chain(...) composes them with RegularForce over K block steps of a frozen schedule,
with torch.utils.checkpoint segments, to differentiate a final-state observable with respect
to the initial conditions.  This module only marshals tensors between library calls (row
gathers and scatters of the active set); every arithmetic step runs in the library.
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
def _or_zeros(g, like):
    return g.contiguous() if g is not None else like.new_zeros(like.shape)


class Predict(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, v, a, j, t_last, t, nbctx):
        xp, vp = nbctx.hermite_predict(t, x.detach().contiguous(), v.detach().contiguous(), a.detach().contiguous(),
                                       j.detach().contiguous(), t_last.contiguous())
        ctx.save_for_backward(t_last)
        ctx.t, ctx.nbctx = t, nbctx
        return xp, vp

    @staticmethod
    def backward(ctx, g_xp, g_vp):
        (t_last,) = ctx.saved_tensors
        like = t_last.new_zeros((t_last.shape[0], 3))
        gx, gv, ga, gj = ctx.nbctx.hermite_predict_backward(ctx.t, t_last, _or_zeros(g_xp, like), _or_zeros(g_vp, like))
        return gx, gv, ga, gj, None, None, None


class Correct(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xp, vp, a0, j0, a1, j1, t_last, t, nbctx):
        d = lambda q: q.detach().contiguous()
        x1, v1 = nbctx.hermite_correct(t, t_last.contiguous(), d(xp), d(vp), d(a0), d(j0), d(a1), d(j1))
        ctx.save_for_backward(t_last)
        ctx.t, ctx.nbctx = t, nbctx
        return x1, v1

    @staticmethod
    def backward(ctx, g_x1, g_v1):
        (t_last,) = ctx.saved_tensors
        like = t_last.new_zeros((t_last.shape[0], 3))
        grads = ctx.nbctx.hermite_correct_backward(ctx.t, t_last, _or_zeros(g_x1, like), _or_zeros(g_v1, like))
        return (*grads, None, None, None)


def block_step(state, m, active, t_next, nbctx):
    """One block step of a frozen schedule: predict all, force on the active set, correct it.

    state = (x, v, a, j, t_last); t_last (FP64, not differentiated) gives each active
    particle's step t_next - t_last.
    """
    x, v, a, j, t_last = state
    xp, vp = Predict.apply(x, v, a, j, t_last, float(t_next), nbctx)
    a1, j1, _ = regular_force(xp, vp, m, active, nbctx)
    act = active.long()
    x1, v1 = Correct.apply(xp[act], vp[act], a[act], j[act], a1, j1, t_last[act].contiguous(), float(t_next), nbctx)
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
