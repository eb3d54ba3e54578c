"""Differentiable fixed-step 6th-order Hermite trajectories on the GPU.

`HermiteStep` is one shared step of the scheme of section 3 (predictor,
evaluation of acceleration, jerk and snap, corrector with the quintic
interpolation's crackle; every particle active, as in the paper's shared
time step) as a torch.autograd.Function: its forward runs the library's
predictor, FP64 all-pairs evaluation and corrector kernels, and its backward
the library's hand-written adjoints of the three (nb_traj_correct_adjoint,
nb_pairs_fp64_adjoint, nb_traj_predict_adjoint) through the C-ABI; torch
only allocates the tensors.  `PairSums` is the evaluation alone (used for
the start-up).  `torch.utils.checkpoint` keeps only every
`checkpoint`-th state, recomputing each segment in the backward pass.
"""
from __future__ import annotations

import ctypes as C

import torch
from torch.utils.checkpoint import checkpoint

from . import NB_OK, NBError, lib

_work_cache: dict = {}


def _workspace(n: int, device) -> torch.Tensor:
    key = (n, device)
    w = _work_cache.get(key)
    if w is None:
        nbytes = int(lib().nb_pairs_workspace_bytes(n))
        w = torch.empty(nbytes, dtype=torch.uint8, device=device)
        _work_cache[key] = w
    return w


def _ptr(t: torch.Tensor):
    return C.c_void_p(t.data_ptr())


def _check(st):
    if st != NB_OK:
        raise NBError(st, lib().nb_last_error(None).decode())


class PairSums(torch.autograd.Function):
    """(acc, jerk, snap) = pair sums over all particles; FP64, CUDA tensors:
    m [n], x, v, a [n, 3]."""

    @staticmethod
    def forward(ctx, m, x, v, a, eps):
        m, x, v, a = (t.contiguous() for t in (m, x, v, a))
        n = m.numel()
        acc = torch.empty_like(x)
        jerk = torch.empty_like(x)
        snap = torch.empty_like(x)
        stream = torch.cuda.current_stream(x.device).cuda_stream
        _check(lib().nb_pairs_fp64(n, _ptr(m), _ptr(x), _ptr(v), _ptr(a), float(eps), _ptr(acc),
                                   _ptr(jerk), _ptr(snap), _ptr(_workspace(n, x.device)),
                                   C.c_void_p(stream)))
        ctx.save_for_backward(m, x, v, a)
        ctx.eps = eps
        return acc, jerk, snap

    @staticmethod
    def backward(ctx, g_acc, g_jerk, g_snap):
        m, x, v, a = ctx.saved_tensors
        n = m.numel()
        zero = torch.zeros_like(x)
        g_acc = zero if g_acc is None else g_acc.contiguous()
        g_jerk = zero if g_jerk is None else g_jerk.contiguous()
        g_snap = zero if g_snap is None else g_snap.contiguous()
        gx, gv, ga = (torch.empty_like(x) for _ in range(3))
        gm = torch.empty_like(m)
        stream = torch.cuda.current_stream(x.device).cuda_stream
        _check(lib().nb_pairs_fp64_adjoint(n, _ptr(m), _ptr(x), _ptr(v), _ptr(a), float(ctx.eps),
                                           _ptr(g_acc), _ptr(g_jerk), _ptr(g_snap), _ptr(gx),
                                           _ptr(gv), _ptr(ga), _ptr(gm), C.c_void_p(stream)))
        return gm, gx, gv, ga, None


class HermiteStep(torch.autograd.Function):
    """One shared step of length h: (x, v, a, j, s, c) -> (x1, v1, A, J, S, c1)
    with m [n] and the state [n, 3], FP64 CUDA tensors."""

    @staticmethod
    def forward(ctx, m, x, v, a, j, s, c, eps, h):
        ctx.set_materialize_grads(False)
        m, x, v, a, j, s, c = (t.contiguous() for t in (m, x, v, a, j, s, c))
        n = m.numel()
        stream = C.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
        xp, vp, ap = (torch.empty_like(x) for _ in range(3))
        _check(lib().nb_traj_predict(n, float(h), *[_ptr(t) for t in (x, v, a, j, s, c, xp, vp, ap)],
                                     stream))
        A, J, S = (torch.empty_like(x) for _ in range(3))
        _check(lib().nb_pairs_fp64(n, _ptr(m), _ptr(xp), _ptr(vp), _ptr(ap), float(eps), _ptr(A),
                                   _ptr(J), _ptr(S), _ptr(_workspace(n, x.device)), stream))
        x1, v1, c1 = (torch.empty_like(x) for _ in range(3))
        _check(lib().nb_traj_correct(n, float(h), *[_ptr(t) for t in (x, v, a, j, s, A, J, S, x1, v1,
                                                                        c1)], stream))
        ctx.save_for_backward(m, xp, vp, ap)
        ctx.eps, ctx.h = eps, h
        return x1, v1, A, J, S, c1

    @staticmethod
    def backward(ctx, gx1, gv1, gA, gJ, gS, gc1):
        m, xp, vp, ap = ctx.saved_tensors
        n = m.numel()
        h = float(ctx.h)
        stream = C.c_void_p(torch.cuda.current_stream(xp.device).cuda_stream)
        opt = lambda t: None if t is None else _ptr(t.contiguous())  # noqa: E731  (None = zero)
        keep = [t.contiguous() for t in (gx1, gv1, gc1, gA, gJ, gS) if t is not None]  # noqa: F841
        gx, gv, ga, gj, gs, gAt, gJt, gSt = (torch.empty_like(xp) for _ in range(8))
        _check(lib().nb_traj_correct_adjoint(n, h, opt(gx1), opt(gv1), opt(gc1), opt(gA), opt(gJ),
                                             opt(gS), *[_ptr(t) for t in (gx, gv, ga, gj, gs, gAt, gJt,
                                                                          gSt)], stream))
        gxp, gvp, gap = (torch.empty_like(xp) for _ in range(3))
        gm = torch.empty_like(m)
        _check(lib().nb_pairs_fp64_adjoint(n, _ptr(m), _ptr(xp), _ptr(vp), _ptr(ap), float(ctx.eps),
                                           _ptr(gAt), _ptr(gJt), _ptr(gSt), _ptr(gxp), _ptr(gvp),
                                           _ptr(gap), _ptr(gm), stream))
        gc = torch.empty_like(xp)
        _check(lib().nb_traj_predict_adjoint(n, h, _ptr(gxp), _ptr(gvp), _ptr(gap), _ptr(gx), _ptr(gv),
                                             _ptr(ga), _ptr(gj), _ptr(gs), _ptr(gc), stream))
        return gm, gx, gv, ga, gj, gs, gc, None, None


def start_state(m, x, v, eps):
    """a and jerk from a pass with zero accelerations, snap from a pass with
    those accelerations, crackle zero (the scheme's start-up)."""
    zero = torch.zeros_like(x)
    a, j, _ = PairSums.apply(m, x, v, zero, eps)
    _, _, s = PairSums.apply(m, x, v, a, eps)
    return x, v, a, j, s, torch.zeros_like(x)


def hermite_step(m, eps, h, x, v, a, j, s, c):
    """One shared step of length h: predict all, evaluate all, correct."""
    return HermiteStep.apply(m, x, v, a, j, s, c, eps, h)


def trajectory(m, x0, v0, eps, h, steps, checkpoint_every=8):
    """Final (x, v) after `steps` shared steps of length h from (x0, v0),
    differentiable in m, x0, v0.  Every `checkpoint_every` steps only the
    state is stored and the segment is recomputed in the backward pass
    (checkpoint_every <= 0: no checkpointing)."""
    state = start_state(m, x0, v0, eps)

    def segment(k, *st):
        for _ in range(k):
            st = hermite_step(m, eps, h, *st)
        return st

    if checkpoint_every <= 0 or not torch.is_grad_enabled():
        state = segment(steps, *state)
        return state[0], state[1]
    done = 0
    while done < steps:
        k = min(checkpoint_every, steps - done)
        state = checkpoint(segment, k, *state, use_reentrant=False)
        done += k
    return state[0], state[1]


def loss_and_grads(m, x0, v0, eps, h, steps, checkpoint_every=8):
    """loss = sum_i m_i |x_i(T)|^2 and its gradients with respect to x0, v0, m."""
    m = m.detach().clone().requires_grad_(True)
    x0 = x0.detach().clone().requires_grad_(True)
    v0 = v0.detach().clone().requires_grad_(True)
    xT, _ = trajectory(m, x0, v0, eps, h, steps, checkpoint_every)
    loss = (m * (xT * xT).sum(dim=1)).sum()
    gx, gv, gm = torch.autograd.grad(loss, (x0, v0, m))
    return loss.detach(), gx, gv, gm
