"""Differentiable fixed-step 6th-order Hermite trajectories on the GPU.

`PairSums` is a torch.autograd.Function whose forward is the library's FP64
all-pairs evaluation (acceleration, jerk and snap, paper section 3 item 4)
and whose backward is the library's hand-written adjoint kernel
(nb_pairs_fp64 / nb_pairs_fp64_adjoint through the C-ABI).  The trajectory
around it (predictor, corrector, quintic interpolation with a shared
power-of-two step, the scheme of section 3 with every particle active as in
the paper's shared time step) is written with torch tensor operations on the
device, so torch's autograd carries the gradient through those linear
stages, and `torch.utils.checkpoint` keeps only every `checkpoint`-th state,
recomputing each segment in the backward pass.
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


def start_state(m, x, v, eps):
    """a and jerk from a pass with zero accelerations, snap from a pass with
    those accelerations, crackle zero (the scheme's start-up)."""
    zero = torch.zeros_like(x)
    a, j, _ = PairSums.apply(m, x, v, zero, eps)
    _, _, s = PairSums.apply(m, x, v, a, eps)
    return x, v, a, j, s, torch.zeros_like(x)


def hermite_step(m, eps, h, x, v, a, j, s, c):
    """One shared step of length h: predict all, evaluate all, correct."""
    h2, h3 = h / 2.0, h / 3.0
    xp = x + h * (v + h2 * (a + h3 * (j + (h / 4.0) * (s + (h / 5.0) * c))))
    vp = v + h * (a + h2 * (j + h3 * (s + (h / 4.0) * c)))
    ap = a + h * (j + h2 * (s + h3 * c))
    A, J, S = PairSums.apply(m, xp, vp, ap, eps)
    v1 = v + h2 * (a + A) - (h * h / 10.0) * (J - j) + (h ** 3 / 120.0) * (s + S)
    x1 = x + h2 * (v + v1) - (h * h / 10.0) * (A - a) + (h ** 3 / 120.0) * (j + J)
    R1 = A - a - h * j - (h * h / 2.0) * s
    R2 = h * (J - j - h * s)
    R3 = h * h * (S - s)
    c1 = (60.0 * R1 - 36.0 * R2 + 9.0 * R3) / h ** 3
    return x1, v1, A, J, S, c1


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
