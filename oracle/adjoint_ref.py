"""FP64 CPU reference for gradients of fixed-step Hermite-6 trajectories.

TEST INFRASTRUCTURE ONLY (same rules as the rest of oracle/).  A plain
restatement in torch CPU double precision: the pair terms in the physics
form of the evaluation step (paper section 3 item 4; self terms masked
out), the Taylor predictor, the two-point Hermite corrector and the quintic
interpolation with a shared step h (section 3), written as vectorised
tensor expressions with no blocking, and differentiated by torch autograd
(reverse mode) without checkpointing.
"""
from __future__ import annotations

import torch


def pair_sums(m, x, v, a, eps):
    """acc, jerk, snap [n, 3]: A = m_j r / R^(3/2), J = m_j v / R^(3/2) - 3 alpha A,
    S = m_j a / R^(3/2) - 6 alpha J - 3 beta A summed over j != i."""
    n = m.shape[0]
    r = x[None, :, :] - x[:, None, :]
    vv = v[None, :, :] - v[:, None, :]
    aa = a[None, :, :] - a[:, None, :]
    R = (r * r).sum(-1) + eps * eps
    off = 1.0 - torch.eye(n, dtype=x.dtype)
    mr3 = off * m[None, :] / (R * torch.sqrt(R))
    alpha = (r * vv).sum(-1) / R
    beta = ((vv * vv).sum(-1) + (r * aa).sum(-1)) / R + alpha * alpha
    A = mr3[..., None] * r
    J = mr3[..., None] * vv - 3.0 * alpha[..., None] * A
    S = mr3[..., None] * aa - 6.0 * alpha[..., None] * J - 3.0 * beta[..., None] * A
    return A.sum(1), J.sum(1), S.sum(1)


def trajectory(m, x0, v0, eps, h, steps):
    zero = torch.zeros_like(x0)
    a, j, _ = pair_sums(m, x0, v0, zero, eps)
    _, _, s = pair_sums(m, x0, v0, a, eps)
    x, v, c = x0, v0, torch.zeros_like(x0)
    for _ in range(steps):
        xp = x + v * h + a * h ** 2 / 2 + j * h ** 3 / 6 + s * h ** 4 / 24 + c * h ** 5 / 120
        vp = v + a * h + j * h ** 2 / 2 + s * h ** 3 / 6 + c * h ** 4 / 24
        ap = a + j * h + s * h ** 2 / 2 + c * h ** 3 / 6
        A, J, S = pair_sums(m, xp, vp, ap, eps)
        v1 = v + h / 2 * (a + A) - h ** 2 / 10 * (J - j) + h ** 3 / 120 * (s + S)
        x1 = x + h / 2 * (v + v1) - h ** 2 / 10 * (A - a) + h ** 3 / 120 * (j + J)
        # quintic through (a, j, s) at both ends: crackle at the end of the step
        R1 = A - a - j * h - s * h ** 2 / 2
        R2 = h * (J - j - s * h)
        R3 = h ** 2 * (S - s)
        c = (60 * R1 - 36 * R2 + 9 * R3) / h ** 3
        x, v, a, j, s = x1, v1, A, J, S
    return x, v


def loss(m, x0, v0, eps, h, steps):
    xT, _ = trajectory(m, x0, v0, eps, h, steps)
    return (m * (xT * xT).sum(1)).sum()


def loss_and_grads(m, x0, v0, eps, h, steps):
    """(loss, d/dx0, d/dv0, d/dm) as numpy arrays."""
    m = torch.as_tensor(m, dtype=torch.float64).clone().requires_grad_(True)
    x0 = torch.as_tensor(x0, dtype=torch.float64).clone().requires_grad_(True)
    v0 = torch.as_tensor(v0, dtype=torch.float64).clone().requires_grad_(True)
    L = loss(m, x0, v0, eps, h, steps)
    gx, gv, gm = torch.autograd.grad(L, (x0, v0, m))
    return float(L.detach()), gx.numpy(), gv.numpy(), gm.numpy()
