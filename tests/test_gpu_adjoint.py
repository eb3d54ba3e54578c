"""Differentiable path on the GPU: the stateless FP64 pair sums, the
hand-written adjoint kernel, and gradients of a checkpointed fixed-step
Hermite trajectory (shared step 2^-10, 64 steps, eps = 1e-3, checkpoints
every 8 steps) against the FP64 CPU reference and central differences."""
import numpy as np
import pytest

import nb_inputs as ni
import oracle as O
from nbhelp import nb_gpu, rel_err

pytestmark = pytest.mark.gpu


def _cuda(*arrs):
    import torch
    return [torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda") for a in arrs]


def test_pair_sums_forward_matches_oracle():
    nb_gpu()
    from paper_1901_08532_gb300 import adjoint as A
    m, x, v = ni.plummer(333, 31, imf="salpeter")
    a = ni.random_state(333, 32)
    got = A.PairSums.apply(*_cuda(m, x, v, a), 1e-3)
    ref = O.evaluate(m, x, v, a, 1e-3)
    for g, r in zip(got, ref):
        assert rel_err(g.cpu().numpy(), r).max() < 1e-12


def test_adjoint_kernel_matches_reference_autograd():
    nb_gpu()
    import torch
    from oracle import adjoint_ref as R
    from paper_1901_08532_gb300 import adjoint as A
    n, eps = 200, 1e-3
    m, x, v = ni.plummer(n, 33, imf="salpeter")
    a = ni.random_state(n, 34)
    gA, gJ, gS = (ni.random_state(n, k) for k in (35, 36, 37))
    ins = _cuda(m, x, v, a)
    for t in ins:
        t.requires_grad_(True)
    outs = A.PairSums.apply(*ins, eps)
    tot = sum((o * g).sum() for o, g in zip(outs, _cuda(gA, gJ, gS)))
    got = torch.autograd.grad(tot, ins)
    cins = [torch.tensor(q, dtype=torch.float64, requires_grad=True) for q in (m, x, v, a)]
    couts = R.pair_sums(*cins, eps)
    ctot = sum((o * torch.tensor(g)).sum() for o, g in zip(couts, (gA, gJ, gS)))
    ref = torch.autograd.grad(ctot, cins)
    # both sides sum 200 terms per particle in FP64 with cancellation (the
    # acceleration gradient most); bound relative to the largest component
    for name, g, r in zip(("m", "x", "v", "a"), got, ref):
        g, r = g.detach().cpu().numpy(), r.numpy()
        assert np.abs(g - r).max() <= 1e-9 * np.abs(r).max(), name


def test_trajectory_gradient_matches_cpu_reference_at_n64():
    nb_gpu()
    from oracle import adjoint_ref as R
    from paper_1901_08532_gb300 import adjoint as A
    n, eps, h, steps = 64, 1e-3, 2.0 ** -10, 64
    m, x, v = ni.plummer(n, 35)
    L, gx, gv, gm = A.loss_and_grads(*_cuda(m, x, v), eps, h, steps, checkpoint_every=8)
    Lr, gxr, gvr, gmr = R.loss_and_grads(m, x, v, eps, h, steps)
    assert abs(float(L) - Lr) <= 1e-12 * abs(Lr)
    for g, r in ((gx, gxr), (gv, gvr), (gm, gmr)):
        g = g.cpu().numpy()
        assert np.abs(g - r).max() <= 1e-8 * np.abs(r).max()


def test_trajectory_gradient_matches_central_differences():
    nb_gpu()
    import torch
    from paper_1901_08532_gb300 import adjoint as A
    n, eps, h, steps, fd = 64, 1e-3, 2.0 ** -10, 64, 1e-6
    m, x, v = ni.plummer(n, 36)
    _, gx, gv, gm = A.loss_and_grads(*_cuda(m, x, v), eps, h, steps)

    def L(mm, xx, vv):
        with torch.no_grad():
            xT, _ = A.trajectory(*_cuda(mm, xx, vv), eps, h, steps, checkpoint_every=0)
            mt = torch.tensor(mm, device="cuda")
            return float((mt * (xT * xT).sum(1)).sum())

    rng = ni.uniform(7, 1, np.arange(24))
    for q in range(24):
        which = q % 3
        arr = (x, v, m)[which]
        k = int(rng[q] * arr.size)
        p, mi = arr.reshape(-1).copy(), arr.reshape(-1).copy()
        p[k] += fd
        mi[k] -= fd
        argp, argm = [m, x, v], [m, x, v]
        idx = (1, 2, 0)[which]
        argp[idx] = p.reshape(arr.shape)
        argm[idx] = mi.reshape(arr.shape)
        num = (L(*argp) - L(*argm)) / (2 * fd)
        g = (gx, gv, gm)[which].cpu().numpy().reshape(-1)[k]
        assert abs(num - g) <= 1e-6 * max(1.0, abs(g)), (which, k, num, g)
