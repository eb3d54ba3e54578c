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


def _state(n, seed):
    return [ni.random_state(n, seed + k, scale=1.0 + k) for k in range(6)]


def test_trajectory_stage_kernels_match_oracle():
    """Predictor and corrector kernels of the differentiable path against the
    oracle's predictor (t_i = 0 to t = h), corrector and interpolation."""
    nb = nb_gpu()
    import torch
    lib = nb.lib()
    n, h = 97, 2.0 ** -7
    x, v, a, j, s, c = _state(n, 50)
    A, J, S = _state(n, 60)[:3]
    dev = _cuda(x, v, a, j, s, c, A, J, S)
    out = [torch.empty_like(dev[0]) for _ in range(6)]
    p = lambda t: t.data_ptr()  # noqa: E731
    assert lib.nb_traj_predict(n, h, *[p(t) for t in dev[:6]], *[p(t) for t in out[:3]], None) == 0
    assert lib.nb_traj_correct(n, h, *[p(t) for t in dev[:5]], *[p(t) for t in dev[6:]],
                               *[p(t) for t in out[3:]], None) == 0
    torch.cuda.synchronize()
    xp, vp, ap = O.predict(h, np.zeros(n), x, v, a, j, s, c)
    for g, r in zip(out[:3], (xp, vp, ap)):
        assert np.abs(g.cpu().numpy() - r).max() <= 1e-15 * np.abs(r).max()
    for i in range(0, n, 7):
        x1, v1 = O.correct(h, x[i], v[i], a[i], j[i], s[i], A[i], J[i], S[i])
        c1, _, _ = O.interpolate(h, a[i], j[i], s[i], A[i], J[i], S[i])
        for g, r in zip(out[3:], (x1, v1, c1)):
            assert np.abs(g[i].cpu().numpy() - r).max() <= 1e-12 * max(1.0, np.abs(r).max())


def test_stage_adjoints_are_the_transposes():
    """The predictor and corrector are linear for a fixed step, so their
    adjoints must satisfy <g, F u> = <F^T g, u> for any cotangents g and
    inputs u (checked with seeded random vectors, to rounding)."""
    nb = nb_gpu()
    import torch
    lib = nb.lib()
    n, h = 301, 2.0 ** -6
    p = lambda t: t.data_ptr()  # noqa: E731
    u = _cuda(*_state(n, 70))                     # x, v, a, j, s, c
    g = _cuda(*_state(n, 80)[:3])                 # cotangents of xp, vp, ap
    F = [torch.empty_like(u[0]) for _ in range(3)]
    assert lib.nb_traj_predict(n, h, *[p(t) for t in u], *[p(t) for t in F], None) == 0
    adj = [torch.zeros_like(u[0]) for _ in range(6)]
    assert lib.nb_traj_predict_adjoint(n, h, *[p(t) for t in g], *[p(t) for t in adj], None) == 0
    torch.cuda.synchronize()
    lhs = sum(float((gi * Fi).sum()) for gi, Fi in zip(g, F))
    rhs = sum(float((ai * ui).sum()) for ai, ui in zip(adj, u))
    assert abs(lhs - rhs) <= 1e-13 * sum(float((ai * ui).abs().sum()) for ai, ui in zip(adj, u))

    u = _cuda(*(_state(n, 90)[:5] + _state(n, 95)[:3]))   # x, v, a, j, s, A, J, S
    g = _cuda(*(_state(n, 100)[:3] + _state(n, 105)[:3]))  # gx1, gv1, gc1, gA_in, gJ_in, gS_in
    F = [torch.empty_like(u[0]) for _ in range(3)]
    assert lib.nb_traj_correct(n, h, *[p(t) for t in u], *[p(t) for t in F], None) == 0
    adj = [torch.empty_like(u[0]) for _ in range(8)]
    assert lib.nb_traj_correct_adjoint(n, h, *[p(t) for t in g], *[p(t) for t in adj], None) == 0
    torch.cuda.synchronize()
    # outputs (x1, v1, c1) with cotangents g[0:3]; A, J, S pass through with g[3:6]
    lhs = sum(float((gi * Fi).sum()) for gi, Fi in zip(g[:3], F))
    lhs += sum(float((gi * ui).sum()) for gi, ui in zip(g[3:], u[5:]))
    rhs = sum(float((ai * ui).sum()) for ai, ui in zip(adj, u))
    scale = sum(float((ai * ui).abs().sum()) for ai, ui in zip(adj, u))
    assert abs(lhs - rhs) <= 1e-13 * scale
    # NULL cotangents count as zero
    adj0 = [torch.empty_like(u[0]) for _ in range(8)]
    assert lib.nb_traj_correct_adjoint(n, h, None, None, None, None, None, None,
                                       *[p(t) for t in adj0], None) == 0
    torch.cuda.synchronize()
    assert all(float(t.abs().max()) == 0.0 for t in adj0)


def test_trajectory_gradient_at_n8192_matches_central_differences():
    """The Plummer N = 8192, eps = 1e-3, shared step 2^-10 trajectory with
    checkpoints every 8 steps (16 steps here): 36 sampled coordinates of the
    gradient of sum m |x(T)|^2 with respect to x0, v0 and m against central
    differences with h = 1e-6 in FP64."""
    nb_gpu()
    import torch
    from paper_1901_08532_gb300 import adjoint as A
    n, eps, h, steps, fd = 8192, 1e-3, 2.0 ** -10, 16, 1e-6
    m, x, v = ni.plummer(n, 5)
    _, gx, gv, gm = A.loss_and_grads(*_cuda(m, x, v), eps, h, steps, checkpoint_every=8)
    grads = [q.cpu().numpy().reshape(-1) for q in (gx, gv, gm)]

    def L(mm, xx, vv):
        # the loss summed exactly rounded (fsum), so that the difference
        # quotient's rounding is that of the trajectory alone
        import math
        with torch.no_grad():
            xT, _ = A.trajectory(*_cuda(mm, xx, vv), eps, h, steps, checkpoint_every=0)
        xT = xT.cpu().numpy()
        return math.fsum(mm * (xT * xT).sum(1))

    L0 = L(m, x, v)
    pick = ni.uniform(11, 1, np.arange(36))
    for q in range(36):
        which = q % 3
        arr = (x, v, m)[which]
        k = int(pick[q] * arr.size)
        args = {}
        for sgn in (1, -1):
            pert = arr.reshape(-1).copy()
            pert[k] += sgn * fd
            call = [m, x, v]
            call[(1, 2, 0)[which]] = pert.reshape(arr.shape)
            args[sgn] = L(*call)
        num = (args[1] - args[-1]) / (2 * fd)
        g = grads[which][k]
        # relative 2e-6, plus the quotient's rounding floor of about 1e-16 |L| / fd
        tol = 2e-6 * abs(g) + 1e-15 * abs(L0) / fd
        assert abs(num - g) <= tol, (which, k, num, g)
