"""Pins for the FP64 CPU reference of trajectory gradients: its pair sums
equal the C oracle's evaluation, its forward trajectory equals the C
oracle's shared-step integration, and its autograd gradient equals central
finite differences of its own forward."""
import numpy as np
import pytest

import nb_inputs as ni
import oracle as O

torch = pytest.importorskip("torch")
from oracle import adjoint_ref as R  # noqa: E402


def test_reference_pair_sums_equal_the_oracle():
    m, x, v = ni.plummer(40, 21, imf="salpeter")
    a = ni.random_state(40, 22)
    got = R.pair_sums(*(torch.tensor(q) for q in (m, x, v, a)), 1e-3)
    ref = O.evaluate(m, x, v, a, 1e-3)
    for g, r in zip(got, ref):
        np.testing.assert_allclose(g.numpy(), r, rtol=1e-12, atol=1e-12 * np.abs(r).max())


def test_reference_trajectory_equals_oracle_shared_steps():
    m, x, v = ni.plummer(32, 23)
    h, steps, eps = 2.0 ** -10, 16, 1e-3
    xT, vT = R.trajectory(torch.tensor(m), torch.tensor(x), torch.tensor(v), eps, h, steps)
    s = O.System(m, x, v, eps, dt_shared=h, dt_max=h)
    s.run_until(h * steps)
    st = s.state()
    np.testing.assert_allclose(xT.numpy(), st["x"], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(vT.numpy(), st["v"], rtol=1e-11, atol=1e-12)


def test_reference_gradient_matches_central_differences():
    n, h, steps, eps, fd = 8, 2.0 ** -8, 16, 1e-3, 1e-6
    m, x, v = ni.plummer(n, 24)
    L0, gx, gv, gm = R.loss_and_grads(m, x, v, eps, h, steps)

    def L(mm, xx, vv):
        return float(R.loss(torch.tensor(mm), torch.tensor(xx), torch.tensor(vv), eps, h, steps))

    for (arr, grad, which) in ((x, gx, 0), (v, gv, 1), (m, gm, 2)):
        flat = arr.reshape(-1)
        for k in range(0, flat.size, max(1, flat.size // 6)):
            p, q = flat.copy(), flat.copy()
            p[k] += fd
            q[k] -= fd
            args_p = [m, x, v]
            args_q = [m, x, v]
            idx = (1, 2, 0)[which]   # x, v, m positions in (m, x, v)
            args_p[idx] = p.reshape(arr.shape)
            args_q[idx] = q.reshape(arr.shape)
            num = (L(*args_p) - L(*args_q)) / (2 * fd)
            g = grad.reshape(-1)[k]
            assert abs(num - g) <= 1e-6 * max(1.0, abs(g)), (which, k, num, g)


@pytest.mark.parametrize("arg", ["m", "x", "v", "a"])
def test_reference_pair_adjoint_matches_complex_step(arg):
    """The pair-level adjoint (autograd of the reference's pair sums, the
    gradient the adjoint kernel is held to) against complex-step
    derivatives: for a direction d of one argument and cotangents w,
    Im(w . f(z + i h d)) / h with h = 1e-30 is the exact directional
    derivative to rounding, with no subtraction and no autograd."""
    n, eps, h = 12, 1e-2, 1e-30
    m, x, v = ni.plummer(n, 31, imf="salpeter")
    a = ni.random_state(n, 32, scale=2.0)
    rng = np.random.default_rng(33)
    w = [torch.tensor(rng.standard_normal((n, 3))) for _ in range(3)]
    base = {"m": m, "x": x, "v": v, "a": a}
    d = rng.standard_normal(base[arg].shape)

    leaves = {k: torch.tensor(q, requires_grad=(k == arg)) for k, q in base.items()}
    out = R.pair_sums(leaves["m"], leaves["x"], leaves["v"], leaves["a"], eps)
    loss = sum((o * wk).sum() for o, wk in zip(out, w))
    (g,) = torch.autograd.grad(loss, leaves[arg])
    adjoint = float((g.numpy() * d).sum())

    cplx = {k: torch.tensor(q + (1j * h * d if k == arg else 0.0), dtype=torch.complex128)
            for k, q in base.items()}
    outc = R.pair_sums(cplx["m"], cplx["x"], cplx["v"], cplx["a"], eps)
    step = float(sum((o.imag * wk).sum() for o, wk in zip(outc, w))) / h
    assert adjoint == pytest.approx(step, rel=1e-11), (arg, adjoint, step)
