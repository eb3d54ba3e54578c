"""The CUDA path against worked examples derived by hand from the closed
forms (tests/golden), through the C-ABI: the pair term of two-particle
systems in every evaluation precision, and the on-device energy and angular
momentum.  Only the softened cases run here (the library requires eps > 0).

Tolerances, relative to the largest component of the expected vector:
FP64 1e-14, EX (double word, about 48 bits) 1e-12, mixed (FP32 pair
arithmetic) 1e-6."""
import numpy as np
import pytest

from nbhelp import load_golden, nb_gpu

pytestmark = pytest.mark.gpu

PAIRS = [c for c in load_golden("pair_worked_examples.txt") if c["eps"] > 0]
SYSTEMS = [c for c in load_golden("energy_worked_examples.txt") if c["eps"] > 0]
TOL = {0: 1e-14, 1: 1e-6, 3: 1e-12}


@pytest.mark.parametrize("prec", [0, 1, 3])
@pytest.mark.parametrize("case", PAIRS, ids=[c["name"] for c in PAIRS])
def test_pair_worked_example_on_the_gpu(case, prec):
    nb = nb_gpu()
    m = np.array([2.0 * case["m_j"], case["m_j"]])
    x = np.stack([case["x_i"], case["x_j"]])
    v = np.stack([case["v_i"], case["v_j"]])
    a = np.stack([case["a_i"], case["a_j"]])
    g = nb.NBody(m, x, v, case["eps"], precision=prec, start_forces=False)
    try:
        g.set_state({"x": x, "v": v, "a": a, "j": np.zeros((2, 3)), "s": np.zeros((2, 3)),
                     "c": np.zeros((2, 3)), "t": np.zeros(2), "dt": np.full(2, 2.0 ** -3)})
        g.predict(0.0)
        got = g.evaluate(np.array([0, 1], dtype=np.int32))
    finally:
        g.close()
    for out, k in zip(got, ("acc", "jerk", "snap")):
        tol = TOL[prec] * np.abs(case[k]).max()
        np.testing.assert_allclose(out[0], case[k], rtol=0, atol=tol, err_msg=k)
        np.testing.assert_allclose(out[1], -2.0 * case[k], rtol=0, atol=2 * tol, err_msg=k)


@pytest.mark.parametrize("case", SYSTEMS, ids=[c["name"] for c in SYSTEMS])
def test_energy_and_angular_momentum_worked_example_on_the_gpu(case):
    nb = nb_gpu()
    b = case["body"]
    g = nb.NBody(b[:, 0].copy(), b[:, 1:4].copy(), b[:, 4:7].copy(), case["eps"])
    try:
        ek, ep = g.energy()
        L, Ln = g.angmom()
    finally:
        g.close()
    assert ek == pytest.approx(case["ekin"], rel=1e-14)
    assert ep == pytest.approx(case["epot"], rel=1e-14)
    np.testing.assert_allclose(L, case["L"], rtol=0, atol=1e-13)
    assert Ln == pytest.approx(case["Lnorm"], rel=1e-14)
