"""The FP64 oracle against worked examples derived by hand from the closed
forms (tests/golden): one softened pair term (acceleration, jerk, snap) and
the energy and angular momentum of small systems.

Tolerance: 2e-15 of the largest component of the expected vector (about
nine ulps): the snap's three terms cancel to a fifth of their size in the
"general" cases, so the exact result carries a few ulps of rounding; a
dropped term, a wrong sign or a wrong coefficient is off by O(1)."""
import numpy as np
import pytest

import oracle as O
from nbhelp import load_golden

PAIRS = load_golden("pair_worked_examples.txt")
SYSTEMS = load_golden("energy_worked_examples.txt")


def test_fixtures_parse():
    assert len(PAIRS) == 6 and len(SYSTEMS) == 3
    for c in PAIRS:
        assert all(c[k].shape == (3,) for k in ("x_i", "v_i", "a_i", "x_j", "v_j", "a_j",
                                                 "acc", "jerk", "snap"))


@pytest.mark.parametrize("case", PAIRS, ids=[c["name"] for c in PAIRS])
def test_oracle_pair_matches_worked_example(case):
    got = O.pair(case["x_i"], case["v_i"], case["a_i"], case["x_j"], case["v_j"],
                 case["a_j"], case["m_j"], case["eps"])
    for g, k in zip(got, ("acc", "jerk", "snap")):
        np.testing.assert_allclose(g, case[k], rtol=0, atol=2e-15 * np.abs(case[k]).max(), err_msg=k)


@pytest.mark.parametrize("case", PAIRS, ids=[c["name"] for c in PAIRS])
def test_oracle_evaluation_of_the_two_body_system(case):
    """The evaluation sum of a two-particle system is the pair term on i, and
    minus the pair term (times m_i / m_j) on j."""
    m = np.array([2.0 * case["m_j"], case["m_j"]])
    x = np.stack([case["x_i"], case["x_j"]])
    v = np.stack([case["v_i"], case["v_j"]])
    a = np.stack([case["a_i"], case["a_j"]])
    got = O.evaluate(m, x, v, a, case["eps"], [0, 1])
    for g, k in zip(got, ("acc", "jerk", "snap")):
        tol = 2e-15 * np.abs(case[k]).max()
        np.testing.assert_allclose(g[0], case[k], rtol=0, atol=tol, err_msg=k)
        np.testing.assert_allclose(g[1], -2.0 * case[k], rtol=0, atol=2 * tol, err_msg=k)


@pytest.mark.parametrize("case", SYSTEMS, ids=[c["name"] for c in SYSTEMS])
def test_oracle_energy_and_angular_momentum_match_worked_example(case):
    b = case["body"]
    ek, ep = O.energy(b[:, 0], b[:, 1:4], b[:, 4:7], case["eps"])
    assert ek == pytest.approx(case["ekin"], rel=1e-15)
    assert ep == pytest.approx(case["epot"], rel=1e-15)
    L, Ln = O.angmom(b[:, 0], b[:, 1:4], b[:, 4:7])
    np.testing.assert_allclose(L, case["L"], rtol=0, atol=1e-14)
    assert Ln == pytest.approx(case["Lnorm"], rel=1e-15)
