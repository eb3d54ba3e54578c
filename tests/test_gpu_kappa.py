"""Condition numbers of the evaluation's sums (nb_evaluate_kappa, section 3
item 4: a, jerk and snap are sums of pair terms) against the oracle's, and
the mixed path's error over a whole population in units of them (the
kappa-normalised reading of its 1e-6 bound)."""
import numpy as np
import pytest

import nb_inputs as ni
import oracle as O
from nbhelp import nb_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_kappa_matches_the_oracle(prec):
    """sum_j |A_ij|, |J_ij|, |S_ij| for 333 listed particles of a Plummer
    model with Salpeter masses and a seeded acceleration field, from the
    FP64, mixed and EX contexts' own j-buffers, within 1e-5 of the oracle's;
    the whole population's values agree bit for bit on the listed ones."""
    nb = nb_gpu()
    n, eps = 1000, 1e-4
    m, x, v = ni.plummer(n, 41, imf="salpeter")
    a = ni.random_state(n, 42, scale=2.0)
    g = nb.NBody(m, x, v, eps, precision=prec, start_forces=False)
    g.set_state({"a": a})
    g.predict(0.0)
    act = ni.active_subset(n, 333, 43)
    got = g.evaluate_kappa(act)
    every = g.evaluate_kappa(None)
    g.close()
    ref = O.evaluate_kappa(m, x, v, a, eps, act)
    for gq, eq, rq in zip(got, every, ref):
        np.testing.assert_allclose(gq, rq, rtol=1e-5, atol=0)
        np.testing.assert_array_equal(eq[act], gq)


def test_kappa_arguments():
    nb = nb_gpu()
    m, x, v = ni.plummer(64, 44)
    g = nb.NBody(m, x, v, 1e-3, precision=nb.NB_MIXED, start_forces=False)
    with pytest.raises(nb.NBError) as e:
        g.evaluate_kappa(None)
    assert e.value.status == nb.NB_ESTATE
    g.predict(0.0)
    for bad in (np.array([0, 64], dtype=np.int32), np.array([-1], dtype=np.int32)):
        with pytest.raises(nb.NBError) as e:
            g.evaluate_kappa(bad)
        assert e.value.status == nb.NB_EINVAL
    empty = g.evaluate_kappa(np.zeros(0, dtype=np.int32))
    assert all(q.size == 0 for q in empty)
    # the context's own evaluation is untouched: evaluate, kappa, evaluate again
    first = g.evaluate(None)
    g.evaluate_kappa(np.arange(10, dtype=np.int32))
    again = g.evaluate(None)
    for f, s in zip(first, again):
        np.testing.assert_array_equal(f, s)
    g.close()


def test_mixed_error_over_a_whole_population_in_units_of_kappa():
    """Plummer N = 65536 with Salpeter masses, eps = 1e-4, a seeded
    acceleration field, every particle active in the automatic launch
    shape: the mixed sums against the FP64 GPU path (error about 1e-15), in
    units of their condition numbers.  Acceleration and jerk within 1e-6 for
    every particle; snap within 1e-6 for all but a ten-thousandth and within
    1.25e-6 for all (its pair terms' own FP32 rounding: at N = 2^20, 9 of
    1,048,576 snaps lie between 1e-6 and 1.11e-6).  The EX arithmetic, against
    the FP64 path on the same double-word-rounded inputs, within 1e-12 of them
    for every particle."""
    nb = nb_gpu()
    n, eps = 65536, 1e-4
    m, x, v = ni.plummer(n, 45, imf="salpeter")
    a = ni.random_state(n, 46, scale=2.0)
    out = {}
    for prec in (nb.NB_FP64, nb.NB_MIXED, nb.NB_EX, "fp64_dw"):
        if prec == "fp64_dw":
            # the FP64 path on the inputs rounded to double words, as EX holds them
            def dw(q):
                h = q.astype(np.float32).astype(np.float64)
                return h + (q - h).astype(np.float32).astype(np.float64)
            g = nb.NBody(dw(m), dw(x), dw(v), eps, precision=nb.NB_FP64, start_forces=False)
            g.set_state({"a": dw(a)})
        else:
            g = nb.NBody(m, x, v, eps, precision=prec, start_forces=False)
            g.set_state({"a": a})
        g.predict(0.0)
        out[prec] = g.evaluate(None)
        if prec == nb.NB_MIXED:
            kap = g.evaluate_kappa(None)
        g.close()
    ratios = []
    for q in range(3):
        d = np.abs(out[nb.NB_MIXED][q] - out[nb.NB_FP64][q]).max(axis=1)
        ratios.append(d / kap[q])
    assert ratios[0].max() <= 1e-6 and ratios[1].max() <= 1e-6, (ratios[0].max(), ratios[1].max())
    assert (ratios[2] > 1e-6).mean() <= 1e-4 and ratios[2].max() <= 1.25e-6, ratios[2].max()
    # EX arithmetic (double-word FP32) against FP64 on the same double-word
    # inputs: within 1e-12 of each condition number for every particle (at
    # N = 2^20 at most 8.1e-13)
    for q in range(3):
        r = np.abs(out[nb.NB_EX][q] - out["fp64_dw"][q]).max(axis=1) / kap[q]
        assert r.max() <= 1e-12, (q, r.max())
