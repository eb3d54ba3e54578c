"""Block-step integration at full size: Plummer N = 65536, equal masses,
eps = 1e-4, seed 2, dt_max = 2^-4, to t = 1/16 (the integration workload of
the benchmark; section 2 block steps, section 3 stages).  The oracle cannot
integrate 65536 particles in a test's time, so it checks the start-up
forces of sampled particles one by one, and the run is held to properties
that hold at any size: FP64 and EX arithmetic take the same block steps
(same times and active counts at every step), end on the same state, and
conserve energy to a bound well above both runs' error."""
import numpy as np

import pytest

import nb_inputs as ni
import oracle as O
from nbhelp import check_parity, nb_gpu, rel_err

pytestmark = pytest.mark.gpu


def test_full_size_integration_fp64_and_ex_agree():
    nb = nb_gpu()
    n, eps, t_end = 65536, 1e-4, 1.0 / 16
    m, x, v = ni.plummer(n, 2)
    pick = ni.active_subset(n, 128, 22)
    zero = np.zeros((pick.size, 3))
    # start-up pass with zero accelerations: a and jerk of the sampled particles
    ref_a, ref_j, _ = O.evaluate(m, x, v, np.zeros_like(x), eps, pick)
    kap_a, kap_j, _ = O.evaluate_kappa(m, x, v, np.zeros_like(x), eps, pick)
    runs = {}
    for prec in (nb.NB_FP64, nb.NB_EX):
        g = nb.NBody(m, x, v, eps, precision=prec, dt_max=2.0 ** -4)
        st0 = g.state()
        # FP64: 1e-12 per component of |ref|; EX: 1e-12 of sum_j |T_ij|
        for f, r, kq in (("a", ref_a, kap_a), ("j", ref_j, kap_j)):
            mode = 0 if prec == nb.NB_FP64 else 1
            assert check_parity(mode, st0[f][pick], r, kq, tol_mixed=1e-12) <= 1.0, (prec, f)
        assert np.all(st0["c"][pick] == zero) and np.all(st0["t"] == 0.0)
        E0 = sum(g.energy())
        steps, (lt, ln) = g.run_until(t_end, log_cap=1 << 16)
        E1 = sum(g.energy())
        runs[prec] = (steps, lt, ln, g.state(), abs((E1 - E0) / E0))
        g.close()
    (s64, t64, n64, st64, de64), (sex, tex, nex, stex, deex) = runs[nb.NB_FP64], runs[nb.NB_EX]
    assert s64 == sex and 1000 < s64 < (1 << 16)
    np.testing.assert_array_equal(t64, tex)
    np.testing.assert_array_equal(n64, nex)
    assert n64.min() >= 1 and n64[-1] == n and np.all(np.diff(t64) > 0) and t64[-1] == t_end
    assert np.all(st64["t"] == t_end) and np.all(stex["t"] == t_end)
    np.testing.assert_array_equal(st64["dt"], stex["dt"])
    for f in ("x", "v"):
        assert rel_err(stex[f], st64[f]).max() < 1e-9, f
    assert de64 < 1e-9 and deex < 1e-9, (de64, deex)
