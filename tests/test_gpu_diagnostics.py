"""Device diagnostics stream (nb_run_diag) and the single-precision control
mode (NB_SP) against the FP64 CPU oracle.

The energy and angular momentum of section 3 item 3 are sampled on the device
at synchronisation times; Eq. 1 turns them into the relative errors that the
paper's precision study plots against time for DP, EX and SP arithmetic.
"""
import numpy as np
import pytest

import nb_inputs as ni
import oracle as O
from nbhelp import check_parity, nb_gpu, rel_err

pytestmark = pytest.mark.gpu


def test_run_diag_samples_match_oracle_energy_and_angular_momentum():
    """Plummer N=1024 FP64 block steps to t=1/8, a sample every 2^-5."""
    nb = nb_gpu()
    m, x, v = ni.plummer(1024, 4, imf="salpeter")
    eps, dt_max = 1e-4, 2.0 ** -5
    g = nb.NBody(m, x, v, eps, dt_max=dt_max)
    steps, d = g.run_diag(0.125, dt_max)
    assert d["t"].tolist() == [0.0, 1 / 32, 2 / 32, 3 / 32, 4 / 32]
    assert d["steps"][0] == 0 and d["steps"][-1] == steps
    ref = O.System(m, x, v, eps, dt_max=dt_max)
    done = 0
    for k, t in enumerate(d["t"]):
        if t > 0:
            done += ref.run_until(t)[0]
        assert d["steps"][k] == done
        st = ref.state()
        ek, ep = O.energy(m, st["x"], st["v"], eps)
        L, la = O.angmom(m, st["x"], st["v"])
        assert abs(d["ekin"][k] - ek) < 1e-11 * abs(ek)
        assert abs(d["epot"][k] - ep) < 1e-11 * abs(ep)
        assert np.abs(d["L"][k] - L).max() < 1e-11 * la
        assert abs(d["labs"][k] - la) < 1e-11 * la
    g.close()


def test_run_diag_trajectory_is_run_until_bit_for_bit():
    nb = nb_gpu()
    m, x, v = ni.plummer(700, 6)
    a = nb.NBody(m, x, v, 1e-3, dt_max=2.0 ** -4)
    b = nb.NBody(m, x, v, 1e-3, dt_max=2.0 ** -4)
    sa, _ = a.run_until(0.25)
    sb, d = b.run_diag(0.25, 2.0 ** -3)
    assert sa == sb and len(d["t"]) == 3
    for k in ("x", "v", "a", "j", "s", "c", "t", "dt"):
        np.testing.assert_array_equal(a.state()[k], b.state()[k])
    # a second call continues from the synchronisation time reached
    _, d2 = b.run_diag(0.5, 2.0 ** -2)
    assert d2["t"].tolist() == [0.25, 0.5]
    assert d2["ekin"][0] == d["ekin"][-1] and d2["epot"][0] == d["epot"][-1]
    a.close()
    b.close()


def test_run_diag_capacity_and_argument_errors():
    nb = nb_gpu()
    m, x, v = ni.plummer(128, 2)
    g = nb.NBody(m, x, v, 1e-3, dt_max=2.0 ** -4)
    steps, d = g.run_diag(0.25, 2.0 ** -4, cap=2)
    assert len(d["t"]) == 2 and d["t"].tolist() == [0.0, 2.0 ** -4]
    for bad in ((0.5, 2.0 ** -5), (0.3, 2.0 ** -4), (0.5, 0.0), (0.5, -1.0), (0.125, 2.0 ** -3)):
        with pytest.raises(nb.NBError):
            g.run_diag(*bad)
    t, _ = g.step()                             # now between synchronisation times
    assert t % 2.0 ** -4 != 0.0
    with pytest.raises(nb.NBError):
        g.run_diag(0.5, 2.0 ** -4)
    g.close()


def test_single_precision_mode_is_fp32_positions_within_kappa_bound():
    """NB_SP drops the low FP32 half of every position: the evaluation equals
    the oracle on positions rounded to FP32, within the FP32 pair-arithmetic
    bound 1e-6 sum_j |T_ij|; it is measurably worse than NB_MIXED once the
    system sits away from the origin."""
    nb = nb_gpu()
    n, eps = 1000, 1e-4
    m, x, v = ni.plummer(n, 13, imf="salpeter")
    x = x + np.array([3.0, -2.0, 1.0])
    a = ni.random_state(n, 113, scale=2.0)
    act = ni.active_subset(n, 333, 9)
    out = {}
    for prec in (nb.NB_MIXED, nb.NB_SP):
        g = nb.NBody(m, x, v, eps, precision=prec, start_forces=False)
        g.set_state({"x": x, "v": v, "a": a, "j": np.zeros((n, 3)), "s": np.zeros((n, 3)),
                     "c": np.zeros((n, 3)), "t": np.zeros(n), "dt": np.full(n, 2.0 ** -3)})
        g.predict(0.0)
        out[prec] = g.evaluate(act)
        g.close()
    x32 = x.astype(np.float32).astype(np.float64)
    ref32 = O.evaluate(m, x32, v, a, eps, act)
    kap32 = O.evaluate_kappa(m, x32, v, a, eps, act)
    for got, r, k in zip(out[nb.NB_SP], ref32, kap32):
        assert check_parity(1, got, r, k) <= 1.0
    ref = O.evaluate(m, x, v, a, eps, act)
    err_mixed = rel_err(out[nb.NB_MIXED][0], ref[0]).max()
    err_sp = rel_err(out[nb.NB_SP][0], ref[0]).max()
    assert err_sp > 10 * err_mixed


def test_single_precision_ensemble_is_rejected():
    nb = nb_gpu()
    m, x, v = ni.plummer(64, 3)
    with pytest.raises(nb.NBError):
        nb.Ensemble([64], m, x, v, 1e-3, precision=nb.NB_SP)
