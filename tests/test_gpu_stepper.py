"""The device-resident block stepper (active sets of up to 128 particles scheduled, evaluated
and corrected inside one cooperative launch) against the host-driven path
and the FP64 oracle.  The stepper sums the pair terms in another order
(per-block slices), so results agree to rounding and the step decisions are
the same."""
import numpy as np
import pytest

import nb_inputs as ni
import oracle as O
from nbhelp import nb_gpu, rel_err

pytestmark = pytest.mark.gpu


def _run(nb, m, x, v, eps, t_end, device, **kw):
    g = nb.NBody(m, x, v, eps, device_steps=device, **kw)
    steps, log = g.run_until(t_end, log_cap=1 << 20)
    st, act, cnt = g.state(), g.active(), g.counters()
    g.close()
    return steps, log, st, act, cnt


@pytest.mark.parametrize("prec", [0, 3])
def test_stepper_takes_the_host_paths_decisions(prec):
    """FP64 and EX: identical step logs, active set of the last step and
    interaction counts; states equal to rounding."""
    nb = nb_gpu()
    m, x, v = ni.plummer(2000, 21)
    a = _run(nb, m, x, v, 1e-4, 0.125, True, precision=prec)
    b = _run(nb, m, x, v, 1e-4, 0.125, False, precision=prec)
    assert a[0] == b[0]
    np.testing.assert_array_equal(a[1][0], b[1][0])
    np.testing.assert_array_equal(a[1][1], b[1][1])
    assert (a[1][1] <= 128).sum() > 0.5 * a[0]       # most steps ran in the stepper
    for k in ("x", "v"):
        assert rel_err(a[2][k], b[2][k]).max() < 1e-12, k
    for k in ("a", "j", "s"):
        assert rel_err(a[2][k], b[2][k]).max() < 1e-10, k
    np.testing.assert_array_equal(a[2]["t"], b[2]["t"])
    np.testing.assert_array_equal(a[2]["dt"], b[2]["dt"])
    np.testing.assert_array_equal(np.sort(a[3]), np.sort(b[3]))
    assert a[4][1] == b[4][1]                         # interactions
    assert a[4][0] < b[4][0]                          # fewer launches


def test_stepper_fp64_matches_the_oracle_log():
    nb = nb_gpu()
    m, x, v = ni.plummer(700, 22)
    ref = O.System(m, x, v, 1e-4)
    steps_r, (lt_r, ln_r, _) = ref.run_until(0.125, log_cap=100000)
    steps, (lt, ln), st, _, _ = _run(nb, m, x, v, 1e-4, 0.125, True)
    assert steps == steps_r
    np.testing.assert_array_equal(lt, lt_r)
    np.testing.assert_array_equal(ln, ln_r)
    sr = ref.state()
    for k in ("x", "v"):
        assert rel_err(st[k], sr[k]).max() < 1e-10, k


@pytest.mark.parametrize("prec", [1, 2])
def test_stepper_fp32_paths_conserve_energy_like_the_host_path(prec):
    """Mixed and single-precision control: the FP32 rounding may move step
    decisions, so the two paths are compared by their energy error."""
    nb = nb_gpu()
    m, x, v = ni.plummer(1000, 23)
    out = []
    for device in (True, False):
        g = nb.NBody(m, x, v, 1e-3, precision=prec, device_steps=device)
        e0 = sum(g.energy())
        g.run_until(0.125)
        out.append(abs(sum(g.energy()) / e0 - 1.0))
        g.close()
    assert out[0] < 1e-6 and out[1] < 1e-6


def test_stepper_tiny_system_and_log_capacity():
    nb = nb_gpu()
    m, x, v = ni.plummer(5, 24)
    a = _run(nb, m, x, v, 1e-3, 0.25, True)
    b = _run(nb, m, x, v, 1e-3, 0.25, False)
    assert a[0] == b[0]
    np.testing.assert_array_equal(a[1][0], b[1][0])
    g = nb.NBody(m, x, v, 1e-3)
    steps, (lt, ln) = g.run_until(0.25, log_cap=3)
    g.close()
    assert steps == a[0] and lt.size == 3
    np.testing.assert_array_equal(lt, a[1][0][:3])
