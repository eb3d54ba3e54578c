"""Checkpoint and resume of a block-step integration (section 2 block steps,
section 3 Hermite state): run k steps, copy the state out with nb_get_state,
load it into a FRESH context with nb_set_state (start_forces = 0, so the
context computes nothing of its own), run k more steps, and compare with 2k
uninterrupted steps.  Every step depends only on the state (x, v, a, jerk,
snap, crackle, t_i, dt_i), and the kernels sum in a fixed order, so the two
runs must agree bit for bit, decisions included."""
import numpy as np
import pytest

import nb_inputs as ni
from nbhelp import nb_gpu

pytestmark = pytest.mark.gpu

FIELDS = ("x", "v", "a", "j", "s", "c", "t", "dt")


def _assert_same(a, b):
    for k in FIELDS:
        assert np.array_equal(a[k], b[k]), (k, np.abs(a[k] - b[k]).max())


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_resume_after_k_steps_is_bit_exact(prec):
    nb = nb_gpu()
    eps, k = 1e-4, 40
    m, x, v = ni.plummer(1024, 1)
    straight = nb.NBody(m, x, v, eps, precision=prec)
    log_straight = [straight.step() for _ in range(2 * k)]
    ref = straight.state()
    straight.close()

    first = nb.NBody(m, x, v, eps, precision=prec)
    log_first = [first.step() for _ in range(k)]
    ckpt = first.state()
    first.close()

    resumed = nb.NBody(m, x, v, eps, precision=prec, start_forces=False)
    resumed.set_state(ckpt)
    log_second = [resumed.step() for _ in range(k)]
    got = resumed.state()
    resumed.close()

    assert log_first + log_second == log_straight
    _assert_same(got, ref)


@pytest.mark.parametrize("prec", [0, 3])
def test_resume_of_run_until_is_bit_exact(prec):
    """Host-driven integration to t = 1/32, checkpoint, resume in a fresh
    context to t = 1/16, against one run to 1/16 (device_steps off on both,
    because the device-resident stepper sums in another order and its use
    depends on a back-off counter that is not part of the state)."""
    nb = nb_gpu()
    eps = 1e-4
    m, x, v = ni.plummer(512, 3)
    kw = dict(precision=prec, dt_max=2.0 ** -5, device_steps=False)
    straight = nb.NBody(m, x, v, eps, **kw)
    n_straight, _ = straight.run_until(1.0 / 16)
    ref = straight.state()
    straight.close()

    first = nb.NBody(m, x, v, eps, **kw)
    n1, _ = first.run_until(1.0 / 32)
    ckpt = first.state()
    first.close()
    resumed = nb.NBody(m, x, v, eps, start_forces=False, **kw)
    resumed.set_state(ckpt)
    n2, _ = resumed.run_until(1.0 / 16)
    got = resumed.state()
    resumed.close()

    assert n1 + n2 == n_straight
    assert np.all(got["t"] == 1.0 / 16)
    _assert_same(got, ref)
