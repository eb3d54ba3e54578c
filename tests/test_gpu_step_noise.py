"""The step criterion with a rounding floor (nb_config.step_noise).

With FP32 pair arithmetic the evaluated acceleration, jerk and snap carry
rounding of a few 1e-8 of each sum's condition number; the quintic
interpolation divides the residuals' share of it by h^3, h^4, h^5, and once
a close pair takes small steps the interpolated crackle, pop and a^(5) are
mostly rounding, which drives the pair to the smallest step.  With
step_noise set to the arithmetic's rounding level the criterion discounts
the parts of those derivatives below their rounding floor.  Checked here on
a system with a close pair (the 1438-particle member of the 256-system
ensemble): the mixed integration with the floor takes a number of block
steps comparable to FP64's instead of sitting at the 2^-20 floor, and its
energy error stays at the integrator's level.  step_noise = 0 (the default)
is the criterion as is; every other test runs with it."""
import numpy as np
import pytest

import nb_inputs as ni
from nbhelp import nb_gpu

pytestmark = pytest.mark.gpu


def _close_pair_system():
    sizes = ni.ensemble_sizes(256, 4)
    k = int(np.nonzero(sizes == 1438)[0][0])
    return ni.plummer(1438, 1000 + k)


def _run(nb, prec, noise, t_end=2.0 ** -4):
    m, x, v = _close_pair_system()
    g = nb.NBody(m, x, v, 1e-4, precision=prec, step_noise=noise, dt_max=min(t_end, 2.0 ** -4))
    e0 = sum(g.energy())
    steps, _ = g.run_until(t_end)
    e1 = sum(g.energy())
    st = g.state()
    g.close()
    return steps, abs((e1 - e0) / e0), st


def test_mixed_with_rounding_floor_leaves_the_step_floor():
    """FP64 takes 118 block steps to t = 1/16.  Mixed with the criterion as
    is reaches the 2^-20 floor within t = 1/64; with a floor of 4e-7 (about
    2^-21, the relative error of mu = m q q^2 from the two special-function
    estimates) it takes about twice FP64's steps and stays at the
    integrator's energy error."""
    nb = nb_gpu()
    steps64, err64, _ = _run(nb, nb.NB_FP64, 0.0)
    _, _, st0 = _run(nb, nb.NB_MIXED, 0.0, t_end=2.0 ** -6)
    assert st0["dt"].min() == 2.0 ** -20
    steps_m, err_m, st_m = _run(nb, nb.NB_MIXED, 4e-7)
    assert steps_m <= 4 * steps64, (steps_m, steps64)
    assert err_m <= max(100 * err64, 1e-9), (err_m, err64)
    assert np.all(st_m["t"] == 2.0 ** -4)
    # every step stays a power of two dividing t (block-step invariant)
    assert np.all(np.fmod(st_m["t"], st_m["dt"]) == 0.0)


def test_rounding_floor_is_rejected_out_of_range():
    nb = nb_gpu()
    m, x, v = ni.plummer(16, 3)
    for bad in (-1e-9, 2e-3, float("nan")):
        with pytest.raises(nb.NBError) as e:
            nb.NBody(m, x, v, 1e-3, step_noise=bad)
        assert e.value.status == nb.NB_EINVAL


@pytest.mark.parametrize("noise", [0.0, 2e-6])
def test_criterion_discounts_only_the_rounding_floor(noise):
    """One particle (and a far, massless companion) on a constant-snap motion:
    a1, j1, s1 follow a0, j0, s0 exactly, except for a relative error of
    1e-6 planted in a1, loaded through nb_set_forces.  The quintic's
    crackle, pop and a^(5) are then that error divided by h^3, h^4, h^5,
    and the criterion as is halves the step; with a rounding floor of 2e-6,
    above the planted error, they are discounted to zero, so the step stays
    h (it may not double at a time that is not a multiple of 2h).  The
    oracle's interpolation, floors and criterion give the same step."""
    nb = nb_gpu()
    import oracle as O
    h = 2.0 ** -10
    a0, j0, s0 = np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0])
    a1 = (a0 + j0 * h + s0 * h * h / 2) * (1 + 1e-6)
    j1, s1 = j0 + s0 * h, s0
    m = np.array([1.0, 0.0])
    x = np.array([[0.0, 0.0, 0.0], [100.0, 0.0, 0.0]])
    v = np.zeros((2, 3))
    g = nb.NBody(m, x, v, 1e-3, start_forces=False, step_noise=noise, dt_max=2.0 ** -3)
    z = np.zeros((2, 3))
    g.set_state({"x": x, "v": v, "a": np.array([a0, [0, 0, 0]]), "j": np.array([j0, [0, 0, 0]]),
                 "s": np.array([s0, [0, 0, 0]]), "c": z, "t": np.zeros(2), "dt": np.full(2, h)})
    g.predict(h)
    f = np.zeros((9, 1))
    f[0:3, 0], f[3:6, 0], f[6:9, 0] = a1, j1, s1
    g.set_forces(np.array([0], dtype=np.int32), f)
    g.correct(h)
    dt = g.state()["dt"][0]
    g.close()
    c, d, e = O.interpolate(h, a0, j0, s0, a1, j1, s1)
    fl = O.interp_floor(noise, h, a0, j0, s0, a1, j1, s1)
    ref, _ = O.dt_quantise(O.dt_crit_floored(0.4, a1, j1, s1, c, d, e, fl), h, h, dt_max=2.0 ** -3)
    assert dt == ref
    # the planted error alone halves the step; the floor above it keeps h
    assert ref == (h / 2 if noise == 0.0 else h)


@pytest.mark.parametrize("case", ["plummer_1024", "close_pair_1438"])
def test_fp64_with_rounding_floor_takes_the_oracles_decisions(case):
    """FP64 arithmetic with the floor at 4e-7 on both sides (the oracle's
    orc_interp_floor and floored criterion): the GPU takes the oracle's block
    steps (time, active count and active set at every step) and ends on its
    state to 1e-10: Plummer N = 1024 to t = 1/8, and the close-pair system
    to t = 1/16; host-driven steps and nb_run_until alike."""
    nb = nb_gpu()
    import oracle as O
    if case == "plummer_1024":
        (m, x, v), t_end = ni.plummer(1024, 1), 0.125
    else:
        (m, x, v), t_end = _close_pair_system(), 2.0 ** -4
    ref = O.System(m, x, v, 1e-4, dt_max=t_end, step_noise=4e-7)
    steps_r, (lt_r, ln_r, lh_r) = ref.run_until(t_end, log_cap=1 << 17)
    g = nb.NBody(m, x, v, 1e-4, dt_max=t_end, step_noise=4e-7)
    tn, sets = [], []
    while True:
        t, n_act = g.step()
        tn.append(t)
        sets.append(g.active().copy())
        assert sets[-1].size == n_act
        if t == t_end and n_act == m.size:
            break
        assert len(tn) <= steps_r
    st_g = g.state()
    g.close()
    st_r = ref.state()
    assert len(tn) == steps_r
    np.testing.assert_array_equal(tn, lt_r)
    np.testing.assert_array_equal([q.size for q in sets], ln_r)
    assert [O.set_hash(q) for q in sets] == [int(h) for h in lh_r]
    np.testing.assert_array_equal(st_g["t"], st_r["t"])
    np.testing.assert_array_equal(st_g["dt"], st_r["dt"])
    for f in ("x", "v"):
        assert np.abs(st_g[f] - st_r[f]).max() <= 1e-10 * np.abs(st_r[f]).max(), f
    # the same run through nb_run_until (small active sets on the
    # device-resident stepper) takes the same steps
    g = nb.NBody(m, x, v, 1e-4, dt_max=t_end, step_noise=4e-7)
    steps_d, (lt_d, ln_d) = g.run_until(t_end, log_cap=1 << 17)
    st_d = g.state()
    g.close()
    assert steps_d == steps_r
    np.testing.assert_array_equal(lt_d, lt_r)
    np.testing.assert_array_equal(ln_d, ln_r)
    np.testing.assert_array_equal(st_d["dt"], st_r["dt"])
