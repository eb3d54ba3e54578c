"""Extended-precision (EX, double-word FP32) evaluation against the FP64 CPU
oracle, through the C-ABI.

EX represents every predicted x, v, a and m as hi + lo FP32 numbers (about
48 mantissa bits) and computes the whole pair term in double-word
arithmetic.  Two error sources, tested apart:
  * arithmetic: against the oracle evaluated on the double-word-rounded
    inputs, |got - ref|_inf <= 1e-12 sum_j |T_ij| per particle (the
    double-word operations carry about 2^-45 relative error each; a float32
    emulation of the kernel's operation sequence stays below 2.5e-13);
  * representation: the position of a particle at distance |x| from the
    origin is held to 2^-48 |x|, so at the natural coordinates of the
    Plummer model (|x| of order 1) the same bound holds against the oracle
    on the original FP64 inputs.
"""
import numpy as np
import pytest

import nb_inputs as ni
import oracle as O
from nbhelp import check_parity, nb_gpu, rel_err

pytestmark = pytest.mark.gpu

TOL_EX = 1e-12
SHAPES = [
    {},
    {"junroll": 1},
    {"threads": 64, "jtile": 96, "lanes": 4, "split": 3},
    {"threads": 32, "jtile": 64, "lanes": 32, "split": 7, "junroll": 1},
    {"threads": 128, "jtile": 512, "lanes": 2, "split": 2},
    {"threads": 128, "jtile": 60, "lanes": 1, "split": 5, "junroll": 2},
]


def dw(q):
    """Round FP64 values to the double word hi + lo the EX buffer holds."""
    q = np.asarray(q, dtype=np.float64)
    hi = q.astype(np.float32).astype(np.float64)
    lo = (q - hi).astype(np.float32).astype(np.float64)
    return hi + lo


def _system(n, seed, offset=0.0):
    m, x, v = ni.plummer(n, seed, imf="salpeter")
    return m, x + offset, v, ni.random_state(n, seed + 100, scale=2.0)


def _ex_eval(nb, m, x, v, a, eps, act, shape):
    n = m.size
    g = nb.NBody(m, x, v, eps, precision=nb.NB_EX, tiles=shape, start_forces=False)
    g.set_state({"x": x, "v": v, "a": a, "j": np.zeros((n, 3)), "s": np.zeros((n, 3)),
                 "c": np.zeros((n, 3)), "t": np.zeros(n), "dt": np.full(n, 2.0 ** -3)})
    g.predict(0.0)
    out = g.evaluate(act)
    g.close()
    return out


@pytest.mark.parametrize("shape", range(len(SHAPES)))
@pytest.mark.parametrize("n_act", [1, 7, 333, 1000])
@pytest.mark.parametrize("offset", [0.0, 5.0])
def test_ex_arithmetic_against_oracle_on_double_word_inputs(shape, n_act, offset):
    nb = nb_gpu()
    n, eps = 1000, 1e-4
    m, x, v, a = _system(n, 11, offset)
    act = ni.active_subset(n, n_act, 5 + n_act)
    got = _ex_eval(nb, m, x, v, a, eps, act, SHAPES[shape])
    mr, xr, vr, ar = dw(m), dw(x), dw(v), dw(a)
    ref = O.evaluate(mr, xr, vr, ar, eps, act)
    kap = O.evaluate_kappa(mr, xr, vr, ar, eps, act)
    for g, r, k in zip(got, ref, kap):
        assert check_parity(1, g, r, k, tol_mixed=TOL_EX) <= 1.0


def test_ex_against_oracle_at_natural_coordinates_and_beats_mixed():
    nb = nb_gpu()
    n, eps = 1000, 1e-4
    m, x, v, a = _system(n, 12)
    act = ni.active_subset(n, 500, 3)
    got = _ex_eval(nb, m, x, v, a, eps, act, {})
    ref = O.evaluate(m, x, v, a, eps, act)
    kap = O.evaluate_kappa(m, x, v, a, eps, act)
    for g, r, k in zip(got, ref, kap):
        assert check_parity(1, g, r, k, tol_mixed=TOL_EX) <= 1.0
        assert rel_err(g, r).max() < 1e-11
    gm = nb.NBody(m, x, v, eps, precision=nb.NB_MIXED, start_forces=False)
    gm.set_state({"a": a})
    gm.predict(0.0)
    mixed = gm.evaluate(act)
    gm.close()
    for g, mq, r in zip(got, mixed, ref):
        assert rel_err(g, r).max() * 1e4 < rel_err(mq, r).max()


def test_ex_predictor_writes_double_words():
    nb = nb_gpu()
    n = 513
    m, x, v, a = _system(n, 3, offset=2.0)
    j, s, c = (ni.random_state(n, k, scale=4.0) for k in (41, 42, 43))
    t_i = np.where(np.arange(n) % 2 == 0, 0.0, 0.125)
    g = nb.NBody(m, x, v, 1e-4, precision=nb.NB_EX)
    g.set_state({"x": x, "v": v, "a": a, "j": j, "s": s, "c": c, "t": t_i,
                 "dt": np.full(n, 2.0 ** -3)})
    g.predict(0.25)
    got = g.predicted()
    g.close()
    ref = O.predict(0.25, t_i, x, v, a, j, s, c)
    for gq, rq in zip(got, ref):
        # hi + lo of the FP64 prediction: 2^-48 relative, plus the FP64
        # Taylor sum's own rounding
        assert np.all(np.abs(gq - rq) <= 2.0 ** -48 * np.abs(rq) + 1e-15 * (np.abs(rq).max() + 1))


def test_ex_block_steps_against_oracle_replay():
    """EX rounding may move a step-size decision across a power of two; the
    oracle replays the GPU's decisions and the states are compared."""
    nb = nb_gpu()
    m, x, v = ni.plummer(300, 4)
    g = nb.NBody(m, x, v, 1e-4, precision=nb.NB_EX)
    st0 = g.state()
    ref0 = O.System(m, x, v, 1e-4)
    for k in ("a", "j", "s"):
        assert rel_err(st0[k], ref0.state()[k]).max() < 1e-10, k
    ref = ref0       # the oracle from its own start-up; only the decisions come from the GPU
    tn, sets = [], []
    for _ in range(6):
        t_g, n_g = g.step()
        tn.append(t_g)
        sets.append(g.active().copy())
        assert sets[-1].size == n_g
    ref.replay(tn, sets)
    st_r, st_g = ref.state(), g.state()
    g.close()
    for k in ("x", "v"):
        assert rel_err(st_g[k], st_r[k]).max() < 1e-13, k
    for k in ("a", "j", "s"):
        assert rel_err(st_g[k], st_r[k]).max() < 1e-10, k


def test_ex_full_size_sampled_parity():
    """N = 2^20 Plummer with Salpeter masses, eps = 1e-4, active fraction
    2^-10, the automatic launch shape: 16 sampled particles against the
    oracle on the double-word inputs."""
    nb = nb_gpu()
    n, eps = 1 << 20, 1e-4
    m, x, v = ni.plummer(n, 3, imf="salpeter")
    a = ni.random_state(n, 5, scale=2.0)
    g = nb.NBody(m, x, v, eps, precision=nb.NB_EX, start_forces=False)
    g.set_state({"a": a})
    act = ni.active_subset(n, 1024, 77)
    g.predict(0.0)
    got = g.evaluate(act)
    g.close()
    pick = np.arange(0, 1024, 64)
    mr, xr, vr, ar = dw(m), dw(x), dw(v), dw(a)
    ref = O.evaluate(mr, xr, vr, ar, eps, act[pick])
    kap = O.evaluate_kappa(mr, xr, vr, ar, eps, act[pick])
    for gq, rq, kq in zip(got, ref, kap):
        assert check_parity(1, gq[pick], rq, kq, tol_mixed=TOL_EX) <= 1.0


def test_ex_rejects_shapes_it_does_not_have():
    nb = nb_gpu()
    m, x, v = ni.plummer(64, 2)
    g = nb.NBody(m, x, v, 1e-3, precision=nb.NB_EX)
    g.predict(0.0)
    for bad in ({"ki": 2}, {"threads": 256}, {"junroll": 4}):
        g.set_tiles(**bad)
        with pytest.raises(nb.NBError):
            g.evaluate(None)
    g.set_tiles()
    g.evaluate(None)
    g.close()
