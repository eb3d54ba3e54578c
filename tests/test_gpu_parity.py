"""CUDA path against the FP64 CPU oracle, element by element, through the
C-ABI (via the ctypes binding).  Sizes span several j-tiles and i-tiles with
ragged tails; launch shapes cover lane-split and block-split evaluation.

Tolerances per particle:
  FP64 path  |got - ref|_inf <= 1e-12 |ref|_2
  mixed path |got - ref|_inf <= 1e-6 sum_j |T_ij|  (the sum's condition
             number; FP32 pair terms each carry a few 1e-8 relative error)
"""
import numpy as np
import pytest

import nb_inputs as ni
import oracle as O
from nbhelp import check_parity, nb_gpu, rel_err

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-6}
SHAPES = [
    {},                                                      # automatic
    {"ki": 1, "threads": 128, "jtile": 128, "lanes": 1, "split": 1},
    {"ki": 2, "threads": 64, "jtile": 96, "lanes": 4, "split": 3},
    {"ki": 1, "threads": 32, "jtile": 64, "lanes": 32, "split": 7},
    {"ki": 4, "threads": 128, "jtile": 256, "lanes": 2, "split": 2},
    {"ki": 2, "threads": 256, "jtile": 32, "lanes": 8, "split": 1},
    {"ki": 1, "threads": 128, "jtile": 512, "lanes": 1, "split": 1, "junroll": 2},
    {"ki": 2, "threads": 128, "jtile": 60, "lanes": 1, "split": 5, "junroll": 4},
    {"ki": 3, "threads": 128, "jtile": 512, "lanes": 1, "split": 2, "junroll": 4},
    {"ki": 3, "threads": 64, "jtile": 256, "lanes": 2, "split": 1, "junroll": 4},
    {"ki": 2, "threads": 128, "jtile": 512, "lanes": 2, "split": 3, "junroll": 4},
]


def _system(n, seed, imf="equal"):
    m, x, v = ni.plummer(n, seed, imf=imf)
    a = ni.random_state(n, seed + 100, scale=2.0)
    return m, x, v, a


def _shape_for(prec, shape):
    """The mixed kernel takes KI 1, 2 or 3 (at most 128 threads for KI 2 and
    3, KI 3 with four j per inner iteration); KI 4 shapes run there as KI 2
    with two j per inner iteration.  The FP64 kernel runs KI 3 shapes as
    KI 2."""
    shape = dict(shape)
    if prec == 1 and shape.get("ki") == 4:
        shape.update(ki=2, junroll=2)
    if prec == 0 and shape.get("ki") == 3:
        shape.update(ki=2)
    if prec == 1 and shape.get("ki") == 2 and shape.get("threads", 0) > 128:
        shape.update(threads=128)
    return shape


def _gpu_eval(nb, prec, m, x, v, a, eps, active, shape):
    g = nb.NBody(m, x, v, eps, precision=prec, tiles=_shape_for(prec, shape), start_forces=False)
    n = m.size
    g.set_state({"x": x, "v": v, "a": a, "j": np.zeros((n, 3)), "s": np.zeros((n, 3)),
                 "c": np.zeros((n, 3)), "t": np.zeros(n), "dt": np.full(n, 2.0 ** -3)})
    g.predict(0.0)
    out = g.evaluate(active)
    g.close()
    return out


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("shape", range(len(SHAPES)))
@pytest.mark.parametrize("n_act", [1, 7, 333, 1000])
def test_evaluation_matches_oracle(prec, shape, n_act):
    nb = nb_gpu()
    n, eps = 1000, 1e-4
    m, x, v, a = _system(n, 11, imf="salpeter")
    act = ni.active_subset(n, n_act, 5 + n_act)
    got = _gpu_eval(nb, prec, m, x, v, a, eps, act, SHAPES[shape])
    ref = O.evaluate(m, x, v, a, eps, act)
    kap = O.evaluate_kappa(m, x, v, a, eps, act) if prec else (None,) * 3
    for g, r, k in zip(got, ref, kap):
        assert check_parity(prec, g, r, k) <= 1.0


@pytest.mark.parametrize("prec", [0, 1])
def test_predictor_matches_oracle(prec):
    nb = nb_gpu()
    n = 777
    m, x, v, a = _system(n, 3)
    j, s, c = (ni.random_state(n, k, scale=4.0) for k in (41, 42, 43))
    t_i = np.where(np.arange(n) % 3 == 0, 0.0, np.where(np.arange(n) % 3 == 1, 0.125, 0.1875))
    dt = np.where(t_i == 0.1875, 2.0 ** -4, 2.0 ** -3)
    t = 0.25
    g = nb.NBody(m, x, v, 1e-4, precision=prec)
    g.set_state({"x": x, "v": v, "a": a, "j": j, "s": s, "c": c, "t": t_i, "dt": dt})
    g.predict(t)
    got = g.predicted()
    g.close()
    ref = O.predict(t, t_i, x, v, a, j, s, c)
    tol = {0: 4e-16, 1: 1e-7}[prec]
    for q, (gq, rq) in enumerate(zip(got, ref)):
        scale = np.abs(rq).max() + 1.0
        if prec == 1 and q == 0:
            tol_q = 4e-15  # hi + lo position pair carries ~48 bits
        else:
            tol_q = tol
        assert np.abs(gq - rq).max() < tol_q * 8 * scale, (q, np.abs(gq - rq).max())


def test_split_and_lane_shapes_agree_to_rounding_and_are_deterministic():
    nb = nb_gpu()
    n, eps = 2048, 1e-4
    m, x, v, a = _system(n, 21)
    act = ni.active_subset(n, 100, 9)
    outs = [_gpu_eval(nb, 0, m, x, v, a, eps, act, SHAPES[k]) for k in range(len(SHAPES))]
    for o in outs[1:]:
        for g, r in zip(o, outs[0]):
            assert rel_err(g, r).max() < 1e-13
    again = _gpu_eval(nb, 0, m, x, v, a, eps, act, SHAPES[3])
    for g, r in zip(again, outs[3]):
        np.testing.assert_array_equal(g, r)


def test_fp64_block_steps_take_the_oracles_decisions():
    """FP64: same starting steps, same (t_next, active set) at every step,
    same state to 1e-12."""
    nb = nb_gpu()
    m, x, v = ni.plummer(300, 4)
    ref = O.System(m, x, v, 1e-4)
    g = nb.NBody(m, x, v, 1e-4)
    st0_ref, st0 = ref.state(), g.state()
    for k in ("a", "j", "s"):
        assert rel_err(st0[k], st0_ref[k]).max() < 4e-12
    np.testing.assert_array_equal(st0["dt"], st0_ref["dt"])
    for _ in range(3):
        t_r, n_r, h_r = ref.step()
        t_g, n_g = g.step()
        assert (t_g, n_g) == (t_r, n_r)
        assert O.set_hash(g.active()) == h_r
    st_r, st_g = ref.state(), g.state()
    g.close()
    for k in ("x", "v", "a", "j", "s"):
        assert rel_err(st_g[k], st_r[k]).max() < 4e-12, k
    np.testing.assert_array_equal(st_g["t"], st_r["t"])
    np.testing.assert_array_equal(st_g["dt"], st_r["dt"])


def test_mixed_block_steps_against_oracle_replay():
    """Mixed: FP32 rounding may move a step-size decision across a power of
    two, which gives another valid trajectory.  The oracle replays the GPU's
    decisions (t_next and active sets) from its own start-up state (the same
    positions and velocities) and the states are compared."""
    nb = nb_gpu()
    m, x, v = ni.plummer(300, 4)
    g = nb.NBody(m, x, v, 1e-4, precision=nb.NB_MIXED)
    ref = O.System(m, x, v, 1e-4)     # its own start-up; only the decisions come from the GPU
    tn, sets = [], []
    for _ in range(4):
        t_g, n_g = g.step()
        tn.append(t_g)
        sets.append(g.active().copy())
        assert sets[-1].size == n_g
    ref.replay(tn, sets)
    st_r, st_g = ref.state(), g.state()
    g.close()
    for k in ("x", "v"):
        assert rel_err(st_g[k], st_r[k]).max() < 1e-9, k
    # a, jerk, snap: 1e-6 of each sum's condition number sum_j |T_ij|, taken
    # on the replayed state (each particle's forces are from its own last
    # step, a few block steps at most before the state's time)
    kap = O.evaluate_kappa(m, st_r["x"], st_r["v"], st_r["a"], 1e-4)
    for k, kq in zip(("a", "j", "s"), kap):
        assert check_parity(1, st_g[k], st_r[k], kq) <= 1.0, k
    np.testing.assert_array_equal(st_g["t"], st_r["t"])


def test_plummer_1024_block_integration_matches_oracle():
    """Plummer N=1024, eps=1e-4, eta=0.4, dt in [2^-20, 2^-3], FP64, t=0.125."""
    nb = nb_gpu()
    m, x, v = ni.plummer(1024, 1)
    eps = 1e-4
    ref = O.System(m, x, v, eps)
    steps_r, (lt_r, ln_r, _) = ref.run_until(0.125, log_cap=100000)
    g = nb.NBody(m, x, v, eps)
    E0 = sum(g.energy())
    steps_g, (lt_g, ln_g) = g.run_until(0.125, log_cap=100000)
    assert steps_g == steps_r
    np.testing.assert_array_equal(lt_g, lt_r)
    np.testing.assert_array_equal(ln_g, ln_r)
    st_r, st_g = ref.state(), g.state()
    for k in ("x", "v"):
        assert rel_err(st_g[k], st_r[k]).max() < 1e-10, k
    E1 = sum(g.energy())
    E0r = sum(O.energy(m, x, v, eps))
    E1r = sum(O.energy(m, st_r["x"], st_r["v"], eps))
    assert abs(E0 - E0r) < 1e-13 and abs(E1 - E1r) < 1e-12
    assert abs((E1 - E0) / E0) < 1e-9
    g.close()


def test_energy_and_angular_momentum_match_oracle():
    nb = nb_gpu()
    m, x, v = ni.plummer(3000, 8, imf="salpeter")
    g = nb.NBody(m, x, v, 1e-3)
    ek, ep = g.energy()
    L, la = g.angmom()
    g.close()
    ekr, epr = O.energy(m, x, v, 1e-3)
    Lr, lar = O.angmom(m, x, v)
    assert abs(ek - ekr) < 1e-14 * abs(ekr) and abs(ep - epr) < 1e-13 * abs(epr)
    assert np.abs(L - Lr).max() < 1e-13 * lar and abs(la - lar) < 1e-13 * lar


def test_kepler_shared_steps_follow_analytic_orbit():
    nb = nb_gpu()
    from test_oracle_pins import kepler_state
    m, x, v = kepler_state(0.0)
    g = nb.NBody(m, x, v, 1e-12, dt_shared=2.0 ** -7, dt_max=2.0 ** -7)
    steps, _ = g.run_until(2.0)
    st = g.state()
    g.close()
    _, xr, _ = kepler_state(2.0)
    assert steps == 256
    assert np.abs(st["x"] - xr).max() < 1e-9
    ref = O.System(m, x, v, 1e-12, dt_shared=2.0 ** -7, dt_max=2.0 ** -7)
    ref.run_until(2.0)
    assert np.abs(st["x"] - ref.state()["x"]).max() < 1e-13


@pytest.mark.parametrize("prec", [0, 1, 3])
@pytest.mark.parametrize("n", [1, 2, 3, 31, 33])
def test_tiny_systems(n, prec):
    """Sizes below one j-tile and one warp, in FP64, mixed and EX; the step
    decisions must match the oracle's (a, j, s differ only by rounding)."""
    nb = nb_gpu()
    m, x, v = ni.plummer(max(n, 1), 12)
    if n == 1:
        x = np.zeros((1, 3)) + 0.3
        v = np.zeros((1, 3))
        m = np.ones(1)
    g = nb.NBody(m, x, v, 1e-3, precision=prec)
    ref = O.System(m, x, v, 1e-3)
    st_g, st_r = g.state(), ref.state()
    # condition numbers of the start-up sums: a and jerk from the pass with
    # a_j = 0, snap from the pass with the starting accelerations
    kap0 = O.evaluate_kappa(m, x, v, np.zeros_like(x), 1e-3)
    kap1 = O.evaluate_kappa(m, x, v, st_r["a"], 1e-3)
    for k, kq in zip(("a", "j", "s"), (kap0[0], kap0[1], kap1[2])):
        if prec == 1:   # FP32 pair arithmetic: 1e-6 of the sum's condition number
            assert check_parity(1, st_g[k], st_r[k], kq) <= 1.0, k
        else:
            np.testing.assert_allclose(st_g[k], st_r[k], rtol={0: 1e-12, 3: 1e-10}[prec], atol=1e-300)
    if prec == 1 and not np.array_equal(st_g["dt"], st_r["dt"]):
        # FP32 rounding moved a starting step across a power of two: another
        # valid trajectory; the steps may differ by one factor of two only
        assert set(np.unique(st_g["dt"] / st_r["dt"])) <= {0.5, 1.0, 2.0}
        g.close()
        return
    np.testing.assert_array_equal(st_g["dt"], st_r["dt"])
    t_r, n_r, _ = ref.step()
    t_g, n_g = g.step()
    assert (t_g, n_g) == (t_r, n_r)
    g.close()


def test_empty_active_set_and_argument_errors():
    nb = nb_gpu()
    m, x, v = ni.plummer(64, 2)
    g = nb.NBody(m, x, v, 1e-3)
    with pytest.raises(nb.NBError) as e:
        g.evaluate(np.array([0], dtype=np.int32))
    assert e.value.status == nb.NB_ESTATE
    g.predict(0.0)
    out = g.evaluate(np.zeros(0, dtype=np.int32))
    assert all(o.shape == (0, 3) for o in out)
    with pytest.raises(nb.NBError) as e:
        g.evaluate(np.array([64], dtype=np.int32))
    assert e.value.status == nb.NB_EINVAL
    with pytest.raises(nb.NBError) as e:
        g.correct(0.5)
    assert e.value.status == nb.NB_ESTATE
    g.close()
    with pytest.raises(nb.NBError) as e:
        nb.NBody(m, x, v, 0.0)
    assert e.value.status == nb.NB_EINVAL
    bad = x.copy()
    bad[3, 1] = np.nan
    with pytest.raises(nb.NBError) as e:
        nb.NBody(m, bad, v, 1e-3)
    assert e.value.status == nb.NB_ENONFINITE


@pytest.mark.parametrize("device_steps", [True, False])
@pytest.mark.parametrize("prec", [0, 1, 3])
def test_lone_particle_coasts_at_the_largest_step(prec, device_steps):
    """N = 1, the method's degenerate system: no force, so the step
    criterion is 0/0, sets no bound, and the particle moves in a straight
    line at dt_max, exactly as the oracle's lone particle does."""
    nb = nb_gpu()
    x0, v0 = np.array([[0.25, -0.5, 1.0]]), np.array([[0.5, 0.125, -1.0]])
    g = nb.NBody(np.ones(1), x0, v0, 1e-4, precision=prec, device_steps=device_steps)
    steps, _ = g.run_until(0.5)
    st = g.state()
    g.close()
    ref = O.System(np.ones(1), x0, v0, 1e-4)
    ref_steps, _ = ref.run_until(0.5)
    sr = ref.state()
    assert steps == ref_steps == 4
    for f in ("x", "v", "t", "dt"):
        np.testing.assert_array_equal(st[f], sr[f], err_msg=f)
    np.testing.assert_array_equal(st["x"], x0 + 0.5 * v0)


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_sampled_parity(prec):
    """N = 2^20 Plummer with Salpeter masses, eps = 1e-4, active fraction
    2^-10 in the launch shape the benchmark uses: 16 sampled particles
    against the oracle."""
    nb = nb_gpu()
    n, eps = 1 << 20, 1e-4
    m, x, v = ni.plummer(n, 3, imf="salpeter")
    a = ni.random_state(n, 5, scale=2.0)
    g = nb.NBody(m, x, v, eps, precision=prec, start_forces=False)
    g.set_state({"a": a})
    act = ni.active_subset(n, 1024, 77)
    g.predict(0.0)
    got = g.evaluate(act)
    g.close()
    pick = np.arange(0, 1024, 64)
    ref = O.evaluate(m, x, v, a, eps, act[pick])
    kap = O.evaluate_kappa(m, x, v, a, eps, act[pick]) if prec else (None,) * 3
    for gq, rq, kq in zip(got, ref, kap):
        assert check_parity(prec, gq[pick], rq, kq) <= 1.0


def test_bench_headline_launch_sampled_parity():
    """The bench's headline step: N = 2^20 Plummer with Salpeter masses,
    eps = 1e-4, every particle active, the mixed kernel in the automatic
    launch shape (KI 3, 128 threads, j-tile 512, no split), with the seeded
    acceleration field the bench's oracle comparison uses; 256 evenly spread
    particles against the oracle at 1e-6 of sum_j |T_ij|."""
    nb = nb_gpu()
    n, eps = 1 << 20, 1e-4
    m, x, v = ni.plummer(n, 3, imf="salpeter")
    a = ni.random_state(n, 5, scale=2.0)
    g = nb.NBody(m, x, v, eps, precision=nb.NB_MIXED, dt_shared=2.0 ** -10, start_forces=False)
    g.set_state({"a": a})
    shape = g.resolve_tiles(n)
    assert (shape["ki"], shape["threads"], shape["jtile"], shape["split"]) == (3, 128, 512, 1)
    g.predict(0.0)
    got = g.evaluate(None)
    g.close()
    pick = np.linspace(0, n - 1, 256).astype(np.int32)
    ref = O.evaluate(m, x, v, a, eps, pick)
    kap = O.evaluate_kappa(m, x, v, a, eps, pick)
    for gq, rq, kq in zip(got, ref, kap):
        assert check_parity(1, gq[pick], rq, kq) <= 1.0


@pytest.fixture(scope="module")
def large_system():
    n, eps = 1 << 24, 1e-4
    m, x, v = ni.plummer(n, 17, imf="salpeter")
    a = ni.random_state(n, 18, scale=2.0)
    act = ni.active_subset(n, 1024, 19)
    pick = np.array([0, 341, 682, 1023])
    ref = O.evaluate(m, x, v, a, eps, act[pick])
    kap = O.evaluate_kappa(m, x, v, a, eps, act[pick])
    return m, x, v, a, eps, act, pick, ref, kap


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_large_system_sampled_parity(prec, large_system):
    """N = 2^24, sixteen times the benchmark's N (about 6 GB of device
    state), Plummer with Salpeter masses, eps = 1e-4, a seeded acceleration
    field, 1024 active particles in the automatic launch shape: 4 sampled
    particles against the oracle (FP64 1e-12 per component of |ref|; mixed
    1e-6 and EX 1e-12 of sum_j |T_ij|)."""
    nb = nb_gpu()
    m, x, v, a, eps, act, pick, ref, kap = large_system
    g = nb.NBody(m, x, v, eps, precision=prec, start_forces=False)
    g.set_state({"a": a})
    g.predict(0.0)
    got = g.evaluate(act)
    g.close()
    for gq, rq, kq in zip(got, ref, kap):
        if prec == 0:
            assert check_parity(0, gq[pick], rq) <= 1.0
        else:
            assert check_parity(1, gq[pick], rq, kq, tol_mixed=1e-6 if prec == 1 else 1e-12) <= 1.0
