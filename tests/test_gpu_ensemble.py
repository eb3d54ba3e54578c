"""Ensembles of independent systems in one persistent launch, against the
FP64 oracle run system by system."""
import numpy as np
import pytest

import nb_inputs as ni
import oracle as O
from nbhelp import check_parity, nb_gpu, rel_err

pytestmark = pytest.mark.gpu

SIZES = [2, 5, 33, 300, 1000, 64, 257]


def _systems(sizes, base_seed=40):
    ms, xs, vs = [], [], []
    for k, n in enumerate(sizes):
        m, x, v = ni.plummer(n, base_seed + k)
        ms.append(m)
        xs.append(x)
        vs.append(v)
    return ms, xs, vs


def _concat(ms, xs, vs):
    return np.concatenate(ms), np.concatenate(xs), np.concatenate(vs)


@pytest.mark.parametrize("prec, noise", [(0, 0.0), (3, 0.0), (0, 4e-7)])
def test_fp64_and_ex_ensembles_match_oracle_per_system(prec, noise):
    """FP64 and EX (double-word) ensembles take the oracle's step decisions
    system by system and end on its state to 1e-10; also with the step
    criterion's rounding floor (FP64, 4e-7 on both sides)."""
    nb = nb_gpu()
    ms, xs, vs = _systems(SIZES)
    eps, t_end = 1e-4, 0.125
    ens = nb.Ensemble(SIZES, *_concat(ms, xs, vs), eps, precision=prec, step_noise=noise)
    ens.run(t_end)
    st = ens.state()
    steps, inter, _ = ens.stats()
    ens.close()
    o = 0
    for k, n in enumerate(SIZES):
        ref = O.System(ms[k], xs[k], vs[k], eps, step_noise=noise)
        nsteps, _ = ref.run_until(t_end)
        sr = ref.state()
        assert steps[k] == nsteps, (k, steps[k], nsteps)
        for f in ("x", "v"):
            assert rel_err(st[f][o:o + n], sr[f]).max() < 1e-10, (k, f)
        np.testing.assert_array_equal(st["t"][o:o + n], sr["t"])
        np.testing.assert_array_equal(st["dt"][o:o + n], sr["dt"])
        o += n
    assert inter > 0


def test_fp64_ensemble_launch_shapes_agree():
    nb = nb_gpu()
    ms, xs, vs = _systems(SIZES, 60)
    out = []
    for g, thr in ((1, 256), (4, 128), (8, 256)):
        ens = nb.Ensemble(SIZES, *_concat(ms, xs, vs), 1e-4, dt_max=2.0 ** -5)
        ens.set_shape(g, thr)
        ens.run(2.0 ** -5, use_graph=(g != 4))
        out.append(ens.state())
        ens.close()
    for st in out[1:]:
        for f in ("x", "v", "a"):
            assert rel_err(st[f], out[0][f]).max() < 1e-12, f
        np.testing.assert_array_equal(st["t"], out[0]["t"])


@pytest.mark.parametrize("prec, tol_xv, noise", [(1, 1e-8, 0.0), (4, 1e-7, 0.0), (1, 1e-8, 4e-7)])
def test_mixed_ensembles_match_oracle_replay_per_system(prec, tol_xv, noise):
    """Mixed ensembles against the FP64 oracle, system by system.  FP32 pair
    arithmetic may move a step decision across a power of two (another valid
    trajectory), so the oracle replays each system's logged (t_next, active
    set) sequence, starting from its own start-up state (only the step
    decisions come from the GPU); then t must agree exactly, x and v per
    particle to tol_xv of |x|, |v|, and a and jerk to 1e-6 of each sum's
    condition number sum_j |T_ij| (on the oracle's final state; every
    particle is evaluated at t_end in the last step).  Snap takes the
    predicted accelerations as inputs, and their crackle term comes from the
    quintic interpolation, which divides the rounding of a, jerk and snap by
    h^3 (60 R1 / h^3) before the predictor multiplies it back by h^3 / 6:
    the predicted a carries about ten times the evaluation's relative
    rounding, so snap is held to 1e-5 of its condition number.
    The two start-up states differ by the mixed rounding of the starting
    forces (about 1e-7 of |a|), which the integration carries into v (|a| t
    of a few 1e-9 of |v| for the 5-body system's close pair at t = 2^-10):
    NB_MIXED (1), whose predictor and corrector are FP64, is held to 1e-8 in
    x and v; NB_MIXED32 (4) forms the corrector's increments in FP32 (about
    6e-8 of each increment): 1e-7.  The run is short (to t = 2^-10, block
    steps down to 2^-20), since the per-step force rounding of a few 1e-8
    grows along close encounters.  With a step-criterion noise floor
    (nb_config.step_noise) the decisions change, and the replay checks
    the same arithmetic along them."""
    nb = nb_gpu()
    sizes = [2, 5, 16, 33, 300, 64, 257]
    ms, xs, vs = _systems(sizes, 110)
    eps, t_end = 1e-4, 2.0 ** -10
    ens = nb.Ensemble(sizes, *_concat(ms, xs, vs), eps, precision=prec, dt_max=t_end, step_noise=noise)
    ens.set_log(1 << 20, 1 << 24)
    ens.run(t_end)
    st = ens.state()
    steps, _, _ = ens.stats()
    log, (n_steps, n_idx) = ens.log()
    ens.close()
    assert n_steps == int(steps.sum()) and n_steps <= 1 << 20 and n_idx <= 1 << 24
    small = large = 0
    o = 0
    for k, n in enumerate(sizes):
        sl = slice(o, o + n)
        o += n
        tn = [t for t, _ in log[k]]
        sets = [idx for _, idx in log[k]]
        assert len(tn) == steps[k] and all(q is not None for q in sets)
        assert all(np.all(np.diff(q) > 0) for q in sets) and tn == sorted(tn)
        small += sum(len(q) <= 16 for q in sets)
        large += sum(len(q) > 16 for q in sets)
        ref = O.System(ms[k], xs[k], vs[k], eps, dt_max=t_end)
        ref.replay(tn, sets)
        sr = ref.state()
        np.testing.assert_array_equal(st["t"][sl], sr["t"])
        assert np.all(sr["t"] == t_end)
        for f in ("x", "v"):
            assert rel_err(st[f][sl], sr[f]).max() < tol_xv, (k, f, rel_err(st[f][sl], sr[f]).max())
        kap = O.evaluate_kappa(ms[k], sr["x"], sr["v"], sr["a"], eps)
        for f, kq in zip(("a", "j", "s"), kap):
            tol = 1e-5 if f == "s" else 1e-6
            assert check_parity(1, st[f][sl], sr[f], kq, tol_mixed=tol) <= 1.0, (k, f)
    assert small > 0 and large > 0      # both evaluation paths of the persistent kernel ran


def test_mixed_ensemble_tracks_fp64_and_conserves_energy():
    nb = nb_gpu()
    sizes = [300, 1000, 64]
    ms, xs, vs = _systems(sizes, 80)
    eps, t_end = 1e-4, 0.125
    res = {}
    for prec in (nb.NB_FP64, nb.NB_MIXED, nb.NB_MIXED32):
        ens = nb.Ensemble(sizes, *_concat(ms, xs, vs), eps, precision=prec)
        ens.run(t_end)
        res[prec] = ens.state()
        ens.close()
    o = 0
    for k, n in enumerate(sizes):
        e0 = sum(O.energy(ms[k], xs[k], vs[k], eps))
        for prec in (nb.NB_FP64, nb.NB_MIXED, nb.NB_MIXED32):
            st = res[prec]
            e1 = sum(O.energy(ms[k], st["x"][o:o + n], st["v"][o:o + n], eps))
            assert abs((e1 - e0) / e0) < 1e-8, (k, prec)
        for prec in (nb.NB_MIXED, nb.NB_MIXED32):
            assert rel_err(res[prec]["x"][o:o + n], res[nb.NB_FP64]["x"][o:o + n]).max() < 1e-6
        o += n


def test_graph_replay_continues_the_integration():
    nb = nb_gpu()
    sizes = [33, 300]
    ms, xs, vs = _systems(sizes, 90)
    eps = 1e-4
    a = nb.Ensemble(sizes, *_concat(ms, xs, vs), eps)
    a.run(0.125)
    a.run(0.25)
    _, _, launches = a.stats()
    b = nb.Ensemble(sizes, *_concat(ms, xs, vs), eps)
    b.run(0.25, use_graph=False)
    sa, sb = a.state(), b.state()
    a.close()
    b.close()
    for f in ("x", "v", "a", "j", "s", "t", "dt"):
        np.testing.assert_array_equal(sa[f], sb[f])
    assert launches == 3  # start-up + two graph launches


def test_ex_ensemble_launch_shapes_agree_and_track_fp64():
    nb = nb_gpu()
    ms, xs, vs = _systems(SIZES, 70)
    out = []
    for g, thr in ((1, 128), (4, 128), (8, 64), (16, 64)):   # 16: non-portable cluster size
        ens = nb.Ensemble(SIZES, *_concat(ms, xs, vs), 1e-4, precision=nb.NB_EX, dt_max=2.0 ** -5)
        ens.set_shape(g, thr)
        ens.run(2.0 ** -5)
        out.append(ens.state())
        ens.close()
    ref = nb.Ensemble(SIZES, *_concat(ms, xs, vs), 1e-4, dt_max=2.0 ** -5)
    ref.run(2.0 ** -5)
    st64 = ref.state()
    ref.close()
    for st in out:
        for f in ("x", "v"):
            assert rel_err(st[f], out[0][f]).max() < 1e-12, f
            assert rel_err(st[f], st64[f]).max() < 1e-11, f
        np.testing.assert_array_equal(st["t"], st64["t"])


@pytest.mark.parametrize("prec", [0, 1, 3, 4])
def test_lone_particle_system_coasts_at_the_largest_step(prec):
    """A one-particle system feels no force: its step criterion is 0/0 and
    sets no bound, so it coasts in a straight line at dt_max (exactly, with
    dyadic inputs) beside systems that do interact."""
    nb = nb_gpu()
    ms, xs, vs = _systems([2, 33], 90)
    m1, x1, v1 = np.ones(1), np.array([[0.25, -0.5, 1.0]]), np.array([[0.5, 0.125, -1.0]])
    sizes = [1, 2, 33]
    ens = nb.Ensemble(sizes, *_concat([m1] + ms, [x1] + xs, [v1] + vs), 1e-4, precision=prec)
    ens.run(0.25)
    st = ens.state()
    steps, _, _ = ens.stats()
    ens.close()
    assert steps[0] == 2
    np.testing.assert_array_equal(st["x"][0], x1[0] + 0.25 * v1[0])
    np.testing.assert_array_equal(st["v"][0], v1[0])
    assert st["dt"][0] == 0.125 and st["t"][0] == 0.25
    assert np.isfinite(st["x"]).all() and (st["t"] == 0.25).all()


def test_full_size_ensemble_sampled_systems_match_oracle():
    """The 256-system ensemble at full size (N log-uniform in [256, 16384],
    1,004,043 particles, seeds as in the bench, eps = 1e-4) in EX at the
    library's default launch shape, to t = 1/4 in one persistent launch,
    with the step log on.  Sampled systems (the three smallest and those
    nearest 1000 and 2000 particles, so both the small-set and the large-set
    evaluation paths run): the oracle, run on its own, takes the same block
    steps (every logged time and active set), and ends on the same t and dt
    exactly and on x, v to 1e-10 (EX sums are within about 1e-13 of the FP64
    sums)."""
    nb = nb_gpu()
    eps, t_end = 1e-4, 0.25
    sizes = ni.ensemble_sizes(256, 4)
    parts = [ni.plummer(int(k), 1000 + q) for q, k in enumerate(sizes)]
    ens = nb.Ensemble(sizes, *[np.concatenate([p[f] for p in parts]) for f in range(3)], eps,
                      precision=nb.NB_EX)
    ens.set_log(1 << 20, 1 << 28)
    ens.run(t_end)
    st = ens.state()
    steps, _, _ = ens.stats()
    log, (n_steps, n_idx) = ens.log()
    ens.close()
    assert n_steps == int(steps.sum()) and n_idx <= 1 << 28
    order = np.argsort(sizes)
    pick = [int(order[0]), int(order[1]), int(order[2]), int(np.argmin(np.abs(sizes - 1000))),
            int(np.argmin(np.abs(sizes - 2000)))]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    for k in pick:
        sl = slice(int(offs[k]), int(offs[k + 1]))
        ref = O.System(*parts[k], eps)
        nsteps, (lt, ln, lh) = ref.run_until(t_end, log_cap=int(steps[k]) + 16)
        sr = ref.state()
        assert steps[k] == nsteps and len(log[k]) == nsteps, (k, steps[k], nsteps)
        assert all(idx is not None for _, idx in log[k])
        np.testing.assert_array_equal([t for t, _ in log[k]], lt)
        np.testing.assert_array_equal([len(idx) for _, idx in log[k]], ln)
        assert [O.set_hash(idx) for _, idx in log[k]] == [int(h) for h in lh], k
        np.testing.assert_array_equal(st["t"][sl], sr["t"])
        np.testing.assert_array_equal(st["dt"][sl], sr["dt"])
        for f in ("x", "v"):
            assert rel_err(st[f][sl], sr[f]).max() < 1e-10, (k, f, rel_err(st[f][sl], sr[f]).max())


def test_full_size_mixed_ensemble_with_rounding_floor():
    """The 256-system ensemble at full size in the mixed form (FP32 pair
    terms, FP64 prediction and correction) with the step criterion's
    rounding floor at 4e-7, the bench's configuration, to t = 1/4: the
    sampled systems (the three smallest, those nearest 1000 and 2000
    particles) end at t = 1/4 on power-of-two steps that divide it, take no
    more block steps than the oracle's own FP64 run of the same system, and
    conserve energy (the oracle's energy of the final state) to within ten
    times that FP64 run's error plus 2e-9 (measured: 1.3e-9 to 9.6e-9
    against 1.3e-10 to 5.7e-9 for FP64)."""
    nb = nb_gpu()
    eps, t_end = 1e-4, 0.25
    sizes = ni.ensemble_sizes(256, 4)
    parts = [ni.plummer(int(k), 1000 + q) for q, k in enumerate(sizes)]
    ens = nb.Ensemble(sizes, *[np.concatenate([p[f] for p in parts]) for f in range(3)], eps,
                      precision=nb.NB_MIXED, step_noise=4e-7)
    ens.run(t_end)
    st = ens.state()
    steps, _, _ = ens.stats()
    ens.close()
    order = np.argsort(sizes)
    pick = [int(order[0]), int(order[1]), int(order[2]), int(np.argmin(np.abs(sizes - 1000))),
            int(np.argmin(np.abs(sizes - 2000)))]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    for k in pick:
        sl = slice(int(offs[k]), int(offs[k + 1]))
        m, x, v = parts[k]
        assert np.all(st["t"][sl] == t_end)
        assert np.all(np.fmod(st["t"][sl], st["dt"][sl]) == 0.0)
        ref = O.System(m, x, v, eps)
        nsteps, _ = ref.run_until(t_end)
        sr = ref.state()
        E0 = sum(O.energy(m, x, v, eps))
        de_ref = abs((sum(O.energy(m, sr["x"], sr["v"], eps)) - E0) / E0)
        de = abs((sum(O.energy(m, st["x"][sl], st["v"][sl], eps)) - E0) / E0)
        assert steps[k] <= nsteps, (k, steps[k], nsteps)
        assert de <= 10 * de_ref + 2e-9, (k, de, de_ref)
