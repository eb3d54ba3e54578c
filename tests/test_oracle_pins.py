"""Pins for the FP64 CPU oracle: each check ties it to something other than
itself (symbolic derivatives, conservation laws, polynomial exactness,
closed forms, the analytic Kepler orbit), so that a dropped term, a wrong
sign or coefficient, or a transposed operand fails at least one of them.
"""
import math

import numpy as np
import pytest

import nb_inputs as ni
import oracle as O


# --------------------------------------------------------------- pair terms

def _sympy_pair(xi, vi, ai, xj, vj, aj, mj, eps):
    """acc, jerk, snap of a softened pair by symbolic differentiation of
    A(tau) = m r(tau) / (|r(tau)|^2 + eps^2)^(3/2) along
    r(tau) = dx + dv tau + da tau^2 / 2 (sympy, 40 digits)."""
    sp = pytest.importorskip("sympy")
    tau = sp.Symbol("tau")
    R = [sp.Rational(float(xj[k])) - sp.Rational(float(xi[k])) for k in range(3)]
    V = [sp.Rational(float(vj[k])) - sp.Rational(float(vi[k])) for k in range(3)]
    Acc = [sp.Rational(float(aj[k])) - sp.Rational(float(ai[k])) for k in range(3)]
    r = [R[k] + V[k] * tau + Acc[k] * tau ** 2 / 2 for k in range(3)]
    e2 = sp.Rational(float(eps)) ** 2
    den = (r[0] ** 2 + r[1] ** 2 + r[2] ** 2 + e2) ** sp.Rational(3, 2)
    m = sp.Rational(float(mj))
    out = []
    for order in range(3):
        out.append(np.array([float(sp.diff(m * r[k] / den, tau, order).subs(tau, 0).evalf(40))
                             for k in range(3)]))
    return out


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_pair_matches_symbolic_derivatives(seed):
    s = ni.random_state(6, seed)
    xi, vi, ai, xj, vj, aj = s
    mj, eps = 0.37, 0.05
    got = O.pair(xi, vi, ai, xj, vj, aj, mj, eps)
    ref = _sympy_pair(xi, vi, ai, xj, vj, aj, mj, eps)
    for g, r in zip(got, ref):
        np.testing.assert_allclose(g, r, rtol=1e-13, atol=1e-13 * np.abs(r).max())


def test_pair_self_term_is_zero_and_antisymmetric():
    s = ni.random_state(6, 11)
    xi, vi, ai, xj, vj, aj = s
    for q in O.pair(xi, vi, ai, xi, vi, ai, 1.0, 1e-4):
        assert np.all(q == 0.0)
    mi, mj = 0.3, 0.7
    f_ij = O.pair(xi, vi, ai, xj, vj, aj, mj, 0.01)
    f_ji = O.pair(xj, vj, aj, xi, vi, ai, mi, 0.01)
    for a, b in zip(f_ij, f_ji):
        np.testing.assert_allclose(mi * a, -mj * b, rtol=1e-14, atol=1e-15)


# ------------------------------------------------------------ evaluation sum

@pytest.mark.parametrize("lam,tau", [(2.0, 4.0), (0.25, 0.5), (8.0, 0.125)])
def test_units_scaling_law_is_exact(lam, tau):
    """Change of units x -> lam x, t -> tau t (G = 1 kept, so m -> lam^3 /
    tau^2 m, and eps -> lam eps): acc, jerk and snap scale by lam / tau^2,
    lam / tau^3 and lam / tau^4.  With powers of two every rounding scales
    too, so the identity holds bit for bit; a wrong power of q or a
    misplaced factor in any term breaks it."""
    n, eps = 64, 1e-3
    m, x, v = ni.plummer(n, 41, imf="salpeter")
    a = ni.random_state(n, 42, scale=2.0)
    act = ni.active_subset(n, 17, 43)
    ref = O.evaluate(m, x, v, a, eps, act)
    got = O.evaluate(m * lam ** 3 / tau ** 2, x * lam, v * lam / tau, a * lam / tau ** 2,
                     eps * lam, act)
    for k, (g, r) in enumerate(zip(got, ref)):
        np.testing.assert_array_equal(g, r * lam / tau ** (2 + k))


def test_newton_third_law_for_acc_jerk_snap():
    m, x, v = ni.plummer(256, 5, imf="salpeter")
    a = ni.random_state(256, 6)
    acc, jrk, snp = O.evaluate(m, x, v, a, 1e-4)
    for q in (acc, jrk, snp):
        tot = (m[:, None] * q).sum(axis=0)
        scale = (m[:, None] * np.abs(q)).sum()
        assert np.all(np.abs(tot) < 1e-13 * scale)


def test_evaluate_equals_sum_of_pairs_and_skips_self():
    m, x, v = ni.plummer(9, 3)
    a = ni.random_state(9, 4)
    act = np.array([0, 4, 8], dtype=np.int32)
    acc, jrk, snp = O.evaluate(m, x, v, a, 1e-3, act)
    for k, i in enumerate(act):
        tot = [np.zeros(3) for _ in range(3)]
        for j in range(9):
            if j != i:
                for q, t in zip(O.pair(x[i], v[i], a[i], x[j], v[j], a[j], m[j], 1e-3), tot):
                    t += q
        np.testing.assert_allclose(acc[k], tot[0], rtol=1e-13)
        np.testing.assert_allclose(jrk[k], tot[1], rtol=1e-13)
        np.testing.assert_allclose(snp[k], tot[2], rtol=1e-13)


def test_compensated_sum_survives_cancellation():
    """Antipodal pairs around particle 0, in shuffled order, cancel exactly;
    one faint distant particle leaves a result far below the terms' size.
    The oracle's compensated sums must equal the correctly rounded sum of
    its own pair terms (math.fsum) within the error bound of compensated
    summation, 2u|S| + n u^2 sum|x_i| (Higham, Accuracy and Stability of
    Numerical Algorithms, section 4.3), which plain left-to-right summation
    exceeds by orders of magnitude."""
    rng = np.random.default_rng(51)
    k = 100
    d = rng.standard_normal((k, 3)) * rng.uniform(0.5, 2.0, (k, 1))
    xs = np.concatenate([d, -d, [[40.0, 30.0, 0.0]]])
    vs = np.concatenate([rng.standard_normal((k, 3)), np.zeros((k + 1, 3))])
    vs[k:2 * k] = -vs[:k]                                 # antipodal velocities too
    vs[-1] = [0.1, -0.2, 0.3]                             # the faint particle moves
    ms = np.concatenate([rng.uniform(0.5, 1.5, k), np.zeros(k + 1)])
    ms[k:2 * k] = ms[:k]
    ms[-1] = 1e-6
    order = rng.permutation(xs.shape[0])
    x = np.concatenate([[[0.0, 0.0, 0.0]], xs[order]])
    v = np.concatenate([[[0.0, 0.0, 0.0]], vs[order]])
    m = np.concatenate([[1.0], ms[order]])
    a = np.zeros_like(x)
    got = O.evaluate(m, x, v, a, 1e-3, [0])
    terms = [O.pair(x[0], v[0], a[0], x[j], v[j], a[j], m[j], 1e-3) for j in range(1, m.size)]
    u, n = 2.0 ** -53, len(terms)
    for q in range(3):
        exact = np.array([math.fsum(t[q][c] for t in terms) for c in range(3)])
        total = np.array([math.fsum(abs(t[q][c]) for t in terms) for c in range(3)])
        naive = np.zeros(3)
        for t in terms:
            naive += t[q]
        bound = 2 * u * np.abs(exact) + n * u * u * total
        assert np.abs(exact).max() > 0
        assert np.all(np.abs(got[q][0] - exact) <= bound), q
        assert np.abs(naive - exact).max() > 100 * bound.max(), q


def test_jerk_and_snap_are_time_derivatives_of_acc():
    """Along x_k(tau) = x_k + v_k tau + a_k tau^2 / 2 for every particle,
    jerk_i = d acc_i / d tau and snap_i = d^2 acc_i / d tau^2 at tau = 0
    (5-point central differences, h = 2^-10)."""
    n = 48
    m, x, v = ni.plummer(n, 7)
    a0, _, _ = O.evaluate(m, x, v, np.zeros((n, 3)), 1e-2)
    acc, jrk, snp = O.evaluate(m, x, v, a0, 1e-2)
    h = 2.0 ** -10

    def acc_at(tau):
        return O.evaluate(m, x + v * tau + a0 * tau * tau / 2, v, a0, 1e-2)[0]

    Am2, Am1, A0, Ap1, Ap2 = (acc_at(k * h) for k in (-2, -1, 0, 1, 2))
    d1 = (Am2 - 8 * Am1 + 8 * Ap1 - Ap2) / (12 * h)
    d2 = (-Am2 + 16 * Am1 - 30 * A0 + 16 * Ap1 - Ap2) / (12 * h * h)
    np.testing.assert_allclose(A0, acc, rtol=0, atol=0)
    for got, fd in ((jrk, d1), (snp, d2)):
        err = np.abs(got - fd).max(axis=1) / np.linalg.norm(got, axis=1)
        assert err.max() < 1e-6, err.max()


def test_kappa_bounds_the_sum_and_equals_it_without_cancellation():
    m, x, v = ni.plummer(64, 13)
    a = ni.random_state(64, 14)
    act = np.arange(0, 64, 5, dtype=np.int32)
    sums = O.evaluate(m, x, v, a, 1e-3, act)
    kap = O.evaluate_kappa(m, x, v, a, 1e-3, act)
    for s_, k_ in zip(sums, kap):
        assert np.all(np.linalg.norm(s_, axis=1) <= k_ * (1 + 1e-14))
    # two bodies: one term, no cancellation
    ka, kj, ks = O.evaluate_kappa(m[:2], x[:2], v[:2], a[:2], 1e-3, [0])
    A, J, S = O.pair(x[0], v[0], a[0], x[1], v[1], a[1], m[1], 1e-3)
    assert ka[0] == pytest.approx(np.linalg.norm(A), rel=1e-15)
    assert kj[0] == pytest.approx(np.linalg.norm(J), rel=1e-15)
    assert ks[0] == pytest.approx(np.linalg.norm(S), rel=1e-15)
    # a particle at the centre of a symmetric cube of 8 equal masses at rest:
    # the acceleration cancels exactly while kappa is 8 |A_one|
    xc = np.array([[0.0, 0.0, 0.0]] + [[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1)
                                        for sz in (-1, 1)])
    mc = np.ones(9)
    zero = np.zeros((9, 3))
    acc = O.evaluate(mc, xc, zero, zero, 1e-3, [0])[0]
    ka = O.evaluate_kappa(mc, xc, zero, zero, 1e-3, [0])[0]
    assert np.abs(acc).max() < 1e-15
    assert ka[0] == pytest.approx(8 * math.sqrt(3) / (3 + 1e-6) ** 1.5, rel=1e-12)


# ------------------------------------------------------------- polynomials

def _poly_state(coef, t):
    """value and first 5 derivatives of the vector polynomial sum coef[k] t^k."""
    out = []
    c = [np.polynomial.Polynomial(coef[:, d]) for d in range(3)]
    for order in range(8):
        out.append(np.array([p.deriv(order)(t) if order else p(t) for p in c]))
    return out


def test_predictor_exact_for_quintic_trajectories():
    rng_coef = ni.random_state(6, 21)
    ti = np.array([0.25, 0.5])
    t = 0.75
    xs, vs, as_, js, ss, cs = [], [], [], [], [], []
    for k in range(2):
        st = _poly_state(rng_coef * (k + 1), ti[k])
        for lst, q in zip((xs, vs, as_, js, ss, cs), st[:6]):
            lst.append(q)
    xp, vp, ap = O.predict(t, ti, *(np.array(q) for q in (xs, vs, as_, js, ss, cs)))
    for k in range(2):
        st = _poly_state(rng_coef * (k + 1), t)
        np.testing.assert_allclose(xp[k], st[0], rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(vp[k], st[1], rtol=1e-14, atol=1e-14)
        np.testing.assert_allclose(ap[k], st[2], rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("seed", [31, 32])
def test_corrector_exact_for_degree6_positions(seed):
    coef = ni.random_state(7, seed)
    h = 0.125
    s0 = _poly_state(coef, 0.0)
    s1 = _poly_state(coef, h)
    x1, v1 = O.correct(h, s0[0], s0[1], s0[2], s0[3], s0[4], s1[2], s1[3], s1[4])
    np.testing.assert_allclose(v1, s1[1], rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(x1, s1[0], rtol=1e-14, atol=1e-14)


def test_corrector_velocity_exact_for_degree7_and_position_not():
    coef = np.zeros((8, 3))
    coef[7] = [1.0, -2.0, 0.5]
    h = 0.5
    s0 = _poly_state(coef, 0.0)
    s1 = _poly_state(coef, h)
    x1, v1 = O.correct(h, s0[0], s0[1], s0[2], s0[3], s0[4], s1[2], s1[3], s1[4])
    np.testing.assert_allclose(v1, s1[1], rtol=1e-14, atol=1e-14)
    # the position quadrature integrates v = 7 t^6 with an h^7 error term
    assert np.all(np.abs(x1 - s1[0]) > 1e-6 * np.abs(s1[0]))


@pytest.mark.parametrize("seed,h", [(41, 0.125), (42, 0.5), (43, 1.0), (44, 2.0 ** -10)])
def test_interpolation_exact_for_quintic_acceleration(seed, h):
    """Exact for a(t) of degree 5.  The k-th derivative is recovered from
    differences of O(|a|) values divided by h^k, so rounding alone bounds its
    accuracy by about eps_mach |a| / h^k; the tolerance follows that."""
    coef = np.zeros((8, 3))
    coef[2:8] = ni.random_state(6, seed)  # x of degree 7 -> a of degree 5
    s0 = _poly_state(coef, 0.0)
    s1 = _poly_state(coef, h)
    c1, d1, e1 = O.interpolate(h, s0[2], s0[3], s0[4], s1[2], s1[3], s1[4])
    scale = np.abs(np.concatenate([s0[2], s1[2]])).max()
    for k, (got, ref) in zip((3, 4, 5), ((c1, s1[5]), (d1, s1[6]), (e1, s1[7]))):
        tol = 1e-13 * np.abs(ref).max() + 1e3 * 2.2e-16 * scale / h ** k
        assert np.abs(got - ref).max() < tol, (k, np.abs(got - ref).max(), tol)


# --------------------------------------------------------------- time steps

def test_aarseth_criterion_on_circular_motion():
    """x = R (cos wt, sin wt, 0): |a^(k)| = R w^(k+2), so A1 = 2 R w^3,
    A4 = 2 R w^6 and the 6th-order criterion gives exactly eta / w."""
    R, w, t, eta = 1.7, 3.0, 0.3, 0.4

    def deriv(k):
        ph = w * t + k * math.pi / 2
        return R * w ** k * np.array([math.cos(ph), math.sin(ph), 0.0])

    a, j, s, c, d, e = (deriv(k) for k in range(2, 8))
    assert O.dt_crit(eta, a, j, s, c, d, e) == pytest.approx(eta / w, rel=1e-14)


def test_initial_step():
    a = np.array([2.0, 0, 0])
    j = np.array([0, 4.0, 0])
    s = np.array([0, 0, 1.0])
    assert O.dt_initial(0.01, a, j, s) == pytest.approx(0.01 * 0.5, rel=1e-15)
    s = np.array([0, 0, 32.0])
    assert O.dt_initial(0.01, a, j, s) == pytest.approx(0.01 * 0.25, rel=1e-15)


def test_no_force_sets_no_bound():
    """A particle under no force (every derivative exactly zero) gives the
    ratios 0/0: no bound, so the quantised step is dt_max and no floor hit.
    A zero acceleration beside a non-zero jerk still gives the bound 0."""
    z = np.zeros(3)
    assert O.dt_crit(0.4, z, z, z, z, z, z) == math.inf
    assert O.dt_initial(0.01, z, z, z) == math.inf
    assert O.dt_quantise(math.inf, -1, 0.0) == (0.125, False)
    assert O.dt_initial(0.01, z, np.array([0, 1.0, 0]), z) == 0.0
    # one ratio 0/0, the other a real bound: the real bound is taken
    a, s = np.array([4.0, 0, 0]), np.array([0, 0, 1.0])
    assert O.dt_initial(0.01, a, z, s) == pytest.approx(0.02, rel=1e-15)


def test_lone_particle_coasts_at_the_largest_step():
    """N = 1: no force, so straight-line motion at dt_max, exactly."""
    x0, v0 = np.array([[0.25, -0.5, 1.0]]), np.array([[0.5, 0.125, -1.0]])
    sys1 = O.System(np.ones(1), x0, v0, 1e-4)
    steps, _ = sys1.run_until(0.5)
    st = sys1.state()
    assert steps == 4 and sys1.floor_hits == 0
    np.testing.assert_array_equal(st["dt"], [0.125])
    np.testing.assert_array_equal(st["x"], x0 + 0.5 * v0)
    np.testing.assert_array_equal(st["v"], v0)


@pytest.mark.parametrize("crit,old,t1,want,hit", [
    (0.3, -1, 0.0, 0.125, False),          # clamp to dt_max
    (float("inf"), -1, 0.0, 0.125, False),  # unbounded criterion -> dt_max
    (0.001, -1, 0.0, 2.0 ** -10, False),   # largest power of two below
    (2.0 ** -7, -1, 0.0, 2.0 ** -7, False),  # exact power of two is kept
    (1e-9, -1, 0.0, 2.0 ** -20, True),     # floor
    (float("nan"), 2.0 ** -5, 0.0, 2.0 ** -20, True),
    (1.0, 2.0 ** -10, 3 * 2.0 ** -10, 2.0 ** -10, False),  # t1 not commensurate
    (1.0, 2.0 ** -10, 4 * 2.0 ** -10, 2.0 ** -9, False),   # at most doubled
    (2.0 ** -12 * 1.5, 2.0 ** -5, 0.5, 2.0 ** -12, False),  # any decrease allowed
])
def test_quantise_table(crit, old, t1, want, hit):
    got, h = O.dt_quantise(crit, old, t1)
    assert got == want and h == hit


# --------------------------------------------------------------- diagnostics

def test_energy_two_body_closed_form_and_plummer_virial():
    m = np.array([0.25, 0.75])
    x = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    v = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    ek, ep = O.energy(m, x, v, 0.0)
    assert ek == pytest.approx(0.5 * 0.25 + 0.5 * 0.75 * 4.0, rel=1e-15)
    assert ep == pytest.approx(-0.25 * 0.75 / 5.0, rel=1e-15)
    m, x, v = ni.plummer(1024, 1)
    ek, ep = O.energy(m, x, v, 1e-4)
    assert abs(ek + ep + 0.25) < 0.02 and abs(ek / -ep - 0.5) < 0.03


def test_angular_momentum_two_body():
    m = np.array([1.0, 2.0])
    x = np.array([[1.0, 0, 0], [0, 1.0, 0]])
    v = np.array([[0, 1.0, 0], [0, 0, 3.0]])
    L, la = O.angmom(m, x, v)
    np.testing.assert_allclose(L, [6.0, 0.0, 1.0])
    assert la == pytest.approx(7.0)


# ------------------------------------------------------------------- Kepler

def kepler_state(t, m1=0.5, m2=0.5, a=1.0, e=0.5):
    """Two bodies on an ellipse (G = 1), pericentre at t = 0, analytic."""
    mu = m1 + m2
    n = math.sqrt(mu / a ** 3)
    M = n * t
    E = M
    for _ in range(60):
        E -= (E - e * math.sin(E) - M) / (1 - e * math.cos(E))
    dE = n / (1 - e * math.cos(E))
    b = a * math.sqrt(1 - e * e)
    r = np.array([a * (math.cos(E) - e), b * math.sin(E), 0.0])
    u = np.array([-a * math.sin(E) * dE, b * math.cos(E) * dE, 0.0])
    x = np.array([-m2 / mu * r, m1 / mu * r])
    v = np.array([-m2 / mu * u, m1 / mu * u])
    return np.array([m1, m2]), x, v


def _kepler_error(dt, T):
    m, x, v = kepler_state(0.0)
    s = O.System(m, x, v, 1e-12, dt_shared=dt, dt_max=dt)
    s.run_until(T)
    st = s.state()
    _, xr, vr = kepler_state(T)
    return np.abs(st["x"] - xr).max()


def test_kepler_matches_analytic_orbit_with_sixth_order_convergence():
    T = 2.0
    errs = [_kepler_error(2.0 ** -k, T) for k in (5, 6, 7)]
    assert errs[2] < 1e-9
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    for p in orders:
        assert 5.5 < p < 6.6, orders


def test_kepler_energy_over_an_orbit():
    m, x, v = kepler_state(0.0)
    s = O.System(m, x, v, 1e-12, dt_shared=2.0 ** -10, dt_max=2.0 ** -10)
    E0 = sum(O.energy(m, x, v, 1e-12))
    s.run_until(8.0)
    st = s.state()
    E1 = sum(O.energy(m, st["x"], st["v"], 1e-12))
    assert abs((E1 - E0) / E0) < 1e-12


def test_kepler_block_steps_follow_analytic_orbit():
    m, x, v = kepler_state(0.0)
    s = O.System(m, x, v, 1e-12, eta=0.1)
    s.run_until(2.0)
    st = s.state()
    _, xr, _ = kepler_state(2.0)
    assert np.abs(st["x"] - xr).max() < 1e-7


# ------------------------------------------------------------ block stepping

def test_block_step_invariants_and_plummer_energy():
    m, x, v = ni.plummer(1024, 1)
    eps = 1e-4
    E0 = sum(O.energy(m, x, v, eps))
    s = O.System(m, x, v, eps)
    steps, (lt, ln, lh) = s.run_until(0.125, log_cap=100000)
    assert steps == lt.size and np.all(ln >= 1) and np.all(np.diff(lt) > 0)
    st = s.state()
    dt = st["dt"]
    assert np.all(st["t"] == 0.125)
    k = np.log2(dt)
    assert np.all(k == np.round(k)) and dt.min() >= 2.0 ** -20 and dt.max() <= 0.125
    assert np.all(np.mod(st["t"], dt) == 0.0)
    E1 = sum(O.energy(m, st["x"], st["v"], eps))
    assert abs((E1 - E0) / E0) < 1e-9


def test_shared_mode_activates_everyone_and_hash_is_sum_of_mixes():
    m, x, v = ni.plummer(32, 2)
    s = O.System(m, x, v, 1e-3, dt_shared=2.0 ** -8)
    t, na, h = s.step()
    assert t == 2.0 ** -8 and na == 32
    assert h == O.set_hash(range(32))


def test_replay_of_own_log_reproduces_state():
    m, x, v = ni.plummer(64, 9)
    a = O.System(m, x, v, 1e-3)
    b = O.System(m, x, v, 1e-3)
    tn, sets = [], []
    for _ in range(12):
        before = a.state()
        t, na, h = a.step()
        due = np.nonzero(before["t"] + before["dt"] == t)[0]
        assert due.size == na and O.set_hash(due) == h
        tn.append(t)
        sets.append(due)
    b.replay(tn, sets)
    sa, sb = a.state(), b.state()
    for k in ("x", "v", "a", "j", "s", "c", "t"):
        np.testing.assert_array_equal(sa[k], sb[k])


# ------------------------------------- step criterion with rounding floors
#
# The floors (orc_interp_floor) bound how far the interpolated crackle, pop
# and a^(5) move when each input vector carries a relative error up to
# `noise`.  They are pinned here against the interpolation itself, which is
# pinned above (exact on quintics): its response to single inputs gives the
# linear maps the floors must reproduce.

_SLOTS = ("a0", "j0", "s0", "a1", "j1", "s1")


def _responses(h):
    """Per input slot, the interpolation's response (c1, d1, e1) to that
    input alone set to the unit vector along x: a [6][3] array."""
    out = np.zeros((6, 3))
    for k in range(6):
        ins = [np.zeros(3) for _ in range(6)]
        ins[k][0] = 1.0
        c, d, e = O.interpolate(h, *ins)
        out[k] = c[0], d[0], e[0]
    return out


def _rand_inputs(rng, scale=1.0):
    return [rng.normal(size=3) * scale * 10.0 ** rng.uniform(-3, 3) for _ in range(6)]


def test_floor_is_zero_without_noise_and_the_criterion_reduces():
    rng = np.random.default_rng(61)
    for _ in range(200):
        h = 2.0 ** -int(rng.integers(3, 21))
        ins = _rand_inputs(rng)
        fl = O.interp_floor(0.0, h, *ins)
        assert np.all(fl == 0.0)
        a, j, s, c, d, e = _rand_inputs(rng)
        assert O.dt_crit_floored(0.4, a, j, s, c, d, e, fl) == O.dt_crit(0.4, a, j, s, c, d, e)


@pytest.mark.parametrize("h", [2.0 ** -3, 2.0 ** -11, 2.0 ** -20])
def test_floor_is_tight_for_inputs_of_one_residual(h):
    """a0 and a1 enter only the first residual, j1 only the second, s1 only
    the third: with that input alone, of norm L, the worst error (noise L
    along the input) moves (c1, d1, e1) by exactly the floors."""
    resp = _responses(h)
    rng = np.random.default_rng(62)
    noise = 4e-7
    for slot in (0, 3, 4, 5):
        for L in (1e-3, 1.0, 7.5e4):
            u = rng.normal(size=3)
            ins = [np.zeros(3) for _ in range(6)]
            ins[slot] = L * u / np.linalg.norm(u)
            fl = O.interp_floor(noise, h, *ins)
            np.testing.assert_allclose(fl, np.abs(resp[slot]) * noise * L, rtol=1e-12, atol=0)


@pytest.mark.parametrize("h", [2.0 ** -3, 2.0 ** -11, 2.0 ** -20])
def test_floor_propagates_independent_residual_bounds(h):
    """Every input, alone: its coefficients in the three residuals follow
    from the interpolation (its response solved against the responses to the
    residuals alone, i.e. to a1, j1 / h, s1 / h^2), each residual's error is
    bounded by noise times |coefficient| times the input's norm, and the
    floors are those bounds through the absolute values of the map from
    residuals to (c1, d1, e1).  Over several inputs at once the floors add."""
    resp = _responses(h)
    G = np.stack([resp[3], resp[4] / h, resp[5] / (h * h)], axis=1)   # [3 outputs][3 residuals]
    noise = 1e-6
    rng = np.random.default_rng(63)
    total = np.zeros(3)
    ins_all = [np.zeros(3) for _ in range(6)]
    for slot in range(6):
        coef = np.linalg.solve(G, resp[slot])
        L = 10.0 ** rng.uniform(-2, 2)
        ins = [np.zeros(3) for _ in range(6)]
        ins[slot] = L * rng.normal(size=3)
        ins[slot] *= L / np.linalg.norm(ins[slot])
        ins_all[slot] = ins[slot]
        want = np.abs(G) @ (noise * np.abs(coef) * L)
        fl = O.interp_floor(noise, h, *ins)
        np.testing.assert_allclose(fl, want, rtol=1e-10, atol=0)
        total += fl
    np.testing.assert_allclose(O.interp_floor(noise, h, *ins_all), total, rtol=1e-12, atol=0)


def test_floor_bounds_every_perturbation_within_the_noise():
    """Random inputs, each input vector moved by a random vector of norm up
    to noise times its own: the interpolated derivatives move by no more
    than the floors (vector norms), and aligned moves come close to them."""
    rng = np.random.default_rng(64)
    noise = 1e-6
    worst = 0.0
    for _ in range(400):
        h = 2.0 ** -int(rng.integers(3, 21))
        ins = _rand_inputs(rng)
        pert = []
        for q in ins:
            dq = rng.normal(size=3)
            pert.append(q + dq / np.linalg.norm(dq) * noise * np.linalg.norm(q) * rng.uniform())
        fl = O.interp_floor(noise, h, *pert)
        base = O.interpolate(h, *ins)
        moved = O.interpolate(h, *pert)
        for b, m_, f in zip(base, moved, fl):
            r = np.linalg.norm(m_ - b) / f
            assert r <= 1.0 + 1e-6
            worst = max(worst, r)
    assert worst > 0.05


def test_floored_criterion_discounts_only_what_is_below_the_floor():
    """Exact constant-snap motion (all residuals zero) with every input moved
    by up to noise of its norm: the derivatives the interpolation then shows
    are rounding only, the floored criterion sets no bound, while the plain
    criterion (and the floored one at 1e-4 of the noise) does."""
    rng = np.random.default_rng(65)
    noise = 1e-6
    for _ in range(100):
        h = 2.0 ** -int(rng.integers(3, 21))
        a0, j0, s0 = (rng.normal(size=3) for _ in range(3))
        a1, j1, s1 = a0 + j0 * h + s0 * h * h / 2, j0 + s0 * h, s0.copy()
        ins = []
        for q in (a0, j0, s0, a1, j1, s1):
            dq = rng.normal(size=3)
            ins.append(q + dq / np.linalg.norm(dq) * 0.9 * noise * np.linalg.norm(q))
        c, d, e = O.interpolate(h, *ins)
        a, j, s = ins[3:]
        assert math.isfinite(O.dt_crit(0.4, a, j, s, c, d, e))
        assert O.dt_crit_floored(0.4, a, j, s, c, d, e, O.interp_floor(noise, h, *ins)) == math.inf
        assert math.isfinite(O.dt_crit_floored(0.4, a, j, s, c, d, e,
                                               O.interp_floor(noise * 1e-4, h, *ins)))


def test_block_steps_with_rounding_floors():
    """The integrator with floors (4e-7, the level set for FP32 pair terms):
    the run ends with every particle at t_end on steps that are powers of two
    dividing t, takes no more block steps than without floors, conserves
    energy as well, and noise = 0 is the criterion as is."""
    m, x, v = ni.plummer(256, 12)
    eps = 1e-4
    E0 = sum(O.energy(m, x, v, eps))
    plain = O.System(m, x, v, eps)
    zero = O.System(m, x, v, eps, step_noise=0.0)
    n_plain, (lt0, _, lh0) = plain.run_until(0.125, log_cap=1 << 16)
    n_zero, (lt1, _, lh1) = zero.run_until(0.125, log_cap=1 << 16)
    assert n_zero == n_plain and np.all(lt0 == lt1) and np.all(lh0 == lh1)
    fl = O.System(m, x, v, eps, step_noise=4e-7)
    n_fl, _ = fl.run_until(0.125)
    st = fl.state()
    assert np.all(st["t"] == 0.125) and np.all(np.mod(st["t"], st["dt"]) == 0.0)
    k = np.log2(st["dt"])
    assert np.all(k == np.round(k))
    assert n_fl <= n_plain
    E1 = sum(O.energy(m, st["x"], st["v"], eps))
    assert abs((E1 - E0) / E0) < 1e-9
