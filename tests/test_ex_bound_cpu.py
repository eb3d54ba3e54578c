"""Where the EX parity bound comes from: a float32 emulation of the
double-word operation sequence of the extended-precision pair term (TwoSum,
Fast2Sum and FMA TwoProd on FP32 numbers, unnormalised intermediates, the
accurate sum for position differences, one Newton step on an rsqrt estimate
carrying 2^-22 relative error) against the FP64 oracle on the
double-word-rounded inputs.  The GPU parity tests hold the kernel to
1e-12 sum_j |T_ij|; the emulated sequence stays below 2.5e-13 of it, close to
the origin or 100 units away (no dependence on the position scale).

The emulation is written here from the published transformations; it shares
nothing with the CUDA source.  fma(a, b, c) is emulated as the FP64 sum of
the exact product of two FP32 numbers and c, rounded to FP32."""
import numpy as np
import pytest

import nb_inputs as ni
import oracle as O

F = np.float32


def f32(x):
    return np.asarray(x, dtype=np.float32)


def add(a, b):
    return f32(a + b)


def sub(a, b):
    return f32(a - b)


def mul(a, b):
    return f32(a * b)


def fma(a, b, c):
    return f32(a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64))


def two_sum(a, b):
    s = add(a, b)
    bb = sub(s, a)
    return s, add(sub(a, sub(s, bb)), sub(b, bb))


def fast_two_sum(a, b):
    s = add(a, b)
    return s, sub(b, sub(s, a))


def dw_add(x, y):           # sloppy sum, unnormalised result
    s, e = two_sum(x[0], y[0])
    return s, add(e, add(x[1], y[1]))


def dw_add_accurate(x, y):  # both parts through TwoSum
    sh, sl = two_sum(x[0], y[0])
    th, tl = two_sum(x[1], y[1])
    vh, vl = fast_two_sum(sh, add(sl, th))
    return vh, add(tl, vl)


def dw_mul(x, y):
    p = mul(x[0], y[0])
    e = fma(x[1], y[0], fma(x[0], y[1], fma(x[0], y[0], -p)))
    return p, e


def dw_mulc(x, c):
    p = mul(x[0], c)
    return p, fma(x[1], c, fma(x[0], c, -p))


def dw_sqr(x):
    p = mul(x[0], x[0])
    return p, fma(add(x[0], x[0]), x[1], fma(x[0], x[0], -p))


def dw_mad(x, y, z):
    p, e = dw_mul(x, y)
    s, t = two_sum(p, z[0])
    return s, add(t, add(e, z[1]))


def dw_rsqrt(r, rng):
    q0 = f32(1.0 / np.sqrt(r[0].astype(np.float64)))
    q0 = f32(q0 * (1.0 + (rng.random(q0.shape) - 0.5) * 2.0 ** -22))   # estimate error
    t = dw_mul(r, (mul(q0, q0), fma(q0, q0, -mul(q0, q0))))
    d = sub(sub(F(1.0), t[0]), t[1])
    return fast_two_sum(q0, mul(mul(q0, d), F(0.5)))


def split(q):
    q = np.asarray(q, dtype=np.float64)
    h = f32(q)
    return h, f32(q - h.astype(np.float64))


def value(x):
    return x[0].astype(np.float64) + x[1].astype(np.float64)


def emulate(m, x, v, a, eps, act, seed=1):
    """acc, jerk, snap of the listed particles, emulated double words."""
    rng = np.random.default_rng(seed)
    n = m.size
    xs = [split(x[:, d]) for d in range(3)]
    vs = [split(v[:, d]) for d in range(3)]
    as_ = [split(a[:, d]) for d in range(3)]
    ms = split(m)
    e2 = tuple(np.full(n, c, dtype=np.float32) for c in split(np.float64(eps) ** 2))
    out = np.zeros((3, len(act), 3))
    m3, two = F(-3.0), F(2.0)
    for k, i in enumerate(act):
        def neg(s):
            return np.full(n, -s[0][i], dtype=np.float32), np.full(n, -s[1][i], dtype=np.float32)
        r = [dw_add_accurate(xs[d], neg(xs[d])) for d in range(3)]
        dv = [dw_add(vs[d], neg(vs[d])) for d in range(3)]
        da = [dw_add(as_[d], neg(as_[d])) for d in range(3)]
        R = dw_mad(r[0], r[0], dw_mad(r[1], r[1], dw_mad(r[2], r[2], e2)))
        rv = dw_mad(r[0], dv[0], dw_mad(r[1], dv[1], dw_mul(r[2], dv[2])))
        sv = dw_mad(r[0], da[0], dw_mad(r[1], da[1], dw_mad(r[2], da[2], dw_mad(
            dv[0], dv[0], dw_mad(dv[1], dv[1], dw_sqr(dv[2]))))))
        q = dw_rsqrt(R, rng)
        q2 = dw_sqr(q)
        mu = dw_mul(dw_mul(ms, q), q2)
        al = dw_mul(rv, q2)
        be = dw_mad(al, al, dw_mul(sv, q2))
        na3 = dw_mulc(al, m3)
        na6 = (mul(na3[0], two), mul(na3[1], two))
        nb3 = dw_mulc(be, m3)
        for d in range(3):
            u = dw_mad(na3, r[d], dv[d])
            w = dw_mad(na6, u, dw_mad(nb3, r[d], da[d]))
            for o, t in enumerate((r[d], u, w)):
                out[o, k, d] = value(dw_mul(mu, t)).sum()
    return out


@pytest.mark.parametrize("offset", [0.0, 100.0])
def test_emulated_ex_sequence_is_within_a_quarter_of_the_parity_bound(offset):
    n, eps = 300, 1e-4
    m, x, v = ni.plummer(n, 17, imf="salpeter")
    x = x + offset
    a = ni.random_state(n, 117, scale=2.0)
    act = ni.active_subset(n, 24, 3)
    rnd = lambda q: value(split(q))
    mr, xr, vr, ar = rnd(m), rnd(x), rnd(v), rnd(a)
    got = emulate(mr, xr, vr, ar, eps, act)
    ref = O.evaluate(mr, xr, vr, ar, eps, act)
    kap = O.evaluate_kappa(mr, xr, vr, ar, eps, act)
    for o in range(3):
        ratio = (np.abs(got[o] - ref[o]).max(axis=1) / kap[o]).max()
        assert ratio < 2.5e-13, (o, ratio)


def test_plain_sloppy_position_difference_would_not_be_enough():
    """With the sloppy sum for the position differences too, the error grows
    with the distance from the origin (2^-48 |x| / |r|), which is why the
    accurate sum is used there."""
    n, eps = 200, 1e-4
    m, x, v = ni.plummer(n, 18)
    x = x + 100.0
    a = ni.random_state(n, 118, scale=2.0)
    act = ni.active_subset(n, 12, 4)
    rnd = lambda q: value(split(q))
    mr, xr, vr, ar = rnd(m), rnd(x), rnd(v), rnd(a)
    global dw_add_accurate
    keep = dw_add_accurate
    try:
        dw_add_accurate = dw_add
        got = emulate(mr, xr, vr, ar, eps, act)
    finally:
        dw_add_accurate = keep
    ref = O.evaluate(mr, xr, vr, ar, eps, act)
    kap = O.evaluate_kappa(mr, xr, vr, ar, eps, act)
    worst = max((np.abs(got[o] - ref[o]).max(axis=1) / kap[o]).max() for o in range(3))
    assert worst > 1e-12
