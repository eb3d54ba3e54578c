"""Where the mixed path's parity bound comes from: a float32 emulation of the
operation sequence of the mixed pair term against the FP64 oracle.

The sequence: positions as hi + lo FP32 pairs, x - x_i formed as
(x_hi - x_i,hi) + (x_lo - x_i,lo); velocities and accelerations as single
FP32 numbers; the dot products and the u, w terms as FP32 fused
multiply-adds; q = R^(-1/2) and q^2 = 1/R from two hardware estimates,
modelled as the exact values times (1 + delta) with |delta| up to the
documented worst cases (2^-22.9 for rsqrt.approx.f32, 2^-23 for
rcp.approx.f32), each term accumulated in FP32 over blocks of 128 j (two
interleaved lanes of 64 terms, the kernel's running sums between folds)
and the block sums added without further error.  The GPU parity tests hold the kernel to
1e-6 sum_j |T_ij|; the emulated sequence must stay below it.

The emulation is written here from the description above; it shares
nothing with the CUDA source.  fma(a, b, c) is emulated as the FP64 sum of
the exact product of two FP32 numbers and c, rounded to FP32."""
import numpy as np
import pytest

import nb_inputs as ni
import oracle as O

F = np.float32


def f32(q):
    return np.asarray(q, dtype=np.float32)


def fma(a, b, c):
    return f32(a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64))


def estimate(exact, rel, rng):
    """An estimate within `rel` relative error of the exact value."""
    return f32(exact * (1.0 + rng.uniform(-rel, rel, exact.shape)))


def emulate(m, x, v, a, eps, act, fold=128, seed=5, single_estimate=False):
    rng = np.random.default_rng(seed)
    xh = f32(x)
    xl = f32(x - xh.astype(np.float64))
    vf, af, mf = f32(v), f32(a), f32(m)
    e2 = F(np.float64(eps) ** 2)
    n = m.size
    out = np.zeros((3, len(act), 3))
    for k, i in enumerate(act):
        r = f32(f32(xh - xh[i]) + f32(xl - xl[i]))           # [n, 3]
        dv = f32(vf - vf[i])
        da = f32(af - af[i])
        R = fma(r[:, 0], r[:, 0], fma(r[:, 1], r[:, 1], fma(r[:, 2], r[:, 2], np.full(n, e2))))
        rv = fma(r[:, 0], dv[:, 0], fma(r[:, 1], dv[:, 1], f32(r[:, 2] * dv[:, 2])))
        sv = fma(r[:, 0], da[:, 0], fma(r[:, 1], da[:, 1], fma(r[:, 2], da[:, 2], fma(
            dv[:, 0], dv[:, 0], fma(dv[:, 1], dv[:, 1], f32(dv[:, 2] * dv[:, 2]))))))
        Rd = R.astype(np.float64)
        q = estimate(1.0 / np.sqrt(Rd), 2.0 ** -22.9, rng)
        q2 = f32(q * q) if single_estimate else estimate(1.0 / Rd, 2.0 ** -23, rng)
        mu = f32(f32(mf * q) * q2)
        al = f32(rv * q2)
        be = fma(al, al, f32(sv * q2))
        na3, na6, nb3 = f32(al * F(-3)), f32(al * F(-6)), f32(be * F(-3))
        u = fma(na3[:, None], r, dv)
        w = fma(na6[:, None], u, fma(nb3[:, None], r, da))
        for o, t in enumerate((r, u, w)):
            # the product is rounded before it is added: one rounding more than
            # the kernel's fused multiply-add, so the emulation errs high
            term = f32(mu[:, None] * t)                       # [n, 3]
            for j0 in range(0, n, fold):
                blk = term[j0:j0 + fold]
                for lane in (0, 1):                           # FP32 running sums per lane
                    part = np.cumsum(blk[lane::2], axis=0, dtype=np.float32)
                    if len(part):
                        out[o, k] += part[-1].astype(np.float64)
    return out


def _ratio(got, m, x, v, a, eps, act):
    ref = O.evaluate(m, x, v, a, eps, act)
    kap = O.evaluate_kappa(m, x, v, a, eps, act)
    return max(float((np.abs(got[o] - ref[o]).max(axis=1) / kap[o]).max()) for o in range(3))


@pytest.mark.parametrize("seed", [11, 12])
def test_emulated_mixed_sequence_is_within_the_parity_bound(seed):
    n, eps = 4096, 1e-4
    m, x, v = ni.plummer(n, seed, imf="salpeter")
    a = ni.random_state(n, seed + 100, scale=2.0)
    act = ni.active_subset(n, 24, seed)
    got = emulate(m, x, v, a, eps, act)
    assert _ratio(got, m, x, v, a, eps, act) < 1e-6


def test_a_single_estimate_is_not_enough():
    """With q^2 = q q from the rsqrt estimate alone, the estimate's error
    enters alpha and beta twice and the snap's cancelling terms amplify it:
    the bound is broken (the kernel therefore takes q^2 from its own rcp
    estimate)."""
    n, eps, worst = 4096, 1e-4, 0.0
    for seed in (11, 12):
        m, x, v = ni.plummer(n, seed, imf="salpeter")
        a = ni.random_state(n, seed + 100, scale=2.0)
        act = ni.active_subset(n, 24, seed)
        got = emulate(m, x, v, a, eps, act, single_estimate=True)
        worst = max(worst, _ratio(got, m, x, v, a, eps, act))
    assert worst > 1e-6


def test_hi_lo_positions_are_needed():
    """With single FP32 positions (the SP control: no low parts), the
    close pairs of a Plummer core break the bound."""
    n, eps = 4096, 1e-4
    m, x, v = ni.plummer(n, 13, imf="salpeter")
    a = ni.random_state(n, 113, scale=2.0)
    act = ni.active_subset(n, 24, 13)
    x1 = f32(x).astype(np.float64)        # the SP control's positions
    got = emulate(m, x1, v, a, eps, act)  # its low parts are zero
    assert _ratio(got, m, x, v, a, eps, act) > 1e-6
