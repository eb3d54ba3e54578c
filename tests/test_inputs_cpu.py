"""Pins for the seeded input generators (nb_inputs), the one module the oracle
and the CUDA path share: the random source against the published SplitMix64
output, and each workload against the closed form it samples (Plummer's
cumulative mass and speed distribution, the Salpeter power law, the
log-uniform ensemble sizes).  Statistical checks use Kolmogorov-Smirnov
distances at about the 1 % level for their sample sizes; every seed is
fixed, so each test is deterministic."""
import math

import numpy as np
import pytest

import nb_inputs as ni

KS_1PCT = 1.63   # sqrt(n) x the KS distance exceeded with probability 1 %


def _ks(sample, cdf):
    s = np.sort(np.asarray(sample))
    n = s.size
    f = cdf(s)
    return max(np.max(np.arange(1, n + 1) / n - f), np.max(f - np.arange(n) / n)) * math.sqrt(n)


def test_splitmix64_matches_its_published_output():
    """SplitMix64 (Steele, Lea and Flood 2014) seeded with 1234567: the
    first five outputs of the reference implementation.  The k-th draw of a
    stream is the finaliser of key + (k + 1) * gamma, i.e. exactly that
    sequence when the key is the seed."""
    with np.errstate(over="ignore"):
        z = np.uint64(1234567) + (np.arange(5, dtype=np.uint64) + np.uint64(1)) * ni._GAMMA
    assert [int(q) for q in ni._mix64(z)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_uniform_draws():
    u = ni.uniform(7, 3, np.arange(200000))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert _ks(u, lambda q: q) < KS_1PCT
    assert np.array_equal(u[1000:1010], ni.uniform(7, 3, np.arange(1000, 1010)))   # counter-based
    w = ni.uniform(7, 4, np.arange(200000))                                          # another stream
    assert abs(np.corrcoef(u, w)[0, 1]) < 0.01


def test_plummer_cumulative_mass_profile():
    """Equal masses: the fraction of particles inside r follows
    M(<r) = r^3 / (r^2 + a^2)^(3/2) / 0.999 (the outer 0.1 % is cut), with the
    scale a = 3 pi / 16 of Henon units."""
    n = 40000
    _, x, _ = ni.plummer(n, 21)
    a = 3.0 * math.pi / 16.0
    r = np.linalg.norm(x, axis=1)
    assert _ks(r, lambda s: np.minimum(1.0, (s / a) ** 3 / (1 + (s / a) ** 2) ** 1.5 / 0.999)) < KS_1PCT


def test_plummer_speeds_and_isotropy():
    """q = |v| / v_esc(r) has density ~ q^2 (1 - q^2)^(7/2) on [0, 1], whose
    CDF is the regularised incomplete beta function I_{q^2}(3/2, 9/2);
    directions are isotropic; the centre of mass is at rest at the origin."""
    special = pytest.importorskip("scipy.special")
    n = 40000
    m, x, v = ni.plummer(n, 22)
    a = 3.0 * math.pi / 16.0
    r = np.linalg.norm(x, axis=1) / a
    v_esc = math.sqrt(2.0) * (1.0 + r * r) ** -0.25 * math.sqrt(16.0 / (3.0 * math.pi))
    q = np.linalg.norm(v, axis=1) / v_esc
    assert _ks(np.clip(q, 0, 1), lambda s: special.betainc(1.5, 4.5, s * s)) < KS_1PCT
    cz = x[:, 2] / np.linalg.norm(x, axis=1)            # cos(theta) uniform on [-1, 1]
    assert _ks(cz, lambda s: (s + 1) / 2) < KS_1PCT
    assert np.abs((m[:, None] * x).sum(0)).max() < 1e-12
    assert np.abs((m[:, None] * v).sum(0)).max() < 1e-12


def test_salpeter_quantiles_and_range():
    """Inverse-CDF sampling of dN/dm ~ m^-2.35 on [0.1, 100]: total mass 1,
    a dynamic range of at most 1000, and scale-free quantile ratios
    m(F) / m(1/2) equal to the closed form
    m(F) = (lo^p + F (hi^p - lo^p))^(1/p), p = 1 - 2.35, within 4 standard
    deviations of the sample quantiles (sd of ln m(F) =
    sqrt(F (1 - F) / n) |d ln m / dF|)."""
    n = 200000
    m = ni.salpeter_masses(n, 8)
    assert m.sum() == pytest.approx(1.0, rel=1e-12)
    assert m.max() / m.min() <= 1000.0 * (1 + 1e-12)
    p, lo, hi = 1 - 2.35, 0.1, 100.0

    def quantile(f):
        return (lo ** p + f * (hi ** p - lo ** p)) ** (1 / p)

    def sd_log(f):
        dlnm = (hi ** p - lo ** p) / (p * (lo ** p + f * (hi ** p - lo ** p)))
        return math.sqrt(f * (1 - f) / n) * abs(dlnm)

    med = np.quantile(m, 0.5)
    for f in (0.1, 0.25, 0.75, 0.9, 0.99):
        got = math.log(np.quantile(m, f) / med)
        want = math.log(quantile(f) / quantile(0.5))
        assert abs(got - want) < 4 * math.hypot(sd_log(f), sd_log(0.5)), f


def test_ensemble_sizes_are_log_uniform():
    s = ni.ensemble_sizes(40000, 9)
    assert s.min() >= 256 and s.max() <= 16384
    lo, hi = math.log(256), math.log(16384)
    assert _ks(np.log(s), lambda q: np.clip((q - lo) / (hi - lo), 0, 1)) < KS_1PCT
    # the 256-cluster ensemble workload (seed 4)
    assert ni.ensemble_sizes(256, 4).sum() == 1004043


def test_active_subsets():
    for n, k in ((1000, 0), (1000, 1), (1000, 333), (1000, 1000), (1 << 16, 4096)):
        a = ni.active_subset(n, k, 5)
        assert a.dtype == np.int32 and a.size == k
        assert np.all(np.diff(a) > 0) and (k == 0 or (a[0] >= 0 and a[-1] < n))
    a = ni.active_subset(1 << 16, 4096, 5)
    assert _ks(a / (1 << 16), lambda q: q) < KS_1PCT
    with pytest.raises(ValueError):
        ni.active_subset(10, 11, 1)
