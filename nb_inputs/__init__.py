"""Seeded synthetic inputs for the direct N-body hot path.

This module is the only code shared by the FP64 oracle (``oracle/``) and the
CUDA path (``paper_1901_08532_gb300``): it draws initial conditions and
random selections and holds none of the integrator's arithmetic (no pair
force, predictor, corrector, time-step or scheduler code).

Random numbers come from a counter-based form of SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the
k-th draw of a stream with key K is the SplitMix64 finaliser applied to
K + (k + 1) * 0x9E3779B97F4A7C15 (mod 2^64).  Every draw is therefore a pure
function of (seed, stream, index), so any subset of particles can be
regenerated without replaying a sequence, and numpy evaluates it vectorised.

Workloads (the paper gives no initial model; section 3 only says its accuracy
test used 4096 particles):

* Plummer sphere sampled as in Aarseth, Henon and Wielen (1974), A&A 37, 183,
  scaled to Henon units (G = M = 1, E = -1/4 up to sampling noise).
* Salpeter (1955) initial mass function, slope 2.35 on [0.1, 100], normalised
  to total mass 1.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "uniform",
    "plummer",
    "salpeter_masses",
    "active_subset",
    "ensemble_sizes",
    "random_state",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream identifiers (arbitrary distinct constants)
_S_RADIUS, _S_POSDIR_Z, _S_POSDIR_PHI = 1, 2, 3
_S_SPEED_Q, _S_SPEED_Y, _S_VELDIR_Z, _S_VELDIR_PHI = 4, 5, 6, 7
_S_MASS, _S_ACTIVE, _S_ENSEMBLE, _S_STATE = 8, 9, 10, 11


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output finaliser (Stafford's Mix13 variant)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    s = np.array([(seed * 0x100000001B3 + stream * 0xC2B2AE3D27D4EB4F) & 0xFFFFFFFFFFFFFFFF],
                 dtype=np.uint64)
    return _mix64(s)[0]


def uniform(seed: int, stream: int, index) -> np.ndarray:
    """U[0,1) doubles with 53 random bits, one per entry of ``index``."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _key(seed, stream) + (idx + np.uint64(1)) * _GAMMA
    u = _mix64(z) >> np.uint64(11)
    return u.astype(np.float64) * (1.0 / 9007199254740992.0)


def _isotropic(seed: int, s_z: int, s_phi: int, idx: np.ndarray, radius: np.ndarray) -> np.ndarray:
    z = 2.0 * uniform(seed, s_z, idx) - 1.0
    phi = 2.0 * math.pi * uniform(seed, s_phi, idx)
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    out = np.empty((idx.size, 3))
    out[:, 0] = radius * rho * np.cos(phi)
    out[:, 1] = radius * rho * np.sin(phi)
    out[:, 2] = radius * z
    return out


def salpeter_masses(n: int, seed: int, slope: float = 2.35, m_lo: float = 0.1,
                    m_hi: float = 100.0) -> np.ndarray:
    """Masses from dN/dm ~ m^-slope on [m_lo, m_hi] by inverse CDF, normalised to sum 1."""
    idx = np.arange(n, dtype=np.uint64)
    x = uniform(seed, _S_MASS, idx)
    p = 1.0 - slope
    lo, hi = m_lo ** p, m_hi ** p
    m = (lo + x * (hi - lo)) ** (1.0 / p)
    return m / m.sum()


def plummer(n: int, seed: int, imf: str = "equal", henon_units: bool = True):
    """Plummer sphere of ``n`` particles; returns (m[n], x[n,3], v[n,3]) in FP64.

    Radii from the cumulative mass X = r^3 (1 + r^2)^(-3/2) (scale a = 1,
    G = M = 1): r = (X^(-2/3) - 1)^(-1/2), with X uniform on [0, 0.999) (the
    outer 0.1 % of the mass is cut, as Aarseth, Henon and Wielen do).  Speeds
    v = q v_esc(r), v_esc = sqrt(2) (1 + r^2)^(-1/4), with q drawn by von
    Neumann rejection from g(q) = q^2 (1 - q^2)^(7/2) (g < 0.1 on [0, 1]).
    Directions are isotropic.  Henon units: x *= 3 pi / 16,
    v *= sqrt(16 / (3 pi)).  The mass-weighted centre of mass and its velocity
    are then subtracted.  No energy-based rescaling is applied.
    """
    if n <= 0:
        raise ValueError("n must be positive")
    idx = np.arange(n, dtype=np.uint64)
    if imf == "equal":
        m = np.full(n, 1.0 / n)
    elif imf == "salpeter":
        m = salpeter_masses(n, seed)
    else:
        raise ValueError(f"unknown imf {imf!r}")

    xm = 0.999 * uniform(seed, _S_RADIUS, idx)
    with np.errstate(divide="ignore"):
        r = 1.0 / np.sqrt(xm ** (-2.0 / 3.0) - 1.0)
    r = np.where(xm > 0.0, r, 0.0)
    x = _isotropic(seed, _S_POSDIR_Z, _S_POSDIR_PHI, idx, r)

    q = np.empty(n)
    todo = np.arange(n)
    attempt = 0
    while todo.size:
        ctr = np.uint64(attempt) * np.uint64(n) + todo.astype(np.uint64)
        qq = uniform(seed, _S_SPEED_Q, ctr)
        yy = 0.1 * uniform(seed, _S_SPEED_Y, ctr)
        ok = yy < qq * qq * (1.0 - qq * qq) ** 3.5
        q[todo[ok]] = qq[ok]
        todo = todo[~ok]
        attempt += 1
    speed = q * math.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
    v = _isotropic(seed, _S_VELDIR_Z, _S_VELDIR_PHI, idx, speed)

    if henon_units:
        x *= 3.0 * math.pi / 16.0
        v *= math.sqrt(16.0 / (3.0 * math.pi))
    mt = m.sum()
    x -= (m[:, None] * x).sum(axis=0) / mt
    v -= (m[:, None] * v).sum(axis=0) / mt
    return m, np.ascontiguousarray(x), np.ascontiguousarray(v)


def active_subset(n_total: int, n_active: int, seed: int) -> np.ndarray:
    """Sorted int32 indices of a seeded uniform random subset of size n_active."""
    if not 0 <= n_active <= n_total:
        raise ValueError("n_active out of range")
    keys = uniform(seed, _S_ACTIVE, np.arange(n_total, dtype=np.uint64))
    sel = np.argpartition(keys, n_active - 1)[:n_active] if 0 < n_active < n_total else (
        np.arange(n_total) if n_active == n_total else np.arange(0))
    return np.sort(sel).astype(np.int32)


def ensemble_sizes(n_clusters: int, seed: int, n_lo: int = 256, n_hi: int = 16384) -> np.ndarray:
    """Cluster sizes round(exp(U[ln n_lo, ln n_hi])) (log-uniform), int64."""
    u = uniform(seed, _S_ENSEMBLE, np.arange(n_clusters, dtype=np.uint64))
    return np.rint(np.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo)))).astype(np.int64)


def random_state(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """n x 3 doubles uniform on [-scale, scale), for derivative test data."""
    u = uniform(seed, _S_STATE, np.arange(3 * n, dtype=np.uint64)).reshape(n, 3)
    return scale * (2.0 * u - 1.0)
