"""FP64 CPU oracle for the 6th-order Hermite block-time-step N-body method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package; the CUDA
library and its Python binding never do.  The arithmetic lives in
``nb_oracle.c`` (plain single-threaded C99, IEEE double, no FMA
contraction), which is compiled on first use with the host C compiler.

Every function mirrors a C entry point; arrays are numpy float64 with
vectors laid out as [n, 3].
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = C.POINTER(C.c_double)
_i32 = C.POINTER(C.c_int32)
_i64 = C.POINTER(C.c_int64)
_u64 = C.POINTER(C.c_uint64)


def build(force: bool = False) -> str:
    """Compile liboracle.so with the host gcc; returns its path.

    NB_ORACLE_LIB, when set, names an already-built library to load instead
    (the mutation tests use it to load deliberately broken copies)."""
    alt = os.environ.get("NB_ORACLE_LIB")
    if alt:
        return alt
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "nb_oracle.h"))):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class orc_params(C.Structure):
    _fields_ = [("eta", C.c_double), ("eta_s", C.c_double), ("dt_min", C.c_double),
                ("dt_max", C.c_double), ("dt_shared", C.c_double), ("step_noise", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_pair.argtypes = [_d] * 6 + [C.c_double, C.c_double, _d, _d, _d]
            L.orc_evaluate.argtypes = [C.c_int64, _d, _d, _d, _d, C.c_double, C.c_int64,
                                       _i32, _d, _d, _d]
            L.orc_evaluate_kappa.argtypes = [C.c_int64, _d, _d, _d, _d, C.c_double, C.c_int64,
                                             _i32, _d, _d, _d]
            L.orc_predict.argtypes = [C.c_int64, C.c_double] + [_d] * 10
            L.orc_correct.argtypes = [C.c_double] + [_d] * 10
            L.orc_interpolate.argtypes = [C.c_double] + [_d] * 9
            L.orc_dt_crit.argtypes = [C.c_double] + [_d] * 6
            L.orc_dt_crit.restype = C.c_double
            L.orc_interp_floor.argtypes = [C.c_double, C.c_double] + [_d] * 7
            L.orc_dt_crit_floored.argtypes = [C.c_double] + [_d] * 7
            L.orc_dt_crit_floored.restype = C.c_double
            L.orc_dt_initial.argtypes = [C.c_double, _d, _d, _d]
            L.orc_dt_initial.restype = C.c_double
            L.orc_dt_quantise.argtypes = [C.c_double] * 5 + [C.POINTER(C.c_int)]
            L.orc_dt_quantise.restype = C.c_double
            L.orc_energy.argtypes = [C.c_int64, _d, _d, _d, C.c_double, _d, _d]
            L.orc_angmom.argtypes = [C.c_int64, _d, _d, _d, _d, _d]
            L.orc_create.argtypes = [C.c_int64, _d, _d, _d, C.c_double, C.POINTER(orc_params)]
            L.orc_create.restype = C.c_void_p
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_step.argtypes = [C.c_void_p, _d, _u64]
            L.orc_step.restype = C.c_int64
            L.orc_run_until.argtypes = [C.c_void_p, C.c_double, C.c_int64, _d, _i64, _u64]
            L.orc_run_until.restype = C.c_int64
            L.orc_replay.argtypes = [C.c_void_p, C.c_int64, _d, _i64, _i32]
            L.orc_replay.restype = C.c_int64
            L.orc_get_state.argtypes = [C.c_void_p] + [_d] * 8
            L.orc_set_state.argtypes = [C.c_void_p] + [_d] * 8
            L.orc_floor_hits.argtypes = [C.c_void_p]
            L.orc_floor_hits.restype = C.c_int64
            L.orc_hash_index.argtypes = [C.c_int64]
            L.orc_hash_index.restype = C.c_uint64
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(_d)


def _f(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def pair(xi, vi, ai, xj, vj, aj, mj, eps):
    """Acceleration, jerk and snap on i from j (three length-3 arrays)."""
    ins = [_f(q, 3) for q in (xi, vi, ai, xj, vj, aj)]
    out = [np.zeros(3) for _ in range(3)]
    lib().orc_pair(*[_p(q) for q in ins], float(mj), float(eps), *[_p(q) for q in out])
    return tuple(out)


def evaluate(m, x, v, a, eps, active=None):
    """(acc, jerk, snap), each [n_act, 3], for the active list (default: all)."""
    m = _f(m)
    n = m.size
    x, v, a = _f(x, (n, 3)), _f(v, (n, 3)), _f(a, (n, 3))
    act = np.arange(n, dtype=np.int32) if active is None else np.ascontiguousarray(
        active, dtype=np.int32)
    out = [np.zeros((act.size, 3)) for _ in range(3)]
    lib().orc_evaluate(n, _p(m), _p(x), _p(v), _p(a), float(eps), act.size,
                       act.ctypes.data_as(_i32), *[_p(q) for q in out])
    return tuple(out)


def evaluate_kappa(m, x, v, a, eps, active=None):
    """(sum_j |A_ij|, sum_j |J_ij|, sum_j |S_ij|), each [n_act], for the active list."""
    m = _f(m)
    n = m.size
    x, v, a = _f(x, (n, 3)), _f(v, (n, 3)), _f(a, (n, 3))
    act = np.arange(n, dtype=np.int32) if active is None else np.ascontiguousarray(
        active, dtype=np.int32)
    out = [np.zeros(act.size) for _ in range(3)]
    lib().orc_evaluate_kappa(n, _p(m), _p(x), _p(v), _p(a), float(eps), act.size,
                             act.ctypes.data_as(_i32), *[_p(q) for q in out])
    return tuple(out)


def predict(t, ti, x, v, a, j, s, c):
    """Predicted (x, v, a) of every particle at time t."""
    ti = _f(ti)
    n = ti.size
    ins = [_f(q, (n, 3)) for q in (x, v, a, j, s, c)]
    out = [np.zeros((n, 3)) for _ in range(3)]
    lib().orc_predict(n, float(t), _p(ti), *[_p(q) for q in ins], *[_p(q) for q in out])
    return tuple(out)


def correct(h, x0, v0, a0, j0, s0, a1, j1, s1):
    """Corrected (x1, v1) of one particle over a step h."""
    ins = [_f(q, 3) for q in (x0, v0, a0, j0, s0, a1, j1, s1)]
    x1, v1 = np.zeros(3), np.zeros(3)
    lib().orc_correct(float(h), *[_p(q) for q in ins], _p(x1), _p(v1))
    return x1, v1


def interpolate(h, a0, j0, s0, a1, j1, s1):
    """(crackle, 4th, 5th derivative of a) at the end of the step."""
    ins = [_f(q, 3) for q in (a0, j0, s0, a1, j1, s1)]
    out = [np.zeros(3) for _ in range(3)]
    lib().orc_interpolate(float(h), *[_p(q) for q in ins], *[_p(q) for q in out])
    return tuple(out)


def dt_crit(eta, a, j, s, c, d, e):
    return lib().orc_dt_crit(float(eta), *[_p(_f(q, 3)) for q in (a, j, s, c, d, e)])


def interp_floor(noise, h, a0, j0, s0, a1, j1, s1):
    """Rounding floors (of |c1|, |d1|, |e1|) for inputs with relative error `noise`."""
    out = np.zeros(3)
    lib().orc_interp_floor(float(noise), float(h), *[_p(_f(q, 3)) for q in (a0, j0, s0, a1, j1, s1)],
                           _p(out))
    return out


def dt_crit_floored(eta, a, j, s, c, d, e, floor):
    return lib().orc_dt_crit_floored(float(eta), *[_p(_f(q, 3)) for q in (a, j, s, c, d, e, floor)])


def dt_initial(eta_s, a, j, s):
    return lib().orc_dt_initial(float(eta_s), *[_p(_f(q, 3)) for q in (a, j, s)])


def dt_quantise(dt_crit_value, dt_old, t1, dt_min=2.0 ** -20, dt_max=2.0 ** -3):
    hit = C.c_int(0)
    r = lib().orc_dt_quantise(float(dt_crit_value), float(dt_old), float(t1), float(dt_min),
                              float(dt_max), C.byref(hit))
    return r, bool(hit.value)


def energy(m, x, v, eps):
    """(kinetic, potential) energy."""
    m = _f(m)
    n = m.size
    ek, ep = C.c_double(), C.c_double()
    lib().orc_energy(n, _p(m), _p(_f(x, (n, 3))), _p(_f(v, (n, 3))), float(eps),
                     C.byref(ek), C.byref(ep))
    return ek.value, ep.value


def angmom(m, x, v):
    """(L vector, sum of m |x cross v|)."""
    m = _f(m)
    n = m.size
    L = np.zeros(3)
    la = C.c_double()
    lib().orc_angmom(n, _p(m), _p(_f(x, (n, 3))), _p(_f(v, (n, 3))), _p(L), C.byref(la))
    return L, la.value


def hash_index(i: int) -> int:
    return int(lib().orc_hash_index(int(i)))


def set_hash(indices) -> int:
    """Order-independent hash of an active set (sum of per-index mixes mod 2^64)."""
    h = 0
    for i in np.asarray(indices).ravel():
        h = (h + hash_index(int(i))) & 0xFFFFFFFFFFFFFFFF
    return h


class System:
    """The whole integrator: block (or shared) time steps from t = 0."""

    def __init__(self, m, x, v, eps, eta=0.4, eta_s=0.01, dt_min=2.0 ** -20,
                 dt_max=2.0 ** -3, dt_shared=0.0, step_noise=0.0):
        m = _f(m)
        self.n = m.size
        self.params = orc_params(eta, eta_s, dt_min, dt_max, dt_shared, step_noise)
        self._h = lib().orc_create(self.n, _p(m), _p(_f(x, (self.n, 3))),
                                   _p(_f(v, (self.n, 3))), float(eps), C.byref(self.params))
        if not self._h:
            raise MemoryError("orc_create failed")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def step(self):
        """One block step; returns (t_next, n_act, set_hash)."""
        t = C.c_double()
        h = C.c_uint64()
        na = lib().orc_step(self._h, C.byref(t), C.byref(h))
        return t.value, int(na), int(h.value)

    def run_until(self, t_end, log_cap=0):
        lt = np.zeros(max(log_cap, 1))
        ln = np.zeros(max(log_cap, 1), dtype=np.int64)
        lh = np.zeros(max(log_cap, 1), dtype=np.uint64)
        steps = lib().orc_run_until(self._h, float(t_end), int(log_cap), _p(lt),
                                    ln.ctypes.data_as(_i64), lh.ctypes.data_as(_u64))
        k = min(steps, log_cap)
        return int(steps), (lt[:k], ln[:k], lh[:k])

    def replay(self, t_next, active_sets):
        t_next = _f(t_next)
        offs = np.zeros(len(active_sets) + 1, dtype=np.int64)
        offs[1:] = np.cumsum([len(a) for a in active_sets])
        idx = np.ascontiguousarray(np.concatenate([np.asarray(a, dtype=np.int32)
                                                   for a in active_sets]) if active_sets
                                   else np.zeros(1, np.int32), dtype=np.int32)
        return lib().orc_replay(self._h, len(active_sets), _p(t_next), offs.ctypes.data_as(_i64),
                                idx.ctypes.data_as(_i32))

    def state(self):
        """dict of x, v, a, j, s, c ([n,3]) and t, dt ([n])."""
        n = self.n
        out = {k: np.zeros((n, 3)) for k in ("x", "v", "a", "j", "s", "c")}
        out["t"] = np.zeros(n)
        out["dt"] = np.zeros(n)
        lib().orc_get_state(self._h, *[_p(out[k]) for k in ("x", "v", "a", "j", "s", "c",
                                                             "t", "dt")])
        return out

    def set_state(self, st):
        n = self.n
        arrs = [_f(st[k], (n, 3)) for k in ("x", "v", "a", "j", "s", "c")] + [
            _f(st["t"]), _f(st["dt"])]
        lib().orc_set_state(self._h, *[_p(q) for q in arrs])

    def energy(self, m, eps):
        st = self.state()
        return energy(m, st["x"], st["v"], eps)

    @property
    def floor_hits(self):
        return int(lib().orc_floor_hits(self._h))
