"""GB300 (sm_103a) direct N-body hot path: 6th-order Hermite predictor,
evaluation (acceleration, jerk, snap) and corrector with block time steps.

This module is a thin ctypes binding over the C-ABI library ``libnb.so``
(declared in ``include/nb.h``): it only marshals arguments.  Every step of
the path runs in the library's CUDA kernels; there is no CPU fallback.  If
the library has not been built, importing the module raises ImportError
(build it with ``python -m paper_1901_08532_gb300.build`` or
``__graft_entry__.build()``).

PyTorch is used only for device memory and streams: device tensors are
passed by ``data_ptr()`` and work is issued on
``torch.cuda.current_stream()``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libnb.so is not built ({LIB_PATH}); run paper_1901_08532_gb300/build.py")

_lib = C.CDLL(LIB_PATH)

NB_OK, NB_EINVAL, NB_ECUDA, NB_ENOMEM, NB_ENONFINITE, NB_ETIMEOUT, NB_ESTATE = 0, -1, -2, -3, -4, -5, -6
NB_FP64, NB_MIXED, NB_SP, NB_EX, NB_MIXED32 = 0, 1, 2, 3, 4
_STATUS = {NB_EINVAL: "NB_EINVAL", NB_ECUDA: "NB_ECUDA", NB_ENOMEM: "NB_ENOMEM",
           NB_ENONFINITE: "NB_ENONFINITE", NB_ETIMEOUT: "NB_ETIMEOUT", NB_ESTATE: "NB_ESTATE"}


class NBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Tiles(C.Structure):
    _fields_ = [("ki", C.c_int32), ("threads", C.c_int32), ("jtile", C.c_int32),
                ("lanes", C.c_int32), ("split", C.c_int32), ("junroll", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Config(C.Structure):
    _fields_ = [("precision", C.c_int32), ("eta", C.c_double), ("eta_s", C.c_double),
                ("dt_min", C.c_double), ("dt_max", C.c_double), ("dt_shared", C.c_double),
                ("tiles", Tiles), ("start_forces", C.c_int32), ("stream", C.c_void_p),
                ("device_steps", C.c_int32), ("step_noise", C.c_double)]


_d = C.POINTER(C.c_double)
_i32 = C.POINTER(C.c_int32)
_i64 = C.POINTER(C.c_int64)
_vp = C.c_void_p

_lib.nb_config_default.argtypes = [C.POINTER(Config)]
_lib.nb_config_default.restype = None
_lib.nb_init.argtypes = [C.POINTER(C.c_void_p), C.c_int64, _d, _d, _d, C.c_double, C.POINTER(Config)]
_lib.nb_predict.argtypes = [_vp, C.c_double]
_lib.nb_get_predicted.argtypes = [_vp, _d, _d, _d]
_lib.nb_evaluate.argtypes = [_vp, _vp, C.c_int64, C.c_int, _vp, _vp, _vp, C.c_int]
_lib.nb_correct.argtypes = [_vp, C.c_double]
_lib.nb_schedule.argtypes = [_vp, _d, _i64]
_lib.nb_evaluate_partial.argtypes = [_vp, _vp, C.c_int64, C.c_int, C.c_int64, C.c_int64, _vp, C.c_int]
_lib.nb_set_forces.argtypes = [_vp, _vp, C.c_int64, C.c_int, _vp, C.c_int]
_lib.nb_evaluate_kappa.argtypes = [_vp, _vp, C.c_int64, C.c_int, _vp, C.c_int]
_lib.nb_step.argtypes = [_vp, _d, _i64]
_lib.nb_run_until.argtypes = [_vp, C.c_double, _i64, C.c_int64, _d, _i64]
_lib.nb_run_diag.argtypes = [_vp, C.c_double, C.c_double, C.c_int64, _d, _i64, _i64]
_lib.nb_energy.argtypes = [_vp, _d, _d]
_lib.nb_angmom.argtypes = [_vp, _d, _d]
_lib.nb_get_state.argtypes = [_vp] + [_d] * 8
_lib.nb_set_state.argtypes = [_vp] + [_d] * 8
_lib.nb_get_active.argtypes = [_vp, _i32, C.c_int64, _i64]
_lib.nb_set_tiles.argtypes = [_vp, C.POINTER(Tiles)]
_lib.nb_inject_fault.argtypes = [_vp, C.c_int32]
_lib.nb_inject_fault.restype = C.c_int
_lib.nb_resolve_tiles.argtypes = [_vp, C.c_int64, C.POINTER(Tiles)]
_lib.nb_counters.argtypes = [_vp, _i64, _d]
_lib.nb_evaluate_fp64_static.argtypes = [_vp, C.c_int64, _vp, C.c_int64, C.c_double, C.c_int32,
                                         _vp, _vp]
_lib.nb_evaluate_fp64_static.restype = C.c_int
_lib.nb_ensemble_init.argtypes = [C.POINTER(C.c_void_p), C.c_int32, _i64, _d, _d, _d, C.c_double,
                                  C.POINTER(Config)]
_lib.nb_ensemble_set_shape.argtypes = [_vp, C.c_int32, C.c_int32, C.c_int32]
_lib.nb_ensemble_get_shape.argtypes = [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
_lib.nb_ensemble_run.argtypes = [_vp, C.c_double, C.c_int]
_lib.nb_ensemble_get_state.argtypes = [_vp] + [_d] * 8
_lib.nb_ensemble_stats.argtypes = [_vp, _i64, _d, _i64]
_lib.nb_ensemble_set_log.argtypes = [_vp, C.c_int64, C.c_int64]
_lib.nb_ensemble_get_log.argtypes = [_vp, _i32, _d, _i32, _i64, _i32, _i64, _i64]
_lib.nb_ensemble_last_error.argtypes = [_vp]
_lib.nb_ensemble_last_error.restype = C.c_char_p
_lib.nb_ensemble_free.argtypes = [_vp]
_lib.nb_ensemble_free.restype = None
for _f in ("nb_ensemble_init", "nb_ensemble_set_shape", "nb_ensemble_get_shape", "nb_ensemble_run",
           "nb_ensemble_get_state", "nb_ensemble_stats", "nb_ensemble_set_log", "nb_ensemble_get_log"):
    getattr(_lib, _f).restype = C.c_int
_lib.nb_pairs_workspace_bytes.argtypes = [C.c_int64]
_lib.nb_pairs_workspace_bytes.restype = C.c_size_t
_lib.nb_pairs_fp64.argtypes = [C.c_int64, _vp, _vp, _vp, _vp, C.c_double, _vp, _vp, _vp, _vp, _vp]
_lib.nb_pairs_fp64.restype = C.c_int
_lib.nb_pairs_fp64_adjoint.argtypes = [C.c_int64, _vp, _vp, _vp, _vp, C.c_double, _vp, _vp, _vp,
                                       _vp, _vp, _vp, _vp, _vp]
_lib.nb_pairs_fp64_adjoint.restype = C.c_int
_lib.nb_traj_predict.argtypes = [C.c_int64, C.c_double] + [_vp] * 9 + [_vp]
_lib.nb_traj_predict_adjoint.argtypes = [C.c_int64, C.c_double] + [_vp] * 9 + [_vp]
_lib.nb_traj_correct.argtypes = [C.c_int64, C.c_double] + [_vp] * 11 + [_vp]
_lib.nb_traj_correct_adjoint.argtypes = [C.c_int64, C.c_double] + [_vp] * 14 + [_vp]
for _f in ("nb_traj_predict", "nb_traj_predict_adjoint", "nb_traj_correct", "nb_traj_correct_adjoint"):
    getattr(_lib, _f).restype = C.c_int
_lib.nb_peak_probe.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, _d, _d, _d, _d]
_lib.nb_peak_probe.restype = C.c_int
_lib.nb_last_error.argtypes = [_vp]
_lib.nb_last_error.restype = C.c_char_p
_lib.nb_free.argtypes = [_vp]
_lib.nb_free.restype = None
for _f in ("nb_init", "nb_predict", "nb_get_predicted", "nb_evaluate", "nb_correct", "nb_step", "nb_run_until",
           "nb_schedule", "nb_evaluate_partial", "nb_set_forces", "nb_evaluate_kappa",
           "nb_run_diag",
           "nb_energy", "nb_angmom", "nb_get_state", "nb_set_state", "nb_get_active",
           "nb_set_tiles", "nb_resolve_tiles", "nb_counters"):
    getattr(_lib, _f).restype = C.c_int

EXPORTED = ("nb_config_default", "nb_init", "nb_predict", "nb_get_predicted", "nb_evaluate", "nb_correct", "nb_step",
            "nb_schedule", "nb_evaluate_partial", "nb_set_forces", "nb_evaluate_kappa",
            "nb_run_until", "nb_run_diag", "nb_energy", "nb_angmom", "nb_get_state", "nb_set_state",
            "nb_get_active", "nb_set_tiles", "nb_resolve_tiles", "nb_counters", "nb_inject_fault",
            "nb_evaluate_fp64_static", "nb_last_error", "nb_free", "nb_ensemble_init",
            "nb_ensemble_set_shape", "nb_ensemble_get_shape", "nb_ensemble_run", "nb_ensemble_get_state",
            "nb_ensemble_stats", "nb_ensemble_set_log", "nb_ensemble_get_log",
            "nb_ensemble_last_error", "nb_ensemble_free", "nb_pairs_workspace_bytes", "nb_pairs_fp64",
            "nb_pairs_fp64_adjoint", "nb_traj_predict", "nb_traj_predict_adjoint", "nb_traj_correct",
            "nb_traj_correct_adjoint", "nb_peak_probe")

PROBE_KINDS = ("ffma", "ffma2", "dfma", "rsqrt", "rcp", "ffma2+rsqrt", "ffma2+rsqrt_noftz",
               "ffma2+rsqrt+rcp", "ffma2_3reg")


def lib():
    """The loaded ctypes library (for direct C-ABI calls)."""
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(shape) if shape is not None else a


def _ptr(a):
    return a.ctypes.data_as(_d)


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def peak_probe(kind, blocks_per_sm=4, threads=256, iters=4096):
    """Throughput of one CUDA-core pipe on the current device (nb_peak_probe):
    kind is a name from PROBE_KINDS or its index.  Returns a dict with
    operations per clock per SM (FMA = 1 operation; an f32x2 FMA = 2),
    special-function estimates per clock per SM (mixed kinds), operations
    per second over the whole GPU, and the SM clock the launch ran at."""
    k = PROBE_KINDS.index(kind) if isinstance(kind, str) else int(kind)
    per_clk, per_s, est, mhz = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    st = _lib.nb_peak_probe(k, int(blocks_per_sm), int(threads), int(iters), C.byref(per_clk),
                            C.byref(per_s), C.byref(est), C.byref(mhz))
    if st != NB_OK:
        raise NBError(st, _lib.nb_last_error(None).decode())
    return {"kind": PROBE_KINDS[k], "ops_per_clk_per_sm": per_clk.value,
            "est_per_clk_per_sm": est.value, "ops_per_s": per_s.value, "sm_mhz": mhz.value}


class NBody:
    """One N-body system on the current CUDA device (a libnb context).

    m[n], x[n,3], v[n,3] are host arrays (copied); eps > 0.  precision is
    NB_FP64, NB_MIXED, NB_SP or NB_EX (NB_SP NBody only).  stream: a torch.cuda.Stream or raw cudaStream_t
    (default: torch's current stream).  device_steps: run_until / run_diag run
    block steps with at most 128 active particles in the device-resident
    stepper (one cooperative launch per run of such steps).
    """

    def __init__(self, m, x, v, eps, precision=NB_FP64, eta=0.4, eta_s=0.01,
                 dt_min=2.0 ** -20, dt_max=2.0 ** -3, dt_shared=0.0, tiles=None, stream=None,
                 start_forces=True, device_steps=True, step_noise=0.0):
        m = _f64(m)
        n = m.size
        x, v = _f64(x, (n, 3)), _f64(v, (n, 3))
        cfg = Config()
        _lib.nb_config_default(C.byref(cfg))
        cfg.precision, cfg.eta, cfg.eta_s = precision, eta, eta_s
        cfg.dt_min, cfg.dt_max, cfg.dt_shared = dt_min, dt_max, dt_shared
        if tiles:
            for k, val in dict(tiles).items():
                setattr(cfg.tiles, k, int(val))
        cfg.start_forces = 1 if start_forces else 0
        cfg.device_steps = 1 if device_steps else 0
        cfg.step_noise = float(step_noise)
        cfg.stream = _stream_handle(stream)
        self.n = n
        self.precision = precision
        self._ctx = C.c_void_p()
        st = _lib.nb_init(C.byref(self._ctx), n, _ptr(m), _ptr(x), _ptr(v), float(eps), C.byref(cfg))
        if st != NB_OK:
            raise NBError(st, _lib.nb_last_error(None).decode())

    def _check(self, st):
        if st != NB_OK:
            raise NBError(st, _lib.nb_last_error(self._ctx).decode())

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            _lib.nb_free(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._ctx.value

    # --- the three stages -------------------------------------------------
    def predict(self, t):
        self._check(_lib.nb_predict(self._ctx, float(t)))

    def predicted(self):
        """(x, v, a) [n, 3] of the evaluation buffer from the last predict()."""
        out = [np.zeros((self.n, 3)) for _ in range(3)]
        self._check(_lib.nb_get_predicted(self._ctx, *[_ptr(q) for q in out]))
        return tuple(out)

    def evaluate(self, active=None, out=None):
        """Acceleration, jerk, snap of the active particles.

        active: None (all), a host int32 array, or a CUDA int32 tensor.
        out: None -> returns three numpy [n_act, 3] arrays; "device" ->
        returns three CUDA float64 tensors; False -> keeps results for
        correct() only and returns None.
        """
        if active is None:
            aptr, n_act, on_dev = None, self.n, 0
        elif _is_torch(active) and active.is_cuda:
            assert active.dtype.__str__() == "torch.int32" and active.is_contiguous()
            aptr, n_act, on_dev = active.data_ptr(), active.numel(), 1
        else:
            active = np.ascontiguousarray(active, dtype=np.int32)
            aptr, n_act, on_dev = active.ctypes.data, active.size, 0
        if out is False:
            self._check(_lib.nb_evaluate(self._ctx, aptr, n_act, on_dev, None, None, None, 0))
            return None
        if out == "device":
            import torch
            res = [torch.empty((n_act, 3), dtype=torch.float64, device="cuda") for _ in range(3)]
            self._check(_lib.nb_evaluate(self._ctx, aptr, n_act, on_dev,
                                         *[r.data_ptr() for r in res], 1))
            return tuple(res)
        res = [np.empty((n_act, 3)) for _ in range(3)]
        self._check(_lib.nb_evaluate(self._ctx, aptr, n_act, on_dev,
                                     *[r.ctypes.data for r in res], 0))
        return tuple(res)

    def correct(self, t):
        self._check(_lib.nb_correct(self._ctx, float(t)))

    # --- the block step taken apart (multi-device evaluation) --------------
    def schedule(self):
        """Next block time and active count (nb_schedule); active() lists the set."""
        t = C.c_double()
        na = C.c_int64()
        self._check(_lib.nb_schedule(self._ctx, C.byref(t), C.byref(na)))
        return t.value, int(na.value)

    @staticmethod
    def _active_arg(active, n):
        if active is None:
            return None, n, 0, None
        if _is_torch(active) and active.is_cuda:
            return active.data_ptr(), active.numel(), 1, active
        active = np.ascontiguousarray(active, dtype=np.int32)
        return active.ctypes.data, active.size, 0, active

    def evaluate_partial(self, active, j_lo, j_hi, out="device"):
        """FP64 partial sums [9, n_act] of the active set against predicted
        j in [j_lo, j_hi) (nb_evaluate_partial): a CUDA tensor (out="device")
        or a numpy array (out="host")."""
        aptr, n_act, on_dev, keep = self._active_arg(active, self.n)
        if out == "device":
            import torch
            part = torch.empty((9, n_act), dtype=torch.float64, device="cuda")
            pptr, pdev = part.data_ptr(), 1
        else:
            part = np.empty((9, n_act))
            pptr, pdev = part.ctypes.data, 0
        self._check(_lib.nb_evaluate_partial(self._ctx, aptr, n_act, on_dev, int(j_lo), int(j_hi),
                                             pptr, pdev))
        return part

    def set_forces(self, active, f):
        """Load a, jerk, snap [9, n_act] (CUDA tensor or host array) of the
        active set as the evaluation for correct() (nb_set_forces)."""
        aptr, n_act, on_dev, keep = self._active_arg(active, self.n)
        if _is_torch(f) and f.is_cuda:
            assert f.dtype.__str__() == "torch.float64" and f.is_contiguous()
            fptr, fdev = f.data_ptr(), 1
        else:
            f = np.ascontiguousarray(f, dtype=np.float64)
            fptr, fdev = f.ctypes.data, 0
        self._check(_lib.nb_set_forces(self._ctx, aptr, n_act, on_dev, fptr, fdev))

    def evaluate_kappa(self, active=None):
        """Condition numbers (sum_j |A_ij|, sum_j |J_ij|, sum_j |S_ij|) of the
        active particles' sums at the last prediction, three numpy arrays
        [n_act] (nb_evaluate_kappa)."""
        aptr, n_act, on_dev, keep = self._active_arg(active, self.n)
        out = np.zeros((3, max(1, n_act)))
        self._check(_lib.nb_evaluate_kappa(self._ctx, aptr, n_act, on_dev, out.ctypes.data, 0))
        return tuple(out[q, :n_act].copy() for q in range(3))

    # --- integration --------------------------------------------------------
    def step(self):
        t = C.c_double()
        na = C.c_int64()
        self._check(_lib.nb_step(self._ctx, C.byref(t), C.byref(na)))
        return t.value, int(na.value)

    def run_until(self, t_end, log_cap=0):
        steps = C.c_int64()
        lt = np.zeros(max(1, log_cap))
        ln = np.zeros(max(1, log_cap), dtype=np.int64)
        self._check(_lib.nb_run_until(self._ctx, float(t_end), C.byref(steps), int(log_cap),
                                      _ptr(lt), ln.ctypes.data_as(_i64)))
        k = min(int(steps.value), log_cap)
        return int(steps.value), (lt[:k], ln[:k])

    def run_diag(self, t_end, dt_diag, cap=None):
        """Integrate to t_end, sampling energy and angular momentum on the
        device at the current time and every multiple of dt_diag.  Returns
        (steps, samples) with samples a dict of arrays: t, ekin, epot, L [k, 3],
        labs, steps."""
        if cap is None:
            cap = int(t_end / dt_diag) + 1 if dt_diag > 0 else 1
        cap = max(1, cap)
        out = np.zeros((cap, 8))
        ns, steps = C.c_int64(), C.c_int64()
        self._check(_lib.nb_run_diag(self._ctx, float(t_end), float(dt_diag), cap, _ptr(out),
                                     C.byref(ns), C.byref(steps)))
        k = min(cap, int(ns.value))
        o = out[:k]
        return int(steps.value), {"t": o[:, 0].copy(), "ekin": o[:, 1].copy(), "epot": o[:, 2].copy(),
                                  "L": o[:, 3:6].copy(), "labs": o[:, 6].copy(),
                                  "steps": o[:, 7].astype(np.int64)}

    # --- diagnostics and state ---------------------------------------------
    def energy(self):
        ek, ep = C.c_double(), C.c_double()
        self._check(_lib.nb_energy(self._ctx, C.byref(ek), C.byref(ep)))
        return ek.value, ep.value

    def angmom(self):
        L = np.zeros(3)
        la = C.c_double()
        self._check(_lib.nb_angmom(self._ctx, _ptr(L), C.byref(la)))
        return L, la.value

    def state(self):
        n = self.n
        out = {k: np.zeros((n, 3)) for k in ("x", "v", "a", "j", "s", "c")}
        out["t"] = np.zeros(n)
        out["dt"] = np.zeros(n)
        self._check(_lib.nb_get_state(self._ctx, *[_ptr(out[k]) for k in
                                                   ("x", "v", "a", "j", "s", "c", "t", "dt")]))
        return out

    def set_state(self, st):
        n = self.n
        args = []
        for k in ("x", "v", "a", "j", "s", "c"):
            args.append(_ptr(_f64(st[k], (n, 3))) if k in st else None)
        for k in ("t", "dt"):
            args.append(_ptr(_f64(st[k])) if k in st else None)
        keep = [a for a in args]  # noqa: F841  (arrays stay alive through the call)
        self._check(_lib.nb_set_state(self._ctx, *args))

    def active(self):
        na = C.c_int64()
        self._check(_lib.nb_get_active(self._ctx, None, 0, C.byref(na)))
        idx = np.zeros(max(1, na.value), dtype=np.int32)
        self._check(_lib.nb_get_active(self._ctx, idx.ctypes.data_as(_i32), na.value, C.byref(na)))
        return idx[:na.value]

    def inject_fault(self, kind=1):
        """Test hook: make the next evaluation's first tile wait run out."""
        self._check(_lib.nb_inject_fault(self._ctx, int(kind)))

    def set_tiles(self, **tiles):
        t = Tiles()
        for k, val in tiles.items():
            setattr(t, k, int(val))
        self._check(_lib.nb_set_tiles(self._ctx, C.byref(t)))

    def resolve_tiles(self, n_act):
        t = Tiles()
        self._check(_lib.nb_resolve_tiles(self._ctx, int(n_act), C.byref(t)))
        return t.as_dict()

    def counters(self):
        la = C.c_int64()
        it = C.c_double()
        self._check(_lib.nb_counters(self._ctx, C.byref(la), C.byref(it)))
        return int(la.value), float(it.value)


class Ensemble:
    """Independent systems advanced together in one persistent launch.

    sizes: particle count of each system; m, x, v: the systems' particles
    concatenated (host arrays).  Same precision/step parameters as NBody.
    """

    def __init__(self, sizes, m, x, v, eps, precision=NB_FP64, eta=0.4, eta_s=0.01,
                 dt_min=2.0 ** -20, dt_max=2.0 ** -3, dt_shared=0.0, stream=None, step_noise=0.0):
        sizes = np.ascontiguousarray(sizes, dtype=np.int64)
        m = _f64(m)
        n = m.size
        assert sizes.sum() == n
        x, v = _f64(x, (n, 3)), _f64(v, (n, 3))
        cfg = Config()
        _lib.nb_config_default(C.byref(cfg))
        cfg.precision, cfg.eta, cfg.eta_s = precision, eta, eta_s
        cfg.dt_min, cfg.dt_max, cfg.dt_shared = dt_min, dt_max, dt_shared
        cfg.step_noise = float(step_noise)
        if stream is not None:
            cfg.stream = _stream_handle(stream)
        self.sizes = sizes
        self.n = n
        self.precision = precision
        self._e = C.c_void_p()
        st = _lib.nb_ensemble_init(C.byref(self._e), sizes.size, sizes.ctypes.data_as(_i64), _ptr(m),
                                   _ptr(x), _ptr(v), float(eps), C.byref(cfg))
        if st != NB_OK:
            raise NBError(st, _lib.nb_ensemble_last_error(None).decode())

    def _check(self, st):
        if st != NB_OK:
            raise NBError(st, _lib.nb_ensemble_last_error(self._e).decode())

    def set_shape(self, ctas_per_system=None, threads=128, jtile=None):
        """Blocks per system, threads per block, j-tile length (None: the
        library's default for the precision and device)."""
        self._check(_lib.nb_ensemble_set_shape(self._e, int(ctas_per_system or 0), int(threads or 0),
                                               int(jtile or 0)))

    def shape(self):
        """(blocks per system, threads per block, j-tile) in use."""
        g, t, j = C.c_int32(), C.c_int32(), C.c_int32()
        self._check(_lib.nb_ensemble_get_shape(self._e, C.byref(g), C.byref(t), C.byref(j)))
        return g.value, t.value, j.value

    def run(self, t_end, use_graph=True):
        self._check(_lib.nb_ensemble_run(self._e, float(t_end), 1 if use_graph else 0))

    def state(self):
        n = self.n
        out = {k: np.zeros((n, 3)) for k in ("x", "v", "a", "j", "s", "c")}
        out["t"] = np.zeros(n)
        out["dt"] = np.zeros(n)
        self._check(_lib.nb_ensemble_get_state(self._e, *[_ptr(out[k]) for k in
                                                          ("x", "v", "a", "j", "s", "c", "t", "dt")]))
        return out

    def stats(self):
        steps = np.zeros(self.sizes.size, dtype=np.int64)
        it = C.c_double()
        la = C.c_int64()
        self._check(_lib.nb_ensemble_stats(self._e, steps.ctypes.data_as(_i64), C.byref(it),
                                           C.byref(la)))
        return steps, float(it.value), int(la.value)

    def set_log(self, step_cap, idx_cap):
        """Record every block step from now on (step_cap steps, idx_cap active
        indices kept); 0, 0 turns the log off."""
        self._log_caps = (int(step_cap), int(idx_cap))
        self._check(_lib.nb_ensemble_set_log(self._e, int(step_cap), int(idx_cap)))

    def log(self):
        """The step log per system: {system: [(t, active indices within the
        system or None if not kept), ...]} in the order the steps were taken,
        and the totals (steps, indices) recorded."""
        sc, ic = getattr(self, "_log_caps", (0, 0))
        sys_ = np.zeros(max(1, sc), dtype=np.int32)
        t = np.zeros(max(1, sc))
        na = np.zeros(max(1, sc), dtype=np.int32)
        off = np.zeros(max(1, sc), dtype=np.int64)
        idx = np.zeros(max(1, ic), dtype=np.int32)
        ns, ni = C.c_int64(), C.c_int64()
        self._check(_lib.nb_ensemble_get_log(self._e, sys_.ctypes.data_as(_i32), _ptr(t),
                                             na.ctypes.data_as(_i32), off.ctypes.data_as(_i64),
                                             idx.ctypes.data_as(_i32), C.byref(ns), C.byref(ni)))
        out = {}
        for k in range(min(sc, int(ns.value))):
            rec = idx[off[k]:off[k] + na[k]].copy() if off[k] >= 0 else None
            out.setdefault(int(sys_[k]), []).append((float(t[k]), rec))
        return out, (int(ns.value), int(ni.value))

    def close(self):
        if getattr(self, "_e", None) and self._e.value:
            _lib.nb_ensemble_free(self._e)
            self._e = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
