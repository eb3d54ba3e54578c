"""Argument checking of the C-ABI, which happens on the host before any CUDA
call, so it runs without a GPU: every rejected call returns its status and a
message, and nothing is allocated."""
import ctypes as C

import numpy as np
import pytest

nb = pytest.importorskip("paper_1901_08532_gb300")
lib = nb.lib()


def _cfg(**kw):
    cfg = nb.Config()
    lib.nb_config_default(C.byref(cfg))
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


def _init(n=8, eps=1e-3, m=None, x=None, v=None, **kw):
    m = np.full(n, 1.0 / max(n, 1)) if m is None else m
    x = np.random.default_rng(1).random((max(n, 1), 3)) if x is None else x
    v = np.zeros((max(n, 1), 3)) if v is None else v
    ctx = C.c_void_p()
    st = lib.nb_init(C.byref(ctx), n, m.ctypes.data_as(C.POINTER(C.c_double)),
                     x.ctypes.data_as(C.POINTER(C.c_double)), v.ctypes.data_as(C.POINTER(C.c_double)),
                     float(eps), C.byref(_cfg(**kw)))
    return st, ctx, lib.nb_last_error(None).decode()


def test_config_defaults():
    cfg = _cfg()
    assert cfg.precision == nb.NB_FP64 and cfg.eta == 0.4 and cfg.eta_s == 0.01
    assert cfg.dt_min == 2.0 ** -20 and cfg.dt_max == 2.0 ** -3 and cfg.dt_shared == 0.0
    assert cfg.start_forces == 1 and cfg.device_steps == 1 and not cfg.stream
    assert cfg.step_noise == 0.0


@pytest.mark.parametrize("kw, msg", [
    ({"n": 0}, "n must be"),
    ({"eps": 0.0}, "eps"),
    ({"eps": -1.0}, "eps"),
    ({"eps": float("nan")}, "eps"),
    ({"eps": 2.0 ** -41, "precision": 1}, "FP32"),
    ({"eps": 2.0 ** -41, "precision": 3}, "FP32"),
    ({"precision": 7}, "precision"),
    ({"eta": 0.0}, "eta"),
    ({"dt_min": 2.0 ** -2, "dt_max": 2.0 ** -3}, "dt_min"),
    ({"dt_max": 0.1}, "powers of two"),
    ({"dt_shared": 0.3}, "dt_shared"),
    ({"step_noise": -1e-7}, "step_noise"),
    ({"step_noise": 0.01}, "step_noise"),
])
def test_invalid_arguments_are_rejected_before_any_cuda_call(kw, msg):
    st, ctx, err = _init(**kw)
    assert st == nb.NB_EINVAL and not ctx.value
    assert msg in err


def test_too_many_particles_are_rejected_before_the_arrays_are_read():
    """n above 2^29 (about 190 GB of device state) is refused from n alone:
    the host arrays passed here hold one particle and are never read."""
    one = np.zeros(3)
    p = one.ctypes.data_as(C.POINTER(C.c_double))
    for n in ((1 << 29) + 1, 1 << 31, 1 << 40):
        ctx = C.c_void_p()
        st = lib.nb_init(C.byref(ctx), n, p, p, p, 1e-3, C.byref(_cfg()))
        assert st == nb.NB_EINVAL and not ctx.value
        assert "n must be" in lib.nb_last_error(None).decode()


def test_invalid_tiles_are_rejected():
    cfg_tiles = {"lanes": 3}
    cfg = _cfg()
    for k, v in cfg_tiles.items():
        setattr(cfg.tiles, k, v)
    m, x, v = np.ones(4), np.zeros((4, 3)), np.zeros((4, 3))
    ctx = C.c_void_p()
    st = lib.nb_init(C.byref(ctx), 4, m.ctypes.data_as(C.POINTER(C.c_double)),
                     x.ctypes.data_as(C.POINTER(C.c_double)), v.ctypes.data_as(C.POINTER(C.c_double)),
                     1e-3, C.byref(cfg))
    assert st == nb.NB_EINVAL and "lanes" in lib.nb_last_error(None).decode()


@pytest.mark.parametrize("bad", ["mass", "x", "v"])
def test_non_finite_or_negative_inputs(bad):
    n = 6
    m, x, v = np.full(n, 0.1), np.zeros((n, 3)), np.zeros((n, 3))
    if bad == "mass":
        m[2] = -1.0
    elif bad == "x":
        x[3, 1] = np.inf
    else:
        v[0, 0] = np.nan
    st, ctx, _ = _init(n=n, m=m, x=x, v=v)
    assert st == nb.NB_ENONFINITE and not ctx.value


def test_null_contexts_are_rejected():
    for name, args in (("nb_predict", (None, 0.0)), ("nb_correct", (None, 0.0)),
                       ("nb_step", (None, None, None)), ("nb_energy", (None, None, None)),
                       ("nb_run_until", (None, 1.0, None, 0, None, None)),
                       ("nb_run_diag", (None, 1.0, 0.5, 0, None, None, None))):
        assert getattr(lib, name)(*args) == nb.NB_EINVAL, name


def test_ensemble_rejects_single_precision_and_bad_sizes():
    n = 8
    m, x, v = np.full(n, 0.1), np.random.default_rng(2).random((n, 3)), np.zeros((n, 3))
    sizes = np.array([4, 4], dtype=np.int64)
    d = C.POINTER(C.c_double)
    e = C.c_void_p()
    st = lib.nb_ensemble_init(C.byref(e), 2, sizes.ctypes.data_as(C.POINTER(C.c_int64)),
                              m.ctypes.data_as(d), x.ctypes.data_as(d), v.ctypes.data_as(d), 1e-3,
                              C.byref(_cfg(precision=2)))
    assert st == nb.NB_EINVAL and not e.value
    st = lib.nb_ensemble_init(C.byref(e), 0, sizes.ctypes.data_as(C.POINTER(C.c_int64)),
                              m.ctypes.data_as(d), x.ctypes.data_as(d), v.ctypes.data_as(d), 1e-3,
                              C.byref(_cfg()))
    assert st == nb.NB_EINVAL and not e.value


@pytest.mark.parametrize("jrec, act, out, n, n_act, split, msg", [
    (0x1008, 0x2000, 0x3000, 1000, 10, 0, b"aligned"),     # jrec only 8-byte aligned
    (0x1000, 0x2002, 0x3000, 1000, 10, 0, b"aligned"),     # active not 4-byte aligned
    (0x1000, 0x2000, 0x3004, 1000, 10, 0, b"aligned"),     # out not 8-byte aligned
    (0x1000, 0x2000, 0x3000, 1 << 24, 1, 200000, b"65535"),  # too many j-chunks
    (0x1000, 0x2000, 0x3000, 1 << 16, 1 << 14, 64, b"static scratch"),  # partials too large
    (0x1000, 0x2000, 0x3000, 1 << 20, 600000, 2, b"static scratch"),    # more than 4096 i-tiles
    (0x1000, 0x2000, 0x3000, 1000, 1001, 0, b"invalid argument"),       # n_act > n
])
def test_static_entry_rejects_before_any_cuda_call(jrec, act, out, n, n_act, split, msg):
    """The allocation-free entry point checks pointers' alignment and the
    explicit split on the host and returns NB_EINVAL without launching: the
    pointers here are not device memory, and no GPU is needed."""
    lib.nb_evaluate_fp64_static.restype = C.c_int
    st = lib.nb_evaluate_fp64_static(C.c_void_p(jrec), n, C.c_void_p(act), n_act, 1e-3, split,
                                     C.c_void_p(out), None)
    assert st == nb.NB_EINVAL
    assert msg in lib.nb_last_error(None)
