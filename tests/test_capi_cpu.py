"""The C-ABI library builds, loads without a GPU, exports every entry point
declared in include/nb.h, and rejects bad arguments before touching CUDA."""
import ctypes as C
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_nb_build", os.path.join(ROOT, "paper_1901_08532_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return C.CDLL(mod.build())


def _declared():
    text = open(os.path.join(ROOT, "include", "nb.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nb_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    lib = _lib()
    names = _declared()
    assert "nb_init" in names and "nb_evaluate" in names and len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    _lib()
    import paper_1901_08532_gb300 as nb
    assert sorted(nb.EXPORTED) == _declared()


def test_init_rejects_bad_arguments_without_a_gpu():
    import paper_1901_08532_gb300 as nb
    lib = nb.lib()
    ctx = C.c_void_p()
    m = np.ones(4)
    x = np.zeros((4, 3))
    p = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))  # noqa: E731
    assert lib.nb_init(C.byref(ctx), 0, p(m), p(x), p(x), 1e-3, None) == nb.NB_EINVAL
    assert b"n must be" in lib.nb_last_error(None)
    cfg = nb.Config()
    lib.nb_config_default(C.byref(cfg))
    assert cfg.eta == 0.4 and cfg.dt_max == 0.125 and cfg.dt_min == 2.0 ** -20
    assert cfg.start_forces == 1
    cfg.dt_max = 0.3
    assert lib.nb_init(C.byref(ctx), 4, p(m), p(x), p(x), 1e-3, C.byref(cfg)) == nb.NB_EINVAL
    lib.nb_config_default(C.byref(cfg))
    cfg.tiles.lanes = 3
    assert lib.nb_init(C.byref(ctx), 4, p(m), p(x), p(x), 1e-3, C.byref(cfg)) == nb.NB_EINVAL
    bad = x.copy()
    bad[1, 2] = np.inf
    assert lib.nb_init(C.byref(ctx), 4, p(m), p(bad), p(x), 1e-3, None) == nb.NB_ENONFINITE
    assert ctx.value is None
    lib.nb_free(None)


def test_every_declaration_is_documented():
    """Each entry point in include/nb.h is preceded by its own comment (the
    operation, argument meaning and layout, ownership, errors)."""
    lines = open(os.path.join(ROOT, "include", "nb.h")).read().splitlines()
    decl = re.compile(r"^(nb_status|void|const char \*)\s*\**\s*(nb_[a-z_0-9]+)\s*\(")
    found, bad = 0, []
    for k, line in enumerate(lines):
        m = decl.match(line)
        if not m:
            continue
        found += 1
        j = k - 1
        while j >= 0 and not lines[j].strip():
            j -= 1
        if not lines[j].rstrip().endswith("*/"):
            bad.append(m.group(2))
    assert found >= 30 and not bad, bad
