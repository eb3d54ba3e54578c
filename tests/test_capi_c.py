"""The C-ABI from plain C: include/nb.h compiles as C99 (and as C++),
a C program links against libnb.so, and (on a GPU) that program reproduces
the softened_general worked example of tests/golden through nb_evaluate,
its closed-form energy through nb_energy, and integrates with nb_run_until."""
import os
import subprocess

import numpy as np
import pytest

from nbhelp import load_golden

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "capi_example.c")
OUT = os.path.join(ROOT, "tests", "_build")


def _libpath():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "_nb_build", os.path.join(ROOT, "paper_1901_08532_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()


def _build_example():
    lib = _libpath()
    os.makedirs(OUT, exist_ok=True)
    exe = os.path.join(OUT, "capi_example")
    libdir = os.path.dirname(lib)
    subprocess.run(["gcc", "-std=c99", "-O1", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    "-I", os.path.join(ROOT, "include"), SRC, "-o", exe,
                    "-L", libdir, "-l:" + os.path.basename(lib), "-Wl,-rpath," + libdir],
                   check=True, capture_output=True, text=True)
    return exe


def test_header_is_c99_and_cxx_and_the_example_links():
    subprocess.run(["g++", "-std=c++17", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    "-fsyntax-only", "-x", "c++", "-I", os.path.join(ROOT, "include"), SRC],
                   check=True, capture_output=True, text=True)
    assert os.access(_build_example(), os.X_OK)


def _run(prec):
    exe = _build_example()
    res = subprocess.run([exe, str(prec)], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr
    out = {}
    for line in res.stdout.splitlines():
        key, *vals = line.split()
        out[key] = np.array([float(q) for q in vals])
    return out


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1, 3])
def test_c_program_reproduces_the_worked_example(prec):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    case = next(c for c in load_golden("pair_worked_examples.txt") if c["name"] == "softened_general")
    out = _run(prec)
    tol = {0: 1e-14, 1: 1e-6, 3: 1e-12}[prec]
    for k in ("acc", "jerk", "snap"):
        np.testing.assert_allclose(out[k], case[k], rtol=0, atol=tol * np.abs(case[k]).max(), err_msg=k)
    # m_i = 2 m_j: the pair term on j is -2 times the one on i
    np.testing.assert_allclose(out["acc_j"], -2.0 * case["acc"], rtol=0,
                               atol=2 * tol * np.abs(case["acc"]).max())
    assert out["ekin"][0] == pytest.approx(12.5, rel=1e-15)
    assert out["epot"][0] == pytest.approx(-10.0, rel=1e-14)
    assert out["steps"][0] >= 2
    np.testing.assert_array_equal(out["t"], [0.25, 0.25])
