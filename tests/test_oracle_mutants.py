"""The oracle's pins must catch plausible mistakes: each case below plants
one error in a copy of the oracle's C source (on the CPU), builds it, and
requires the pin suite to fail against it."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "nb_oracle.c")

MUTANTS = {
    "jerk_coefficient": ("jrk[k] = mr3 * v[k] - 3.0 * alpha", "jrk[k] = mr3 * v[k] - 2.0 * alpha"),
    "snap_operand": ("- 6.0 * alpha * jrk[k]", "- 6.0 * alpha * acc[k]"),
    "beta_dropped_term": ("/ R + alpha * alpha;", "/ R;"),
    "acc_difference_sign": ("a[k] = aj[k] - ai[k];", "a[k] = ai[k] - aj[k];"),
    "corrector_coefficient": ("h * h / 10.0 * (j1[k] - j0[k])", "h * h / 12.0 * (j1[k] - j0[k])"),
    "corrector_uses_v0_twice": ("h / 2.0 * (v0[k] + v1[k])", "h / 2.0 * (v0[k] + v0[k])"),
    "predictor_crackle": ("c[q] * d5 / 120.0", "c[q] * d5 / 100.0"),
    "interp_crackle": ("c1[k] = (y[0] + y[1] + y[2] / 2.0) / h3;", "c1[k] = (y[0] + y[1] + y[2]) / h3;"),
    "aarseth_swapped": ("sqrt(norm3(c) * norm3(e)) + norm3(d)", "sqrt(norm3(c) * norm3(d)) + norm3(e)"),
    "kinetic_half": ("0.5 * m[i] * dot3", "m[i] * dot3"),
    "quantise_off_by_one": ("p = ldexp(1.0, ex - 1);", "p = ldexp(1.0, ex);"),
    "compensation_dropped": ("return s->sum + s->comp; }", "return s->sum; }"),
    "potential_unsoftened": ("m[j] / sqrt(dot3(r, r) + eps * eps));", "m[j] / sqrt(dot3(r, r)));"),
    "softening_not_squared": ("double R = dot3(r, r) + eps * eps;", "double R = dot3(r, r) + eps;"),
    "angmom_z_sign": ("r[0] * u[1] - r[1] * u[0]};", "r[1] * u[0] - r[0] * u[1]};"),
    "no_force_floor": ("norm3(d);\n    if (A1 == 0.0 && A4 == 0.0)\n        return INFINITY;\n", "norm3(d);\n"),
    "floor_rho1_drops_j0": ("norm3(a0) + h * norm3(j0) + h * h / 2.0 * norm3(s0));",
                            "norm3(a0) + h * h / 2.0 * norm3(s0));"),
    "floor_rho2_power_of_h": ("rho[1] = noise * h * (norm3(j1)", "rho[1] = noise * (norm3(j1)"),
    "floor_rho3_drops_s0": ("rho[2] = noise * h * h * (norm3(s1) + norm3(s0));",
                            "rho[2] = noise * h * h * norm3(s1);"),
    "floor_signed_map": ("fabs(G[q][1]) * rho[1]", "G[q][1] * rho[1]"),
    "floor_map_crackle": ("G[0][k] = y[0] + y[1] + y[2] / 2.0;", "G[0][k] = y[0] + y[1] + y[2];"),
    "floored_norm_sign": ("double nd = fmax(norm3(d) - floor[1], 0.0);", "double nd = fmax(norm3(d) + floor[1], 0.0);"),
}
PIN_FILES = ("test_oracle_pins.py", "test_golden_cpu.py")


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    mut = tmp_path / "mut.c"
    mut.write_text(src.replace(old, new))
    (tmp_path / "nb_oracle.h").write_text(open(os.path.join(ROOT, "oracle", "nb_oracle.h")).read())
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                    str(mut), "-o", str(so), "-lm"], check=True)
    env = dict(os.environ, NB_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "--basetemp", str(tmp_path / "inner")]
                       + [os.path.join(ROOT, "tests", f) for f in PIN_FILES],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
