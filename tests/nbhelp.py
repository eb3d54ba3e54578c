"""Shared helpers for the parity tests (error metrics, GPU import, the
worked-example fixtures under tests/golden)."""
import pathlib

import numpy as np
import pytest


def rel_err(got, ref):
    """Per-particle error: largest component error over the reference vector
    norm, |got - ref|_inf / |ref|_2 (rows of [n, 3] arrays)."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    den = np.linalg.norm(ref, axis=1)
    den = np.where(den > 0, den, 1.0)
    return np.abs(got - ref).max(axis=1) / den


def check_parity(prec, got, ref, kappa=None, tol64=1e-12, tol_mixed=1e-6):
    """FP64 (prec 0): |got - ref|_inf <= tol64 |ref|_2 per particle.
    Mixed (prec 1): |got - ref|_inf <= tol_mixed * kappa per particle, with
    kappa = sum_j |T_ij| the condition number of the sum (the FP32 pair terms
    each carry rounding errors of a few 1e-8 relative to |T_ij|).  Returns
    the worst ratio to the bound."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    if prec == 0:
        return float((rel_err(got, ref) / tol64).max()) if len(ref) else 0.0
    assert kappa is not None
    err = np.abs(got - ref).max(axis=1)
    bound = tol_mixed * np.asarray(kappa, dtype=np.float64)
    # a sum with no terms (kappa = 0, e.g. a lone particle) must be exact
    ratio = np.where(bound > 0, err / np.where(bound > 0, bound, 1.0), np.where(err > 0, np.inf, 0.0))
    return float(ratio.max()) if len(ref) else 0.0


def nb_gpu():
    """The CUDA package, or skip when no GPU is present."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1901_08532_gb300 as nb
    return nb


_GOLDEN = pathlib.Path(__file__).resolve().parent / "golden"


def _value(tok):
    """One number of a fixture: integer, decimal, fraction p/q or a closed
    form built from numbers, + - * / and sqrt(), evaluated in FP64 (true
    division of exact integers is correctly rounded).  Anything else in the
    expression is rejected."""
    import ast
    import math
    import operator

    ops = {ast.Add: operator.add, ast.Sub: operator.sub, ast.Mult: operator.mul,
           ast.Div: operator.truediv}

    def ev(node):
        if isinstance(node, ast.Expression):
            return ev(node.body)
        if isinstance(node, ast.Constant) and type(node.value) in (int, float):
            return node.value
        if isinstance(node, ast.UnaryOp) and isinstance(node.op, (ast.USub, ast.UAdd)):
            x = ev(node.operand)
            return -x if isinstance(node.op, ast.USub) else x
        if isinstance(node, ast.BinOp) and type(node.op) in ops:
            return ops[type(node.op)](ev(node.left), ev(node.right))
        if (isinstance(node, ast.Call) and isinstance(node.func, ast.Name)
                and node.func.id == "sqrt" and len(node.args) == 1 and not node.keywords):
            return math.sqrt(ev(node.args[0]))
        raise ValueError(f"unsupported fixture value {tok!r}")

    return float(ev(ast.parse(tok, mode="eval")))


def load_golden(name):
    """The cases of a text fixture under tests/golden: a list of dicts with
    "name", scalars (one value), vectors (three values) and, for "body"
    lines, an [n, 7] array (m, x, y, z, vx, vy, vz)."""
    cases = []
    for raw in (_GOLDEN / name).read_text().splitlines():
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        key, rest = line.split(None, 1)
        if key == "case":
            cases.append({"name": rest.strip(), "body": []})
            continue
        case = cases[-1]
        if key == "body":
            case["body"].append([_value(t) for t in rest.split()])
        elif key in ("epot", "Lnorm", "ekin", "m_j", "eps"):
            case[key] = _value(rest.strip())
        else:
            case[key] = np.array([_value(t) for t in rest.split()])
    for case in cases:
        case["body"] = np.array(case["body"]) if case["body"] else None
    return cases
