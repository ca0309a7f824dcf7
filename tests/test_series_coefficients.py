"""The short power series the constitutive kernels use for ln x near 1 (Mercator's series of
ln(1 + u)) and exp x near 0 (the exponential series), read from the CUDA source and evaluated here
in FP64 by the same Horner scheme: over the ranges the kernels admit them (|x - 1| <= 1/32 and
|x| <= 1/16) they must agree with the library log and exp to a few units in the last place, so a
wrong sign, a dropped term or a misplaced coefficient fails.  The ranges themselves are checked
against the kernel's guards."""
import math
import pathlib
import re

import numpy as np
import pytest

SRC = pathlib.Path(__file__).resolve().parents[1] / "paper_2307_16894_gb300" / "csrc" / "material.cuh"


def _body(name, arg="x"):
    s = SRC.read_text()
    i = s.index("double %s(double %s)" % (name, arg))
    j = s.index("\n}\n", i)
    return s[i:j]


def _num(expr):
    expr = expr.strip()
    assert re.fullmatch(r"-?[0-9.]+(\s*/\s*[0-9.]+)?", expr), expr
    if "/" in expr:
        a, b = expr.split("/")
        return float(a) / float(b)
    return float(expr)


def _guard(body, var):
    return float(re.search(r"fabs\(%s\) <= ([0-9.]+)" % var, body).group(1))


def _horner(name, var):
    body = _body(name, var)
    seed = re.search(r"double p = ([^;]+);", body).group(1)
    steps = re.findall(r"p = fma\(%s, p, ([^)]+)\);" % var, body)
    return [_num(seed)] + [_num(c) for c in steps], body


def _eval(coef, t):
    p = np.full_like(t, coef[0])
    for c in coef[1:]:
        p = t * p + c
    return p


def test_log_near1_series():
    coef, body = _horner("log1p_series", "u")
    assert "return u * p;" in body
    for name, arg, fallback in (("log_near1", "x", "return log(x);"), ("log1p_near0", "u", "return log1p(u);")):
        b = _body(name, arg)
        assert _guard(b, "u") == 1 / 32 and "return log1p_series(u);" in b and fallback in b
    guard = 1 / 32
    assert len(coef) == 11                                     # terms u .. u^11
    x = np.linspace(1 - guard, 1 + guard, 100_001)
    u = x - 1.0
    got = u * _eval(coef, u)
    ref = np.log1p(u)
    nz = np.abs(ref) > 0
    assert np.max(np.abs(got[nz] - ref[nz]) / np.abs(ref[nz])) < 1e-15
    assert np.all(got[~nz] == 0.0)


def test_exp_near0_series():
    coef, body = _horner("exp_near0", "x")
    guard = _guard(body, "x")
    assert guard == 1 / 16
    assert "return fma(x, p, 1.0);" in body and "return exp(x);" in body
    assert len(coef) == 9                                      # terms x .. x^9 (plus the 1)
    assert coef == pytest.approx([1 / math.factorial(k) for k in range(9, 0, -1)], rel=1e-15)
    x = np.linspace(-guard, guard, 100_001)
    got = x * _eval(coef, x) + 1.0
    assert np.max(np.abs(got - np.exp(x)) / np.exp(x)) < 1e-15


def test_series_truncation_bounds():
    """Remainders of the truncated series at the range ends, from their closed forms: the first
    omitted terms bound the error (alternating / geometric tails) far below FP64 rounding."""
    u = 1 / 32
    tail_log = sum(u ** k / k for k in range(12, 40))           # |ln(1+u) - sum_{k<=11}| <= this
    assert tail_log / math.log1p(-u).__abs__() < 1e-16
    x = 1 / 16
    tail_exp = sum(x ** k / math.factorial(k) for k in range(10, 30))
    assert tail_exp / math.exp(-x) < 1e-16
