"""Planted mistakes in the oracle: each case copies the C oracle (material point of Appendix A,
reduced step of Sec. 3.2-3.3, polar split, shape sensitivities), plants ONE plausible mistake
(a dropped term or factor, a wrong sign, a transposed operand, a reversed product, a broken
derivative rule), builds the copy and runs the oracle's pins against it; at least one pin must
fail.  A control build of the unchanged sources passes them all, so every failure below is the
planted mistake's.  Mistakes that no computation can see (a transposed major-symmetric
tangent, a transposed symmetric stiffness) are not planted."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORC = os.path.join(ROOT, "oracle")
SOURCES = ["orc_material.c", "orc_rom.c"]
PINS = ["tests/test_oracle_material.py", "tests/test_oracle_rom.py", "tests/test_oracle_sensitivity.py"]

M, R = "orc_material.c", "orc_rom.c"
# (name, file, original text (must occur exactly once), planted text)
MISTAKES = [
    # material point, Appendix A
    ("lame_lambda_dropped", M, "m_scld(m_eye(), treps), lam / 1.0)", "m_scld(m_eye(), treps), 0.0)"),
    ("deviator_keeps_mean", M, "dmat s = m_sub(sig_tr, m_scld(m_eye(), mean));", "dmat s = sig_tr; (void)mean;"),
    ("von_mises_factor_dropped", M, "dual q_tr = scl(snorm, sqrt(1.5));", "dual q_tr = scl(snorm, 1.0);"),
    ("return_map_2G_for_3G", M, "double g = q_tr.v - 3.0 * G * x - sy;", "double g = q_tr.v - 2.0 * G * x - sy;"),
    ("flow_direction_factor_dropped", M, "dvd(cst(1.0), snorm)), sqrt(1.5));", "dvd(cst(1.0), snorm)), 1.0);"),
    ("plastic_update_reversed", M, "Fpnew = m_mul(m_exp(m_scld(r, dg)), Fpn);",
     "Fpnew = m_mul(Fpn, m_exp(m_scld(r, dg)));"),
    ("plastic_update_sign", M, "Fpnew = m_mul(m_exp(m_scld(r, dg)), Fpn);",
     "Fpnew = m_mul(m_exp(m_scld(r, scl(dg, -1.0))), Fpn);"),
    ("pk1_plastic_factor_transposed", M, "sig), m_tr(m_inv(Fpnew)));", "sig), m_inv(Fpnew));"),
    ("hardening_slope_wrong", M, "ph->H_or_k * pow(base, ph->p - 1.0);", "ph->H_or_k * pow(base, ph->p);"),
    ("dual_product_rule_term_dropped", M, "mk(a.v * b.v, a.d * b.v + a.v * b.d)", "mk(a.v * b.v, a.d * b.v)"),
    ("log_series_coefficient", M, "m_scl(term, 1.0 / (2.0 * j + 1.0))", "m_scl(term, 1.0 / (2.0 * j))"),
    # reduced step, Eqs. forcevector_ecm, stiffnessmatrix_ecm, eff_stress_1, eff_stiffness_1
    ("force_without_det_F_mu", R, "const double wJ = s->w[i] * s->J[i];", "const double wJ = s->w[i];"),
    ("kinematics_F_mu_inverse_transposed", R, "H[a * d + rr] * Finv[(size_t)i * d2 + rr * d + b];",
     "H[a * d + rr] * Finv[(size_t)i * d2 + b * d + rr];"),
    ("stiffness_without_det_F_mu", R, "K[j * n + k] += wJ * sum;", "K[j * n + k] += s->w[i] * sum;"),
    ("abar_fluctuation_dropped", R, "tt += s.gF[((size_t)i * n + j) * d2 + c] * qkl[j];", "(void)qkl;"),
    ("abar_tangent_problem_sign", R, "qkl[j] = -sum;", "qkl[j] = sum;"),
    ("pbar_without_volume", R, "Pbar[c] = sum / omega;", "Pbar[c] = sum;"),
    ("lu_solve_permutation_dropped", R,
     "for (int k = 0; k < n; ++k) { int p = piv[k]; if (p != k) { double t = b[k]; b[k] = b[p]; b[p] = t; } }",
     "(void)piv;"),
    # full-order FE element loops (Eqs. weakform-dep-mapped, Dweakform-dep), the brute-force reference
    ("fe_force_without_det_F_mu", R, "const double wJ = a->gw[g] * a->J[qp];", "const double wJ = a->gw[g];"),
    ("fe_shape_gradient_not_pulled_back", R, "s += a->dN[(g * nen + node) * d + rr] * Fi[rr * d + b];",
     "s += (rr == b) * a->dN[(g * nen + node) * d + rr];"),
    ("fe_kinematics_not_pulled_back", R, "s += H[i * d + rr] * Fi[rr * d + j];", "s += H[i * d + rr] * (rr == j);"),
    ("fe_stiffness_tangent_indices_swapped", R, "A[(i * d + b) * d2 + k * d + l]", "A[(i * d + l) * d2 + k * d + b]"),
    # shape sensitivities, Eq. eff_sensitivities_full
    ("sensitivity_det_derivative_dropped", R, "rhs[j] -= w[i] * (J[i] * (t1 + t2) + dJk * t3);",
     "rhs[j] -= w[i] * (J[i] * (t1 + t2)); (void)dJk; (void)t3;"),
    # polar split of the macro deformation (Sec. 4)
    ("polar_spin_sign_2d", R, "double om = (M[2] - M[1]) / trU;", "double om = (M[1] - M[2]) / trU;"),
]


def build_copy(dest, mistake=None):
    """Copy the C oracle to dest, plant `mistake` (name, file, original, planted) and build it
    with the oracle's own compiler flags; returns the library path."""
    src = os.path.join(dest, "src")
    os.makedirs(src)
    for f in SOURCES + ["orc.h"]:
        shutil.copy(os.path.join(ORC, f), src)
    if mistake is not None:
        _, fname, old, new = mistake
        path = os.path.join(src, fname)
        text = open(path).read()
        assert text.count(old) == 1, "the original text must occur exactly once: %r" % old
        open(path, "w").write(text.replace(old, new))
    so = os.path.join(dest, "liborc_copy.so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", so]
                   + [os.path.join(src, f) for f in SOURCES] + ["-lm"], check=True, capture_output=True)
    return so


def run_pins(so):
    """The oracle's pins, in a fresh interpreter that loads the library copy; stops at the
    first failing pin."""
    env = dict(os.environ, ORACLE_LIB=so)
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]
                          + PINS, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)


def test_control_copy_passes_pins(tmp_path):
    r = run_pins(build_copy(str(tmp_path)))
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("mistake", MISTAKES, ids=[m[0] for m in MISTAKES])
def test_planted_mistake_fails_a_pin(tmp_path, mistake):
    r = run_pins(build_copy(str(tmp_path), mistake))
    # exit code 1: a pin failed (not a crash, a collection error or an interruption)
    assert r.returncode == 1, "planted mistake %s was not caught:\n%s" % (mistake[0], r.stdout[-3000:])
    assert " failed" in r.stdout


# The MLP oracle (learned Newton start) is plain numpy: a planted copy of the module is loaded
# from its text and the MLP pins run against it in this process.
MLP_MISTAKES = [
    ("gelu_grad_second_term_dropped",
     " + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)", ""),
    ("input_standardisation_inverted", "h = (X - xm) / xs", "h = (X - xm) * xs"),
    ("output_scale_dropped", "return out * ys + ym", "return out + ym"),
    ("loss_gradient_factor_dropped", "d = 2.0 * r / r.size", "d = r / r.size"),
    ("backprop_through_gelu_value", "d = d * gelu_grad(zs[l])", "d = d * gelu(zs[l])"),
    ("bias_gradient_mean", "gb = d.sum(0)", "gb = d.mean(0)"),
    ("bias_dropped_in_forward", "z = h @ W.T + b", "z = h @ W.T"),
]


def _planted_mlp(old, new):
    import types
    text = open(os.path.join(ORC, "mlp.py")).read()
    assert text.count(old) == 1, "the original text must occur exactly once: %r" % old
    mod = types.ModuleType("planted_mlp")
    exec(compile(text.replace(old, new), "planted_mlp.py", "exec"), mod.__dict__)
    return mod


def _mlp_pins():
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import test_oracle_mlp
    return test_oracle_mlp, [getattr(test_oracle_mlp, f) for f in dir(test_oracle_mlp) if f.startswith("test_")]


def test_mlp_control_copy_passes_pins(monkeypatch):
    mod, pins = _mlp_pins()
    monkeypatch.setattr(mod, "mlp", _planted_mlp("import numpy as np", "import numpy as np"))
    for pin in pins:
        pin()


@pytest.mark.parametrize("mistake", MLP_MISTAKES, ids=[m[0] for m in MLP_MISTAKES])
def test_planted_mlp_mistake_fails_a_pin(monkeypatch, mistake):
    mod, pins = _mlp_pins()
    monkeypatch.setattr(mod, "mlp", _planted_mlp(mistake[1], mistake[2]))
    failed = []
    for pin in pins:
        try:
            pin()
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, "planted mistake %s was not caught" % mistake[0]
