"""Two-scale accuracy measure of the paper's second example (Sec. 4.2): the compliance
C_k = int_Gamma T u_y dx of every load step and its relative error eps_C against the full
FE^2 solution, in which every macro Gauss point carries the full-order micro problem.

Pins: with the full basis and full Gauss quadrature the reduced model is the full-order
model written in another basis, so the reduced FE^2 reproduces the full FE^2 compliance at
every step of a loading-unloading program (eps_C at the Newton tolerance); the loading
programs, the Sobol training samples and the error-bounded ECM stop are checked against
their definitions."""
import numpy as np
import pytest

import oracle
from oracle import fe, reduction
from oracle.build_roms import MATRIX, phase_2d
from paper_2307_16894_gb300 import fe2, inputs

from test_fe2 import OracleMicro
from test_oracle_rom import full_rom


def test_load_programs():
    T = fe2.load_levels(80.0, 10, unload=True)
    assert np.allclose(T, [16, 32, 48, 64, 80, 64, 48, 32, 16, 0])
    assert np.allclose(fe2.load_levels(80.0, 4), [20, 40, 60, 80])
    U = np.array([[1.01, 0.004], [0.004, 0.98]])
    P = inputs.load_unload_path(U, 40)
    assert P.shape == (40, 2, 2)
    assert np.allclose(P[19], U) and np.allclose(P[-1], np.eye(2)) and np.allclose(P[9], np.eye(2) + 0.5 * (U - np.eye(2)))
    assert np.allclose(P[20:39], P[18::-1])                                          # the ramp down mirrors the ramp up


def test_sobol_samples():
    rng = [(0.995, 1.005), (0.98, 1.0), (-0.005, 0.005), (0.2, 0.35)]
    a = inputs.sobol_samples(20, rng, 2307)
    b = inputs.sobol_samples(20, rng, 2307)
    assert a.shape == (20, 4) and np.array_equal(a, b)
    lo, hi = np.array(rng).T
    assert np.all(a >= lo) and np.all(a <= hi)
    # low discrepancy: every coordinate has points in both halves of its range
    mid = (lo + hi) / 2
    assert np.all((a < mid).sum(0) >= 5) and np.all((a > mid).sum(0) >= 5)


def test_compliance_error_definition():
    eps, mean = fe2.compliance_error([1.0, 2.0, 3.0, 0.0], [2.0, 2.0, -4.0, 0.0])
    assert np.allclose(eps[:3], [0.5, 0.0, 1.75]) and np.isnan(eps[3])
    assert mean == pytest.approx((0.5 + 0.0 + 1.75) / 3)


def test_ecm_error_bound():
    """With an error bound instead of a point count, ECM stops at the first set whose
    integration error is <= epsilon; a tighter bound needs at least as many points."""
    rng = np.random.default_rng(5)
    x = np.linspace(0, 1, 400)
    Fint = np.array([np.cos(np.pi * k * x + rng.uniform(0, 1)) for k in range(12)])
    wq = np.full(400, 1 / 400)
    res = {}
    for tol in (1e-1, 1e-2, 1e-3):
        sel, w, err = reduction.ecm_greedy(Fint, wq, tol=tol)
        assert err <= tol and np.all(w > 0) and len(set(sel.tolist())) == len(sel)
        res[tol] = len(sel)
    assert res[1e-1] <= res[1e-2] <= res[1e-3]
    with pytest.raises(ValueError):
        reduction.ecm_greedy(Fint, wq)


@pytest.fixture(scope="module")
def tiny_two_scale():
    mesh = fe.Mesh(2, 4, phase_2d)
    Gq = inputs.map_gradients(inputs.map_modes(2, 1, 7), mesh.X.reshape(-1, 2))
    rom = full_rom(mesh, [MATRIX])
    rom["Gmu"] = Gq.reshape(rom["m"], 4, 1)
    rom["tol_abs"] = 1e-9
    macro = fe2.BeamMesh(nx=2, ny=1)
    coef = inputs.map_coefficients(2, fe2.beam_mu(macro))
    geo = [fe.geometry(Gq, c) for c in coef]
    Finv = np.stack([g[0] for g in geo]).reshape(len(coef), mesh.nq, 2, 2)
    J = np.stack([g[1] for g in geo]).reshape(len(coef), mesh.nq)
    return mesh, rom, macro, coef, Finv, J


def test_full_basis_two_scale_equals_full_fe2(tiny_two_scale):
    """Full basis + full quadrature: the reduced FE^2 is the full FE^2 (compliance and macro
    displacement) over a load-unload program with plastic flow.  (The macro iteration counts
    may differ by one where the macro residual sits at its stop tolerance: the two micro
    solvers stop at different Newton tolerances.)"""
    mesh, rom, macro, coef, Finv, J = tiny_two_scale
    full = fe.FullMicro(mesh, [MATRIX], Finv, J, tol_rel=1e-12, tol_abs=1e-10)
    ref = fe2.solve(macro, full, 80.0, 6, unload=True)
    red = OracleMicro(rom, coef)
    out = fe2.solve(macro, red, 80.0, 6, unload=True)
    assert full.xi.max() > 1e-3                        # the micro problems yielded
    eps, mean = fe2.compliance_error(out["compliance"], ref["compliance"])
    assert ref["compliance"][-1] == 0.0 and np.isnan(eps[-1])
    assert mean <= 1e-8, eps
    scale = np.abs(ref["u"][2]).max()
    assert np.abs(out["u"][-1] - ref["u"][-1]).max() <= 1e-8 * scale
    assert np.abs(ref["u"][-1]).max() > 1e-3 * scale   # permanent deformation after unloading
    assert np.abs(np.array(out["macro_its"]) - np.array(ref["macro_its"])).max() <= 1


def test_full_micro_matches_path_solver(tiny_two_scale):
    """One macro point of FullMicro, stepped along a path, is the full-order path solver."""
    mesh, rom, macro, coef, Finv, J = tiny_two_scale
    path = [np.array([[1.0 + 0.002 * k, 0.001 * k], [0.0, 1.0 - 0.003 * k]]) for k in range(1, 4)]
    fo = fe.solve_path(mesh, [MATRIX], Finv[0].reshape(-1, 2, 2), J[0].reshape(-1), path, tol_rel=1e-12,
                       tol_abs=1e-10, want_Abar=True)
    fm = fe.FullMicro(mesh, [MATRIX], Finv[:1], J[:1], tol_rel=1e-12, tol_abs=1e-10)
    for k, F in enumerate(path):
        P, A, st = fm.step(F[None])
        assert st[0] == 0
        assert np.abs(P[0] - fo["Pbar"][k]).max() <= 1e-9 * np.abs(fo["Pbar"][k]).max()
        assert np.abs(A[0] - fo["Abar"][k]).max() <= 1e-8 * np.abs(fo["Abar"][k]).max()
    assert fo["n_yield"][-1] > 0
