"""FE^2 driver (macro Q8 beam, reduced RVE at every macro Gauss point): the macro element
passes the patch test, the traction has the prescribed resultant, and with the FP64 oracle as
the micro solver the macro Newton converges quadratically; on the GPU (gpu-marked test) the
library's micro solver reproduces the oracle-driven two-scale solution."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2307_16894_gb300 import fe2, inputs, workload

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


class OracleMicro:
    """micro solver on the FP64 oracle (test infrastructure)"""

    def __init__(self, rom, coef):
        d, n, m = rom["d"], rom["n"], rom["m"]
        B = len(coef)
        self.rom = rom
        Gmu = rom["Gmu"].reshape(m, d, d, -1)
        Fm = np.eye(d)[None, None] + np.einsum("iack,bk->biac", Gmu, coef)
        self.Finv, self.J = np.linalg.inv(Fm), np.abs(np.linalg.det(Fm))
        self.q = np.zeros((B, n))
        self.Fp = np.tile(np.eye(3), (B, m, 1, 1)).copy()
        self.xi = np.zeros((B, m))
        self.saved = None

    def save(self):
        self.saved = (self.q.copy(), self.Fp.copy(), self.xi.copy())

    def restore(self):
        self.q[:], self.Fp[:], self.xi[:] = self.saved

    def step(self, F):
        o = oracle.rom_batch(self.rom, self.Finv, self.J, F, self.q, self.Fp, self.xi, 1e-10, self.rom["tol_abs"], 25)
        return o["Pbar"], o["Abar"], o["status"]


def test_paper_example2_mesh():
    """the macro mesh of the paper's second example: 200 Q8 elements, 800 quadrature points,
    1322 degrees of freedom on a W x H = 2 x 1 structure (tests/golden/paper_example2_macro.json)"""
    g = json.load(open(os.path.join(GOLDEN, "paper_example2_macro.json")))
    m = fe2.BeamMesh(L=g["W"], H=g["H"], nx=20, ny=10)
    assert (m.ne, m.nq, m.ndof) == (g["elements"], g["quadrature_points"], g["dofs"])
    # resultant of T(x) = Tbar (1 - (2x/W - 1)^2) per unit Tbar: 2 W / 3, compressive
    assert np.allclose(m.f_unit.reshape(-1, 2).sum(0), [0.0, -2.0 * g["W"] / 3.0], atol=1e-13)


def test_patch_and_traction():
    m = fe2.BeamMesh(nx=4, ny=2)
    assert np.allclose(m.f_unit.reshape(-1, 2).sum(0), [0.0, -4.0 / 3.0], atol=1e-14)
    lam, G = 1.0, 0.5
    A = np.zeros((2, 2, 2, 2))
    for i, j, k, l in np.ndindex(2, 2, 2, 2):
        A[i, j, k, l] = lam * (i == j) * (k == l) + G * ((i == k) * (j == l) + (i == l) * (j == k))
    E = np.array([[0.01, 0.002], [0.003, -0.004]])
    u = (m.X @ E.T).ravel()
    assert np.abs(m.deformation_gradients(u) - (np.eye(2) + E)).max() <= 1e-15
    P = np.einsum("ijkl,kl->ij", A, E)
    f, K = m.assemble(np.tile(P, (m.nq, 1, 1)), np.tile(A.reshape(4, 4), (m.nq, 1, 1)))
    interior = [m.ids[I, J] for I in range(1, 2 * m.nx) for J in range(1, 2 * m.ny) if m.ids[I, J] >= 0]
    assert np.abs(f.reshape(-1, 2)[interior]).max() <= 1e-15   # constant stress: no interior force
    assert np.abs(K @ u - f).max() <= 1e-15


def test_element_arrays_and_free_assembly():
    """Element force and stiffness against their definitions written out entry by entry,
    f_(a i) = sum_q w_q P_ij dN_a/dX_j and K_(a i)(b k) = sum_q w_q dN_a/dX_j A_ijkl dN_b/dX_l,
    and the free-free CSR assembly against slicing the full matrix."""
    m = fe2.BeamMesh(nx=3, ny=2)
    rng = np.random.default_rng(3)
    P = rng.standard_normal((m.nq, 2, 2))
    A = rng.standard_normal((m.nq, 4, 4))
    fe, Ke = m.element_arrays(P, A)
    A6 = A.reshape(m.ne, 4, 2, 2, 2, 2)
    P4 = P.reshape(m.ne, 4, 2, 2)
    for e in (0, m.ne - 1):
        for a, i in np.ndindex(8, 2):
            ref = sum(m.wdet[e, q] * P4[e, q, i, j] * m.dNdX[e, q, a, j] for q in range(4) for j in range(2))
            assert abs(fe[e, 2 * a + i] - ref) <= 1e-13
            for b, k in np.ndindex(8, 2):
                ref = sum(m.wdet[e, q] * m.dNdX[e, q, a, j] * A6[e, q, i, j, k, l] * m.dNdX[e, q, b, l]
                          for q in range(4) for j in range(2) for l in range(2))
                assert abs(Ke[e, 2 * a + i, 2 * b + k] - ref) <= 1e-12
    f1, K1 = m.assemble(P, A)
    f2, K2 = m.assemble_free(P, A)
    assert np.abs(f1 - f2).max() <= 1e-14
    assert np.abs(K1[m.free][:, m.free].toarray() - K2.toarray()).max() <= 1e-13


def test_fe2_oracle_quadratic_convergence():
    """2 x 1 macro elements (8 macro points) on the 2D porous RVE model, compressed into the
    plastic range in 4 steps; within every step the macro residual contracts quadratically (the
    consistent effective stiffness Abar of the micro problem)."""
    rom = workload.load_model(workload.WORKLOADS["c2"]["model"])
    mesh = fe2.BeamMesh(nx=2, ny=1)
    coef = inputs.map_coefficients(2, fe2.beam_mu(mesh))
    micro = OracleMicro(rom, coef)
    u = np.zeros(2 * mesh.nn)
    for k in range(1, 5):
        fext = 80.0 * k / 4 * mesh.f_unit
        micro.save()
        res = []
        for it in range(10):
            if it:
                micro.restore()
            P, A, st = micro.step(mesh.deformation_gradients(u))
            assert (st == 0).all(), (k, it)
            f, K = mesh.assemble(P, A)
            R = (f - fext)[mesh.free]
            res.append(np.linalg.norm(R) / np.linalg.norm(fext[mesh.free]))
            if res[-1] <= 1e-10:     # the noise floor of micro solves at tolerance 1e-10 is ~1e-11
                break
            u[mesh.free] += np.linalg.solve(K[mesh.free][:, mesh.free].toarray(), -R)
        print("step", k, "macro residuals:", ["%.1e" % r for r in res])
        assert res[-1] <= 1e-10
        for a, b in zip(res[:-1], res[1:]):   # quadratic once in the convergence zone
            if a < 1e-3:
                assert b <= 100 * a * a + 1e-11, (a, b)   # (1e-11: the micro noise floor)
    assert micro.xi.max() > 0          # the load reaches the plastic range


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol,unload", [("fp64", 1e-9, False), ("fp32", 1e-6, False), ("fp64", 1e-9, True)])
def test_fe2_gpu_vs_oracle(prec, tol, unload):
    """monotonic loading to Tbar = 80 in 5 steps; and the load-unload program (up to 80 and
    back to 0 in 6 steps: elastic unloading of plastically deformed micro problems)"""
    import __graft_entry__
    __graft_entry__.build()
    rom = workload.load_model(workload.WORKLOADS["c2"]["model"])
    mesh = fe2.BeamMesh(nx=4, ny=2)
    coef = inputs.map_coefficients(2, fe2.beam_mu(mesh))
    nsteps = 6 if unload else 5
    ref = fe2.solve(mesh, OracleMicro(rom, coef), 80.0, nsteps, unload=unload)
    gm = fe2.RomMicro(rom, coef, prec)
    out = fe2.solve(mesh, gm, 80.0, nsteps, unload=unload)
    gm.close()
    tip_err = np.abs(np.array(out["tip"]) - np.array(ref["tip"])).max() / np.abs(np.array(ref["tip"])).max()
    u_err = np.abs(out["u"][-1] - ref["u"][-1]).max() / np.abs(ref["u"][-1]).max()
    print(prec, "tip %.2e u %.2e macro its" % (tip_err, u_err), out["macro_its"], ref["macro_its"])
    assert u_err <= tol and tip_err <= tol
    assert fe2.compliance_error(out["compliance"], ref["compliance"])[1] <= tol
    if prec == "fp64":
        assert out["macro_its"] == ref["macro_its"]


def test_q8_shape_functions():
    """partition of unity, nodal interpolation and derivatives vs central differences"""
    for xi, eta in [(0.3, -0.7), (-0.2, 0.9), (0.0, 0.0)]:
        N, dN = fe2.q8_shape(xi, eta)
        assert abs(N.sum() - 1.0) <= 1e-14 and np.abs(dN.sum(0)).max() <= 1e-14
        h = 1e-6
        fd = np.stack([(fe2.q8_shape(xi + h, eta)[0] - fe2.q8_shape(xi - h, eta)[0]) / (2 * h),
                       (fe2.q8_shape(xi, eta + h)[0] - fe2.q8_shape(xi, eta - h)[0]) / (2 * h)], 1)
        assert np.abs(fd - dN).max() <= 1e-8
    for a, (xa, ea) in enumerate(fe2.Q8_XI):
        N, _ = fe2.q8_shape(xa, ea)
        assert np.abs(N - np.eye(8)[a]).max() <= 1e-14
