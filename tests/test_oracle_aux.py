"""Pins of the oracle's auxiliary geometry problem (Sec. 3.4, Eqs. auxiliary_problem and
reduced_aux_problem), against facts that do not come from the oracle itself:

* the element stiffness of the auxiliary elasticity (E = 1, nu = 0.25 as the paper takes them)
  has the rigid motions as its null space, and the energy of a homogeneous strain on one element
  equals the closed form 1/2 (lam (tr eps)^2 + 2 G eps:eps) h^d with lam = G = 0.4;
* det F_mu is a null Lagrangian integrated exactly by the Gauss rule of the bilinear / trilinear
  elements, so sum_q w_q det F_mu equals the area or volume of the mapped region: in 2D the unit
  cell minus the void scaled by (1 + theta)^2; in 3D the whole cell (its boundary is fixed) and the
  inclusion scaled by prod_k (1 + theta_k);
* theta = 0 leaves the parent domain unchanged;
* with boundary data linear in theta, N_p reduced modes and the DEIM interpolation reproduce the
  full-order map at parameters outside the training set (to rounding), and A_hat is symmetric
  positive definite;
* the stored model files: the reduced data they hold reproduce their full-order map Gmu."""
import os

import numpy as np
import pytest

from oracle import aux, build_roms
from paper_2307_16894_gb300 import workload


@pytest.fixture(scope="module")
def a2():
    return aux.AuxProblem(2, 16, build_roms.phase_2d, "void", build_roms.VOID_R)


@pytest.fixture(scope="module")
def a3():
    return aux.AuxProblem(3, 8, build_roms.phase_3d, "inclusion", build_roms.INCL_R)


@pytest.mark.parametrize("d", [2, 3])
def test_element_stiffness_rigid_modes_and_energy(d, a2, a3):
    A = a2 if d == 2 else a3
    mesh, Ke, h = A.mesh, A.Ke, 1.0 / A.N
    # nodal coordinates of the first element from its Gauss points (Nv is square and invertible)
    loc = np.linalg.solve(mesh.Nv, mesh.X[0])
    for k in range(d):                                     # translations
        u = np.zeros((mesh.nen, d))
        u[:, k] = 1.0
        assert np.abs(Ke @ u.ravel()).max() < 1e-12
    for a in range(d):                                     # infinitesimal rotations
        for b in range(a + 1, d):
            W = np.zeros((d, d))
            W[a, b], W[b, a] = 1.0, -1.0
            assert np.abs(Ke @ (loc @ W.T).ravel()).max() < 1e-12
    # E = 1, nu = 0.25: lam = G = 0.4; eps:C:eps = 1.2 for a unit uniaxial strain, 1.6 for the
    # shear eps_12 = eps_21 = 1
    uniax = np.zeros((d, d))
    uniax[0, 0] = 1.0
    shear = np.zeros((d, d))
    shear[0, 1] = shear[1, 0] = 1.0
    for eps, density in ((uniax, 1.2), (shear, 1.6)):
        u = (loc @ eps.T).ravel()
        assert abs(0.5 * u @ Ke @ u - 0.5 * density * h ** d) < 1e-13


def test_mapped_area_2d(a2):
    wq = np.tile(a2.mesh.gw, a2.mesh.ne)
    void_cells = a2.N ** 2 - a2.mesh.ne
    for theta in (-0.25, 0.0, 0.1, 0.27):
        F = np.eye(2) + a2.grad_at_gauss(a2.solve([theta]))
        det = np.linalg.det(F)
        assert det.min() > 0
        assert abs((wq * det).sum() - (1.0 - (1 + theta) ** 2 * void_cells / a2.N ** 2)) < 1e-13
        if theta == 0.0:
            assert np.abs(F - np.eye(2)).max() == 0.0


def test_mapped_volume_3d(a3):
    wq = np.tile(a3.mesh.gw, a3.mesh.ne)
    inc = np.repeat(a3.mesh.el_phase == 1, a3.mesh.ngp)
    v_incl = inc.sum() / a3.mesh.ngp / a3.N ** 3
    for theta in ([0.2, -0.3, 0.1], [-0.35, 0.35, 0.0]):
        F = np.eye(3) + a3.grad_at_gauss(a3.solve(theta))
        det = np.linalg.det(F)
        assert det.min() > 0
        assert abs((wq * det).sum() - 1.0) < 1e-13
        assert abs((wq * det)[inc].sum() - np.prod(1 + np.array(theta)) * v_incl) < 1e-14
        # the inclusion is mapped affinely: F = I + diag(theta) there
        assert np.abs(F[inc] - (np.eye(3) + np.diag(theta))).max() < 1e-13


@pytest.mark.parametrize("d", [2, 3])
def test_reduced_problem_exact_for_linear_data(d, a2, a3):
    A = a2 if d == 2 else a3
    rng = np.random.default_rng(3)
    train = rng.uniform(-0.3, 0.3, (2 * A.n_p + 2, A.n_p))
    red = A.reduce(train)
    assert red["Psi"].shape[1] == A.n_p and len(red["P"]) == A.n_p
    assert np.allclose(red["Ahat"], red["Ahat"].T, atol=1e-15) and np.linalg.eigvalsh(red["Ahat"]).min() > 0
    GL, GP = A.reduced_fields(red)
    for theta in rng.uniform(-0.35, 0.35, (3, A.n_p)):
        dh = A.reduced_solve(red, theta)
        u = A.solve(theta)
        Fr = np.einsum("qabk,k->qab", GL, theta) + np.einsum("qabj,j->qab", GP, dh)
        Ff = A.grad_at_gauss(u)
        assert np.abs(Fr - Ff).max() < 1e-12
        # the DEIM reconstruction of the forcing equals its projection
        b = -(A.KFD @ A.lifting(theta)[A.D])
        assert np.abs(red["Mdeim"] @ (red["S"] @ theta) - red["Psi"].T @ b).max() < 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("name", ["rom_a1", "rom_a3"])
def test_model_files_reduced_data_reproduce_map(name):
    if not os.path.exists(os.path.join(workload.DATA, name + ".npz")):
        pytest.skip("model file absent")
    rom = workload.load_model(name)
    d, m = rom["d"], rom["m"]
    rng = np.random.default_rng(5)
    for mu in rng.uniform(0.16, 0.34, (3, len(rom["aux_mu_ref"]))):
        theta = aux.theta_of_mu(mu, rom["aux_mu_ref"])
        dh = np.linalg.solve(rom["aux_Ahat"], rom["aux_Mdeim"] @ (rom["aux_S"] @ theta))
        Fr = np.einsum("ick,k->ic", rom["aux_GL"], theta) + np.einsum("icj,j->ic", rom["aux_Gpsi"], dh)
        Ff = np.einsum("ick,k->ic", rom["Gmu"], theta)
        assert Fr.shape == (m, d * d) and np.abs(Fr - Ff).max() < 1e-11
