"""Pins of the oracle's material point (Appendix A of arXiv 2307.16894) against
facts fixed by the mathematics: closed forms, textbook special cases,
invariants, finite differences."""
import json
import os

import numpy as np
import pytest

import oracle

MAT = dict(E=70e3, nu=0.3, law="power", s0=100.0, k=10.0, p=0.2)
# the matrix material of the paper's first example (tests/golden/paper_example1_material.json)
_EX1 = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                   "paper_example1_material.json")))["matrix"]
LIN = dict(E=_EX1["E"], nu=_EX1["nu"], law="linear", s0=_EX1["sigma_y0"], k=_EX1["H"], p=1.0)
ELAST = dict(E=700e3, nu=0.3, law="power", s0=np.inf, k=0.0, p=1.0)


def lame(ph):
    E, nu = ph["E"], ph["nu"]
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def iso_D(ph):
    lam, G = lame(ph)
    D = np.zeros((3, 3, 3, 3))
    for i, j, k, l in np.ndindex(3, 3, 3, 3):
        D[i, j, k, l] = lam * (i == j) * (k == l) + G * ((i == k) * (j == l) + (i == l) * (j == k))
    return D.reshape(9, 9)


def mat1(F, ph, Fp=None, xi=0.0, tangent=True, d=3):
    Fp = np.eye(3) if Fp is None else Fp
    P, A, P33, Fpn, xin, pl = oracle.material(d, F[None], Fp[None], np.array([xi]), 0, [ph], tangent)
    return P[0], (A[0] if A is not None else None), Fpn[0], xin[0], pl[0]


def rand_rot(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


@pytest.mark.parametrize("ph", [MAT, LIN, ELAST])
def test_zero_state(ph):
    P, A, Fpn, xin, pl = mat1(np.eye(3), ph)
    assert np.all(P == 0.0)
    assert np.allclose(A, iso_D(ph), rtol=0, atol=1e-10 * np.abs(iso_D(ph)).max())
    assert not pl and xin == 0.0


@pytest.mark.parametrize("ph", [MAT, LIN])
def test_elastic_limit(ph):
    rng = np.random.default_rng(3)
    H = rng.standard_normal((3, 3))
    dlt = 1e-6 * ph["s0"] / ph["E"]
    P, _, _, _, pl = mat1(np.eye(3) + dlt * H, ph, tangent=False)
    expect = (iso_D(ph) @ (0.5 * (H + H.T)).ravel()).reshape(3, 3) * dlt
    assert not pl
    assert np.abs(P - expect).max() <= 1e-5 * np.abs(expect).max()


def j2_principal(e, ph, ep=np.zeros(3), xi=0.0):
    """Textbook small-strain J2 radial return (Simo & Hughes 1998, Box 3.2) on principal
    strains, solved for dgamma by bisection -- independent of the oracle."""
    lam, G = lame(ph)
    ee = e - ep
    sig = lam * ee.sum() + 2 * G * ee
    s = sig - sig.mean()
    q = np.sqrt(1.5) * np.linalg.norm(s)

    def sy(x):
        if ph["law"] == "linear":
            return ph["s0"] + ph["k"] * x
        return ph["s0"] * (1 + ph["k"] * x) ** ph["p"]

    if q - sy(xi) <= 1e-12 * sy(xi):
        return sig, ep, xi
    lo, hi = 0.0, (q - sy(xi)) / (3 * G)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if q - 3 * G * mid - sy(xi + mid) > 0:
            lo = mid
        else:
            hi = mid
    dg = 0.5 * (lo + hi)
    r = np.sqrt(1.5) * s / np.linalg.norm(s)
    return sig - 2 * G * dg * r, ep + dg * r, xi + dg


@pytest.mark.parametrize("ph", [MAT, LIN])
def test_proportional_closed_form(ph):
    """Principal stretches with fixed axes: the model is small-strain J2 on e = ln(lambda)."""
    lams = [np.array([1.0 + 0.01 * t, 1.0 - 0.004 * t, 1.0 + 0.002 * t]) for t in range(1, 6)]
    Fp, xi = np.eye(3), 0.0
    ep, xr = np.zeros(3), 0.0
    for lm in lams:
        P, _, Fp, xi, pl = mat1(np.diag(lm), ph, Fp, xi, tangent=False)
        sig, ep, xr = j2_principal(np.log(lm), ph, ep, xr)
        assert np.abs(np.diag(P) - sig / lm).max() <= 1e-12 * np.abs(sig).max()
        assert np.abs(P - np.diag(np.diag(P))).max() <= 1e-12 * np.abs(sig).max()
        assert abs(xi - xr) <= 1e-12 * max(xr, 1e-3)
        assert np.allclose(Fp, np.diag(np.exp(ep)), rtol=1e-12, atol=1e-14)
    assert xi > 0


def test_linear_hardening_one_step():
    """Linear hardening: dgamma = f / (3G + H) in closed form (Eq. j2_2 with Eq. j2_4)."""
    ph = LIN
    lam, G = lame(ph)
    lm = np.array([1.05, 0.98, 1.0])
    P, _, _, xi, pl = mat1(np.diag(lm), ph, tangent=False)
    e = np.log(lm)
    sig = lam * e.sum() + 2 * G * e
    q = np.sqrt(1.5) * np.linalg.norm(sig - sig.mean())
    assert pl and abs(xi - (q - ph["s0"]) / (3 * G + ph["k"])) <= 1e-14


@pytest.mark.parametrize("ph", [MAT, ELAST])
def test_objectivity(ph):
    rng = np.random.default_rng(5)
    F = np.eye(3) + 0.03 * rng.standard_normal((3, 3))
    Fp = np.eye(3)
    if ph is MAT:
        _, _, Fp, xi0, _ = mat1(F, ph, tangent=False)
        F = F @ (np.eye(3) + 0.01 * rng.standard_normal((3, 3)))
    else:
        xi0 = 0.0
    P, A, Fpn, xin, _ = mat1(F, ph, Fp, xi0)
    Q = rand_rot(rng)
    P2, A2, Fpn2, xin2, _ = mat1(Q @ F, ph, Fp, xi0)
    sc = np.abs(P).max()
    assert np.abs(P2 - Q @ P).max() <= 1e-12 * sc
    A4 = A.reshape(3, 3, 3, 3)
    At = np.einsum("ia,ajbl,kb->ijkl", Q, A4, Q).reshape(9, 9)
    assert np.abs(A2 - At).max() <= 1e-10 * np.abs(A).max()
    assert np.abs(Fpn2 - Fpn).max() <= 1e-13 and abs(xin2 - xin) <= 1e-15


def test_invariants_det_and_monotone_xi():
    rng = np.random.default_rng(7)
    Fp, xi = np.eye(3), 0.0
    F = np.eye(3)
    for _ in range(12):
        F = F @ (np.eye(3) + 0.004 * rng.standard_normal((3, 3)))
        _, _, Fpn, xin, _ = mat1(F, MAT, Fp, xi, tangent=False)
        assert abs(np.linalg.det(Fpn) - 1.0) <= 1e-13
        assert xin >= xi
        Fp, xi = Fpn, xin
    assert xi > 0


def test_elastic_unloading_slope():
    """From a plastic state, a small reversal is elastic with the isotropic D slope in log strain."""
    lm = np.array([1.04, 1.0, 1.0])
    _, _, Fp, xi, pl = mat1(np.diag(lm), MAT, tangent=False)
    assert pl
    lm2 = lm * np.array([1 - 1e-5, 1.0, 1.0])
    P1, A, _, _, pl1 = mat1(np.diag(lm), MAT, Fp, xi)
    P2, _, _, xi2, pl2 = mat1(np.diag(lm2), MAT, Fp, xi, tangent=False)
    assert not pl2 and xi2 == xi
    lam, G = lame(MAT)
    de = np.log(lm2) - np.log(lm)
    dsig = lam * de.sum() + 2 * G * de
    # tau = P F^T along principal axes -> sigma_a = P_a lambda_a
    got = np.diag(P2) * lm2 - np.diag(P1) * lm
    assert np.abs(got - dsig).max() <= 1e-6 * np.abs(dsig).max()


@pytest.mark.parametrize("ph", [MAT, LIN, ELAST])
def test_tangent_fd_and_symmetry(ph):
    rng = np.random.default_rng(11)
    F = np.eye(3) + 0.02 * rng.standard_normal((3, 3))
    _, _, Fp, xi, _ = mat1(F, ph, tangent=False)
    F = F @ (np.eye(3) + 0.005 * rng.standard_normal((3, 3)))
    P, A, _, _, _ = mat1(F, ph, Fp, xi)
    h = 1e-6 * np.linalg.norm(F)
    Afd = np.zeros((9, 9))
    for kl in range(9):
        e = np.zeros(9)
        e[kl] = h
        Pp = mat1((F.ravel() + e).reshape(3, 3), ph, Fp, xi, tangent=False)[0]
        Pm = mat1((F.ravel() - e).reshape(3, 3), ph, Fp, xi, tangent=False)[0]
        Afd[:, kl] = ((Pp - Pm) / (2 * h)).ravel()
    sc = np.abs(A).max()
    assert np.abs(A - Afd).max() <= 1e-7 * sc
    assert np.abs(A - A.T).max() <= 1e-12 * sc


def test_plane_strain_block():
    rng = np.random.default_rng(13)
    F2 = np.eye(2) + 0.02 * rng.standard_normal((2, 2))
    F3 = np.eye(3)
    F3[:2, :2] = F2
    P3, A3, Fp3, xi3, _ = mat1(F3, MAT)
    P2, A2, _, _, _ = (lambda r: (r[0][0], r[1][0], r[3][0], r[4][0], r[5][0]))(
        oracle.material(2, F3[None], np.eye(3)[None], np.zeros(1), 0, [MAT]))
    assert np.array_equal(P2, P3[:2, :2])
    A34 = A3.reshape(3, 3, 3, 3)[:2, :2, :2, :2].reshape(4, 4)
    assert np.array_equal(A2, A34)
    assert np.abs(Fp3[:2, 2]).max() == 0 and np.abs(Fp3[2, :2]).max() == 0


def _two_step_nonproportional(ph):
    """Plastic stretch along x, then a plastic shear: F^p after the second step is a product
    of two non-commuting flow exponentials, so it is neither symmetric nor coaxial with the
    second flow direction."""
    F1 = np.diag([1.08, 0.96, 0.98])
    F2 = F1 @ np.array([[1.0, 0.12, 0.0], [0.0, 1.0, 0.04], [0.0, 0.0, 1.0]])
    _, _, Fp1, xi1, pl1 = mat1(F1, ph, tangent=False)
    P2, _, Fp2, xi2, pl2 = mat1(F2, ph, Fp=Fp1, xi=xi1, tangent=False)
    assert pl1 and pl2 and xi2 > xi1 > 0
    assert np.abs(Fp2 - Fp2.T).max() > 1e-4      # the case is non-trivial
    return F2, P2, Fp2, xi2


@pytest.mark.parametrize("ph", [MAT, LIN])
def test_committed_state_reproduces_stress(ph):
    """The return map lands on the yield surface, and the committed history (F^p, xi) is
    the one that produced the returned stress: evaluating the same F again from it gives
    the same P and no further plastic flow (Eqs. j2_2, j2_4, j2_10)."""
    F2, P2, Fp2, xi2 = _two_step_nonproportional(ph)
    P3, _, Fp3, xi3, _ = mat1(F2, ph, Fp=Fp2, xi=xi2, tangent=False)
    assert np.abs(P3 - P2).max() <= 1e-10 * np.abs(P2).max()
    assert np.abs(Fp3 - Fp2).max() <= 1e-12 and abs(xi3 - xi2) <= 1e-12 * xi2


@pytest.mark.parametrize("ph", [MAT, LIN, ELAST])
def test_kirchhoff_stress_symmetric(ph):
    """Balance of angular momentum: the Kirchhoff stress tau = P F^T is symmetric, also after
    non-proportional plastic flow with a non-symmetric F^p."""
    if np.isinf(ph["s0"]):
        F2 = np.array([[1.05, 0.2, 0.0], [-0.1, 0.97, 0.03], [0.02, 0.0, 1.01]])
        P2 = mat1(F2, ph, tangent=False)[0]
    else:
        F2, P2, _, _ = _two_step_nonproportional(ph)
    tau = P2 @ F2.T
    assert np.abs(tau - tau.T).max() <= 1e-12 * np.abs(tau).max()
