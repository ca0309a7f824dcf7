"""Pins of the oracle's FE model, POD, ECM and online reduced solve (Secs. 2-3 of
arXiv 2307.16894) against facts fixed by the mathematics: patch tests, null
Lagrangians, orthonormality, brute-force full-order solves, finite differences,
objectivity, the linear limit."""
import numpy as np
import pytest

import oracle
from oracle import fe, reduction
from oracle.build_roms import MATRIX, INCLUSION, phase_2d
from paper_2307_16894_gb300 import inputs

LIN = dict(E=10.0, nu=0.3, law="linear", s0=0.2, k=5.0, p=1.0)


def iso_D2(ph):
    E, nu = ph["E"], ph["nu"]
    lam, G = E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))
    D = np.zeros((2, 2, 2, 2))
    for i, j, k, l in np.ndindex(2, 2, 2, 2):
        D[i, j, k, l] = lam * (i == j) * (k == l) + G * ((i == k) * (j == l) + (i == l) * (j == k))
    return D.reshape(4, 4)


def full_rom(mesh, phases):
    """Full basis (identity on the FE dofs) with full Gauss quadrature."""
    d = mesh.d
    G = np.zeros((mesh.ne, mesh.ngp, d * d, mesh.ndof))
    for e in range(mesh.ne):
        for g in range(mesh.ngp):
            for node in range(mesh.nen):
                nid = mesh.conn[e, node]
                for a in range(d):
                    dof = mesh.dofmap[nid, a]
                    if dof >= 0:
                        for r in range(d):
                            G[e, g, a * d + r, dof] = mesh.dN[g, node, r]
    m = mesh.ne * mesh.ngp
    return dict(d=d, n=mesh.ndof, m=m, G=G.reshape(m, d * d, mesh.ndof), w=np.tile(mesh.gw, mesh.ne),
                phase=np.repeat(mesh.el_phase, mesh.ngp), phases=phases, omega=1.0)


def run_rom(rom, Finv, J, path, tol_rel=1e-12, tol_abs=1e-12, polar_split=True, max_ls=6, max_iter=40):
    d, n, m = rom["d"], rom["n"], rom["m"]
    q = np.zeros((1, n))
    Fp = np.tile(np.eye(3), (1, m, 1, 1)).copy()
    xi = np.zeros((1, m))
    outs = []
    for Fb in path:
        o = oracle.rom_batch(rom, Finv[None], J[None], Fb[None], q, Fp, xi, tol_rel, tol_abs, max_iter,
                             max_ls=max_ls, polar_split=polar_split)
        assert o["status"][0] == 0
        o["q"] = q[0].copy()
        o["xi"] = xi[0].copy()
        outs.append(o)
    return outs, (q, Fp, xi)


def test_patch_homogeneous():
    """Homogeneous material, mu = 0 (F_mu = I): w = 0 and Pbar = P(Fbar) on a plastic path."""
    mesh = fe.Mesh(2, 4, lambda c: 0)
    Finv = np.tile(np.eye(2), (mesh.nq, 1, 1))
    J = np.ones(mesh.nq)
    path = [np.array([[1.0 + 0.004 * k, 0.002 * k], [0.001 * k, 1.0 - 0.003 * k]]) for k in range(1, 5)]
    out = fe.solve_path(mesh, [MATRIX], Finv, J, path)
    Fp, xi = np.eye(3), 0.0
    for k, Fb in enumerate(path):
        assert np.abs(out["w"][k]).max() <= 1e-12
        F3 = np.eye(3)
        F3[:2, :2] = Fb
        P, _, _, Fpn, xin, pl = oracle.material(2, F3[None], Fp[None], np.array([xi]), 0, [MATRIX], False)
        Fp, xi = Fpn[0], xin[0]
        assert np.abs(out["Pbar"][k] - P[0]).max() <= 1e-11 * np.abs(P).max()
    assert xi > 0


def test_geometry_null_lagrangian():
    """int det F_mu dX^p = |cell| = 1 for a periodic displacement of the map (up to quadrature)."""
    for d, npar, N in ((2, 1, 32), (3, 3, 12)):
        mesh = fe.Mesh(d, N, lambda c: 0)
        modes = inputs.map_modes(d, npar, 5)
        Gq = inputs.map_gradients(modes, mesh.X.reshape(-1, d))
        coef = np.full(npar, 0.33)
        _, J = fe.geometry(Gq, coef)
        vol = np.sum(np.tile(mesh.gw, mesh.ne) * J)
        assert abs(vol - 1.0) < 2e-3
        assert np.abs(Gq).max() <= 0.3 + 1e-2


def test_map_gradient_is_gradient():
    """Gmu = grad d (central differences of the generator's displacement field)."""
    modes = inputs.map_modes(3, 3, 9)
    X = np.random.default_rng(0).uniform(0, 1, (5, 3))
    G = inputs.map_gradients(modes, X)
    h = 1e-6
    for b in range(3):
        e = np.zeros(3)
        e[b] = h
        fd = (inputs.map_displacement(modes, X + e) - inputs.map_displacement(modes, X - e)) / (2 * h)
        assert np.abs(G[:, :, b, :] - fd).max() < 1e-6


@pytest.fixture(scope="module")
def tiny():
    mesh = fe.Mesh(2, 4, phase_2d)
    modes = inputs.map_modes(2, 1, 7)
    Gq = inputs.map_gradients(modes, mesh.X.reshape(-1, 2))
    Finv, J = fe.geometry(Gq, np.array([0.3]))
    return mesh, Finv, J


def test_rom_full_basis_equals_fe(tiny):
    """Full basis + full quadrature reproduces the brute-force FE solve (q, Pbar, Abar)."""
    mesh, Finv, J = tiny
    phases = [MATRIX]
    path = [np.array([[1.0 + 0.003 * k, 0.001 * k], [0.001 * k, 1.0 - 0.002 * k]]) for k in range(1, 3)]
    fo = fe.solve_path(mesh, phases, Finv, J, path, tol_rel=1e-13, tol_abs=1e-10, want_Abar=True)
    rom = full_rom(mesh, phases)
    ro, _ = run_rom(rom, Finv.reshape(-1, 2, 2), J.reshape(-1), path, tol_rel=1e-13, tol_abs=1e-10,
                    polar_split=False)
    for k in range(len(path)):
        sc = np.abs(fo["Pbar"][k]).max()
        assert np.abs(ro[k]["Pbar"][0] - fo["Pbar"][k]).max() <= 1e-9 * sc
        assert np.abs(ro[k]["q"] - fo["w"][k]).max() <= 1e-9 * np.abs(fo["w"][k]).max()
        assert np.abs(ro[k]["Abar"][0] - fo["Abar"][k]).max() <= 1e-8 * np.abs(fo["Abar"][k]).max()
        assert ro[k]["n_yield"][0] == fo["n_yield"][k]
    assert fo["n_yield"][-1] > 0


@pytest.fixture(scope="module")
def small_rom(tiny):
    """A POD/ECM model on the tiny mesh: n = 6, m = 20, from two training paths."""
    mesh, Finv, J = tiny
    snaps_w, snaps_W = [], []
    for seed in (1, 2):
        path = inputs.training_path_2d(seed, 8)
        o = fe.solve_path(mesh, [MATRIX], Finv, J, path)
        snaps_w += o["w"]
        snaps_W += o["W"]
    Phi, lam, MV = reduction.displacement_pod(mesh, snaps_w, 6)
    Bm, _ = reduction.stress_pod(mesh, snaps_W, 8)
    gP = reduction.basis_gradients(mesh, Phi)
    wq = np.tile(mesh.gw, mesh.ne)
    Fint = reduction.ecm_integrands(gP, Bm)
    sel, w, err = reduction.ecm_greedy(Fint, wq, 20)
    rom = dict(d=2, n=6, m=20, G=gP[sel].reshape(20, 4, 6), w=w, phase=np.zeros(20, np.int32),
               phases=[MATRIX], omega=1.0)
    return dict(rom=rom, Phi=Phi, MV=MV, snaps=np.stack(snaps_w, 1), lam=lam, sel=sel, w=w, err=err,
                Fint=Fint, wq=wq, Bm=Bm, Finv=Finv.reshape(-1, 2, 2)[sel], J=J.reshape(-1)[sel], mesh=mesh)


def test_pod_orthonormal_and_projection(small_rom):
    s = small_rom
    Phi, MV, S = s["Phi"], s["MV"], s["snaps"]
    assert np.abs(Phi.T @ MV @ Phi - np.eye(Phi.shape[1])).max() <= 1e-12
    errs = []
    for n in range(1, Phi.shape[1] + 1):
        P = Phi[:, :n]
        R = S - P @ (P.T @ (MV @ S))
        errs.append(np.einsum("ij,ij->", R, MV @ R))
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-12) for i in range(len(errs) - 1))
    # the projection error equals the sum of the discarded eigenvalues (method of snapshots)
    assert abs(errs[-1] - s["lam"][Phi.shape[1]:].sum()) <= 1e-8 * s["lam"].sum()


def test_stress_pod_orthonormal(small_rom):
    Bm, mesh = small_rom["Bm"], small_rom["mesh"]
    wq = np.tile(mesh.gw, mesh.ne)
    Gm = np.einsum("q,lqab,mqab->lm", wq, Bm, Bm)
    assert np.abs(Gm - np.eye(len(Bm))).max() <= 1e-12


def test_ecm_weights(small_rom):
    s = small_rom
    assert np.all(s["w"] > 0) and len(np.unique(s["sel"])) == len(s["sel"])
    assert abs(s["w"].sum() - s["wq"].sum()) <= 0.05 * s["wq"].sum()
    # the selected rule integrates the fitted integrands better than the rule that
    # spreads the same total weight uniformly over the same points
    ex = s["Fint"] @ s["wq"]
    e_ecm = np.linalg.norm(s["Fint"][:, s["sel"]] @ s["w"] - ex)
    e_uni = np.linalg.norm(s["Fint"][:, s["sel"]] @ np.full(len(s["sel"]), s["wq"].sum() / len(s["sel"])) - ex)
    assert e_ecm < e_uni
    assert s["err"] < 0.5


def test_rom_zero_load(small_rom):
    s = small_rom
    outs, _ = run_rom(s["rom"], s["Finv"], s["J"], [np.eye(2)], tol_abs=1e-12)
    assert outs[0]["iters"][0] == 0 and np.all(outs[0]["Pbar"] == 0) and np.all(outs[0]["q"] == 0)


def test_rom_abar_fd_and_schur(small_rom):
    """Abar (d^2 reduced tangent solves) vs central differences of the whole step, and vs
    the Schur form (sum wJA - B^T K^-1 B)/|Omega| built from the converged point tangents."""
    s = small_rom
    rom = s["rom"]
    Fa = np.array([[1.006, 0.002], [0.001, 0.995]])
    Fb = np.array([[1.012, 0.004], [0.003, 0.990]])
    outs, (q, Fp, xi) = run_rom(rom, s["Finv"], s["J"], [Fa])
    base = (q.copy(), Fp.copy(), xi.copy())

    def step(F):
        qq, ff, xx = base[0].copy(), base[1].copy(), base[2].copy()
        return oracle.rom_batch(rom, s["Finv"][None], s["J"][None], F[None], qq, ff, xx, 1e-13, 1e-13, 40,
                                polar_split=False), qq
    o, qs = step(Fb)
    A = o["Abar"][0]
    h = 1e-7
    Afd = np.zeros((4, 4))
    for kl in range(4):
        e = np.zeros(4)
        e[kl] = h
        Pp = step(Fb + e.reshape(2, 2))[0]["Pbar"][0]
        Pm = step(Fb - e.reshape(2, 2))[0]["Pbar"][0]
        Afd[:, kl] = ((Pp - Pm) / (2 * h)).ravel()
    assert np.abs(A - Afd).max() <= 1e-5 * np.abs(A).max()
    # Schur form from the converged state
    m, n = rom["m"], rom["n"]
    Fi, J = s["Finv"], s["J"]
    H = np.einsum("icn,n->ic", rom["G"], qs[0]).reshape(m, 2, 2)
    F = Fb[None] + H @ Fi
    F3 = np.tile(np.eye(3), (m, 1, 1))
    F3[:, :2, :2] = F
    _, Aq, _, _, _, _ = oracle.material(2, F3, base[1][0], base[2][0], 0, [MATRIX])
    gF = np.einsum("iarn,irb->inab", rom["G"].reshape(m, 2, 2, n), Fi).reshape(m, n, 4)
    wJ = rom["w"] * J
    K = np.einsum("i,inc,icd,ikd->nk", wJ, gF, Aq, gF)
    Bm = np.einsum("i,inc,icd->nd", wJ, gF, Aq)
    A0 = np.einsum("i,icd->cd", wJ, Aq)
    As = A0 - Bm.T @ np.linalg.solve(K, Bm)
    assert np.abs(A - As).max() <= 1e-10 * np.abs(A).max()


def test_rom_objectivity(small_rom):
    """With the polar split, Pbar(R Fbar) = R Pbar(Fbar) and Abar rotates accordingly."""
    s = small_rom
    Fb = np.array([[1.006, 0.002], [0.004, 0.995]])
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    o1, _ = run_rom(s["rom"], s["Finv"], s["J"], [Fb])
    o2, _ = run_rom(s["rom"], s["Finv"], s["J"], [R @ Fb])
    P1, P2 = o1[0]["Pbar"][0], o2[0]["Pbar"][0]
    assert np.abs(P2 - R @ P1).max() <= 1e-11 * np.abs(P1).max()
    A1 = o1[0]["Abar"][0].reshape(2, 2, 2, 2)
    A2 = o2[0]["Abar"][0].reshape(2, 2, 2, 2)
    # dP2 = R dP1 for dF2 = R dF1  ->  A2_ijkl = R_ia A1_ajbl R_kb
    At = np.einsum("ia,ajbl,kb->ijkl", R, A1, R)
    assert np.abs(A2 - At).max() <= 1e-9 * np.abs(A1).max()
    # Abar of the polar split vs central differences on the rotated input
    h = 1e-7
    F2 = R @ Fb
    for kl in range(4):
        e = np.zeros(4)
        e[kl] = h
        Pp = run_rom(s["rom"], s["Finv"], s["J"], [F2 + e.reshape(2, 2)])[0][0]["Pbar"][0]
        Pm = run_rom(s["rom"], s["Finv"], s["J"], [F2 - e.reshape(2, 2)])[0][0]["Pbar"][0]
        fd = ((Pp - Pm) / (2 * h)).ravel()
        assert np.abs(o2[0]["Abar"][0][:, kl] - fd).max() <= 1e-5 * np.abs(A2).max()


def test_rom_quadratic_convergence(small_rom):
    s = small_rom
    Fb = np.array([[1.004, 0.001], [0.0, 0.997]])
    res = []
    for it in range(0, 6):
        q = np.zeros((1, 6))
        Fp = np.tile(np.eye(3), (1, 20, 1, 1)).copy()
        xi = np.zeros((1, 20))
        o = oracle.rom_batch(s["rom"], s["Finv"][None], s["J"][None], Fb[None], q, Fp, xi, 1e-300, 0.0, it,
                             max_ls=0, polar_split=False)
        res.append(o["res"][0])
    r = np.array(res) / res[0]
    # last steps before round-off: the error exponent roughly doubles
    k = [i for i in range(1, len(r) - 1) if r[i + 1] > 1e-13]
    assert len(k) >= 1
    i = k[-1]
    assert np.log(r[i + 1]) / np.log(r[i]) > 1.6


def test_linear_limit_homogeneous():
    """Homogeneous cell, tiny strain: Pbar = D : eps (plane strain), Abar = D."""
    mesh = fe.Mesh(2, 4, lambda c: 0)
    ph = [LIN]
    rom = full_rom(mesh, ph)
    Finv = np.tile(np.eye(2), (rom["m"], 1, 1))
    J = np.ones(rom["m"])
    eps = np.array([[2e-5, 5e-6], [5e-6, -1e-5]])
    outs, _ = run_rom(rom, Finv, J, [np.eye(2) + eps], polar_split=False)
    D = iso_D2(LIN)
    expect = (D @ eps.ravel()).reshape(2, 2)
    assert np.abs(outs[0]["Pbar"][0] - expect).max() <= 1e-4 * np.abs(expect).max()
    assert np.abs(outs[0]["Abar"][0] - D).max() <= 1e-4 * np.abs(D).max()


def test_rom_cubature_scale_invariance(small_rom):
    """Scaling all cubature weights and the cell volume |Omega^p| by the same factor scales
    f and K alike and leaves the solution, Pbar and Abar unchanged (Eqs. forcevector_ecm,
    eff_stress_1, eff_stiffness_1: every cubature sum enters divided by |Omega^p| or as a
    homogeneous equation)."""
    s = small_rom
    path = [np.array([[1.0 + 0.004 * k, 0.002 * k], [0.001 * k, 1.0 - 0.003 * k]]) for k in range(1, 4)]
    ref, _ = run_rom(s["rom"], s["Finv"], s["J"], path, tol_rel=1e-12, tol_abs=1e-14)
    rom2 = dict(s["rom"], w=2.5 * s["rom"]["w"], omega=2.5 * s["rom"]["omega"])
    out, _ = run_rom(rom2, s["Finv"], s["J"], path, tol_rel=1e-12, tol_abs=1e-14)
    assert ref[-1]["n_yield"][0] > 0
    for a, b in zip(out, ref):
        assert np.abs(a["q"] - b["q"]).max() <= 1e-10 * np.abs(b["q"]).max()
        assert np.abs(a["Pbar"] - b["Pbar"]).max() <= 1e-10 * np.abs(b["Pbar"]).max()
        assert np.abs(a["Abar"] - b["Abar"]).max() <= 1e-9 * np.abs(b["Abar"]).max()
        assert a["iters"][0] == b["iters"][0]


@pytest.mark.parametrize("d,N", [(2, 16), (3, 6)])
def test_vp_gram_matrix_closed_form(d, N):
    """The V^p inner product (Eq. Vdotproduct: mass plus gradient term) on the full cell:
    a constant field has norm^2 = volume = 1, and the interpolant of u_0 = sin(2 pi X_1) has
    exactly the norm^2 of a piecewise-linear function of X_1 on the node spacing,
    sum_cells h/3 (a^2 + a b + b^2) + sum_cells (b - a)^2 / h (the other directions have
    unit extent and the 2x2(x2) Gauss rule integrates these products exactly)."""
    mesh = fe.Mesh(d, N, lambda c: 0, fix_node=False)
    MV = mesh.mass_and_laplace()
    h = 1.0 / N
    ids = np.arange(mesh.nnode)
    x = (ids % N) * h                                    # node ids run x fastest
    const = np.zeros(mesh.ndof)
    const[mesh.dofmap[:, 0]] = 1.0
    assert abs(const @ (MV @ const) - 1.0) <= 1e-12
    u = np.zeros(mesh.ndof)
    u[mesh.dofmap[:, 0]] = np.sin(2 * np.pi * x)
    a = np.sin(2 * np.pi * np.arange(N) * h)
    b = np.sin(2 * np.pi * (np.arange(N) + 1) * h)
    exact = np.sum(h / 3.0 * (a * a + a * b + b * b)) + np.sum((b - a) ** 2 / h)
    assert abs(u @ (MV @ u) - exact) <= 1e-12 * exact
    # the two components are orthogonal and weighted alike
    v = np.zeros(mesh.ndof)
    v[mesh.dofmap[:, 1]] = np.sin(2 * np.pi * x)
    assert abs(u @ (MV @ v)) <= 1e-12 * exact and abs(v @ (MV @ v) - exact) <= 1e-12 * exact
