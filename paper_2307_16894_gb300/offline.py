"""Offline stage on the device (the offline stage of Algorithm 1; Sec. 3.1-3.2).

Seeded training samples -> full-order training solves (rom_fe_train) -> POD of the fluctuation
snapshots in the V^p inner product (Eq. Vdotproduct) and of the weighted-stress snapshots in
L^2(Omega^p) (rom_pod) -> the ECM integrands dphi_i/dX^p : B_l (rom_ecm_integrands) -> the
empirical cubature (rom_ecm) -> the arrays the online stage loads: basis gradients G at the
selected points, positive weights, phases, geometric-map gradients and the Newton tolerance
scale.  Every solve, Gram product, eigenproblem, integrand and cubature step runs in
libpodecm.so; this module assembles the sparse V^p Gram matrix of the grid (setup data) and
moves arrays between host and device.
"""
import numpy as np
import scipy.sparse as sp

from . import binding


def vp_gram(grid):
    """The V^p Gram matrix on the grid's fluctuation dofs (Eq. Vdotproduct): for each element
    the Gauss sums of N_a N_b (mass) and dN_a . dN_b (gradient term), times the identity on the
    d components, assembled over the element dofs."""
    d, nen = grid.d, grid.nen
    mass = np.einsum("g,ga,gb->ab", grid.gw, grid.Nv, grid.Nv)
    grad = np.einsum("g,gar,gbr->ab", grid.gw, grid.dN, grid.dN)
    blk = np.kron(mass + grad, np.eye(d))                                  # [nen d, nen d]
    ed = grid.edof
    ii = np.repeat(ed[:, :, None], nen * d, axis=2)
    jj = np.repeat(ed[:, None, :], nen * d, axis=1)
    ok = (ii >= 0) & (jj >= 0)
    vals = np.broadcast_to(blk, ii.shape)[ok]
    return sp.csr_matrix((vals, (ii[ok], jj[ok])), shape=(grid.ndof, grid.ndof))


def build(grid, phases, Gq, coef, paths, n, L, m=None, tol=None, volume_weight=10.0, train_tol=(1e-10, 1e-9),
          max_iter=40):
    """The reduced model of a parameterised RVE family.

    grid: mesh.Grid of the parent domain; phases: material table; Gq [nq, d, d, n_par]: the
    geometric-map gradients at every Gauss point; coef [S, n_par] and paths [S, steps, d, d]: the
    training samples; n POD modes, L stress modes, m cubature points (or the error bound tol).
    Returns the model dict (the layout of the model files) and the training record."""
    import torch
    d, nq, ndof = grid.d, grid.nq, grid.ndof
    d2 = d * d
    tr = binding.fe_train(grid, phases, Gq, coef, paths, tol_rel=train_tol[0], tol_abs=train_tol[1],
                          max_iter=max_iter)
    Sw = torch.as_tensor(np.ascontiguousarray(tr["w"].reshape(-1, ndof)), device="cuda")
    Phi, lam_w, _ = binding.pod(Sw, n, M=vp_gram(grid))
    wq = np.tile(grid.gw, grid.ne)
    SW = torch.as_tensor(np.ascontiguousarray(tr["W"].reshape(-1, nq * d2)), device="cuda")
    Bm, lam_W, _ = binding.pod(SW, L, wdiag_d=torch.as_tensor(np.repeat(wq, d2), device="cuda"))
    gradPhi, F = binding.ecm_integrands(grid, Phi, Bm.reshape(L, nq, d2))
    sel, wsel, err, rank = binding.ecm(F, torch.as_tensor(wq, device="cuda"), m=m, tol=tol,
                                       volume_weight=volume_weight)
    G = gradPhi.cpu().numpy()[sel]                                        # [m, d2, n]
    mm = len(sel)
    phase = grid.el_phase[sel // grid.ngp].astype(np.int32)
    Gmu = np.ascontiguousarray(np.asarray(Gq).reshape(nq, d2, -1)[sel])
    s0 = min(p["s0"] for p in phases)
    # Newton tolerance scale: 1e-12 of sum_i w_i |G_i|_F sigma_y0 (the residual floor of a step
    # whose start residual vanishes)
    tol_abs = 1e-12 * float(np.sum(wsel * np.linalg.norm(G.reshape(mm, -1), axis=1))) * s0
    rom = dict(d=d, n=n, m=mm, G=G, w=wsel, phase=phase, qp_index=sel, X=grid.X.reshape(-1, d)[sel], Gmu=Gmu,
               omega=1.0, ecm_err=err, tol_abs=tol_abs,
               ph_E=np.array([p["E"] for p in phases]), ph_nu=np.array([p["nu"] for p in phases]),
               ph_law=np.array([1 if p["law"] == "power" else 0 for p in phases], np.int32),
               ph_s0=np.array([p["s0"] for p in phases]), ph_k=np.array([p["k"] for p in phases]),
               ph_p=np.array([p["p"] for p in phases]), lam_w=lam_w.cpu().numpy()[:n],
               lam_W=lam_W.cpu().numpy()[:L], n_snap=int(Sw.shape[0]), ecm_rank=rank)
    return rom, tr
