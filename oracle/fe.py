"""ORACLE — test infrastructure only.

Full-order finite-element model of the micro problem on the parent domain
(Sec. 2.1-2.2 of arXiv 2307.16894): periodic fluctuation field w on the unit
cell [0,1]^d, mapped weak form (Eq. weakform-dep-mapped), its linearisation
(Eq. Dweakform-dep), Newton (Eq. full_newton, stop rule ||f||_2 <= tol),
effective stress (Eq. eff_stress_full) and effective stiffness by the d^2
tangent problems (Eqs. eff_stiffness_full, tangentproblem).

Discretisation (the paper uses T6 elements; the synthetic workloads use
structured grids): Q4 with 2x2 Gauss points in 2D (plane strain), hex8 with
2x2x2 Gauss points in 3D.  Void elements (element centroid inside the void)
are removed; nodes used only by removed elements carry no unknowns; one node
is fixed to remove the rigid translation of the periodic field.
"""
import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fe_elements

PHASE_VOID = -1


class Mesh:
    """Structured periodic mesh of N^d cells on [0,1]^d.

    phase_fn(centroid[d]) -> -1 (void, removed), 0 (matrix) or 1 (inclusion)."""

    def __init__(self, d, N, phase_fn):
        self.d, self.N = d, N
        h = 1.0 / N
        self.h = h
        corners = list(itertools.product((0, 1), repeat=d))
        if d == 2:
            corners = [(0, 0), (1, 0), (1, 1), (0, 1)]
        else:
            base = [(0, 0), (1, 0), (1, 1), (0, 1)]
            corners = [c + (0,) for c in base] + [c + (1,) for c in base]
        self.nen = len(corners)
        loc = np.array(corners, dtype=float) * 2.0 - 1.0          # reference coords of the nodes
        g1 = 1.0 / np.sqrt(3.0)
        gps = np.array(list(itertools.product((-g1, g1), repeat=d)))
        self.ngp = len(gps)
        # shape-function gradients on the reference cube, mapped to X^p: d/dX = (2/h) d/dxi
        dN = np.zeros((self.ngp, self.nen, d))
        Nv = np.zeros((self.ngp, self.nen))
        for g, xi in enumerate(gps):
            for a, xa in enumerate(loc):
                fac = np.prod([(1.0 + xa[c] * xi[c]) / 2.0 for c in range(d)])
                Nv[g, a] = fac
                for r in range(d):
                    dN[g, a, r] = (xa[r] / 2.0) * np.prod([(1.0 + xa[c] * xi[c]) / 2.0 for c in range(d) if c != r]) * (2.0 / h)
        self.dN, self.Nv = dN, Nv
        self.gw = np.full(self.ngp, (h / 2.0) ** d)
        cells = np.array(list(itertools.product(range(N), repeat=d)))[:, ::-1]   # x fastest
        cent = (cells + 0.5) * h
        phase = np.array([phase_fn(c) for c in cent], dtype=np.int64)
        keep = phase != PHASE_VOID
        self.cells = cells[keep]
        self.el_phase = phase[keep].astype(np.int32)
        self.ne = len(self.cells)
        strides = N ** np.arange(d)
        conn = np.zeros((self.ne, self.nen), dtype=np.int64)
        for a, c in enumerate(corners):
            conn[:, a] = (((self.cells + np.array(c)) % N) * strides).sum(1)
        self.conn = conn.astype(np.int32)
        self.nnode = N ** d
        used = np.zeros(self.nnode, bool)
        used[self.conn.ravel()] = True
        fixed = int(self.conn[0, 0])
        dofmap = -np.ones((self.nnode, d), dtype=np.int64)
        k = 0
        for nid in range(self.nnode):
            if used[nid] and nid != fixed:
                dofmap[nid] = np.arange(k, k + d)
                k += d
        self.dofmap = dofmap.astype(np.int32)
        self.ndof = k
        # Gauss-point positions in X^p
        xnode = np.zeros((self.ne, self.nen, d))
        for a, c in enumerate(corners):
            xnode[:, a, :] = (self.cells + np.array(c)) * h
        self.X = np.einsum("ga,ead->egd", Nv, xnode)               # [ne, ngp, d]
        self.nq = self.ne * self.ngp
        # element dof table and COO pattern
        edof = self.dofmap[self.conn].reshape(self.ne, self.nen * d)
        self.edof = edof
        ii = np.repeat(edof[:, :, None], edof.shape[1], axis=2)
        jj = np.repeat(edof[:, None, :], edof.shape[1], axis=1)
        mask = (ii >= 0) & (jj >= 0)
        self._coo = (ii[mask], jj[mask], mask)

    def assemble_vec(self, fe):
        f = np.zeros(self.ndof)
        m = self.edof >= 0
        np.add.at(f, self.edof[m], fe[m])
        return f

    def assemble_mat(self, Ke):
        ii, jj, mask = self._coo
        return sp.csr_matrix((Ke[mask], (ii, jj)), shape=(self.ndof, self.ndof))

    def grad_field(self, wdofs):
        """dw/dX^p at every Gauss point: [ne, ngp, d, d] (row = component)."""
        u = np.where(self.edof >= 0, wdofs[np.maximum(self.edof, 0)], 0.0).reshape(self.ne, self.nen, self.d)
        return np.einsum("ead,gar->egdr", u, self.dN)

    def mass_and_laplace(self):
        """V^p Gram matrix (Eq. Vdotproduct on the parent domain): mass + gradient terms."""
        d, nen = self.d, self.nen
        Me = np.einsum("g,ga,gb->ab", self.gw, self.Nv, self.Nv)
        Le = np.einsum("g,gar,gbr->ab", self.gw, self.dN, self.dN)
        blk = np.kron(Me + Le, np.eye(d))
        return self.assemble_mat(np.broadcast_to(blk, (self.ne, nen * d, nen * d)).copy())


def geometry(Gmu_q, coef):
    """F_mu = I + sum_k coef_k Gmu_k at every point; returns (Finv, J) with J = |det F_mu|."""
    d = Gmu_q.shape[-2]
    Fm = np.eye(d) + np.einsum("...abk,k->...ab", Gmu_q, np.atleast_1d(coef))
    det = np.linalg.det(Fm)
    if np.any(det <= 0):
        raise ValueError("det F_mu <= 0")
    return np.linalg.inv(Fm), np.abs(det)


def _newton(mesh, phases, Finv, J, Fb, w, Fp, xi, tol_rel, tol_abs, max_iter, nthreads):
    """Newton on f(w) = 0 at fixed history (Eq. full_newton), with a backtracking
    line search on ||f||_2 (halving, up to 10 times) for robustness of the
    training solves.  Returns (w, res, iters) or None when it fails."""
    res = fe_elements(mesh, phases, Finv, J, Fb, w, Fp, xi, want_K=True, nthreads=nthreads)
    f = mesh.assemble_vec(res["fe"])
    rn = np.linalg.norm(f)
    r0 = rn
    for it in range(max_iter + 1):
        if not np.isfinite(rn):
            return None
        if rn <= max(tol_rel * r0, tol_abs):
            return w, res, it
        if it == max_iter:
            return None
        K = mesh.assemble_mat(res["Ke"])
        dw = spla.spsolve(K.tocsc(), -f)
        if not np.all(np.isfinite(dw)):
            return None
        step = 1.0
        for _ in range(11):
            wt = w + step * dw
            rt = fe_elements(mesh, phases, Finv, J, Fb, wt, Fp, xi, want_K=True, nthreads=nthreads)
            ft = mesh.assemble_vec(rt["fe"])
            rnt = np.linalg.norm(ft)
            if np.isfinite(rnt) and rnt < rn:
                break
            step *= 0.5
        w, res, f, rn = wt, rt, ft, rnt
    return None


def solve_path(mesh, phases, Finv, J, Fbar_path, tol_rel=1e-10, tol_abs=1e-9, max_iter=40, nthreads=None,
               want_snapshots=True, want_Abar=False, verbose=False, max_split=8):
    """Full-order Newton along a macro load path (Sec. 2.1); each step starts from the
    previous solution.  A step whose Newton fails is split into two half increments
    (recursively, up to max_split levels; the paper notes that small load steps can be
    needed, Appendix A).  Returns per-step fluctuation w, weighted stress
    W = P F_mu^-T J (Eq. forcevector_rewritten) at all Gauss points, Pbar and optionally Abar."""
    d = mesh.d
    nq = mesh.nq
    Fp = np.tile(np.eye(3).ravel(), (nq, 1))
    xi = np.zeros(nq)
    w = np.zeros(mesh.ndof)
    Finv_q = Finv.reshape(nq, d, d)
    Jq = J.reshape(nq)
    out = dict(w=[], W=[], Pbar=[], Abar=[], iters=[], n_yield=[], substeps=[])
    omega = 1.0
    Fprev = np.eye(d)
    for k, Fb in enumerate(Fbar_path):
        # queue of sub-targets between Fprev and Fb
        todo = [(Fb, 0)]
        nsub = 0
        while todo:
            Ft, lev = todo[-1]
            sol = _newton(mesh, phases, Finv, J, Ft, w, Fp, xi, tol_rel, tol_abs, max_iter, nthreads)
            if sol is None:
                if lev >= max_split:
                    raise RuntimeError("FE Newton failed at step %d even after %d splits" % (k, lev))
                Fmid = 0.5 * (Fprev + Ft)
                todo.append((Fmid, lev + 1))
                continue
            w, res, it = sol
            Fp, xi = res["Fp_tr"], res["xi_tr"]
            Fprev = Ft
            todo.pop()
            nsub += 1
        if verbose:
            print("  step %d: %d sub-steps, last %d its, plastic %d" % (k, nsub, it, res["plastic"].sum()), flush=True)
        gwq = np.tile(mesh.gw, mesh.ne)
        P = res["Pq"].reshape(nq, d, d)
        out["Pbar"].append(np.einsum("q,q,qab->ab", gwq, Jq, P) / omega)       # Eq. eff_stress_full
        out["iters"].append(it)
        out["substeps"].append(nsub)
        out["n_yield"].append(int(res["plastic"].sum()))
        if want_snapshots:
            out["w"].append(w.copy())
            out["W"].append(np.einsum("qab,qcb->qac", P, Finv_q) * Jq[:, None, None])
        if want_Abar:
            K = mesh.assemble_mat(res["Ke"])
            out["Abar"].append(effective_stiffness(mesh, K, res["Aq"], Finv, J))
    return out


def effective_stiffness(mesh, K, Aq, Finv, J):
    """Abar by the d^2 tangent problems, Eqs. tangentproblem and eff_stiffness_full."""
    d, d2 = mesh.d, mesh.d * mesh.d
    nq = mesh.nq
    A = Aq.reshape(mesh.ne, mesh.ngp, d2, d2)
    Fi = Finv.reshape(mesh.ne, mesh.ngp, d, d)
    Jq = J.reshape(mesh.ne, mesh.ngp)
    gN = np.einsum("gar,egrb->egab", mesh.dN, Fi)                 # dN/dX^p F_mu^-1
    wJ = mesh.gw[None, :] * Jq
    lu = spla.splu(K.tocsc())
    Abar = np.zeros((d2, d2))
    for kl in range(d2):
        # b = -( int (d dw F^-1) : A J ) : E_kl
        Akl = A[:, :, :, kl].reshape(mesh.ne, mesh.ngp, d, d)     # [i,b] of A_{ib,kl}
        fe = -np.einsum("eg,egab,egib->eai", wJ, gN, Akl).reshape(mesh.ne, mesh.nen * d)
        b = mesh.assemble_vec(fe)
        qkl = lu.solve(b)
        gq = np.einsum("egmr,egrn->egmn", mesh.grad_field(qkl), Fi).reshape(mesh.ne, mesh.ngp, d2)
        dF = gq.copy()
        dF[:, :, kl] += 1.0
        Abar[:, kl] = np.einsum("eg,egij,egj->i", wJ, A, dF)
    return Abar
