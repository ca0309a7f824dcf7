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
import os

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fe_elements

PHASE_VOID = -1


class Mesh:
    """Structured periodic mesh of N^d cells on [0,1]^d.

    phase_fn(centroid[d]) -> -1 (void, removed), 0 (matrix) or 1 (inclusion)."""

    def __init__(self, d, N, phase_fn, fix_node=True):
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
        fixed = int(self.conn[0, 0]) if fix_node else -1
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


class FFTPreconditioner:
    """Approximate inverse of the periodic stiffness matrix by the homogeneous isotropic
    reference operator K0 on the same structured grid: K0 is block-circulant, so
    K0^-1 r is one FFT, a 3x3 (2x2) solve per frequency and one inverse FFT (zero
    frequency removed).  Used as the preconditioner of conjugate gradients for the
    full-order training solves on large meshes (no void elements)."""

    def __init__(self, mesh, E, nu):
        d, N = mesh.d, mesh.N
        full = Mesh(d, N, lambda c: 0, fix_node=False)
        Finv = np.tile(np.eye(d), (full.nq, 1, 1))
        J = np.ones(full.nq)
        res = fe_elements(full, [dict(E=E, nu=nu, law="power", s0=np.inf, k=0.0, p=1.0)], Finv, J, np.eye(d),
                          np.zeros(full.ndof), np.tile(np.eye(3).ravel(), (full.nq, 1)), np.zeros(full.nq))
        K0 = full.assemble_mat(res["Ke"])
        # dof index of (node, c) in the full mesh is 3 node + c (all nodes used)
        shape = (N,) * d
        sym = np.zeros(shape + (d, d), dtype=complex)
        for c in range(d):
            col = K0[:, c].toarray().ravel().reshape(N ** d, d)            # stencil around node 0
            g = col.reshape(shape[::-1] + (d,))                              # [z][y][x] ordering of node ids
            g = np.moveaxis(g, -1, 0)
            sym[..., :, c] = np.moveaxis(np.fft.fftn(g, axes=tuple(range(1, d + 1))), 0, -1)
        zero = (0,) * d
        sym[zero] = np.eye(d)
        inv = np.linalg.inv(sym)
        inv[zero] = 0.0
        self.inv, self.d, self.N, self.mesh = inv, d, N, mesh
        nid = np.repeat(np.arange(mesh.nnode), d)
        comp = np.tile(np.arange(d), mesh.nnode)
        dof = mesh.dofmap.reshape(-1)
        keep = dof >= 0
        self.pos = (nid[keep] * d + comp[keep])[np.argsort(dof[keep])]

    def apply(self, r):
        d, N = self.d, self.N
        full = np.zeros(N ** d * d)
        full[self.pos] = r
        g = np.moveaxis(full.reshape((N,) * d + (d,)), -1, 0)
        gh = np.fft.fftn(g, axes=tuple(range(1, d + 1)))
        uh = np.einsum("...ab,b...->a...", self.inv, gh)
        u = np.real(np.fft.ifftn(uh, axes=tuple(range(1, d + 1))))
        return np.moveaxis(u, 0, -1).reshape(-1)[self.pos]


def geometry(Gmu_q, coef):
    """F_mu = I + sum_k coef_k Gmu_k at every point; returns (Finv, J) with J = |det F_mu|."""
    d = Gmu_q.shape[-2]
    Fm = np.eye(d) + np.einsum("...abk,k->...ab", Gmu_q, np.atleast_1d(coef))
    det = np.linalg.det(Fm)
    if np.any(det <= 0):
        raise ValueError("det F_mu <= 0")
    return np.linalg.inv(Fm), np.abs(det)


def _linsolve(K, b, precond):
    if precond is None:
        return spla.spsolve(K.tocsc(), b)
    M = spla.LinearOperator(K.shape, matvec=precond.apply)
    x, info = spla.cg(K.tocsr(), b, rtol=1e-11, atol=0.0, maxiter=4000, M=M)
    return x if info == 0 else np.full_like(b, np.nan)


def _newton(mesh, phases, Finv, J, Fb, w, Fp, xi, tol_rel, tol_abs, max_iter, nthreads, precond=None):
    """Newton on f(w) = 0 at fixed history (Eq. full_newton), with a backtracking
    line search on ||f||_2 (halving, up to 10 times) for robustness of the
    training solves; trial points are evaluated without the tangent.  Returns
    (w, res, iters) or None when it fails."""
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
        if res["Ke"] is None:
            res = fe_elements(mesh, phases, Finv, J, Fb, w, Fp, xi, want_K=True, nthreads=nthreads)
        K = mesh.assemble_mat(res["Ke"])
        dw = _linsolve(K, -f, precond)
        if not np.all(np.isfinite(dw)):
            return None
        step = 1.0
        for _ in range(11):
            wt = w + step * dw
            rt = fe_elements(mesh, phases, Finv, J, Fb, wt, Fp, xi, want_K=False, nthreads=nthreads)
            ft = mesh.assemble_vec(rt["fe"])
            rnt = np.linalg.norm(ft)
            if np.isfinite(rnt) and rnt < rn:
                break
            step *= 0.5
        w, res, f, rn = wt, rt, ft, rnt
    return None


def solve_path(mesh, phases, Finv, J, Fbar_path, tol_rel=1e-10, tol_abs=1e-9, max_iter=40, nthreads=None,
               want_snapshots=True, want_Abar=False, verbose=False, max_split=8, precond=None):
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
            sol = _newton(mesh, phases, Finv, J, Ft, w, Fp, xi, tol_rel, tol_abs, max_iter, nthreads, precond)
            if sol is None:
                if lev >= max_split:
                    raise RuntimeError("FE Newton failed at step %d even after %d splits" % (k, lev))
                Fmid = 0.5 * (Fprev + Ft)
                todo.append((Fmid, lev + 1))
                continue
            w, res, it = sol
            Fp_prev_step, xi_prev_step = Fp, xi
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
            if res["Ke"] is None:
                res = fe_elements(mesh, phases, Finv, J, Fprev, w, Fp_prev_step, xi_prev_step, want_K=True,
                                  nthreads=nthreads)
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


class FullMicro:
    """Full-order micro problems at B macro points: the reference model of the two-scale
    comparison of Sec. 4.2 (the "full FE^2" solution).  Every point has its own geometry
    (F_mu^-1 and J at all Gauss points, from its mu), fluctuation field w and history
    (F^p, xi).  step(F) solves Eq. full_newton at every point from its current state and
    returns the effective stress (Eq. eff_stress_full) and stiffness (Eqs. tangentproblem,
    eff_stiffness_full, with the tangent at the converged fluctuation); the converged
    fluctuation and the trial history become the point's state.  save()/restore() bracket
    the macro iterations of a load step, as for the reduced model, so the history is
    committed only at macro convergence.

    Finv: [B, nq, d, d], J: [B, nq] (fe.geometry per point); omega: |Omega^p|."""

    def __init__(self, mesh, phases, Finv, J, omega=1.0, tol_rel=1e-10, tol_abs=1e-9, max_iter=40,
                 nthreads=None):
        self.mesh, self.phases = mesh, phases
        self.Finv, self.J, self.omega = Finv, J, omega
        B = len(J)
        self.w = np.zeros((B, mesh.ndof))
        self.Fp = np.tile(np.eye(3).ravel(), (B, mesh.nq, 1))
        self.xi = np.zeros((B, mesh.nq))
        self.tol_rel, self.tol_abs, self.max_iter, self.nthreads = tol_rel, tol_abs, max_iter, nthreads
        self.saved = None
        self.newton_iters = 0

    def save(self):
        self.saved = (self.w.copy(), self.Fp.copy(), self.xi.copy())

    def restore(self):
        self.w[:], self.Fp[:], self.xi[:] = self.saved

    def _point(self, b, F):
        mesh, d = self.mesh, self.mesh.d
        sol = _newton(mesh, self.phases, self.Finv[b], self.J[b], F, self.w[b], self.Fp[b], self.xi[b],
                      self.tol_rel, self.tol_abs, self.max_iter, 1)
        if sol is None:
            return None
        w, res, it = sol
        if res["Ke"] is None:
            res = fe_elements(mesh, self.phases, self.Finv[b], self.J[b], F, w, self.Fp[b], self.xi[b],
                              want_K=True, nthreads=1)
        K = mesh.assemble_mat(res["Ke"])
        Abar = effective_stiffness(mesh, K, res["Aq"], self.Finv[b], self.J[b])
        gwq = np.tile(mesh.gw, mesh.ne)
        Pbar = np.einsum("q,q,qab->ab", gwq, self.J[b], res["Pq"].reshape(mesh.nq, d, d)) / self.omega
        return Pbar, Abar, w, res["Fp_tr"], res["xi_tr"], it

    def step(self, F):
        """The points are independent: they run on a thread pool (the element routines and
        the sparse factorisations run outside the interpreter lock), one thread per point."""
        from concurrent.futures import ThreadPoolExecutor
        d = self.mesh.d
        B = len(F)
        Pbar = np.zeros((B, d, d))
        Abar = np.zeros((B, d * d, d * d))
        status = np.zeros(B, np.int32)
        with ThreadPoolExecutor(self.nthreads or os.cpu_count() or 1) as ex:
            results = list(ex.map(lambda b: self._point(b, F[b]), range(B)))
        for b, r in enumerate(results):
            if r is None:
                status[b] = 1
                continue
            Pbar[b], Abar[b], self.w[b], self.Fp[b], self.xi[b], it = r
            self.newton_iters += it
        return Pbar, Abar, status
