"""ORACLE — test infrastructure only (tests, smoke() and the CPU-baseline leg of bench.py).

The auxiliary geometry problem of Sec. 3.4 (Eqs. auxiliary_problem and reduced_aux_problem;
the geometry steps of the offline and online stages of Algorithm 1), in plain FP64 numpy/scipy.

Full-order problem.  The parent-to-physical map is Phi_mu(X) = X + d(X), with d the
displacement of a linear-elastic body on the parent domain Omega^p (Eq. auxiliary_problem,
small strain, E_aux = 1, nu_aux = 0.25 as the paper takes them; plane strain in 2D).  The
outer boundary of the cell is fixed (d = 0) and d is prescribed on the part of the interior
that the parameters describe.  Here:
  * 2D porous cell: the void of parent radius r_p (its elements are removed) is mapped to a
    void of radius mu; on the nodes of the void boundary d = theta (X - X_c), theta = mu/r_p - 1;
  * 3D inclusion cell: the spherical inclusion of parent radius r_p becomes an ellipsoid with
    semi-axes mu_k; on every node of the inclusion d_k = theta_k (X - X_c)_k, theta_k = mu_k/r_p - 1
    (the inclusion itself is mapped affinely).
The discretisation is the RVE's own: Q4 (2x2 Gauss) or hex8 (2x2x2 Gauss) on the structured
parent grid.  F_mu = I + dd/dX^p at the Gauss points.

Reduced problem (Eq. reduced_aux_problem).  The free-dof part of d is approximated in the span
of N_p modes Psi (POD of full-order solutions at training parameters); the remainder is the
lifting L(theta) (the prescribed values on the Dirichlet nodes, zero elsewhere):
    A_hat = Psi^T K_FF Psi,   b(theta) = -K_FD L_D(theta),   b_hat = Psi^T b(theta),
with b_hat evaluated by the discrete empirical interpolation method: U = POD basis of b
snapshots, P = greedy interpolation rows, b_hat ~ Psi^T U (P^T U)^-1 b(theta)[P].  Then
    A_hat d_hat = b_hat(theta),   F_mu = I + grad L(theta) + sum_j d_hat_j grad psi_j.
The boundary data here are linear in theta, so b(theta)[P] = S theta with a stored
n_deim x N_p matrix S and grad L(theta) = sum_k theta_k grad L_k, and N_p modes reproduce the
full-order solution exactly (to rounding); the DEIM step interpolates b exactly as well.
"""
import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fe

E_AUX, NU_AUX = 1.0, 0.25


def elastic_tensor(d, E=E_AUX, nu=NU_AUX):
    """Isotropic small-strain stiffness C_irjs = lam d_ir d_js + G (d_ij d_rs + d_is d_rj)
    (plane strain in 2D)."""
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    G = E / (2 * (1 + nu))
    I = np.eye(d)
    return (lam * np.einsum("ir,js->irjs", I, I) + G * (np.einsum("ij,rs->irjs", I, I) +
                                                       np.einsum("is,rj->irjs", I, I)))


class AuxProblem:
    """Full-order auxiliary problem on the structured parent grid of an RVE family.

    kind "void": 2D, phase_fn marks void cells with -1 (removed); "inclusion": 3D, phase_fn
    marks inclusion cells with 1.  r_p: parent radius, X_c = (0.5, ...)."""

    def __init__(self, d, N, phase_fn, kind, r_p, E=E_AUX, nu=NU_AUX):
        self.d, self.N, self.kind, self.r_p = d, N, kind, r_p
        self.Xc = np.full(d, 0.5)
        self.n_p = 1 if kind == "void" else d
        mesh = fe.Mesh(d, N, phase_fn, fix_node=False)
        self.mesh = mesh
        h = 1.0 / N
        ids = np.arange(N ** d)
        idx = np.stack([(ids // N ** c) % N for c in range(d)], axis=1)      # node id = sum idx_c N^c
        self.Xn = idx * h
        used = np.zeros(N ** d, bool)
        used[mesh.conn.ravel()] = True
        outer = (idx == 0).any(axis=1)
        inner = np.zeros(N ** d, bool)
        cells = np.array(list(itertools.product(range(N), repeat=d)))[:, ::-1]
        cphase = np.array([phase_fn((c + 0.5) * h) for c in cells])
        corners = np.array(list(itertools.product((0, 1), repeat=d)))
        strides = N ** np.arange(d)
        mark = cphase == (-1 if kind == "void" else 1)
        for c in corners:
            inner[(((cells[mark] + c) % N) * strides).sum(1)] = True
        inner &= used & ~outer
        self.used, self.outer, self.inner = used, outer, inner
        # dofs of the used nodes: node-major, component-minor
        dof = -np.ones((N ** d, d), np.int64)
        nodes = np.nonzero(used)[0]
        dof[nodes] = np.arange(len(nodes) * d).reshape(-1, d)
        self.dof = dof
        self.ndof = len(nodes) * d
        dirich = np.zeros(self.ndof, bool)
        dirich[dof[used & (outer | inner)].ravel()] = True
        self.D = np.nonzero(dirich)[0]
        self.F = np.nonzero(~dirich)[0]
        # element stiffness (the same for every element of the structured grid)
        C = elastic_tensor(d, E, nu)
        Ke = np.einsum("g,gar,irjs,gbs->aibj", mesh.gw, mesh.dN, C, mesh.dN).reshape(mesh.nen * d, mesh.nen * d)
        self.Ke = Ke
        edof = dof[mesh.conn].reshape(mesh.ne, mesh.nen * d)
        ii = np.repeat(edof[:, :, None], edof.shape[1], axis=2).ravel()
        jj = np.repeat(edof[:, None, :], edof.shape[1], axis=1).ravel()
        self.K = sp.csr_matrix((np.broadcast_to(Ke, (mesh.ne,) + Ke.shape).ravel(), (ii, jj)),
                               shape=(self.ndof, self.ndof))
        self.KFF = self.K[self.F][:, self.F].tocsc()
        self.KFD = self.K[self.F][:, self.D].tocsr()
        self._lu = spla.splu(self.KFF)

    # ---- boundary data and full-order solution
    def boundary_map(self, k):
        """T_k of the linear boundary data g(theta)(X) = sum_k theta_k T_k (X - X_c)."""
        return np.eye(self.d) if self.kind == "void" else np.diag(np.eye(self.d)[k])

    def lifting(self, theta):
        """nodal vector (all dofs): the prescribed values on the interior Dirichlet nodes, zero elsewhere"""
        u = np.zeros((self.N ** self.d, self.d))
        T = sum(t * self.boundary_map(k) for k, t in enumerate(np.atleast_1d(theta)))
        u[self.inner] = (self.Xn[self.inner] - self.Xc) @ T.T
        out = np.zeros(self.ndof)
        out[self.dof[self.used].ravel()] = u[self.used].ravel()
        return out

    def solve(self, theta):
        """full-order solution (all dofs) of Eq. auxiliary_problem for the shape parameters theta"""
        u = self.lifting(theta)
        u[self.F] = self._lu.solve(-(self.KFD @ u[self.D]))
        return u

    def grad_at_gauss(self, u):
        """du/dX^p at every Gauss point of the kept elements: [nq, d, d] (row = component)"""
        mesh = self.mesh
        ue = u[self.dof[mesh.conn]]                                     # [ne, nen, d]
        return np.einsum("ead,gar->egdr", ue, mesh.dN).reshape(mesh.nq, self.d, self.d)

    def unit_gradients(self):
        """grad d of the full-order solutions for theta = e_k: [nq, d, d, N_p]; by linearity
        F_mu = I + sum_k theta_k of these at every Gauss point."""
        return np.stack([self.grad_at_gauss(self.solve(np.eye(self.n_p)[k])) for k in range(self.n_p)], axis=-1)

    # ---- reduced basis and DEIM (offline), reduced solve (online)
    def reduce(self, thetas, tol=1e-10):
        """RB + DEIM data of Eq. reduced_aux_problem from full-order solutions at the training
        parameters thetas [n_train, N_p]."""
        S_u = np.stack([self.solve(t)[self.F] for t in thetas], axis=1)
        Uu, su, _ = np.linalg.svd(S_u, full_matrices=False)
        r = int(np.sum(su > tol * su[0]))
        Psi = Uu[:, :r]
        Ahat = Psi.T @ (self.KFF @ Psi)
        S_b = np.stack([-(self.KFD @ self.lifting(t)[self.D]) for t in thetas], axis=1)
        Ub, sb, _ = np.linalg.svd(S_b, full_matrices=False)
        rb = int(np.sum(sb > tol * sb[0]))
        U = Ub[:, :rb]
        P = deim_indices(U)
        Mdeim = (Psi.T @ U) @ np.linalg.inv(U[P])
        # b(theta)[P] = S theta (linear boundary data)
        S = np.stack([-(self.KFD[P] @ self.lifting(np.eye(self.n_p)[k])[self.D]) for k in range(self.n_p)], axis=1)
        return dict(Psi=Psi, Ahat=Ahat, U=U, P=P, Mdeim=Mdeim, S=S, sigma_u=su, sigma_b=sb)

    def reduced_solve(self, red, theta):
        """d_hat of Eq. reduced_aux_problem: A_hat d_hat = M_deim S theta"""
        bhat = red["Mdeim"] @ (red["S"] @ np.atleast_1d(theta))
        return np.linalg.solve(red["Ahat"], bhat)

    def reduced_fields(self, red):
        """gradients at every Gauss point of the lifting per theta_k [nq, d, d, N_p] and of the
        modes psi_j [nq, d, d, r]"""
        GL = np.stack([self.grad_at_gauss(self.lifting(np.eye(self.n_p)[k])) for k in range(self.n_p)], axis=-1)
        GP = []
        for j in range(red["Psi"].shape[1]):
            u = np.zeros(self.ndof)
            u[self.F] = red["Psi"][:, j]
            GP.append(self.grad_at_gauss(u))
        return GL, np.stack(GP, axis=-1)


def deim_indices(U):
    """Greedy DEIM interpolation rows of the basis U (Chaturantabut and Sorensen's selection):
    the first row maximises |u_1|; row l maximises the residual of interpolating u_l at the rows
    already chosen."""
    P = [int(np.argmax(np.abs(U[:, 0])))]
    for l in range(1, U.shape[1]):
        c = np.linalg.solve(U[P, :l], U[P, l])
        r = U[:, l] - U[:, :l] @ c
        P.append(int(np.argmax(np.abs(r))))
    return np.array(P, dtype=np.int64)


def theta_of_mu(mu, r_p):
    """shape parameters of the boundary data: theta = mu / r_p - 1 (radius or semi-axes)"""
    return np.asarray(mu, dtype=np.float64) / r_p - 1.0
