"""Two-scale FE^2 driver with the reduced RVE model at every macro Gauss point (Sec. 4.2,
first-order homogenisation of Sec. 2): a 2D plane-strain macro structure [0, W] x [0, H]
(W = 2, H = 1) of 8-node serendipity (Q8) elements with 2 x 2 Gauss points (20 x 10 elements:
the 200 elements, 800 quadrature points and 1322 degrees of freedom of the paper's second
example), supported on Y = 0 and compressed by the distributed load
T(X) = Tbar (1 - (2 X / W - 1)^2) on Y = H (Tbar ramped up, and optionally back down to zero
as in the paper's loading program), solved by Newton's method on the macro displacement; the
compliance C = int_Gamma T u_y dx of every load step is the paper's accuracy measure.
At every macro Gauss point the effective stress Pbar and stiffness Abar come from the reduced
micro problem (one batched rom_step over all macro points per macro iteration, with a
per-point geometry parameter mu(X)).  The micro history is committed only at macro
convergence: the micro states are saved at the start of a load step and restored before
every macro iteration.

The micro solver is an object with save(), restore() and step(F [B, d, d]) -> (Pbar [B, d, d],
Abar [B, d*d, d*d], status [B]); RomMicro wraps a library context and state.

usage: python -m paper_2307_16894_gb300.fe2 [--nx 20 --ny 10 --steps 50 --T 80 --precision fp32 --unload]
"""
import argparse
import json
import time

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# Q8 reference nodes: corners counter-clockwise, then the mid-sides of the edges 1-2, 2-3, 3-4, 4-1
Q8_XI = np.array([[-1, -1], [1, -1], [1, 1], [-1, 1], [0, -1], [1, 0], [0, 1], [-1, 0]], float)


def q8_shape(xi, eta):
    """N [8] and dN/d(xi, eta) [8, 2] of the serendipity quadrilateral"""
    N = np.zeros(8)
    dN = np.zeros((8, 2))
    for a in range(4):
        xa, ea = Q8_XI[a]
        N[a] = 0.25 * (1 + xi * xa) * (1 + eta * ea) * (xi * xa + eta * ea - 1)
        dN[a, 0] = 0.25 * xa * (1 + eta * ea) * (2 * xi * xa + eta * ea)
        dN[a, 1] = 0.25 * ea * (1 + xi * xa) * (xi * xa + 2 * eta * ea)
    for a in range(4, 8):
        xa, ea = Q8_XI[a]
        if xa == 0:
            N[a] = 0.5 * (1 - xi * xi) * (1 + eta * ea)
            dN[a] = [-xi * (1 + eta * ea), 0.5 * ea * (1 - xi * xi)]
        else:
            N[a] = 0.5 * (1 + xi * xa) * (1 - eta * eta)
            dN[a] = [0.5 * xa * (1 - eta * eta), -eta * (1 + xi * xa)]
    return N, dN


class BeamMesh:
    """[0, L] x [0, H] in nx x ny rectangular Q8 elements; 2 x 2 Gauss points per element;
    the edge Y = 0 is fixed, the edge Y = H carries the load."""

    def __init__(self, L=2.0, H=1.0, nx=20, ny=10):
        self.L, self.H, self.nx, self.ny = L, H, nx, ny
        hx, hy = L / nx, H / ny
        ids = -np.ones((2 * nx + 1, 2 * ny + 1), int)
        X = []
        for I in range(2 * nx + 1):
            for J in range(2 * ny + 1):
                if I % 2 == 1 and J % 2 == 1:
                    continue                      # element centres are not Q8 nodes
                ids[I, J] = len(X)
                X.append((I * hx / 2, J * hy / 2))
        self.X = np.array(X)
        self.nn = len(X)
        conn = []
        for ex in range(nx):
            for ey in range(ny):
                I, J = 2 * ex, 2 * ey
                conn.append([ids[I, J], ids[I + 2, J], ids[I + 2, J + 2], ids[I, J + 2],
                             ids[I + 1, J], ids[I + 2, J + 1], ids[I + 1, J + 2], ids[I, J + 1]])
        self.conn = np.array(conn)
        self.ne = len(conn)
        g = 1.0 / np.sqrt(3.0)
        self.dNdX = np.zeros((self.ne, 4, 8, 2))   # per element and Gauss point
        self.wdet = np.full((self.ne, 4), hx * hy / 4)
        self.Xq = np.zeros((self.ne, 4, 2))
        for e in range(self.ne):
            xe = self.X[self.conn[e]]
            for q, (xi, eta) in enumerate([(-g, -g), (g, -g), (g, g), (-g, g)]):
                N, dN = q8_shape(xi, eta)
                self.dNdX[e, q] = dN / np.array([hx / 2, hy / 2])
                self.Xq[e, q] = N @ xe
        self.nq = self.ne * 4
        self.ids = ids
        # gradient operator: vec(grad u)[2 i + j] = sum_(a, i') Bop[e, q, 2 i + j, 2 a + i'] u_e[2 a + i']
        self.Bop = np.zeros((self.ne, 4, 4, 16))
        for i in range(2):
            for j in range(2):
                self.Bop[:, :, 2 * i + j, i::2] = self.dNdX[:, :, :, j]
        self.BopT_w = self.Bop.transpose(0, 1, 3, 2) * self.wdet[:, :, None, None]
        # the edge Y = 0 is fixed; the edge Y = H carries t_y(X) = -(1 - (2 X / L - 1)^2) per unit
        # Tbar (consistent nodal forces, 3-point Gauss rule per quadratic edge)
        self.fixed = np.zeros((self.nn, 2), bool)
        self.fixed[ids[:, 0][ids[:, 0] >= 0]] = True
        self.free = np.flatnonzero(~self.fixed.ravel())
        f = np.zeros((self.nn, 2))
        s3 = np.sqrt(0.6)
        for ex in range(nx):
            nodes = [ids[2 * ex, 2 * ny], ids[2 * ex + 1, 2 * ny], ids[2 * ex + 2, 2 * ny]]
            x0 = ex * hx
            for s, wg in ((-s3, 5 / 9), (0.0, 8 / 9), (s3, 5 / 9)):
                Nl = [0.5 * s * (s - 1), 1 - s * s, 0.5 * s * (s + 1)]
                x = x0 + (s + 1) * hx / 2
                t = -(1.0 - (2.0 * x / L - 1.0) ** 2)
                for a in range(3):
                    f[nodes[a], 1] += wg * hx / 2 * Nl[a] * t
        self.f_unit = f.ravel()
        self.ndof = 2 * self.nn
        # sparsity of the element stiffness scatter
        dofs = (2 * self.conn[:, :, None] + np.arange(2)[None, None]).reshape(self.ne, 16)
        self.dofs = dofs
        self.rows = np.repeat(dofs, 16, axis=1).ravel()
        self.cols = np.tile(dofs, (1, 16)).ravel()
        # CSR pattern of the free-free block, built once: every element-matrix entry that
        # couples two free dofs has a slot (slot[keep]); assembly is one weighted bincount
        fmap = -np.ones(self.ndof, int)
        fmap[self.free] = np.arange(len(self.free))
        r, c = fmap[self.rows], fmap[self.cols]
        self.keep = (r >= 0) & (c >= 0)
        nf = len(self.free)
        key = r[self.keep] * nf + c[self.keep]
        uniq, self.slot = np.unique(key, return_inverse=True)
        self.ff_indices = (uniq % nf).astype(np.int32)
        self.ff_indptr = np.concatenate([[0], np.cumsum(np.bincount(uniq // nf, minlength=nf))]).astype(np.int32)

    def deformation_gradients(self, u):
        """F = I + grad u at every Gauss point, [ne * 4, 2, 2]"""
        ue = u.reshape(self.nn, 2)[self.conn]                       # [ne, 8, 2]
        F = np.eye(2)[None, None] + np.einsum("eai,eqaj->eqij", ue, self.dNdX)
        return F.reshape(-1, 2, 2)

    def element_arrays(self, P, A):
        """element force vectors [ne, 16] and stiffness matrices [ne, 16, 16] from Pbar [nq, 2, 2]
        and Abar [nq, 4, 4] (index (ij, kl)), 2 x 2 Gauss rule"""
        P = P.reshape(self.ne, 4, 4, 1)
        A = A.reshape(self.ne, 4, 4, 4)
        fe = np.matmul(self.BopT_w, P)[..., 0].sum(1)
        Ke = np.matmul(np.matmul(self.BopT_w, A), self.Bop).sum(1)
        return fe, Ke

    def assemble(self, P, A):
        """internal force and tangent (all dofs) from Pbar [nq, 2, 2], Abar [nq, 4, 4]"""
        fe, Ke = self.element_arrays(P, A)
        f = np.zeros(2 * self.nn)
        np.add.at(f, self.dofs, fe)
        K = sp.coo_matrix((Ke.ravel(), (self.rows, self.cols)), shape=(2 * self.nn, 2 * self.nn)).tocsr()
        return f, K

    def assemble_free(self, P, A):
        """internal force (all dofs) and the free-free block of the tangent (CSR, the pattern
        built once in the constructor)"""
        fe, Ke = self.element_arrays(P, A)
        f = np.bincount(self.dofs.ravel(), weights=fe.ravel(), minlength=self.ndof)
        data = np.bincount(self.slot, weights=Ke.ravel()[self.keep], minlength=len(self.ff_indices))
        nf = len(self.free)
        return f, sp.csr_matrix((data, self.ff_indices, self.ff_indptr), shape=(nf, nf))


def load_levels(T_max, nsteps, unload=False):
    """Tbar at every load step: a linear ramp from 0 to T_max over nsteps, or (unload) the
    loading program of the paper's second example (Sec. 4.2): up to T_max over the first
    half of the steps, back down to 0 over the second half."""
    k = np.arange(1, nsteps + 1)
    if not unload:
        return T_max * k / nsteps
    h = nsteps // 2
    return T_max * np.where(k <= h, k / h, (nsteps - k) / max(nsteps - h, 1))


def solve(mesh, micro, T_max, nsteps, unload=False, tol=1e-8, max_it=25, verbose=False):
    """Load steps Tbar_k from load_levels(); Newton on the free macro dofs until
    ||f_int - f_ext|| <= tol max_{j <= k} ||f_ext,j|| (the largest load applied so far, so
    that steps back at zero load have a scale).  Returns the displacement history, the
    compliance C_k = f_ext,k . u_k = int_Gamma T u_y dx of every load step (Sec. 4.2; exact
    for the finite-element displacement with the consistent load vector) and statistics."""
    u = np.zeros(2 * mesh.nn)
    free = mesh.free
    out = dict(u=[], tip=[], compliance=[], macro_its=[], T=[])
    ref = 0.0
    for k, T in enumerate(load_levels(T_max, nsteps, unload), start=1):
        fext = T * mesh.f_unit
        ref = max(ref, np.linalg.norm(fext[free]))
        micro.save()
        for it in range(max_it + 1):
            F = mesh.deformation_gradients(u)
            if it > 0:
                micro.restore()
            P, A, status = micro.step(F)
            if (status != 0).any():
                raise RuntimeError("micro problem did not converge at load step %d, macro iteration %d" % (k, it))
            fint, Kff = mesh.assemble_free(P, A)
            R = (fint - fext)[free]
            rn = np.linalg.norm(R)
            if verbose:
                print("step %d it %d |R| %.3e" % (k, it, rn))
            if rn <= tol * ref:
                break
            if it == max_it:
                raise RuntimeError("macro Newton did not converge at load step %d" % k)
            du = spla.splu(Kff.tocsc(), permc_spec="MMD_AT_PLUS_A").solve(-R)
            u[free] += du
        out["u"].append(u.copy())
        tip = mesh.ids[mesh.nx, 2 * mesh.ny]            # mid-span node of the loaded edge
        out["tip"].append(u.reshape(-1, 2)[tip].copy())
        out["compliance"].append(float(fext @ u))
        out["macro_its"].append(it)
        out["T"].append(float(T))
    return out


def compliance_error(C, C_ref):
    """Relative compliance error per load step, eps_C,k = |C_k - C_ref,k| / |C_ref,k|, and
    its mean over the load steps (Sec. 4.2).  Steps with C_ref,k = 0 (no load applied: the
    last step of the unloading program) have no relative error and are left out of the mean."""
    C, C_ref = np.asarray(C, float), np.asarray(C_ref, float)
    keep = C_ref != 0.0
    eps = np.full(len(C), np.nan)
    eps[keep] = np.abs(C[keep] - C_ref[keep]) / np.abs(C_ref[keep])
    return eps, float(eps[keep].mean())


class RomMicro:
    """Micro solver on the library: one context and state for all macro Gauss points."""

    def __init__(self, rom, coef, precision="fp32", device=0):
        from . import binding
        self.ctx = binding.Context(rom["d"], device)
        self.ctx.load_basis(rom["G"])
        self.ctx.load_cubature(rom["w"], rom["phase"], rom["phases"], rom["omega"])
        self.ctx.set_geometry(rom["Gmu"], coef)
        self.st = self.ctx.state_create(len(coef))
        mixed = precision != "fp64"
        self.opts = binding.make_opts(1e-9 if mixed else 1e-10, rom["tol_abs"], 50 if mixed else 25, 6, precision,
                                      "plain")
        self.saved = None
        self.micro_iters = 0
        self.micro_solves = 0

    def save(self):
        self.saved = self.st.export(history=True)

    def restore(self):
        self.st.import_(*self.saved)

    def step(self, F):
        P, A, info = self.ctx.step(self.st, self.opts, F)
        self.micro_iters += int(info["iters"].sum())
        self.micro_solves += len(F)
        return P, A, info["status"]

    def close(self):
        self.st.close()
        self.ctx.close()


def beam_mu(mesh, lo=0.2, hi=0.35):
    """geometry parameter of the RVE at every macro Gauss point: graded along the beam"""
    x = mesh.Xq.reshape(-1, 2)[:, 0] / mesh.L
    return (lo + (hi - lo) * x)[:, None]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=20)
    ap.add_argument("--ny", type=int, default=10)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--T", type=float, default=80.0)
    ap.add_argument("--unload", action="store_true", help="load to T over the first half of the steps, "
                    "unload to 0 over the second half (the paper's loading program)")
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "tf32", "bf16"])
    ap.add_argument("--model", default="c2")
    args = ap.parse_args()
    from . import inputs, workload
    rom = workload.load_model(workload.WORKLOADS[args.model]["model"])
    mesh = BeamMesh(nx=args.nx, ny=args.ny)
    coef = inputs.map_coefficients(2, beam_mu(mesh))
    micro = RomMicro(rom, coef, args.precision)
    t0 = time.perf_counter()
    out = solve(mesh, micro, args.T, args.steps, unload=args.unload)
    t = time.perf_counter() - t0
    print(json.dumps(dict(macro_elements=mesh.ne, macro_points=mesh.nq, load_steps=args.steps, unload=args.unload,
                          precision=args.precision, seconds=t, load_steps_per_s=args.steps / t,
                          micro_solves=micro.micro_solves, micro_solves_per_s=micro.micro_solves / t,
                          macro_iterations=int(sum(out["macro_its"])),
                          micro_newton_iters_mean=micro.micro_iters / max(micro.micro_solves, 1),
                          tip_displacement=[float(v) for v in out["tip"][-1]],
                          compliance=out["compliance"][-1])))
    micro.close()


if __name__ == "__main__":
    main()
