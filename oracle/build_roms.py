"""ORACLE — offline ROM construction (the offline stage of Algorithm 1).

Writes data/rom_<name>.npz for the synthetic workloads: seeded training load
paths -> full-order FE solves on the parent mesh (Sec. 2) -> POD of the
fluctuation (V^p) and of the weighted stress (L^2) -> ECM points and weights
(Sec. 3.2) -> basis gradients G_i = dphi_j/dX^p at the selected points.  The
geometric map Gmu_k at the points comes from the seeded input generator, or,
for the families marked map="aux", from the auxiliary linear-elasticity problem
of Sec. 3.4 (oracle/aux.py): then Gmu_k = grad d of its full-order solution for
theta = e_k (the map is linear in theta = mu / r_p - 1), and the file also holds
the reduced auxiliary problem (RB operator, DEIM matrices, gradients of the
lifting and of the RB modes at the selected points) that the library solves on
the device.
Every stored value is produced by this script from oracle code only.

usage: python -m oracle.build_roms c1 [c2 c3 ...]
"""
import os
import sys
import time

import numpy as np

from . import aux, fe, reduction
from paper_2307_16894_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DATA = os.path.join(ROOT, "data")

MATRIX = dict(E=70e3, nu=0.3, law="power", s0=100.0, k=10.0, p=0.2)      # sigma_y = 100 (1 + 10 xi)^0.2
INCLUSION = dict(E=700e3, nu=0.3, law="power", s0=np.inf, k=0.0, p=1.0)  # elastic, stiffness ratio 10

VOID_R = 0.275           # parent void radius (2D family)
INCL_R = 0.25            # parent inclusion radius (3D family)


def phase_2d(c):
    return -1 if np.hypot(c[0] - 0.5, c[1] - 0.5) < VOID_R else 0


def phase_3d(c):
    return 1 if np.linalg.norm(np.asarray(c) - 0.5) < INCL_R else 0


CONFIGS = {
    # 2D 16x16 Q4, void, n=8, m=40, L=20, three 20-step training paths (seeds 1001-1003), map seed 7
    "c1": dict(d=2, N=16, n=8, m=40, L=20, map_seed=7, phases=[MATRIX],
               train=[("u2d", 1001 + i, 20) for i in range(3)], mu_range=(0.2, 0.35)),
    # 2D 64x64 Q4, same void, n=24 (32 modes kept for truncation), m=160, five 25-step paths
    "c2": dict(d=2, N=64, n=32, n_use=24, m=160, L=20, map_seed=7, phases=[MATRIX],
               train=[("stretch", 2001 + i, 25) for i in range(5)], mu_range=(0.2, 0.35)),
    # 3D 24^3 hex8, spherical elastic inclusion (stiffness ratio 10), n=64 (96 kept), m=600
    "c3": dict(d=3, N=24, n=96, n_use=64, m=600, L=20, map_seed=11, phases=[MATRIX, INCLUSION],
               train=[("stretch", 3001 + i, 20) for i in range(8)], mu_range=(0.15, 0.35),
               fft_pcg=True, tol_rel=1e-9, parallel=True),
    # the two-scale accuracy family (second example of Sec. 4.2, its sampling scheme): 2D 32x32 Q4, same
    # void; N_train = 20 Sobol samples of (Uxx, Uyy, Uxy, mu), each applied with the 40-step load-unload
    # amplitude; 40 POD modes kept, L = 20, ECM to integration error epsilon = 0.01.  The stretch ranges
    # cover the macro states of the compressed structure (|Ubar - I| of order 1e-2).
    # the auxiliary-problem families (Sec. 3.4): the map comes from the reduced linear-elasticity
    # problem of the void (2D, 16x16 Q4, radius mu in [0.2, 0.35]) or of the inclusion (3D, 12^3 hex8,
    # semi-axes mu in [0.15, 0.35]^3)
    "a1": dict(d=2, N=16, n=8, m=40, L=20, map="aux", phases=[MATRIX], map_seed=0,
               train=[("u2d", 5001 + i, 20) for i in range(3)], mu_range=(0.2, 0.35)),
    "a3": dict(d=3, N=12, n=16, m=100, L=20, map="aux", phases=[MATRIX, INCLUSION], map_seed=0,
               train=[("stretch", 6001 + i, 15) for i in range(4)], mu_range=(0.15, 0.35), parallel=True),
    "e2": dict(d=2, N=32, n=40, m=None, ecm_tol=0.01, L=20, map_seed=7, phases=[MATRIX],
               train=[("sobol", i, 40) for i in range(20)], mu_range=(0.2, 0.35), parallel=True,
               sobol=dict(n=20, seed=2307, ranges=[(0.995, 1.005), (0.98, 1.0), (-0.005, 0.005), (0.2, 0.35)])),
}


def aux_problem(cfg):
    """the auxiliary geometry problem (Sec. 3.4) of a family with map = "aux" on its parent grid"""
    d = cfg["d"]
    return aux.AuxProblem(d, cfg["N"], phase_2d if d == 2 else phase_3d, "void" if d == 2 else "inclusion",
                          VOID_R if d == 2 else INCL_R)


def map_fields(cfg, mesh):
    """Gmu_k at every Gauss point [nq, d, d, n_par] and the map coefficients of a parameter mu"""
    d = cfg["d"]
    if cfg.get("map") == "aux":
        A = aux_problem(cfg)
        return A.unit_gradients(), (lambda mu: aux.theta_of_mu(mu, A.r_p))
    modes = inputs.map_modes(d, 1 if d == 2 else 3, cfg["map_seed"])
    return inputs.map_gradients(modes, mesh.X.reshape(-1, d)), (lambda mu: inputs.map_coefficients(d, mu))


def aux_reduced(cfg, sel):
    """reduced auxiliary problem (RB + DEIM, Eq. reduced_aux_problem) trained on 2 N_p + 2 seeded
    shapes of the family's range, with its fields at the selected points"""
    A = aux_problem(cfg)
    rng = np.random.default_rng(7)
    mus = rng.uniform(*cfg["mu_range"], size=(2 * A.n_p + 2, A.n_p))
    red = A.reduce(aux.theta_of_mu(mus, A.r_p))
    GL, GP = A.reduced_fields(red)
    d = cfg["d"]
    m = len(sel)
    return dict(aux_Ahat=red["Ahat"], aux_Mdeim=red["Mdeim"], aux_S=red["S"], aux_P=red["P"],
                aux_mu_ref=np.full(A.n_p, A.r_p), aux_GL=GL[sel].reshape(m, d * d, -1),
                aux_Gpsi=GP[sel].reshape(m, d * d, -1), aux_sigma=red["sigma_u"][:A.n_p + 1])


def build(name, verbose=True, nthreads=None):
    cfg = CONFIGS[name]
    d, N = cfg["d"], cfg["N"]
    t0 = time.time()
    mesh = fe.Mesh(d, N, phase_2d if d == 2 else phase_3d)
    Gq, _ = map_fields(cfg, mesh)                                        # [nq, d, d, npar]
    modes = None
    if verbose:
        print("[%s] mesh ne=%d ndof=%d nq=%d" % (name, mesh.ne, mesh.ndof, mesh.nq), flush=True)
    snaps_w, snaps_W, train_info = [], [], []
    jobs = [(name, kind, seed, nst) for kind, seed, nst in cfg["train"]]
    if cfg.get("parallel"):
        import multiprocessing as mp
        nproc = min(len(jobs), os.cpu_count() or 1)
        with mp.get_context("spawn").Pool(nproc) as pool:
            results = pool.starmap(_train_path, [j + (max(1, (os.cpu_count() or 1) // nproc), verbose) for j in jobs])
    else:
        results = [_train_path(*j, nthreads, verbose) for j in jobs]
    for out, info in results:
        snaps_w += out["w"]
        snaps_W += out["W"]
        train_info.append(info)
    # keep the snapshots (outside the repo) so that the reduction can be redone without the FE solves
    np.savez(os.path.join(ROOT, "oracle", "_build", "snapshots_%s.npz" % name), w=np.stack(snaps_w),
             W=np.stack(snaps_W).astype(np.float32))
    n, L, m = cfg["n"], cfg["L"], cfg["m"]
    n = min(n, reduction.snapshot_rank(mesh, snaps_w))
    if verbose:
        print("[%s] POD modes kept: %d" % (name, n), flush=True)
    Phi, lam_w, MV = reduction.displacement_pod(mesh, snaps_w, n)
    Bm, lam_W = reduction.stress_pod(mesh, snaps_W, L)
    gradPhi = reduction.basis_gradients(mesh, Phi)                     # [nq, d, d, n]
    wq = np.tile(mesh.gw, mesh.ne)
    n_use = cfg.get("n_use", n)
    Fint = reduction.ecm_integrands(gradPhi[..., :n_use], Bm)
    t1 = time.time()
    sel, wsel, err = reduction.ecm_greedy(Fint, wq, m, tol=cfg.get("ecm_tol"))
    if verbose:
        print("[%s] ECM m=%d err=%.3e (%.1fs); sum w=%.6f vs %.6f" % (name, len(sel), err, time.time() - t1,
                                                                     wsel.sum(), wq.sum()), flush=True)
    rom = pack(mesh, cfg, modes, Gq, gradPhi, sel, wsel, err, n_use)
    rom.update(dict(lam_w=lam_w[:n], lam_W=lam_W[:L], n_snap=len(snaps_w)))
    if cfg.get("map") == "aux":
        rom.update(aux_reduced(cfg, sel))
    os.makedirs(DATA, exist_ok=True)
    np.savez_compressed(os.path.join(DATA, "rom_%s.npz" % name), **rom)
    # the full set of basis gradients at all Gauss points is kept out of the repo; the
    # truncated (ragged) variants are refit from it by build_variant()
    np.savez(os.path.join(ROOT, "oracle", "_build", "offline_%s.npz" % name),
             gradPhi=gradPhi, Bm=Bm, wq=wq, el_phase=mesh.el_phase, X=mesh.X.reshape(-1, d), Gq=Gq)
    if verbose:
        print("[%s] done in %.1fs" % (name, time.time() - t0), flush=True)
    return rom


def _train_path(name, kind, seed, nst, nthreads, verbose):
    """One seeded full-order training solve (the training solves of the offline stage of Algorithm 1)."""
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    cfg = CONFIGS[name]
    d, N = cfg["d"], cfg["N"]
    mesh = fe.Mesh(d, N, phase_2d if d == 2 else phase_3d)
    npar = 1 if d == 2 else 3
    Gq, coef_of = map_fields(cfg, mesh)
    if kind == "sobol":
        sc = cfg["sobol"]
        smp = inputs.sobol_samples(sc["n"], sc["ranges"], sc["seed"])[seed]      # (Uxx, Uyy, Uxy, mu)
        mu = smp[3:4]
        path = inputs.load_unload_path(np.array([[smp[0], smp[2]], [smp[2], smp[1]]]), nst)
    else:
        mu = np.random.default_rng(seed).uniform(*cfg["mu_range"], size=npar)
        if kind == "u2d":
            path = inputs.training_path_2d(seed, nst)
        else:
            path = inputs.stretch_path(d, seed, nst, rotate=False)
    Finv, J = fe.geometry(Gq, coef_of(mu))
    precond = fe.FFTPreconditioner(mesh, cfg["phases"][0]["E"], cfg["phases"][0]["nu"]) if cfg.get("fft_pcg") else None
    t1 = time.time()
    out = fe.solve_path(mesh, cfg["phases"], Finv, J, path, nthreads=nthreads, verbose=verbose,
                        tol_rel=cfg.get("tol_rel", 1e-10), precond=precond)
    if verbose:
        print("[%s] training path seed %d done in %.1fs" % (name, seed, time.time() - t1), flush=True)
    return dict(w=out["w"], W=out["W"]), dict(seed=seed, mu=mu, steps=nst, Pbar_last=out["Pbar"][-1])


def pack(mesh, cfg, modes, Gq, gradPhi, sel, wsel, err, n_use):
    d = mesh.d
    G = gradPhi[sel][..., :n_use].reshape(len(sel), d * d, n_use)
    phase = mesh.el_phase[sel // mesh.ngp]
    phases = cfg["phases"]
    Gmu = Gq[sel].reshape(len(sel), d * d, -1)
    s0 = min(p["s0"] for p in phases)
    tol_abs = 1e-12 * float(np.sum(wsel * np.linalg.norm(G.reshape(len(sel), -1), axis=1))) * s0
    return dict(d=d, n=n_use, m=len(sel), G=G, w=wsel, phase=phase.astype(np.int32), qp_index=sel,
                X=mesh.X.reshape(-1, d)[sel], Gmu=Gmu, omega=1.0, ecm_err=err, tol_abs=tol_abs,
                ph_E=np.array([p["E"] for p in phases]), ph_nu=np.array([p["nu"] for p in phases]),
                ph_law=np.array([1 if p["law"] == "power" else 0 for p in phases], np.int32),
                ph_s0=np.array([p["s0"] for p in phases]), ph_k=np.array([p["k"] for p in phases]),
                ph_p=np.array([p["p"] for p in phases]), map_seed=cfg["map_seed"], N=cfg["N"],
                map=cfg.get("map", "synthetic"))


# ragged serving family: basis truncations of the 2D and 3D models with their own ECM rules
VARIANTS = {
    "r2_n16_m100": ("c2", 16, 100), "r2_n24_m150": ("c2", 24, 150), "r2_n32_m200": ("c2", 32, 200),
    "r3_n48_m400": ("c3", 48, 400), "r3_n64_m650": ("c3", 64, 650), "r3_n95_m900": ("c3", 95, 900),
    # two-scale accuracy family: N = 5 .. 40 modes, ECM to epsilon = 0.01 (m = None: set by the error bound)
    # (the base model rom_e2 itself has N = 40)
    "e2_n5": ("e2", 5, None), "e2_n10": ("e2", 10, None), "e2_n20": ("e2", 20, None), "e2_n30": ("e2", 30, None),
}


def build_variant(name, verbose=True):
    """Truncate the base model's POD basis to n modes and run the ECM greedy for m points
    (Sec. 3.2; Q grows with N*L, remark of Sec. 4.1)."""
    base, n, m = VARIANTS[name]
    cfg = CONFIGS[base]
    z = np.load(os.path.join(ROOT, "oracle", "_build", "offline_%s.npz" % base))
    gradPhi, Bm, wq = z["gradPhi"], z["Bm"], z["wq"]
    d = cfg["d"]
    mesh = fe.Mesh(d, cfg["N"], phase_2d if d == 2 else phase_3d)
    t1 = time.time()
    Fint = reduction.ecm_integrands(gradPhi[..., :n], Bm)
    sel, wsel, err = reduction.ecm_greedy(Fint, wq, m, tol=cfg.get("ecm_tol"))
    if verbose:
        print("[%s] ECM m=%d err=%.3e (%.1fs)" % (name, len(sel), err, time.time() - t1), flush=True)
    modes = inputs.map_modes(d, 1 if d == 2 else 3, cfg["map_seed"])
    rom = pack(mesh, cfg, modes, z["Gq"], gradPhi, sel, wsel, err, n)
    np.savez_compressed(os.path.join(DATA, "rom_%s.npz" % name), **rom)
    return rom


def load(path):
    """npz -> dict used by the oracle and by the CUDA binding"""
    z = np.load(path)
    rom = {k: z[k] for k in z.files}
    for k in ("d", "n", "m", "N", "map_seed"):
        rom[k] = int(rom[k])
    rom["omega"] = float(rom["omega"])
    rom["tol_abs"] = float(rom["tol_abs"])
    rom["phases"] = [dict(E=float(E), nu=float(nu), law="power" if law == 1 else "linear", s0=float(s0), k=float(k),
                          p=float(p)) for E, nu, law, s0, k, p in
                     zip(rom["ph_E"], rom["ph_nu"], rom["ph_law"], rom["ph_s0"], rom["ph_k"], rom["ph_p"])]
    return rom


if __name__ == "__main__":
    for nm in sys.argv[1:]:
        if nm in VARIANTS:
            build_variant(nm)
        else:
            build(nm)
