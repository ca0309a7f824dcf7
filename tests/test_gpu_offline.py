"""The offline stage on the device (rom_pod, rom_ecm; the offline stage of Algorithm 1, Sec.
3.1-3.2) against the oracle on the same inputs.  Inputs: the 2D auxiliary-map family (16x16 Q4,
n = 8, L = 20, m = 40), whose three seeded full-order training solves the oracle runs here, and
a larger synthetic integrand set.

* POD of the fluctuation snapshots in the V^p inner product (Eq. Vdotproduct): the device modes
  are V^p-orthonormal (pin: Phi M Phi^T = I), their eigenvalues equal the oracle's and the modes
  equal the oracle's up to sign;
* POD of the weighted-stress snapshots in L^2(Omega^p): the same;
* ECM greedy on identical integrands (the oracle's POD modes and stress modes): the device selects
  the same points in the same order (the greedy depends only on the row space of the integrands,
  not on the orthonormal basis chosen for it), with the same weights and integration error."""
import time

import numpy as np
import pytest

from oracle import build_roms, fe, reduction
from paper_2307_16894_gb300 import binding

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def a1_offline():
    cfg = build_roms.CONFIGS["a1"]
    mesh = fe.Mesh(2, cfg["N"], build_roms.phase_2d)
    snaps_w, snaps_W = [], []
    for kind, seed, nst in cfg["train"]:
        out, _ = build_roms._train_path("a1", kind, seed, nst, 1, False)
        snaps_w += out["w"]
        snaps_W += out["W"]
    return cfg, mesh, np.stack(snaps_w), np.stack([W.reshape(-1) for W in snaps_W])


def align(Phi_dev, Phi_ref):
    """flip the device modes to the sign of the oracle's ([n, N] vs [N, n])"""
    sgn = np.sign(np.einsum("jx,xj->j", Phi_dev, Phi_ref))
    return Phi_dev * sgn[:, None]


def test_pod_fluctuation_vp(a1_offline):
    import torch
    cfg, mesh, S, _ = a1_offline
    n = cfg["n"]
    t0 = time.perf_counter()
    Phi_o, lam_o, MV = reduction.displacement_pod(mesh, list(S), n)
    t_o = time.perf_counter() - t0
    S_d = torch.as_tensor(S, device="cuda")
    t0 = time.perf_counter()
    Phi_d, lam_d, sweeps = binding.pod(S_d, n, M=MV.tocsr())
    torch.cuda.synchronize()
    t_d = time.perf_counter() - t0
    Phi, lam = Phi_d.cpu().numpy(), lam_d.cpu().numpy()
    gram = Phi @ (MV @ Phi.T)
    assert np.abs(gram - np.eye(n)).max() < 1e-10
    assert np.abs(lam[:n] - lam_o[:n]).max() / lam_o[0] < 1e-12
    assert np.abs(lam[:n] / lam_o[:n] - 1).max() < 1e-8
    Phi = align(Phi, Phi_o)
    err = np.abs(Phi - Phi_o.T).max() / np.abs(Phi_o).max()
    print("POD (V^p) ns=%d N=%d: modes %.2e, orthonormality %.2e, %d sweeps; device %.3f s, oracle %.3f s"
          % (S.shape[0], S.shape[1], err, np.abs(gram - np.eye(n)).max(), sweeps, t_d, t_o))
    assert err < 1e-7


def test_pod_stress_l2(a1_offline):
    import torch
    cfg, mesh, _, SW = a1_offline
    L = cfg["L"]
    Bm_o, lam_o = reduction.stress_pod(mesh, [w.reshape(mesh.nq, 2, 2) for w in SW], L)
    wq = np.repeat(np.tile(mesh.gw, mesh.ne), 4)
    Phi_d, lam_d, _ = binding.pod(torch.as_tensor(SW, device="cuda"), L, wdiag_d=torch.as_tensor(wq, device="cuda"))
    Phi, lam = Phi_d.cpu().numpy(), lam_d.cpu().numpy()
    assert np.abs((Phi * wq) @ Phi.T - np.eye(L)).max() < 1e-9
    assert np.abs(lam[:L] / lam_o[:L] - 1).max() < 1e-7
    ref = Bm_o.reshape(L, -1).T                                   # [N, L]
    Phi = align(Phi, ref)
    assert np.abs(Phi - ref.T).max() / np.abs(ref).max() < 1e-6


def test_ecm_same_points(a1_offline):
    import torch
    cfg, mesh, S, SW = a1_offline
    n, L, m = cfg["n"], cfg["L"], cfg["m"]
    Phi_o, _, _ = reduction.displacement_pod(mesh, list(S), n)
    Bm_o, _ = reduction.stress_pod(mesh, [w.reshape(mesh.nq, 2, 2) for w in SW], L)
    gradPhi = reduction.basis_gradients(mesh, Phi_o)
    F = reduction.ecm_integrands(gradPhi, Bm_o)
    wq = np.tile(mesh.gw, mesh.ne)
    t0 = time.perf_counter()
    sel_o, w_o, err_o = reduction.ecm_greedy(F, wq, m)
    t_o = time.perf_counter() - t0
    F_d, wq_d = torch.as_tensor(F, device="cuda"), torch.as_tensor(wq, device="cuda")
    t0 = time.perf_counter()
    sel_d, w_d, err_d, rank = binding.ecm(F_d, wq_d, m=m)
    t_d = time.perf_counter() - t0
    t0 = time.perf_counter()
    sel_2, w_2, _, _ = binding.ecm(F_d, wq_d, m=m)          # a second call: no first-use costs
    t_2 = time.perf_counter() - t0
    assert list(sel_2) == list(sel_d) and np.array_equal(w_2, w_d)
    print("ECM P=%d M=%d m=%d: rank %d, err %.4e (oracle %.4e); device %.3f s (first call %.3f s), oracle %.3f s"
          % (F.shape[0], F.shape[1], m, rank, err_d, err_o, t_2, t_d, t_o))
    assert list(sel_d) == list(sel_o)
    assert np.abs(w_d - w_o).max() <= 1e-9 * w_o.max()
    assert abs(err_d - err_o) <= 1e-9 * max(err_o, 1e-12) + 1e-12


@pytest.mark.parametrize("M,P,m,kmax", [(12000, 240, 80, 5), (16384, 480, 160, 8)])
def test_ecm_synthetic_larger(M, P, m, kmax):
    """Larger integrand sets: P smooth functions (products of low Fourier modes with seeded
    phases) at M scattered points with positive weights; the products span (2 kmax)^2
    trigonometric functions, so the set is rank-deficient (rank 100 and 252).  The second case has the sizes of the 2D workload's model (n L = 24 x 20
    integrands, m = 160)."""
    import torch
    rng = np.random.default_rng(11)
    X = rng.uniform(0, 1, (M, 2))
    wq = rng.uniform(0.5, 1.5, M) / M
    k = rng.integers(1, kmax + 1, (P, 2))
    ph = rng.uniform(0, 2 * np.pi, (P, 2))
    F = np.sin(2 * np.pi * k[:, :1] * X[:, 0] + ph[:, :1]) * np.cos(2 * np.pi * k[:, 1:] * X[:, 1] + ph[:, 1:])
    t0 = time.perf_counter()
    sel_o, w_o, err_o = reduction.ecm_greedy(F, wq, m)
    t_o = time.perf_counter() - t0
    t0 = time.perf_counter()
    sel_d, w_d, err_d, rank = binding.ecm(torch.as_tensor(F, device="cuda"), torch.as_tensor(wq, device="cuda"), m=m)
    t_d = time.perf_counter() - t0
    same = int(np.sum(np.array(sel_d) == np.array(sel_o)))
    print("ECM synthetic P=%d M=%d m=%d: rank %d, %d of %d points in the same order, err %.4e (oracle %.4e); "
          "device %.3f s, oracle %.3f s" % (P, M, m, rank, same, m, err_d, err_o, t_d, t_o))
    assert list(sel_d) == list(sel_o)
    assert np.abs(w_d - w_o).max() <= 1e-8 * w_o.max()
