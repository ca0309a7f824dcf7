"""ORACLE — test infrastructure only.

Offline reduction of arXiv 2307.16894 (Sec. 3.1-3.2, the reduction steps of
the offline stage of Algorithm 1): POD of the fluctuation snapshots in the V^p inner product, POD of
the weighted-stress snapshots W = P F_mu^-T |det F_mu| in L^2(Omega^p), and
the empirical cubature (ECM) greedy that picks Gauss points and positive
weights integrating the N*L products dphi_i/dX^p : B_l (Eq. integral_ecm).
"""
import numpy as np
import scipy.optimize as so


def pod_method_of_snapshots(S, M, n):
    """First n POD modes of the columns of S, orthonormal in the inner product
    <u, v> = u^T M v (method of snapshots, no mean-centring).  Returns (Phi, sigma^2)."""
    C = S.T @ (M @ S)
    C = 0.5 * (C + C.T)
    lam, V = np.linalg.eigh(C)
    order = np.argsort(lam)[::-1]
    lam, V = lam[order], V[:, order]
    if n > np.sum(lam > lam[0] * 1e-14):
        raise ValueError("requested %d POD modes but the snapshot set has rank %d" % (n, np.sum(lam > lam[0] * 1e-14)))
    Phi = S @ (V[:, :n] / np.sqrt(lam[:n]))
    return Phi, lam


def snapshot_rank(mesh, snaps_w, rel=1e-14):
    """number of POD eigenvalues above rel * the largest (numerical rank in V^p)"""
    MV = mesh.mass_and_laplace()
    S = np.stack(snaps_w, axis=1)
    lam = np.linalg.eigvalsh(S.T @ (MV @ S))
    return int(np.sum(lam > lam.max() * rel))


def displacement_pod(mesh, snaps_w, n):
    """POD basis phi_1..phi_n of the fluctuation field, (phi_i, phi_j)_{V^p} = delta_ij
    (Eqs. pod_disp and the orthonormality relation after it)."""
    MV = mesh.mass_and_laplace()
    S = np.stack(snaps_w, axis=1)
    Phi, lam = pod_method_of_snapshots(S, MV, n)
    return Phi, lam, MV


def stress_pod(mesh, snaps_W, L):
    """POD basis B_1..B_L of the weighted stress, int B_m : B_n dX^p = delta_mn
    (Eqs. weighted_stress_pod and pod_P_orthonormal)."""
    d2 = mesh.d * mesh.d
    S = np.stack([W.reshape(-1) for W in snaps_W], axis=1)        # [nq*d2, ns]
    wq = np.repeat(np.tile(mesh.gw, mesh.ne), d2)
    import scipy.sparse as sp
    Bm, lam = pod_method_of_snapshots(S, sp.diags(wq), L)
    return Bm.T.reshape(L, mesh.nq, mesh.d, mesh.d), lam


def basis_gradients(mesh, Phi):
    """dphi_j/dX^p at every Gauss point: [nq, d, d, n] (row index = displacement component)."""
    n = Phi.shape[1]
    out = np.zeros((mesh.nq, mesh.d, mesh.d, n))
    for j in range(n):
        out[..., j] = mesh.grad_field(Phi[:, j]).reshape(mesh.nq, mesh.d, mesh.d)
    return out


def ecm_integrands(gradPhi, Bmodes):
    """Rows f_(i,l)(X_q) = dphi_i/dX^p : B_l at all Gauss points (Eq. integralsbasis)."""
    n = gradPhi.shape[-1]
    L = Bmodes.shape[0]
    return np.einsum("qabi,lqab->ilq", gradPhi, Bmodes).reshape(n * L, -1)


def ecm_greedy(Fint, wq, m=None, volume_weight=10.0, tol=None):
    """Empirical cubature (after Hernandez et al. 2017): greedy choice of Gauss points
    with positive weights so that sum_sel w f ~= sum_all wq f for every integrand row of
    Fint [P, M] and for the constant (volume) integrand.

    The weighted-stress snapshots are equilibrated, so the exact integrals of the rows
    vanish; the constant function fixes the scale (sum w = |Omega^p| of the material).
    The integrand space is replaced by an orthonormal basis (SVD of the
    sqrt(wq)-scaled rows) to which the normalised constant function (scaled by
    volume_weight) is appended.  At each step the candidate most aligned with the
    current integration residual is added and the weights are refit by non-negative
    least squares (points that fall to zero weight leave the set); the loop runs until
    m points are selected, or (m None) until the integration error below is <= tol, the
    error bound epsilon of the ECM (Sec. 3.2).

    Returns (idx, w, err) with err = ||Z_sel w - Z wq|| / ||Z wq|| in the orthonormal
    basis (every basis function has unit L^2 norm, so this is the RMS integration error
    of the N*L integrands relative to the volume term, Eq. integral_ecm)."""
    Mq = Fint.shape[1]
    sw = np.sqrt(wq)
    U, s, Vt = np.linalg.svd(Fint * sw[None, :], full_matrices=False)
    k = int(np.sum(s > s[0] * 1e-10))
    Z = Vt[:k] / sw[None, :]                      # orthonormal basis functions at the points [k, M]
    vol = np.sum(wq)
    Zx = np.vstack([Z, (volume_weight / np.sqrt(vol)) * np.ones((1, Mq))])
    bx = Zx @ wq
    colnorm = np.linalg.norm(Zx, axis=0)
    sel = []
    wsel = np.zeros(0)
    r = bx.copy()
    if m is None and tol is None:
        raise ValueError("ecm_greedy needs m or tol")
    nb = np.linalg.norm(bx)
    limit = 20 * (m if m is not None else Mq)
    guard = 0
    while (len(sel) < m if m is not None else np.linalg.norm(r) > tol * nb) and guard < limit:
        guard += 1
        c = (Zx.T @ r) / colnorm
        c[sel] = -np.inf
        i = int(np.argmax(c))
        cand = sel + [i]
        wn, _ = so.nnls(Zx[:, cand], bx, maxiter=50 * len(cand) + 500)
        keep = wn > 0
        sel = [p for p, kp in zip(cand, keep) if kp]
        wsel = wn[keep]
        r = bx - Zx[:, sel] @ wsel
    err = np.linalg.norm(r) / nb
    if m is not None and len(sel) != m:
        raise RuntimeError("ECM greedy stalled at %d of %d points" % (len(sel), m))
    if m is None and err > tol:
        raise RuntimeError("ECM greedy stalled at error %.3e > %.3e with %d points" % (err, tol, len(sel)))
    return np.array(sel), wsel, err
