"""Seeded synthetic inputs for the hyper-reduced RVE solve.

This module holds no arithmetic of the method itself: it only draws seeded
random numbers and builds the inputs that both the CUDA path and the FP64
oracle consume (macro load paths, geometry parameters, the synthetic
geometric map).  Everything is a pure function of its seed.

Synthetic geometric map (stand-in for the paper's auxiliary problem,
Sec. 3.4, whose output is F_mu, F_mu^-1 and det F_mu at the cubature
points): Phi_mu(X) = X + sum_k c_k d_k(X) with d_k a seeded sum of low
periodic Fourier modes, so F_mu = I + sum_k c_k Gmu_k(X), Gmu_k = grad d_k,
each Gmu_k scaled so that max |(Gmu_k)_ab| = 0.3 on a dense grid.
  2D (one parameter, the void radius mu in [0.2, 0.35]): c_1 = mu.
  3D (three parameters, the inclusion semi-axes mu in [0.15, 0.35]^3):
      c_k = mu_k - 0.25 (the parent inclusion is the sphere of radius 0.25).
"""
import numpy as np

AMPLITUDE = 0.3


def map_modes(d, n_par, seed, n_modes=8):
    """Fourier coefficients of the displacement fields d_k: list (per k) of
    (kvec [M, d] int, amp [M, d], phase [M, d])."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_par):
        kv = []
        while len(kv) < n_modes:
            k = rng.integers(-2, 3, size=d)
            if np.any(k != 0):
                kv.append(k)
        kv = np.array(kv)
        amp = rng.standard_normal((n_modes, d)) / (1.0 + (kv ** 2).sum(1))[:, None]
        ph = rng.uniform(0.0, 2.0 * np.pi, size=(n_modes, d))
        out.append([kv, amp, ph])
    # normalise each Gmu_k on a dense grid
    g = 96 if d == 2 else 24
    axes = [np.arange(g) / g] * d
    X = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, d)
    for mode in out:
        G = _grad(mode, X)
        mode[1] = mode[1] * (AMPLITUDE / np.abs(G).max())
    return out


def _grad(mode, X):
    kv, amp, ph = mode
    arg = 2.0 * np.pi * (X @ kv.T)[:, :, None] + ph[None]          # [P, M, d(component a)]
    c = np.cos(arg) * amp[None]                                    # d/dX of sin
    # (G)_ab = d d_a / d X_b = sum_m amp_ma cos(.) 2 pi k_mb
    return np.einsum("pma,mb->pab", c, 2.0 * np.pi * kv.astype(float))


def map_gradients(modes, X):
    """Gmu_k(X) for all k: [P, d, d, n_par]."""
    return np.stack([_grad(m, np.asarray(X, float)) for m in modes], axis=-1)


def map_displacement(modes, X):
    """d_k(X): [P, d, n_par] (for plots / checks only)."""
    X = np.asarray(X, float)
    res = []
    for kv, amp, ph in modes:
        arg = 2.0 * np.pi * (X @ kv.T)[:, :, None] + ph[None]
        res.append((np.sin(arg) * amp[None]).sum(1))
    return np.stack(res, -1)


def map_coefficients(d, mu):
    """mu (physical geometry parameter) -> coefficients c of F_mu = I + sum c_k Gmu_k."""
    mu = np.asarray(mu, float)
    return mu if d == 2 else mu - 0.25


def rotation(d, rng):
    if d == 2:
        th = rng.uniform(-np.pi, np.pi)
        return np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, c, e = q
    return np.array([[a * a + b * b - c * c - e * e, 2 * (b * c - a * e), 2 * (b * e + a * c)],
                     [2 * (b * c + a * e), a * a - b * b + c * c - e * e, 2 * (c * e - a * b)],
                     [2 * (b * e - a * c), 2 * (c * e + a * b), a * a - b * b - c * c + e * e]])


def uniaxial_path(n_steps=20, inc=0.005):
    """Fbar_k = diag(1 + inc k, 1), k = 1..n_steps (2D)."""
    return np.array([np.diag([1.0 + inc * k, 1.0]) for k in range(1, n_steps + 1)])


def training_path_2d(seed, n_steps, lo=0.9, hi=1.1, shear=0.1):
    """Ubar = [[Uxx, Uxy], [Uxy, Uyy]] drawn uniformly, applied as a linear ramp
    I + (k/n)(Ubar - I), k = 1..n (Sec. 4.1 sampling ranges)."""
    rng = np.random.default_rng(seed)
    uxx, uyy = rng.uniform(lo, hi, 2)
    uxy = rng.uniform(-shear, shear)
    U = np.array([[uxx, uxy], [uxy, uyy]])
    I = np.eye(2)
    return np.array([I + (k / n_steps) * (U - I) for k in range(1, n_steps + 1)])


def sobol_samples(n, ranges, seed):
    """n quasi-random points of the box prod_j [lo_j, hi_j] from a scrambled Sobol sequence
    (seeded): the sampling of the training set of Sec. 4.2.  Returns [n, len(ranges)]."""
    import warnings
    from scipy.stats import qmc
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")          # n need not be a power of two
        z = qmc.Sobol(len(ranges), scramble=True, seed=seed).random(n)
    lo = np.array([r[0] for r in ranges], float)
    hi = np.array([r[1] for r in ranges], float)
    return lo + z * (hi - lo)


def load_unload_path(U, n_steps):
    """A macro stretch Ubar applied with the piecewise-linear amplitude of Sec. 4.2: t rises
    from 0 to 1 over the first half of the steps and falls back to 0 over the second half;
    Fbar_k = I + t_k (Ubar - I), k = 1..n_steps."""
    h = n_steps // 2
    k = np.arange(1, n_steps + 1)
    t = np.where(k <= h, k / h, (n_steps - k) / max(n_steps - h, 1))
    I = np.eye(len(U))
    return np.array([I + tk * (np.asarray(U) - I) for tk in t])


def stretch_path(d, seed, n_steps, lo=0.9, hi=1.15, rotate=True):
    """Random principal stretches in [lo, hi]^d with random principal axes Q, and
    (if rotate) a random macro rotation Rbar; both ramped linearly over n_steps:
    Fbar_k = Rbar(t_k) (I + t_k (Q diag(s) Q^T - I)), t_k = k/n."""
    rng = np.random.default_rng(seed)
    s = rng.uniform(lo, hi, d)
    Q = rotation(d, rng)
    U = Q @ np.diag(s) @ Q.T
    I = np.eye(d)
    if rotate:
        if d == 2:
            th = rng.uniform(-np.pi / 4, np.pi / 4)
            Rt = lambda t: np.array([[np.cos(t * th), -np.sin(t * th)], [np.sin(t * th), np.cos(t * th)]])
        else:
            ax = rng.standard_normal(3)
            ax /= np.linalg.norm(ax)
            th = rng.uniform(-np.pi / 4, np.pi / 4)
            Kx = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
            Rt = lambda t: I + np.sin(t * th) * Kx + (1 - np.cos(t * th)) * Kx @ Kx
    else:
        Rt = lambda t: I
    return np.array([Rt(k / n_steps) @ (I + (k / n_steps) * (U - I)) for k in range(1, n_steps + 1)])


def batch_paths(d, B, n_steps, seed0, lo=0.9, hi=1.15, rotate=True):
    """[B, n_steps, d, d]: instance b uses seed seed0 + b."""
    return np.stack([stretch_path(d, seed0 + b, n_steps, lo, hi, rotate) for b in range(B)])


def batch_mu(d, B, seed0, lo, hi):
    """Geometry parameter per instance, instance b drawn from seed seed0 + b (+ 7 offset stream)."""
    npar = 1 if d == 2 else 3
    return np.stack([np.random.default_rng(seed0 + b + 7_000_000).uniform(lo, hi, npar) for b in range(B)])
