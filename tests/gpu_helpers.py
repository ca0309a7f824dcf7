"""Helpers shared by the GPU parity tests: run the CUDA path (through the C ABI)
and the FP64 oracle on the same seeded inputs."""
import numpy as np

import oracle
from paper_2307_16894_gb300 import binding


def geometry_np(rom, coef):
    d, m = rom["d"], rom["m"]
    Gmu = rom["Gmu"].reshape(m, d, d, -1)
    Fm = np.eye(d)[None, None] + np.einsum("iack,bk->biac", Gmu, np.atleast_2d(coef))
    return np.linalg.inv(Fm), np.abs(np.linalg.det(Fm))


def cpinv_from_fp(Fp, d):
    Fi = np.linalg.inv(Fp)
    C = Fi @ np.swapaxes(Fi, -1, -2)
    if d == 2:
        return np.stack([C[..., 0, 0], C[..., 0, 1], C[..., 1, 1], C[..., 2, 2]], -1)
    return np.stack([C[..., 0, 0], C[..., 0, 1], C[..., 0, 2], C[..., 1, 1], C[..., 1, 2], C[..., 2, 2]], -1)


def torch_stream():
    """cudaStream_t of torch's current stream: contexts that exchange torch tensors with
    the library must run on it so that tensor lifetimes and kernels stay stream-ordered."""
    import torch
    return torch.cuda.current_stream().cuda_stream


class GpuRun:
    def __init__(self, rom, coef, device=0, stream=None):
        self.rom = rom
        d = rom["d"]
        self.ctx = binding.Context(d, device, stream)
        self.ctx.load_basis(rom["G"])
        self.ctx.load_cubature(rom["w"], rom["phase"], rom["phases"], rom["omega"])
        self.ctx.set_geometry(rom["Gmu"], coef)
        self.st = self.ctx.state_create(len(coef))

    def step(self, Fbar, **kw):
        opts = binding.make_opts(**kw)
        return self.ctx.step(self.st, opts, Fbar, want_abar=kw.get("want_abar", True))

    def close(self):
        self.st.close()
        self.ctx.close()


class OracleRun:
    def __init__(self, rom, coef):
        self.rom = rom
        d, n, m = rom["d"], rom["n"], rom["m"]
        B = len(coef)
        self.Finv, self.J = geometry_np(rom, coef)
        self.q = np.zeros((B, n))
        self.dq_prev = np.zeros((B, n))
        self.Fp = np.tile(np.eye(3), (B, m, 1, 1)).copy()
        self.xi = np.zeros((B, m))

    def step(self, Fbar, tol_rel=1e-10, tol_abs=0.0, max_iter=25, max_ls=6, start="plain", polar_split=True,
             sensitivity=False, **kw):
        q0 = self.q.copy()
        qs = self.q + (self.dq_prev if start == "prev" else 0.0)
        sk = {}
        if sensitivity:
            sk["dFinv"], sk["dJ"] = oracle.geometry_derivatives(self.rom, self.Finv, self.J)
        out = oracle.rom_batch(self.rom, self.Finv, self.J, Fbar, qs, self.Fp, self.xi, tol_rel, tol_abs, max_iter,
                               max_ls=max_ls, polar_split=polar_split, **sk)
        ok = out["status"] == 0
        self.dq_prev[ok] = qs[ok] - q0[ok]
        self.q[ok] = qs[ok]
        out["q"] = self.q.copy()
        return out


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)
