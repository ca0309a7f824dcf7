"""Ragged serving of many macro points whose RVE models differ in basis size n and
cubature size m (2D and 3D families), with admission by the device-memory footprint of
the per-instance state and per-step latency percentiles.

Every group (one model) is a context with its own stream and CUDA-graph step; rom_serve
issues all groups of a wave together so that they overlap on the GPU.  Instances that do
not fit the memory budget wait for a later wave of the same step; an instance's latency
for a step is the wave's start offset plus its group's completion time.
"""
import os

import numpy as np

from . import binding, inputs, workload

FAMILY_2D = ["r2_n16_m100", "r2_n24_m150", "r2_n32_m200"]
FAMILY_3D = ["r3_n48_m400", "r3_n64_m650", "r3_n95_m900"]


def available(names):
    return [n for n in names if os.path.exists(os.path.join(workload.DATA, "rom_%s.npz" % n))]


def make_groups(B_total, share_2d=0.75, steps=50, seed0=40_000, path_steps=50):
    """Split B_total instances over the available models (share_2d of them 2D); instance b of
    the whole batch uses seed seed0 + b for its geometry and its path_steps-step load path, of
    which the first `steps` steps are kept."""
    f2, f3 = available(FAMILY_2D), available(FAMILY_3D)
    n2 = int(round(B_total * share_2d)) if f3 else B_total
    n3 = B_total - n2 if f3 else 0
    groups, b0 = [], 0
    for fam, tot in ((f2, n2), (f3, n3)):
        for k, name in enumerate(fam):
            B = tot // len(fam) + (1 if k < tot % len(fam) else 0)
            if B == 0:
                continue
            rom = workload.load_model("rom_" + name)
            d = rom["d"]
            lo, hi = ((0.2, 0.35) if d == 2 else (0.15, 0.35))
            mu = np.stack([inputs.batch_mu(d, 1, seed0 + b0 + b, lo, hi)[0] for b in range(B)])
            paths = np.stack([inputs.stretch_path(d, seed0 + b0 + b, path_steps)[:steps] for b in range(B)])
            groups.append(dict(name=name, rom=rom, B=B, mu=mu, coef=inputs.map_coefficients(d, mu), paths=paths))
            b0 += B
    return groups


class Server:
    def __init__(self, groups, precision="fp32", start="prev", budget_bytes=None, device=0, autotune=True):
        import torch
        self.torch = torch
        self.groups = groups
        self.ctxs, self.states, self.opts, self.waves = [], [], [], []
        free, total = torch.cuda.mem_get_info(device)
        self.budget = budget_bytes if budget_bytes is not None else int(0.8 * free)
        used = 0
        for g in groups:
            rom = g["rom"]
            ctx = binding.Context(rom["d"], device)        # own stream per group
            ctx.load_basis(rom["G"])
            ctx.load_cubature(rom["w"], rom["phase"], rom["phases"], rom["omega"])
            ctx.set_geometry(rom["Gmu"], g["coef"])
            need = ctx.state_bytes(g["B"])
            # admission: a group whose state does not fit the remaining budget waits for the next wave
            g["wave"] = 0 if used + need <= self.budget else 1
            if g["wave"] == 0:
                used += need
            st = ctx.state_create(g["B"])
            tol = 1e-10 if precision == "fp64" else 1e-9
            opts = binding.make_opts(tol_rel=tol, tol_abs=rom["tol_abs"], max_iter=50, max_ls=6, precision=precision,
                                     start=start)
            self.ctxs.append(ctx)
            self.states.append(st)
            self.opts.append(opts)
            d, B = rom["d"], g["B"]
            g["F"] = torch.from_numpy(np.ascontiguousarray(g["paths"].transpose(1, 0, 2, 3))).cuda()
            g["P"] = torch.empty((B, d, d), dtype=torch.float64, device="cuda")
            g["A"] = torch.empty((B, d * d, d * d), dtype=torch.float64, device="cuda")
            g["I"] = torch.empty((B, binding.INFO_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
        self.autotune = autotune
        self.tuned = False
        torch.cuda.synchronize()

    def step(self, k):
        """Load step k for every instance; returns (wall ms, per-instance latency ms [B_total],
        per-instance info)."""
        torch = self.torch
        lat, infos = [], []
        t_wave = 0.0
        for wave in (0, 1):
            idx = [i for i, g in enumerate(self.groups) if g["wave"] == wave]
            if not idx:
                continue
            ms = binding.serve([self.ctxs[i] for i in idx], [self.states[i] for i in idx],
                               [self.opts[i] for i in idx], [self.groups[i]["F"][k] for i in idx],
                               [self.groups[i]["P"] for i in idx], [self.groups[i]["A"] for i in idx],
                               [self.groups[i]["I"] for i in idx])
            for i, t in zip(idx, ms):
                lat.append(np.full(self.groups[i]["B"], t_wave + t))
                infos.append(np.frombuffer(self.groups[i]["I"].cpu().numpy().tobytes(), dtype=binding.INFO_DTYPE))
            t_wave += float(ms.max())
        if self.autotune and not self.tuned:
            for i, g in enumerate(self.groups):
                self.ctxs[i].autotune(self.states[i], self.opts[i])
            self.tuned = True
        return t_wave, np.concatenate(lat), np.concatenate(infos)

    def close(self):
        for s in self.states:
            s.close()
        for c in self.ctxs:
            c.close()
