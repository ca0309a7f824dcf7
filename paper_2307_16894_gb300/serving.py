"""Ragged serving of many macro points whose RVE models differ in basis size n and
cubature size m (2D and 3D families), with admission by the device-memory footprint of
the per-instance state and per-step latency percentiles.

The instances of all groups are split into waves whose states fit the memory budget
(plan_waves; a group may be split across waves).  Every chunk (a group's instances within
one wave) has its own context with the geometry of its instances.  Each wave is one
rom_serve call: ONE CUDA-graph launch in which every chunk's load step runs on its own branch
with its own device-driven Newton loop.  With a single wave the states stay resident between
load steps; with several, each wave's states are created, loaded with the host-resident
history (rom_state_import), stepped, written back (rom_state_export) and freed, so the
device never holds more than one wave's states.  An instance's latency for a step is its
wave's start offset plus the completion time of its chunk's branch.
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


def plan_waves(sizes, per_instance_bytes, budget):
    """Split instances into waves under a memory budget: greedy in group order; a wave takes
    whole groups while they fit and the part of the next group that still fits.  Returns a list
    of waves, each a list of (group, first instance, count)."""
    waves, cur, left = [], [], budget
    for g, (B, per) in enumerate(zip(sizes, per_instance_bytes)):
        if per > budget:
            raise ValueError("one instance of group %d needs %d bytes, more than the budget %d" % (g, per, budget))
        start = 0
        while start < B:
            fit = int(left // per)
            if fit == 0:
                waves.append(cur)
                cur, left = [], budget
                continue
            take = min(B - start, fit)
            cur.append((g, start, take))
            start += take
            left -= take * per
    if cur:
        waves.append(cur)
    return waves


def state_bytes_per_instance(groups, device=0):
    """device bytes of one instance's state for each group (rom_state_bytes, rounded up)"""
    per = []
    for g in groups:
        rom = g["rom"]
        probe = binding.Context(rom["d"], device)
        probe.load_basis(rom["G"])
        probe.load_cubature(rom["w"], rom["phase"], rom["phases"], rom["omega"])
        per.append(-(-probe.state_bytes(g["B"]) // g["B"]))
        probe.close()
    return per


class Server:
    def __init__(self, groups, precision="fp32", start="prev", budget_bytes=None, device=0, autotune=True):
        import torch
        self.torch = torch
        self.groups = groups
        tol = 1e-10 if precision == "fp64" else 1e-9
        per = state_bytes_per_instance(groups, device)
        self.state_bytes_per_instance = per
        free, total = torch.cuda.mem_get_info(device)
        self.budget = budget_bytes if budget_bytes is not None else int(0.8 * free)
        self.waves = plan_waves([g["B"] for g in groups], per, self.budget)
        self.resident = len(self.waves) == 1
        self.chunks = []
        for w, wave in enumerate(self.waves):
            for gi, s0, cnt in wave:
                g = groups[gi]
                rom = g["rom"]
                d = rom["d"]
                ctx = binding.Context(d, device)        # own context (and stream) per chunk
                ctx.load_basis(rom["G"])
                ctx.load_cubature(rom["w"], rom["phase"], rom["phases"], rom["omega"])
                ctx.set_geometry(rom["Gmu"], g["coef"][s0:s0 + cnt])
                opts = binding.make_opts(tol_rel=tol, tol_abs=rom["tol_abs"], max_iter=50, max_ls=6,
                                         precision=precision, start=start)
                nc = 4 if d == 2 else 6
                c = dict(group=gi, start=s0, count=cnt, wave=w, ctx=ctx, opts=opts, state=None,
                         F=torch.from_numpy(np.ascontiguousarray(g["paths"][s0:s0 + cnt].transpose(1, 0, 2, 3))).cuda(),
                         P=torch.empty((cnt, d, d), dtype=torch.float64, device="cuda"),
                         A=torch.empty((cnt, d * d, d * d), dtype=torch.float64, device="cuda"),
                         I=torch.empty((cnt, binding.INFO_DTYPE.itemsize), dtype=torch.uint8, device="cuda"))
                if self.resident:
                    c["state"] = ctx.state_create(cnt)
                else:
                    # host-resident history between waves: a = 0, C^p^-1 = I, xi = 0
                    cp = np.zeros((cnt, rom["m"], nc))
                    for comp in ((0, 2, 3) if d == 2 else (0, 3, 5)):
                        cp[:, :, comp] = 1.0
                    c["hist"] = (np.zeros((cnt, rom["n"])), cp, np.zeros((cnt, rom["m"])))
                self.chunks.append(c)
        for g in groups:
            g["wave"] = min(c["wave"] for c in self.chunks if groups[c["group"]] is g)
        self.autotune = autotune
        self.tuned = False
        torch.cuda.synchronize()

    def step(self, k):
        """Load step k for every instance; returns (wall ms, per-instance latency ms [B_total],
        per-instance info), both in group order."""
        lat = {}
        info = {}
        t_wave = 0.0
        for w in range(len(self.waves)):
            cs = [c for c in self.chunks if c["wave"] == w]
            if not self.resident:
                for c in cs:
                    c["state"] = c["ctx"].state_create(c["count"])
                    c["state"].import_(*c["hist"])
            ms = binding.serve([c["ctx"] for c in cs], [c["state"] for c in cs], [c["opts"] for c in cs],
                               [c["F"][k] for c in cs], [c["P"] for c in cs], [c["A"] for c in cs],
                               [c["I"] for c in cs])
            for c, t in zip(cs, ms):
                key = (c["group"], c["start"])
                lat[key] = np.full(c["count"], t_wave + t)
                info[key] = np.frombuffer(c["I"].cpu().numpy().tobytes(), dtype=binding.INFO_DTYPE).copy()
            if self.autotune and not self.tuned:
                for c in cs:
                    c["ctx"].autotune(c["state"], c["opts"])
            if not self.resident:
                for c in cs:
                    c["hist"] = c["state"].export()
                    c["state"].close()
                    c["state"] = None
            t_wave += float(ms.max())
        self.tuned = True
        keys = sorted(lat)
        return t_wave, np.concatenate([lat[k_] for k_ in keys]), np.concatenate([info[k_] for k_ in keys])

    def pbar(self, gi):
        """Pbar [B, d, d] of group gi after the last step (host)."""
        cs = sorted((c for c in self.chunks if c["group"] == gi), key=lambda c: c["start"])
        return np.concatenate([c["P"].cpu().numpy() for c in cs])

    def close(self):
        for c in self.chunks:
            if c["state"] is not None:
                c["state"].close()
            c["ctx"].close()
