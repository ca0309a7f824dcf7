"""Model files (data/rom_*.npz) and batch inputs of the synthetic workloads.

A model file holds the basis gradients G [m, d*d, n] at the cubature points,
the weights w [m], the phase index [m] and table, the geometric-map
gradients Gmu [m, d*d, n_par] and the Newton tolerance scale.  The batch
inputs (geometry parameters, macro load paths) come from ``inputs``.
"""
import os

import numpy as np

from . import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DATA = os.path.join(ROOT, "data")

# workload definitions: model file, batch size, load steps, seeds, mu range, stretch range
WORKLOADS = {
    "c1": dict(model="rom_c1", B=1, steps=20, seed0=None, mu=(0.3, 0.3), uniaxial=True),
    "c2": dict(model="rom_c2", B=4096, steps=50, seed0=10_000, mu=(0.2, 0.35), stretch=(0.9, 1.15)),
    "c3": dict(model="rom_c3", B=16384, steps=50, seed0=20_000, mu=(0.15, 0.35), stretch=(0.9, 1.15)),
    # geometry from the reduced auxiliary problem (rom_set_geometry_aux): the batch's "coefficients"
    # are the shape parameters mu themselves (the device turns them into the map)
    "a1": dict(model="rom_a1", B=256, steps=20, seed0=50_000, mu=(0.2, 0.35), stretch=(0.9, 1.15), aux=True),
    "a3": dict(model="rom_a3", B=16384, steps=20, seed0=60_000, mu=(0.15, 0.35), stretch=(0.9, 1.15), aux=True),
}


def load_model(name):
    z = np.load(os.path.join(DATA, name + ".npz"))
    rom = {k: z[k] for k in z.files}
    for k in ("d", "n", "m"):
        rom[k] = int(rom[k])
    rom["omega"] = float(rom["omega"])
    rom["tol_abs"] = float(rom["tol_abs"])
    rom["phases"] = [dict(E=float(E), nu=float(nu), law="power" if law == 1 else "linear", s0=float(s0), k=float(k),
                          p=float(p)) for E, nu, law, s0, k, p in
                     zip(rom["ph_E"], rom["ph_nu"], rom["ph_law"], rom["ph_s0"], rom["ph_k"], rom["ph_p"])]
    return rom


def truncate(rom, n):
    """The same model with the first n basis functions (POD modes are ordered)."""
    r = dict(rom)
    r["G"] = np.ascontiguousarray(rom["G"][:, :, :n])
    r["n"] = n
    return r


def batch(name, B=None, steps=None, first=0):
    """(mu [B, n_par], map coefficients [B, n_par], Fbar paths [B, steps, d, d]) of a workload;
    instances first .. first+B-1 of the workload's seeded sequence.  For the auxiliary-geometry
    workloads the coefficients returned are mu (rom_set_geometry_aux takes the shape parameters)."""
    w = WORKLOADS[name]
    rom = load_model(w["model"])
    d = rom["d"]
    B = w["B"] if B is None else B
    steps = w["steps"] if steps is None else steps
    if w.get("uniaxial"):
        mu = np.full((B, 1), w["mu"][0])
        paths = np.broadcast_to(inputs.uniaxial_path(steps), (B, steps, d, d)).copy()
    else:
        mu = np.stack([inputs.batch_mu(d, 1, w["seed0"] + first + b, *w["mu"])[0] for b in range(B)])
        paths = np.stack([inputs.stretch_path(d, w["seed0"] + first + b, steps, *w["stretch"]) for b in range(B)])
    return rom, mu, (mu if w.get("aux") else inputs.map_coefficients(d, mu)), paths


def shard(name, B_per_rank, rank, steps=None):
    """Weak-scaling shard: rank r solves instances r*B .. (r+1)*B - 1 of the workload's seeded
    sequence (instances are independent, so no data exchange is needed)."""
    return batch(name, B=B_per_rank, steps=steps, first=rank * B_per_rank)
