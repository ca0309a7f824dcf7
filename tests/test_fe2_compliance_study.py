"""Compliance error of the reduced two-scale solution against the full FE^2 solution: the
accuracy study of the paper's second example (Sec. 4.2, Table 1) on the synthetic void RVE.

For every model of the two-scale family (N = 5 .. 40 POD modes of one training set of 20
Sobol load-unload samples, ECM to integration error epsilon = 0.01), the FE^2 driver runs
the loading-unloading program with the reduced micro model at every macro Gauss point, and
once with the full-order micro model (the reference).  Prints, per model, N, the cubature
size Q, the mean relative compliance error over the load steps, its maximum, and the run
times of both two-scale solutions on the host cores.

The reduced micro model here is the FP64 oracle (test infrastructure); the library's micro
solver reproduces it on the GPU to rounding (tests/test_fe2.py).

As a test (CPU, about 10 s): the same study on a 2 x 1 macro mesh (8 macro points) over a
10-step loading-unloading program at Tbar = 60; the mean compliance error falls as modes are
added (N = 5, 10, 20, 30), as in the paper's Table 1, and every reduced run is faster than
the full FE^2 run.  As a script, the full study:

usage: python tests/test_fe2_compliance_study.py [--nx 4 --ny 2 --steps 50 --T 60 --out study.json]
"""
import argparse
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from oracle import fe, build_roms                                      # noqa: E402
from paper_2307_16894_gb300 import fe2, inputs, workload               # noqa: E402
from test_fe2 import OracleMicro                                       # noqa: E402

MODELS = ["rom_e2_n5", "rom_e2_n10", "rom_e2_n20", "rom_e2_n30", "rom_e2"]


def full_reference(macro, coef, T, steps):
    cfg = build_roms.CONFIGS["e2"]
    mesh = fe.Mesh(2, cfg["N"], build_roms.phase_2d)
    Gq = inputs.map_gradients(inputs.map_modes(2, 1, cfg["map_seed"]), mesh.X.reshape(-1, 2))
    geo = [fe.geometry(Gq, c) for c in coef]
    Finv = np.stack([g[0] for g in geo]).reshape(len(coef), mesh.nq, 2, 2)
    J = np.stack([g[1] for g in geo]).reshape(len(coef), mesh.nq)
    micro = fe.FullMicro(mesh, cfg["phases"], Finv, J)
    t0 = time.perf_counter()
    out = fe2.solve(macro, micro, T, steps, unload=True)
    return out, time.perf_counter() - t0, dict(ndof=mesh.ndof, nq=mesh.nq)


def test_compliance_error_falls_with_modes():
    macro = fe2.BeamMesh(nx=2, ny=1)
    coef = inputs.map_coefficients(2, fe2.beam_mu(macro))
    ref, t_full, _ = full_reference(macro, coef, 60.0, 10)
    means = []
    for name in MODELS[:4]:                                   # N = 5, 10, 20, 30
        rom = workload.load_model(name)
        t0 = time.perf_counter()
        out = fe2.solve(macro, OracleMicro(rom, coef), 60.0, 10, unload=True)
        t = time.perf_counter() - t0
        eps, mean = fe2.compliance_error(out["compliance"], ref["compliance"])
        assert np.isfinite(mean) and t < t_full, (name, t, t_full)
        means.append(mean)
    assert all(a > b for a, b in zip(means, means[1:])), means
    assert means[0] > 0.05 and means[-1] < 0.01, means


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=4)
    ap.add_argument("--ny", type=int, default=2)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--T", type=float, default=60.0)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    macro = fe2.BeamMesh(nx=args.nx, ny=args.ny)
    coef = inputs.map_coefficients(2, fe2.beam_mu(macro))
    ref, t_full, info = full_reference(macro, coef, args.T, args.steps)
    rows = []
    print("full FE^2: %d macro points, RVE %d dofs / %d Gauss points, %.1f s, macro its %d" %
          (macro.nq, info["ndof"], info["nq"], t_full, sum(ref["macro_its"])), flush=True)
    for name in MODELS:
        rom = workload.load_model(name)
        micro = OracleMicro(rom, coef)
        t0 = time.perf_counter()
        out = fe2.solve(macro, micro, args.T, args.steps, unload=True)
        t = time.perf_counter() - t0
        eps, mean = fe2.compliance_error(out["compliance"], ref["compliance"])
        row = dict(model=name, N=int(rom["n"]), Q=int(rom["m"]), eps_C_mean=mean, eps_C_max=float(np.nanmax(eps)),
                   seconds=t, speedup=t_full / t, macro_its=int(sum(out["macro_its"])))
        rows.append(row)
        print("N=%2d Q=%3d  mean eps_C %.3e  max %.3e  %.2f s (speed-up %.0fx)  macro its %d" %
              (row["N"], row["Q"], mean, row["eps_C_max"], t, row["speedup"], row["macro_its"]), flush=True)
    res = dict(macro_elements=macro.ne, macro_points=macro.nq, load_steps=args.steps, T_max=args.T,
               rve_full=info, full_seconds=t_full, full_macro_its=int(sum(ref["macro_its"])),
               compliance_full=ref["compliance"], models=rows)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
