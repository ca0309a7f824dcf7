"""Shape sensitivities dPbar/dmu (Eq. eff_sensitivities_full) from the GPU (rom_sensitivity) vs
the FP64 oracle's, whose formula is pinned by finite differences (test_oracle_sensitivity.py),
along the first load steps of the 2D and 3D workloads, on the FP64 path and on the
mixed-precision paths (FP32 tangent)."""
import os

import numpy as np
import pytest

from paper_2307_16894_gb300 import workload
from gpu_helpers import GpuRun, OracleRun

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def relmax(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("name,B,steps,prec,tol", [
    ("c2", 16, 8, "fp64", 1e-9), ("c2", 16, 8, "fp32", 1e-4),
    ("c3", 4, 5, "fp64", 1e-9), ("c3", 4, 5, "tf32", 1e-4), ("c3", 4, 5, "fp32", 1e-4)])
def test_sensitivity_vs_oracle(name, B, steps, prec, tol):
    if name == "c3" and not os.path.exists(os.path.join(workload.DATA, "rom_c3.npz")):
        pytest.skip("3D model file not generated")
    rom, mu, coef, paths = workload.batch(name, B=B)
    g = GpuRun(rom, coef)
    o = OracleRun(rom, coef)
    mixed = prec != "fp64"
    worst = 0.0
    for k in range(steps):
        P, A, info = g.step(paths[:, k], tol_rel=1e-9 if mixed else 1e-10, tol_abs=rom["tol_abs"],
                            max_iter=50 if mixed else 25, precision=prec, start="prev")
        S = g.ctx.sensitivity(g.st)
        ref = o.step(paths[:, k], tol_rel=1e-10, tol_abs=rom["tol_abs"], start="prev", sensitivity=True)
        assert (info["status"] == 0).all() and (ref["status"] == 0).all()
        assert np.isfinite(S).all()
        worst = max(worst, relmax(S, ref["dPdmu"]))
    print("%s %s dPbar/dmu max rel error vs oracle: %.2e" % (name, prec, worst))
    assert worst <= tol, worst
    g.close()
