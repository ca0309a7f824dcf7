"""Error of every output of the step against the FP64 oracle, per precision (Pbar, Abar, the
reduced coordinates q and the equivalent plastic strain xi), with the Newton iterations of both
sides: the mixed-precision paths change the Jacobian (and the residual arithmetic), not the
converged answer.  2D: the first 8 load steps of 32 instances of the c2 workload; 3D: the first
6 load steps of 8 instances of the c3 workload.  The measured table is printed (-s)."""
import os

import numpy as np
import pytest

from paper_2307_16894_gb300 import workload
from gpu_helpers import GpuRun, OracleRun, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


CASES = {"c2": (32, 8), "c3": (8, 6)}
PRECS = [("fp64", False), ("fp32", False), ("fp32", True), ("tf32", False), ("tf32", True), ("bf16", False)]


def run_case(name, prec, fp64_residual):
    B, steps = CASES[name]
    rom, mu, coef, paths = workload.batch(name, B=B)
    paths = paths[:, :steps]
    g = GpuRun(rom, coef)
    o = OracleRun(rom, coef)
    mixed = prec != "fp64"
    err = dict(P=0.0, A=0.0, q=0.0, xi=0.0)
    its = np.zeros(2)
    for k in range(steps):
        P, A, info = g.step(paths[:, k], tol_rel=1e-9 if mixed else 1e-10, tol_abs=rom["tol_abs"],
                            max_iter=50 if mixed else 25, precision=prec, start="prev", fp64_residual=fp64_residual)
        ref = o.step(paths[:, k], tol_rel=1e-10, tol_abs=rom["tol_abs"], start="prev")
        assert (info["status"] == 0).all() and (ref["status"] == 0).all(), (name, prec, k)
        a, cp, xi = g.st.export()
        err["P"] = max(err["P"], rel(P, ref["Pbar"]))
        err["A"] = max(err["A"], rel(A, ref["Abar"]))
        err["q"] = max(err["q"], rel(a, o.q))
        err["xi"] = max(err["xi"], rel(xi, o.xi))
        its += (info["iters"].mean(), ref["iters"].mean())
    g.close()
    return err, its / steps


@pytest.mark.parametrize("name", ["c2", "c3"])
def test_errors_per_output(name):
    if name == "c3" and not os.path.exists(os.path.join(workload.DATA, "rom_c3.npz")):
        pytest.skip("3D model file not generated")
    rows = []
    for prec, f64r in PRECS:
        err, its = run_case(name, prec, f64r)
        label = prec + (" + FP64 residual" if f64r else "")
        rows.append((label, err, its))
        if prec == "fp64":
            assert err["P"] <= 1e-11 and err["q"] <= 1e-11 and err["xi"] <= 1e-11, err
            assert err["A"] <= 1e-9, err
        else:
            assert err["P"] <= 1e-7, (label, err)
            assert err["A"] <= 1e-4, (label, err)
    print("\n%s | precision | Pbar | Abar | q | xi | Newton its (GPU / oracle)" % name)
    for label, err, its in rows:
        print("%s | %s | %.1e | %.1e | %.1e | %.1e | %.2f / %.2f" % (name, label, err["P"], err["A"], err["q"],
                                                                     err["xi"], its[0], its[1]))
