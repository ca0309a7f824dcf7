"""Tensor-core (tcgen05) stiffness assembly: K in TF32/BF16 vs the FP32 CUDA-core
assembly on the same tangent, and converged answers of the mixed-precision path vs
the FP64 oracle (the inexact Jacobian changes iteration counts, not the answer)."""
import numpy as np
import pytest

from paper_2307_16894_gb300 import binding, workload
from gpu_helpers import GpuRun, OracleRun, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def first_pass_K(rom, coef, F, precision):
    g = GpuRun(rom, coef)
    g.step(F, tol_rel=1e-9, tol_abs=rom["tol_abs"], max_iter=0, precision=precision)
    K = g.st.stiffness()
    g.close()
    return K


@pytest.mark.parametrize("name,B", [("c1", 1), ("c2", 37)])
def test_tc_stiffness_matches_fp32(name, B):
    rom, mu, coef, paths = workload.batch(name, B=B)
    F = paths[:, 3]
    K32 = first_pass_K(rom, coef, F, "fp32")
    for prec, tol in (("tf32", 3e-3), ("bf16", 3e-2)):
        K = first_pass_K(rom, coef, F, prec)
        err = np.linalg.norm(K - K32, axis=(1, 2)) / np.linalg.norm(K32, axis=(1, 2))
        print(name, prec, "max rel Frobenius error of K:", err.max())
        assert np.isfinite(K).all() and err.max() <= tol, (prec, err.max())


@pytest.mark.parametrize("prec", ["tf32", "bf16"])
def test_tc_converged_answer(prec):
    rom, mu, coef, paths = workload.batch("c2", B=33, steps=12)
    g = GpuRun(rom, coef)
    o = OracleRun(rom, coef)
    its = []
    for k in range(paths.shape[1]):
        P, A, info = g.step(paths[:, k], tol_rel=1e-9, tol_abs=rom["tol_abs"], max_iter=50, precision=prec,
                            start="prev")
        ref = o.step(paths[:, k], tol_rel=1e-10, tol_abs=rom["tol_abs"], start="prev")
        assert (info["status"] == 0).all()
        assert rel(P, ref["Pbar"]) <= 1e-7
        assert rel(A, ref["Abar"]) <= 1e-4
        its.append((info["iters"].mean(), ref["iters"].mean()))
    its = np.array(its)
    print(prec, "mean Newton iterations (mixed, FP64 oracle):", its.mean(0))
    g.close()
