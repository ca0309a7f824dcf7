"""CUDA path vs the FP64 oracle on the 2D porous-RVE workload (64x64 Q4 parent
mesh, n = 24, m = 160): a small batch over the whole 50-step path, and the
full 4096-instance batch in the launch configuration of bench.py checked on
sampled instances."""
import numpy as np
import pytest

from paper_2307_16894_gb300 import workload
from gpu_helpers import GpuRun, OracleRun, cpinv_from_fp, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_c2_small_batch_full_path():
    rom, mu, coef, paths = workload.batch("c2", B=9)
    g = GpuRun(rom, coef)
    o = OracleRun(rom, coef)
    kw = dict(tol_rel=1e-10, tol_abs=rom["tol_abs"], max_iter=25, max_ls=6, start="prev")
    worst = 0.0
    for k in range(paths.shape[1]):
        P, A, info = g.step(paths[:, k], **kw)
        ref = o.step(paths[:, k], **kw)
        assert np.array_equal(info["status"], ref["status"]), k
        assert np.array_equal(info["iters"], ref["iters"]), (k, info["iters"], ref["iters"])
        assert np.array_equal(info["evals"], ref["evals"]), k
        ok = ref["status"] == 0
        assert np.array_equal(info["n_yield"][ok], ref["n_yield"][ok]), k
        worst = max(worst, rel(P[ok], ref["Pbar"][ok]))
        assert rel(A[ok], ref["Abar"][ok]) <= 1e-9, k
    a, cp, xi = g.st.export()
    assert rel(a, o.q) <= 1e-11
    assert rel(cp, cpinv_from_fp(o.Fp, 2)) <= 1e-11
    assert np.abs(xi - o.xi).max() <= 1e-11 * max(o.xi.max(), 1e-3)
    assert worst <= 1e-11
    g.close()


def test_c2_full_batch_sampled():
    """B = 4096 (bench configuration), first 6 load steps; 6 sampled instances vs the oracle."""
    rom, mu, coef, paths = workload.batch("c2")
    B = len(coef)
    sample = np.array([0, 1, 1023, 2048, 3001, B - 1])
    g = GpuRun(rom, coef)
    o = OracleRun(rom, coef[sample])
    kw = dict(tol_rel=1e-10, tol_abs=rom["tol_abs"], max_iter=25, max_ls=6, start="prev")
    for k in range(6):
        P, A, info = g.step(paths[:, k], **kw)
        ref = o.step(paths[sample, k], **kw)
        assert np.array_equal(info["iters"][sample], ref["iters"]), k
        ok = ref["status"] == 0
        assert rel(P[sample][ok], ref["Pbar"][ok]) <= 1e-11
        assert rel(A[sample][ok], ref["Abar"][ok]) <= 1e-9
        # every instance converged, with finite outputs
        assert (info["status"] == 0).mean() >= 0.99
        assert np.isfinite(P[info["status"] == 0]).all()
    a, cp, xi = g.st.export()
    assert rel(a[sample], o.q) <= 1e-11
    g.close()


def test_c2_full_batch_sampled_fp32():
    """B = 4096, FP32 tangent and stiffness (FP64 residual, return map and solve): converged
    Pbar within 1e-7 of the FP64 oracle on sampled instances."""
    rom, mu, coef, paths = workload.batch("c2")
    B = len(coef)
    sample = np.array([5, 777, 2500, B - 2])
    g = GpuRun(rom, coef)
    o = OracleRun(rom, coef[sample])
    for k in range(6):
        P, A, info = g.step(paths[:, k], tol_rel=1e-9, tol_abs=rom["tol_abs"], max_iter=50, max_ls=6,
                            precision="fp32", start="prev")
        ref = o.step(paths[sample, k], tol_rel=1e-10, tol_abs=rom["tol_abs"], max_iter=25, max_ls=6, start="prev")
        assert (info["status"] == 0).mean() >= 0.99
        assert rel(P[sample], ref["Pbar"]) <= 1e-7
        assert rel(A[sample], ref["Abar"]) <= 1e-4
    g.close()
