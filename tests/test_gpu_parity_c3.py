"""3D inclusion RVE (24^3 hex8 parent mesh, n = 64, m = 600): FP64 path vs the oracle on
a small batch, the mixed-precision paths (FP32 CUDA cores, TF32 and BF16 tensor cores)
vs the oracle, and the full 16384-instance batch checked on sampled instances."""
import os

import numpy as np
import pytest

from paper_2307_16894_gb300 import workload
from gpu_helpers import GpuRun, OracleRun, cpinv_from_fp, rel

pytestmark = pytest.mark.gpu
HAVE = os.path.exists(os.path.join(workload.DATA, "rom_c3.npz"))


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.skipif(not HAVE, reason="3D model file not generated")
def test_c3_fp64_small_batch():
    rom, mu, coef, paths = workload.batch("c3", B=3)
    paths = paths[:, :6]      # first 6 steps of the 50-step load paths
    g = GpuRun(rom, coef)
    o = OracleRun(rom, coef)
    kw = dict(tol_rel=1e-10, tol_abs=rom["tol_abs"], max_iter=25, max_ls=6, start="prev")
    for k in range(paths.shape[1]):
        P, A, info = g.step(paths[:, k], **kw)
        ref = o.step(paths[:, k], **kw)
        assert np.array_equal(info["status"], ref["status"]), k
        assert np.array_equal(info["iters"], ref["iters"]), (k, info["iters"], ref["iters"])
        assert np.array_equal(info["n_yield"], ref["n_yield"]), k
        ok = ref["status"] == 0
        assert rel(P[ok], ref["Pbar"][ok]) <= 1e-11
        assert rel(A[ok], ref["Abar"][ok]) <= 1e-9
    a, cp, xi = g.st.export()
    assert rel(a, o.q) <= 1e-11
    assert rel(cp, cpinv_from_fp(o.Fp, 3)) <= 1e-11
    g.close()


@pytest.mark.skipif(not HAVE, reason="3D model file not generated")
@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
def test_c3_mixed_precision(prec):
    rom, mu, coef, paths = workload.batch("c3", B=3)
    paths = paths[:, :5]
    g = GpuRun(rom, coef)
    o = OracleRun(rom, coef)
    for k in range(paths.shape[1]):
        P, A, info = g.step(paths[:, k], tol_rel=1e-9, tol_abs=rom["tol_abs"], max_iter=50, precision=prec,
                            start="prev")
        ref = o.step(paths[:, k], tol_rel=1e-10, tol_abs=rom["tol_abs"], start="prev")
        assert (info["status"] == 0).all()
        print(prec, k, "rel err Pbar %.2e Abar %.2e iters %s vs %s" % (rel(P, ref["Pbar"]), rel(A, ref["Abar"]),
                                                                      info["iters"], ref["iters"]))
        assert rel(P, ref["Pbar"]) <= 1e-7
        assert rel(A, ref["Abar"]) <= 1e-4
    g.close()


@pytest.mark.skipif(not HAVE, reason="3D model file not generated")
def test_c3_full_batch_sampled_tf32():
    """B = 16384 in the bench configuration (TF32 tensor cores), first 3 steps of the 50-step
    paths; every instance converges and 3 sampled instances match the oracle."""
    rom, mu, coef, paths = workload.batch("c3")
    paths = paths[:, :3]
    B = len(coef)
    sample = np.array([0, 8191, B - 1])
    g = GpuRun(rom, coef)
    o = OracleRun(rom, coef[sample])
    for k in range(paths.shape[1]):
        P, A, info = g.step(paths[:, k], tol_rel=1e-9, tol_abs=rom["tol_abs"], max_iter=50, precision="tf32",
                            start="prev")
        ref = o.step(paths[sample, k], tol_rel=1e-10, tol_abs=rom["tol_abs"], start="prev")
        assert (info["status"] == 0).all()
        assert rel(P[sample], ref["Pbar"]) <= 1e-7
    g.close()
