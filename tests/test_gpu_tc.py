"""Tensor-core (tcgen05) stiffness assembly: K in TF32/BF16 vs the FP32 CUDA-core
assembly on the same tangent, and converged answers of the mixed-precision path vs
the FP64 oracle (the inexact Jacobian changes iteration counts, not the answer)."""
import os

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


def first_pass_K_At(rom, coef, F, precision):
    g = GpuRun(rom, coef)
    g.step(F, tol_rel=1e-9, tol_abs=rom["tol_abs"], max_iter=0, precision=precision)
    K = g.st.stiffness()
    At = g.st.tangent(precision == "fp64")
    g.close()
    return K, At


def stiffness_from_tangent(G, At):
    """K_b = sum_i G_i^T At_i G_i in FP64 from the tangent the kernels used (At [B, d^4, m])."""
    m, d2, n = G.shape
    A = At.astype(np.float64).reshape(len(At), d2, d2, m)
    Y = np.einsum("baci,icl->bial", A, G, optimize=True)
    return np.einsum("iaj,bial->bjl", G, Y, optimize=True)


@pytest.mark.skipif(not os.path.exists(os.path.join(workload.DATA, "rom_c3.npz")), reason="3D model file not generated")
@pytest.mark.parametrize("B", [3, 37])
def test_tc3_stiffness(B):
    """3D model (n = 64, m = 600): K of the first Newton pass from the 3D tensor-core kernel (BF16,
    TF32, and the TF32 hi/lo split used for FP32 precision) vs K = sum_i G_i^T At_i G_i evaluated
    in FP64 from the same FP32 tangent; B = 37 leaves partly filled CTAs (8, 4 and 2 instances
    per CTA).  The FP64 path's K is printed for reference (it also differs by the FP32 tangent)."""
    rom, mu, coef, paths = workload.batch("c3", B=B)
    F = paths[:, 3]
    K64, _ = first_pass_K_At(rom, coef, F, "fp64")
    errs = {}
    for prec, tol in (("fp32", 2e-5), ("tf32", 1e-3), ("bf16", 5e-3)):
        K, At = first_pass_K_At(rom, coef, F, prec)
        Kref = stiffness_from_tangent(rom["G"], At)
        err = np.linalg.norm(K - Kref, axis=(1, 2)) / np.linalg.norm(Kref, axis=(1, 2))
        e64 = np.linalg.norm(K - K64, axis=(1, 2)) / np.linalg.norm(K64, axis=(1, 2))
        print("c3 B=%d %s max rel Frobenius error of K: %.3e (vs FP64-path K: %.3e)" % (B, prec, err.max(), e64.max()))
        errs[prec] = (np.isfinite(K).all(), err.max(), tol)
    for prec, (fin, e, tol) in errs.items():
        assert fin and e <= tol, (prec, e)


@pytest.mark.parametrize("model,B", [("rom_c1", 5), ("rom_c2", 37), ("rom_e2", 7), ("rom_e2_n5", 35),
                                     ("rom_e2_n30", 9), ("rom_r2_n16_m100", 17), ("rom_r2_n32_m200", 6)])
def test_tc2_stiffness(model, B):
    """2D models on the packed tensor-core kernel (S = min(16, 128 // n) instances per CTA along
    M, N = n rounded up to 16): K of the first Newton pass in BF16, TF32 and the TF32 hi/lo split
    used for FP32 precision vs K = sum_i G_i^T At_i G_i in FP64 from the same FP32 tangent.  The
    models span n = 5 .. 40 (S = 16 .. 3, N = 16 .. 48), chunk counts with a ragged last chunk
    (m = 457, 205, 326) and batches that leave the last CTA partly filled."""
    from paper_2307_16894_gb300 import inputs
    rom = workload.load_model(model)
    d = rom["d"]
    assert d == 2 and rom["n"] <= 64
    mu = np.stack([inputs.batch_mu(d, 1, 70_000 + b, 0.2, 0.35)[0] for b in range(B)])
    coef = inputs.map_coefficients(d, mu)
    F = np.stack([inputs.stretch_path(d, 70_000 + b, 6)[3] for b in range(B)])
    errs = {}
    for prec, tol in (("fp32", 1e-5), ("tf32", 1e-3), ("bf16", 5e-3)):
        K, At = first_pass_K_At(rom, coef, F, prec)
        Kref = stiffness_from_tangent(rom["G"], At)
        err = np.linalg.norm(K - Kref, axis=(1, 2)) / np.linalg.norm(Kref, axis=(1, 2))
        print("%s n=%d m=%d B=%d %s max rel Frobenius error of K: %.3e" % (model, rom["n"], rom["m"], B, prec,
                                                                          err.max()))
        errs[prec] = (np.isfinite(K).all(), err.max(), tol)
    for prec, (fin, e, tol) in errs.items():
        assert fin and e <= tol, (prec, e)


def residual_check(name, B, prec, fp64_residual=False):
    rom, mu, coef, paths = workload.batch(name, B=B)
    g = GpuRun(rom, coef)
    g.step(paths[:, 3], tol_rel=1e-9, tol_abs=rom["tol_abs"], max_iter=0, precision=prec,
           fp64_residual=fp64_residual)
    r, v = g.st.residual()
    g.close()
    G = rom["G"]
    ref = np.einsum("icj,bci->bj", G, v, optimize=True)
    mag = np.einsum("icj,bci->bj", np.abs(G), np.abs(v), optimize=True)
    return np.abs(r - ref).max(axis=1) / mag.max(axis=1)


@pytest.mark.parametrize("name,B", [("c2", 37), ("c3", 37)])
def test_residual_double_float(name, B):
    """Residual r = sum_i G_i^T v_i: double-float (FP32 pairs) on the tensor-core paths and FP64 on
    the FP64 path vs the FP64 sum of the same v, relative to sum |G v| (~1e-13 expected for the
    pairs, below 1e-11 with the worst-case growth of the FP32 compensation over 5400 terms)."""
    if name == "c3" and not os.path.exists(os.path.join(workload.DATA, "rom_c3.npz")):
        pytest.skip("3D model file not generated")
    for prec, f64, tol in (("tf32", False, 1e-11), ("tf32", True, 1e-13), ("fp64", False, 1e-13)):
        err = residual_check(name, B, prec, f64)
        print("%s B=%d %s%s residual max error / sum|terms|: %.3e" % (name, B, prec, " fp64_residual" if f64 else "",
                                                                      err.max()))
        assert np.isfinite(err).all() and err.max() <= tol, (prec, f64, err.max())


def test_fp64_residual_option_converged_answer():
    """The FP64 residual option on the 3D TF32 path converges to the same answers as the default
    double-float residual (both within the mixed-path tolerance of the FP64 oracle)."""
    if not os.path.exists(os.path.join(workload.DATA, "rom_c3.npz")):
        pytest.skip("3D model file not generated")
    rom, mu, coef, paths = workload.batch("c3", B=9)
    paths = paths[:, :6]   # the first steps of the 50-step paths
    runs = [GpuRun(rom, coef), GpuRun(rom, coef)]
    o = OracleRun(rom, coef)
    for k in range(paths.shape[1]):
        out = [g.step(paths[:, k], tol_rel=1e-9, tol_abs=rom["tol_abs"], max_iter=50, precision="tf32",
                      start="prev", fp64_residual=f64) for g, f64 in zip(runs, (False, True))]
        ref = o.step(paths[:, k], tol_rel=1e-10, tol_abs=rom["tol_abs"], start="prev")
        for P, A, info in out:
            assert (info["status"] == 0).all()
            assert rel(P, ref["Pbar"]) <= 1e-7
        assert rel(out[0][0], out[1][0]) <= 1e-8
    for g in runs:
        g.close()
