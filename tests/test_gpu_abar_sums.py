"""Effective stiffness on the mixed paths, whose sums B = sum_i G_i^T Ahat_i and A0 run on the
tensor cores (k_abar_tc3 for 3D models, k_abar_tcp for 2D; n <= 64), against the FP64 oracle
(Eqs. tangent_problem_red, eff_stiffness_1): models of both dimensions with n from 16 to 64,
chunk counts with a ragged last chunk, and batches that leave the last CTA partly filled (14
instances per 3D CTA, 32 per 2D CTA), on the first 8 load steps of seeded 50-step paths.  The
FP32 tangent bounds the agreement (measured 0.9e-6 .. 7e-6 of Abar; Pbar 7e-12 .. 7e-10)."""
import numpy as np
import pytest

from paper_2307_16894_gb300 import inputs, workload
from gpu_helpers import GpuRun, OracleRun, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("model,B,prec", [("rom_c2", 37, "fp32"), ("rom_e2", 33, "tf32"), ("rom_r2_n16_m100", 70, "fp32"),
                                          ("rom_r2_n32_m200", 5, "bf16"), ("rom_c3", 17, "fp32"),
                                          ("rom_r3_n48_m400", 15, "tf32")])
def test_abar_tensor_core_sums(model, B, prec):
    rom = workload.load_model(model)
    d = rom["d"]
    lo, hi = (0.2, 0.35) if d == 2 else (0.15, 0.35)
    mu = np.stack([inputs.batch_mu(d, 1, 80_000 + b, lo, hi)[0] for b in range(B)])
    coef = inputs.map_coefficients(d, mu)
    paths = np.stack([inputs.stretch_path(d, 80_000 + b, 50)[:8] for b in range(B)])   # first 8 of 50 steps
    g = GpuRun(rom, coef)
    o = OracleRun(rom, coef)
    worst_a, worst_p = 0.0, 0.0
    for k in range(paths.shape[1]):
        P, A, info = g.step(paths[:, k], tol_rel=1e-9, tol_abs=rom["tol_abs"], max_iter=50, max_ls=6, precision=prec,
                            start="prev")
        ref = o.step(paths[:, k], tol_rel=1e-10, tol_abs=rom["tol_abs"], start="prev")
        ok = (info["status"] == 0) & (ref["status"] == 0)
        assert ok.sum() >= B - 1
        worst_p = max(worst_p, rel(P[ok], ref["Pbar"][ok]))
        worst_a = max(worst_a, rel(A[ok], ref["Abar"][ok]))
    g.close()
    print("%s n=%d m=%d B=%d %s: Pbar %.2e, Abar %.2e over 8 load steps" % (model, rom["n"], rom["m"], B, prec,
                                                                          worst_p, worst_a))
    assert worst_p <= 1e-7 and worst_a <= 5e-5
