"""Parity of the configurations the benchmark times, against the FP64 oracle, element by
element on sampled instances, in the benchmark's launch configuration:

* the 2D workload (64x64 Q4 parent mesh, n = 24, m = 160) at its full batch B = 4096 with the
  FP32 stiffness, the double-float residual and the learned Newton start, each load step one
  CUDA-graph launch, over all 50 load steps of the paths;
* the 3D workload (24^3 hex8 parent mesh, n = 64, m = 600) at its full batch B = 16384 with the
  TF32 tensor-core stiffness and the learned start, graph mode, over load steps 0-24;
* the 3D model of the ragged family with n = 95, m = 900, whose stiffness runs on the CUDA
  cores (n > 64), in FP64 and FP32.

The oracle runs the same instances with the previous-step start at Newton tolerance 1e-10
(the converged answer does not depend on the start).  Tolerances: Pbar 1e-7 and q, xi 1e-6
on the mixed paths (the metric's admissibility bound), Abar 1e-4 (the FP32 tangent data); the
FP64 path 1e-11 / 1e-9 with equal iteration counts (Eqs. forcevector_ecm, stiffnessmatrix_ecm,
red_newton, eff_stress_1, eff_stiffness_1)."""
import os

import numpy as np
import pytest

from paper_2307_16894_gb300 import binding, inputs, workload
from gpu_helpers import GpuRun, OracleRun, rel, torch_stream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def device_path(name, steps, prec, sample, mlp=True):
    """The workload's full batch through rom_step_device in graph mode (as the benchmark runs it);
    returns per step the sampled instances' Pbar, Abar and info, and the final state."""
    import torch
    from paper_2307_16894_gb300 import warmstart
    rom, mu, coef, paths = workload.batch(name)          # the 50-step paths, as the benchmark runs them
    B, d = len(coef), rom["d"]
    ctx = binding.Context(d, 0, torch_stream())
    ctx.load_basis(rom["G"])
    ctx.load_cubature(rom["w"], rom["phase"], rom["phases"], rom["omega"])
    ctx.set_geometry(rom["Gmu"], coef)
    start = "prev"
    mpath = os.path.join(workload.DATA, "mlp_%s.npz" % name)
    if mlp and os.path.exists(mpath):
        warmstart.load_into(ctx, mpath, B)
        start = "mlp"
    opts = binding.make_opts(tol_rel=1e-9, tol_abs=rom["tol_abs"], max_iter=50, max_ls=6, precision=prec,
                             start=start)
    ctx.use_graphs(True)
    st = ctx.state_create(B)
    Fd = torch.from_numpy(np.ascontiguousarray(paths.transpose(1, 0, 2, 3))).cuda()
    Pd = torch.empty((B, d, d), dtype=torch.float64, device="cuda")
    Ad = torch.empty((B, d * d, d * d), dtype=torch.float64, device="cuda")
    Id = torch.empty((B, binding.INFO_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
    si = torch.from_numpy(sample).cuda()
    out = []
    for k in steps:
        ctx.step_device(st, opts, Fd[k], Pd, Ad, Id)
        info = np.frombuffer(Id.cpu().numpy().tobytes(), dtype=binding.INFO_DTYPE)
        out.append((Pd.index_select(0, si).cpu().numpy(), Ad.index_select(0, si).cpu().numpy(), info.copy()))
    a, cp, xi = st.export()
    st.close()
    ctx.close()
    return rom, coef, paths, start, out, (a[sample], xi[sample])


def compare_with_oracle(rom, coef, paths, sample, steps, out, final, tol_p=1e-7, tol_a=1e-4):
    """Element-by-element comparison on the sampled instances while both sides agree on
    convergence.  From the first step at which they disagree (one side stalls where the other
    converges) an instance's histories differ, so it leaves the comparison; such instances are
    returned and bounded by the caller."""
    o = OracleRun(rom, coef[sample])
    worst_p = worst_a = 0.0
    alive = np.ones(len(sample), bool)
    compared = 0
    for (P, A, info), k in zip(out, steps):
        ref = o.step(paths[sample, k], tol_rel=1e-10, tol_abs=rom["tol_abs"], max_iter=25, max_ls=6, start="prev")
        st = info["status"][sample]
        alive &= st == ref["status"]
        for j in np.nonzero(alive & (ref["status"] == 0))[0]:
            worst_p = max(worst_p, rel(P[j], ref["Pbar"][j]))
            worst_a = max(worst_a, rel(A[j], ref["Abar"][j]))
            compared += 1
        assert worst_p <= tol_p, (k, worst_p)
        assert worst_a <= tol_a, (k, worst_a)
    a, xi = final
    fin = alive & (out[-1][2]["status"][sample] == 0)
    assert rel(a[fin], o.q[fin]) <= 1e-6
    assert np.abs(xi[fin] - o.xi[fin]).max() <= 1e-6 * max(o.xi[fin].max(), 1e-3)
    return worst_p, worst_a, compared, sample[~alive]


def test_c2_fp32_learned_start_graph_full_path():
    """B = 4096, FP32 stiffness, double-float residual, learned start, graphs; 6 sampled
    instances against the oracle at every one of the 50 load steps."""
    B = workload.WORKLOADS["c2"]["B"]
    sample = np.array([0, 911, 1777, 2048, 3333, B - 1])
    steps = list(range(50))
    rom, coef, paths, start, out, final = device_path("c2", steps, "fp32", sample)
    n_bad = sum(int((info["status"] != 0).sum()) for _, _, info in out)
    assert n_bad <= 0.01 * B * len(steps)
    wp, wa, nc, split = compare_with_oracle(rom, coef, paths, sample, steps, out, final)
    print("c2 fp32 %s start: Pbar %.2e Abar %.2e over 50 steps, %d instance-steps compared, split %s"
          % (start, wp, wa, nc, split))
    assert nc >= 0.8 * len(sample) * len(steps)


@pytest.mark.skipif(not os.path.exists(os.path.join(workload.DATA, "rom_c3.npz")), reason="3D model file absent")
def test_c3_tf32_learned_start_graph_steps_0_24():
    """B = 16384, TF32 tensor-core stiffness, double-float residual, learned start, graphs;
    8 sampled instances against the oracle at every load step 0-24 (the benchmark's warm-up
    and timed steps)."""
    B = workload.WORKLOADS["c3"]["B"]
    sample = np.unique(np.linspace(0, B - 1, 8).round().astype(np.int64))
    steps = list(range(25))
    rom, coef, paths, start, out, final = device_path("c3", steps, "tf32", sample)
    n_bad = sum(int((info["status"] != 0).sum()) for _, _, info in out)
    assert n_bad <= 0.001 * B * len(steps)
    wp, wa, nc, split = compare_with_oracle(rom, coef, paths, sample, steps, out, final)
    print("c3 tf32 %s start: Pbar %.2e Abar %.2e over steps 0-24, %d instance-steps compared, split %s"
          % (start, wp, wa, nc, split))
    # an instance on which one side stalls (the hyper-reduced equilibrium is hard to reach from
    # its history) leaves the comparison; at most one of the eight may do so
    assert len(split) <= 1 and nc >= 0.85 * len(sample) * len(steps)


@pytest.mark.skipif(not os.path.exists(os.path.join(workload.DATA, "rom_r3_n95_m900.npz")),
                    reason="ragged 3D model file absent")
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_3d_cuda_core_assembly_n95(prec):
    """The ragged family's 3D model with n = 95 > 64 (stiffness on the CUDA cores in FP64 or
    FP32) against the oracle: 3 instances, 4 load steps."""
    rom = workload.load_model("rom_r3_n95_m900")
    B = 3
    mu = np.stack([inputs.batch_mu(3, 1, 40_000 + b, 0.15, 0.35)[0] for b in range(B)])
    coef = inputs.map_coefficients(3, mu)
    paths = np.stack([inputs.stretch_path(3, 40_000 + b, 50)[:4] for b in range(B)])
    g = GpuRun(rom, coef)
    o = OracleRun(rom, coef)
    fp64 = prec == "fp64"
    kw = dict(tol_rel=1e-10 if fp64 else 1e-9, tol_abs=rom["tol_abs"], max_iter=25 if fp64 else 50, max_ls=6,
              start="prev", precision=prec)
    for k in range(paths.shape[1]):
        P, A, info = g.step(paths[:, k], **kw)
        ref = o.step(paths[:, k], tol_rel=1e-10, tol_abs=rom["tol_abs"], max_iter=25, max_ls=6, start="prev")
        assert (info["status"] == 0).all() and (ref["status"] == 0).all()
        if fp64:
            assert np.array_equal(info["iters"], ref["iters"]), (k, info["iters"], ref["iters"])
            assert np.array_equal(info["n_yield"], ref["n_yield"]), k
        assert rel(P, ref["Pbar"]) <= (1e-11 if fp64 else 1e-7), (k, rel(P, ref["Pbar"]))
        assert rel(A, ref["Abar"]) <= (1e-9 if fp64 else 1e-4), (k, rel(A, ref["Abar"]))
    a, cp, xi = g.st.export()
    assert rel(a, o.q) <= (1e-11 if fp64 else 1e-6)
    g.close()
