"""Learned Newton start on the GPU: the library's MLP forward/backward kernels vs the
FP64 oracle MLP, training, and the learned start inside the reduced solve (the
converged answer decides the result; the start only changes the iteration count)."""
import numpy as np
import pytest

import oracle.mlp as omlp
from paper_2307_16894_gb300 import binding, warmstart, workload
from gpu_helpers import GpuRun, OracleRun, rel, torch_stream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def make_ctx(n_in, n_out, rows):
    ctx = binding.Context(2, 0, torch_stream())
    ctx.mlp_init(n_in, warmstart.WIDTH, warmstart.DEPTH, n_out, rows)
    return ctx


def test_mlp_grad_matches_oracle():
    import torch
    rng = np.random.default_rng(0)
    n_in, n_out, N = 31, 24, 200
    ctx = make_ctx(n_in, n_out, N)
    p = warmstart.init_params(n_in, warmstart.WIDTH, warmstart.DEPTH, n_out, 3)
    ctx.mlp_params(p)
    X = rng.standard_normal((N, n_in)).astype(np.float32)
    Y = rng.standard_normal((N, n_out)).astype(np.float32)
    norm = (X.mean(0), X.std(0), Y.mean(0), Y.std(0))
    ctx.mlp_norm(*norm)
    shp = omlp.shapes(n_in, warmstart.WIDTH, warmstart.DEPTH, n_out)
    normv = np.concatenate(norm).astype(np.float64)
    L_ref, g_ref = omlp.loss_grad(p.astype(np.float64), shp, X.astype(np.float64), Y.astype(np.float64), normv)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    g = torch.empty(p.size, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    ctx.mlp_loss_grad(Xd, Yd, 0, g, loss)          # FP32 weights
    torch.cuda.synchronize()
    assert abs(loss.item() - L_ref) <= 1e-5 * L_ref
    assert rel(g.cpu().numpy(), g_ref) <= 1e-4
    ctx.mlp_loss_grad(Xd, Yd, 1, g, loss)          # BF16 weights (inference precision)
    torch.cuda.synchronize()
    assert abs(loss.item() - L_ref) <= 2e-2 * L_ref
    assert rel(g.cpu().numpy(), g_ref) <= 5e-2
    out = torch.empty((N, n_out), dtype=torch.float64, device="cuda")
    ctx.mlp_predict(Xd, 0, out)
    torch.cuda.synchronize()
    pr = omlp.predict(p.astype(np.float64), shp, X.astype(np.float64), normv)
    assert rel(out.cpu().numpy(), pr) <= 1e-5
    ctx.close()


@pytest.mark.parametrize("n_in,n_out,N", [(31, 24, 200), (142, 64, 300), (55, 24, 128)])
def test_mlp_predict_tensor_cores(n_in, n_out, N):
    """BF16 inference on the tensor cores (one fused tcgen05 kernel per 128 rows: BF16 weights and
    activations, FP32 accumulation) against the FP64 oracle network with the same FP32 weights;
    the shapes cover the 2D and 3D learned starts (n_in 55 / 142, n_out 24 / 64) and a partly
    filled last CTA."""
    import torch
    rng = np.random.default_rng(1)
    ctx = make_ctx(n_in, n_out, N)
    p = warmstart.init_params(n_in, warmstart.WIDTH, warmstart.DEPTH, n_out, 5)
    dims = [n_in] + [warmstart.WIDTH] * warmstart.DEPTH + [n_out]
    o = 0
    for a, b in zip(dims[:-1], dims[1:]):          # non-zero biases, so that the bias add is exercised
        o += a * b
        p[o:o + b] = rng.uniform(-0.3, 0.3, b).astype(np.float32)
        o += b
    ctx.mlp_params(p)
    X = rng.standard_normal((N, n_in)).astype(np.float32)
    Y = rng.standard_normal((N, n_out)).astype(np.float32)
    norm = (X.mean(0), X.std(0), Y.mean(0), Y.std(0))
    ctx.mlp_norm(*norm)
    shp = omlp.shapes(n_in, warmstart.WIDTH, warmstart.DEPTH, n_out)
    pr = omlp.predict(p.astype(np.float64), shp, X.astype(np.float64), np.concatenate(norm).astype(np.float64))
    out = torch.full((N, n_out), np.nan, dtype=torch.float64, device="cuda")
    ctx.mlp_predict(torch.from_numpy(X).cuda(), 1, out)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    print("n_in %d n_out %d: tensor-core BF16 prediction rel error %.3e" % (n_in, n_out, rel(o, pr)))
    assert np.isfinite(o).all() and rel(o, pr) <= 3e-2
    ctx.close()


def test_mlp_training_reduces_loss():
    import torch
    rng = np.random.default_rng(1)
    n_in, n_out, N = 10, 4, 4096
    X = rng.standard_normal((N, n_in)).astype(np.float32)
    Wt = rng.standard_normal((n_in, n_out)) / np.sqrt(n_in)
    Z = X @ Wt
    Y = (np.sin(Z) + 0.5 * Z + 0.1 * Z ** 2).astype(np.float32)
    ctx = make_ctx(n_in, n_out, 512)
    ctx.mlp_params(warmstart.init_params(n_in, warmstart.WIDTH, warmstart.DEPTH, n_out, 0))
    ctx.mlp_norm(*warmstart.fit_norm(X, Y))
    hist = warmstart.train(ctx, X, Y, torch, epochs=10, batch=256, lr=1e-3)
    print("training history (train, validation):", hist)
    assert hist[-1][1] < 0.1
    ctx.close()


def test_learned_start_same_answer_fewer_iterations():
    """Train on the solver's own trajectories (2D c2 model), then the learned start gives
    the oracle's converged answer with fewer Newton iterations than the plain start."""
    import torch
    rom, mu, coef, paths = workload.batch("c2", B=512, steps=20)
    d, n = rom["d"], rom["n"]
    kw = dict(tol_rel=1e-10, tol_abs=rom["tol_abs"], max_iter=25, max_ls=6)
    g = GpuRun(rom, coef, stream=torch_stream())
    Xtr, Ytr, _ = warmstart.collect(g.ctx, g.st, paths, binding.make_opts(start="prev", **kw), torch)
    g.close()
    n_in = warmstart.n_features(d, 1, n)
    # held-out instances (other seeds)
    rom, mu2, coef2, paths2 = workload.batch("c2", B=64, steps=20, first=3000)
    h = GpuRun(rom, coef2, stream=torch_stream())
    h.ctx.mlp_init(n_in, warmstart.WIDTH, warmstart.DEPTH, n, 4096)
    h.ctx.mlp_params(warmstart.init_params(n_in, warmstart.WIDTH, warmstart.DEPTH, n, 0))
    h.ctx.mlp_norm(*warmstart.fit_norm(Xtr, Ytr))
    warmstart.train(h.ctx, Xtr, Ytr, torch, epochs=30, batch=512, lr=1e-3)
    pl = GpuRun(rom, coef2)
    o = OracleRun(rom, coef2)
    it_mlp, it_plain = [], []
    for k in range(paths2.shape[1]):
        P, A, info = h.step(paths2[:, k], start="mlp", **kw)
        P0, A0, info0 = pl.step(paths2[:, k], start="plain", **kw)
        ref = o.step(paths2[:, k], start="plain", **kw)
        assert (info["status"] == 0).all() and (ref["status"] == 0).all()
        assert rel(P, ref["Pbar"]) <= 1e-8
        it_mlp.append(info["iters"].mean())
        it_plain.append(info0["iters"].mean())
    print("mean Newton iterations: learned start %.3f, plain start %.3f" % (np.mean(it_mlp), np.mean(it_plain)))
    assert np.mean(it_mlp) < np.mean(it_plain)
    h.close()
    pl.close()


def test_learned_start_beats_previous_step_predictor_c3():
    """The trained network of the 3D workload (data/mlp_c3.npz, trained on instances 30000 and
    up) on held-out instances of the workload (B = 4096, the 50-step paths), TF32 stiffness in
    graph mode: over load steps 12-24, where the plastic zone grows, it needs fewer Newton
    iterations and less time than the previous-step predictor (the method without it); the two
    starts are stepped alternately so that both see the same GPU conditions.  The converged Pbar
    of sampled instances matches the FP64 oracle within 1e-7 at every step."""
    import os
    import torch
    path = os.path.join(workload.DATA, "mlp_c3.npz")
    if not os.path.exists(path):
        pytest.skip("trained network absent")
    rom, mu, coef, paths = workload.batch("c3", B=4096)
    B, d = len(coef), 3
    runs = {}
    for start in ("prev", "mlp"):
        ctx = binding.Context(d, 0, torch_stream())
        ctx.load_basis(rom["G"])
        ctx.load_cubature(rom["w"], rom["phase"], rom["phases"], rom["omega"])
        ctx.set_geometry(rom["Gmu"], coef)
        if start == "mlp":
            warmstart.load_into(ctx, path, B)
        ctx.use_graphs(True)
        runs[start] = dict(ctx=ctx, st=ctx.state_create(B),
                           opts=binding.make_opts(tol_rel=1e-9, tol_abs=rom["tol_abs"], max_iter=50, max_ls=6,
                                                  precision="tf32", start=start),
                           P=torch.empty((B, d, d), dtype=torch.float64, device="cuda"),
                           A=torch.empty((B, 81), dtype=torch.float64, device="cuda"),
                           I=torch.empty((B, binding.INFO_DTYPE.itemsize), dtype=torch.uint8, device="cuda"),
                           its=[], ms=0.0)
    Fd = torch.from_numpy(np.ascontiguousarray(paths.transpose(1, 0, 2, 3))).cuda()
    sample = np.array([0, 1365, 2730, B - 1])
    o = OracleRun(rom, coef[sample])
    for k in range(25):
        ref = o.step(paths[sample, k], tol_rel=1e-10, tol_abs=rom["tol_abs"], max_iter=25, start="prev")
        for start, r in runs.items():
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            r["ctx"].step_device(r["st"], r["opts"], Fd[k], r["P"], r["A"], r["I"])
            e1.record()
            torch.cuda.synchronize()
            info = np.frombuffer(r["I"].cpu().numpy().tobytes(), dtype=binding.INFO_DTYPE)
            assert (info["status"] == 0).all(), (start, k)
            ok = ref["status"] == 0
            assert rel(r["P"].cpu().numpy()[sample][ok], ref["Pbar"][ok]) <= 1e-7, (start, k)
            if k >= 12:
                r["its"].append(info["iters"].mean())
                r["ms"] += e0.elapsed_time(e1)
    ip, im = np.mean(runs["prev"]["its"]), np.mean(runs["mlp"]["its"])
    tp, tm = runs["prev"]["ms"], runs["mlp"]["ms"]
    print("c3 steps 12-24, B=%d: Newton iterations prev %.4f, learned %.4f; time prev %.1f ms, learned %.1f ms"
          % (B, ip, im, tp, tm))
    for r in runs.values():
        r["st"].close()
        r["ctx"].close()
    assert im < ip - 0.02
    assert tm < tp
