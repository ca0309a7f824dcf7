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
