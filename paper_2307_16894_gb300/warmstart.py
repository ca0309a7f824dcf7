"""Learned Newton start: data collection from the solver's own trajectories,
training with the library's MLP kernels, and persistence.

Every arithmetic step (solve, features, forward/backward, Adam) runs in
libpodecm.so; this module only moves batches between host and device.
Features of a step: [Ubar_k - Ubar_{k-1}, mu, a_n, a_n - a_{n-1}, mean xi, max xi];
target: the correction of the previous-step increment, (a_k - a_n) - (a_n - a_{n-1}).

The context passed to collect() and train() must have been created on torch's
current stream (binding.Context(d, dev, torch.cuda.current_stream().cuda_stream))
so that the torch tensors handed to the library stay stream-ordered.
"""
import numpy as np

from . import binding

WIDTH, DEPTH = 128, 4      # 4 hidden layers of width 128


def n_features(d, n_par, n):
    return d * d + n_par + 2 * n + 2


def init_params(n_in, width, depth, n_out, seed):
    """He-uniform weights, zero biases, packed as W[out][in] then b[out] per linear map."""
    rng = np.random.default_rng(seed)
    dims = [n_in] + [width] * depth + [n_out]
    out = []
    for l in range(depth + 1):
        fan_in = dims[l]
        lim = np.sqrt(6.0 / fan_in) if l < depth else np.sqrt(3.0 / fan_in)
        out.append(rng.uniform(-lim, lim, dims[l + 1] * dims[l]))
        out.append(np.zeros(dims[l + 1]))
    return np.concatenate(out).astype(np.float32)


def collect(ctx, state, paths, opts, torch, max_steps=None):
    """Run the load paths [B, S, d, d] through rom_step (device buffers) and return
    (X [N, n_in], Y [N, n], iters [N]) for the converged instance-steps."""
    d = ctx.dim
    B, S = paths.shape[:2]
    S = S if max_steps is None else min(S, max_steps)
    n_in = n_features(d, ctx.n_par, ctx.n)
    Fd = torch.from_numpy(np.ascontiguousarray(paths.transpose(1, 0, 2, 3))).cuda()
    Xd = torch.empty((B, n_in), dtype=torch.float32, device="cuda")
    Pd = torch.empty((B, d, d), dtype=torch.float64, device="cuda")
    Ad = torch.empty((B, d * d, d * d), dtype=torch.float64, device="cuda")
    Id = torch.empty((B, binding.INFO_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
    Xs, Ys, its = [], [], []
    for k in range(S):
        ctx.features(state, Fd[k], Xd)
        a0 = state.export(history=False)[0]
        ctx.step_device(state, opts, Fd[k], Pd, Ad, Id)
        ctx.sync()
        a1 = state.export(history=False)[0]
        info = np.frombuffer(Id.cpu().numpy().tobytes(), dtype=binding.INFO_DTYPE)
        ok = info["status"] == 0
        X = Xd.cpu().numpy()
        n = ctx.n
        da_prev = X[:, d * d + ctx.n_par + n:d * d + ctx.n_par + 2 * n].astype(np.float64)
        Xs.append(X[ok])
        Ys.append(((a1 - a0) - da_prev)[ok].astype(np.float32))
        its.append(info["iters"][ok])
    return np.concatenate(Xs), np.concatenate(Ys), np.concatenate(its)


def fit_norm(X, Y):
    xs = X.std(0)
    ys = Y.std(0)
    xs[xs < 1e-12] = 1.0
    ys[ys < 1e-12] = 1.0
    return X.mean(0), xs, Y.mean(0), ys


def train(ctx, X, Y, torch, epochs=20, batch=1024, lr=1e-3, seed=0, val_frac=0.1):
    """Train the context's MLP (already initialised) on (X, Y); returns per-epoch
    (train loss, validation loss) on standardised targets."""
    rng = np.random.default_rng(seed)
    N = len(X)
    perm = rng.permutation(N)
    nv = int(N * val_frac)
    vi, ti = perm[:nv], perm[nv:]
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    Yd = torch.from_numpy(np.ascontiguousarray(Y)).cuda()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    grad = torch.empty(ctx.mlp_params().size, dtype=torch.float32, device="cuda")
    hist = []
    t = 0
    for ep in range(epochs):
        order = rng.permutation(ti)
        tot = 0.0
        nb = 0
        for s in range(0, len(order) - batch + 1, batch):
            idx = torch.from_numpy(order[s:s + batch]).cuda()
            t += 1
            ctx.mlp_train_step(Xd.index_select(0, idx).contiguous(), Yd.index_select(0, idx).contiguous(), lr, t,
                               loss)
            if nb % 16 == 0:
                tot += float(loss.item())
            nb += 1
        vl = 0.0
        if nv:
            for s in range(0, nv, batch):
                idx = torch.from_numpy(vi[s:s + batch]).cuda()
                ctx.mlp_loss_grad(Xd.index_select(0, idx).contiguous(), Yd.index_select(0, idx).contiguous(), 1,
                                  grad, loss)
                vl += float(loss.item()) * len(idx)
            vl /= nv
        hist.append((tot / max(1, (nb + 15) // 16), vl))
    return hist


def save(path, shape, params, norm):
    np.savez(path, shape=np.array(shape), params=params, norm=np.concatenate(norm).astype(np.float32))


def load_into(ctx, path, max_rows):
    z = np.load(path)
    n_in, width, depth, n_out = [int(v) for v in z["shape"]]
    ctx.mlp_init(n_in, width, depth, n_out, max_rows)
    ctx.mlp_params(z["params"])
    nrm = z["norm"]
    ctx.mlp_norm(nrm[:n_in], nrm[n_in:2 * n_in], nrm[2 * n_in:2 * n_in + n_out], nrm[2 * n_in + n_out:])
