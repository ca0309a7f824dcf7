"""Train the learned Newton start on the solver's own trajectories and compare it with
the plain and previous-step starts.

  python -m paper_2307_16894_gb300.train_warmstart --workload c2 --paths 4096 --steps 50 \\
         --epochs 20 --out data/mlp_c2.npz

Training instances are drawn from the workload's seeded sequence starting at --first
(disjoint from the benchmark instances 0 .. B-1); every solve, feature, forward,
backward and Adam step runs in libpodecm.so.  Prints one JSON line with the losses and,
on --eval instances of the benchmark batch, the mean Newton iterations, residual
evaluations and time per step of the plain, previous-step and learned starts.
"""
import argparse
import json
import time

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--paths", type=int, default=4096)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--first", type=int, default=20_000)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--eval", type=int, default=1024)
    ap.add_argument("--out", default=None)
    ap.add_argument("--load", default=None, help="evaluate this trained network (npz) instead of training one")
    ap.add_argument("--eval-steps", type=int, default=0,
                    help="evaluate on the first EVAL_STEPS steps of the load paths (0: all)")
    ap.add_argument("--clip", type=float, default=0.0,
                    help="clip the standardised training targets to +-clip (0: no clipping)")
    args = ap.parse_args()

    import torch
    from . import binding, warmstart, workload

    stream = torch.cuda.current_stream().cuda_stream
    rom, mu, coef, paths = workload.batch(args.workload, B=args.paths, steps=args.steps, first=args.first)
    if args.load:
        coef, paths = coef[:1], paths[:1]
    d, n = rom["d"], rom["n"]
    n_par = coef.shape[1]
    prec = args.precision
    kw = dict(tol_rel=1e-10 if prec == "fp64" else 1e-9, tol_abs=rom["tol_abs"], max_iter=50, max_ls=6,
              precision=prec)

    def make_ctx(c):
        ctx = binding.Context(d, 0, stream)
        ctx.load_basis(rom["G"])
        ctx.load_cubature(rom["w"], rom["phase"], rom["phases"], rom["omega"])
        ctx.set_geometry(rom["Gmu"], c)
        return ctx

    n_in = warmstart.n_features(d, n_par, n)
    if args.load:
        z = np.load(args.load)
        params = z["params"]
        nrm = z["norm"]
        norm = (nrm[:n_in], nrm[n_in:2 * n_in], nrm[2 * n_in:2 * n_in + n], nrm[2 * n_in + n:])
        X, hist, t_collect, t_train = np.zeros((0, n_in)), [], 0.0, 0.0
    else:
        t0 = time.time()
        ctx = make_ctx(coef)
        st = ctx.state_create(len(coef))
        X, Y, _ = warmstart.collect(ctx, st, paths, binding.make_opts(start="prev", **kw), torch)
        st.close()
        t_collect = time.time() - t0
        ctx.mlp_init(n_in, warmstart.WIDTH, warmstart.DEPTH, n, max(args.batch, args.eval))
        params0 = warmstart.init_params(n_in, warmstart.WIDTH, warmstart.DEPTH, n, 0)
        ctx.mlp_params(params0)
        norm = warmstart.fit_norm(X, Y)
        if args.clip > 0:
            Y = np.clip(Y, norm[2] - args.clip * norm[3], norm[2] + args.clip * norm[3]).astype(np.float32)
        ctx.mlp_norm(*norm)
        t0 = time.time()
        hist = warmstart.train(ctx, X, Y, torch, epochs=args.epochs, batch=args.batch, lr=args.lr)
        t_train = time.time() - t0
        params = ctx.mlp_params()
        if args.out:
            warmstart.save(args.out, (n_in, warmstart.WIDTH, warmstart.DEPTH, n), params, norm)
        ctx.close()

    # evaluation on benchmark instances (not seen in training)
    rom, mu_e, coef_e, paths_e = workload.batch(args.workload, B=args.eval, steps=args.steps)
    if args.eval_steps > 0:
        paths_e = paths_e[:, :args.eval_steps]
    ev = {}
    for start in ("plain", "prev", "mlp"):
        c = make_ctx(coef_e)
        if start == "mlp":
            c.mlp_init(n_in, warmstart.WIDTH, warmstart.DEPTH, n, args.eval)
            c.mlp_params(params)
            c.mlp_norm(*norm)
        c.use_graphs(True)
        s = c.state_create(args.eval)
        opts = binding.make_opts(start=start, **kw)
        Fd = torch.from_numpy(np.ascontiguousarray(paths_e.transpose(1, 0, 2, 3))).cuda()
        Pd = torch.empty((args.eval, d, d), dtype=torch.float64, device="cuda")
        Ad = torch.empty((args.eval, d * d, d * d), dtype=torch.float64, device="cuda")
        Id = torch.empty((args.eval, binding.INFO_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
        its, evs, ms, ok = [], [], 0.0, 0
        S = paths_e.shape[1]
        for k in range(S):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            c.step_device(s, opts, Fd[k], Pd, Ad, Id)
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            info = np.frombuffer(Id.cpu().numpy().tobytes(), dtype=binding.INFO_DTYPE)
            its.append(info["iters"].mean())
            evs.append(info["evals"].mean())
            ok += int((info["status"] == 0).sum())
        ev[start] = dict(newton_iters=float(np.mean(its)), evals=float(np.mean(evs)), ms_per_step=ms / S,
                         converged=ok, total=args.eval * S)
        s.close()
        c.close()
    print(json.dumps(dict(workload=args.workload, samples=int(len(X)), collect_s=t_collect, train_s=t_train,
                          loss_history=hist, eval=ev)))


if __name__ == "__main__":
    main()
