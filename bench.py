"""Throughput of the hyper-reduced RVE load step on GB300.

One bench "step" = one load step of the whole hot path for every instance of
the batch: geometry, kinematics, FP64 return map, tangent, force and
stiffness assembly, Newton with line search, effective stress and stiffness,
history commit (all Newton iterations included).  Metric: macro-point ROM
load-steps/s = instances x load steps / time, admissible only if the converged
Pbar is within 1e-7 (relative) of the FP64 oracle.

Default workload: 16384 macro points of the 3D inclusion RVE family (24^3 hex8
parent mesh, ellipsoidal inclusion with semi-axes mu in [0.15, 0.35]^3, POD
n = 64, ECM m = 600), each with its own seeded 50-step load path (principal
stretches 0.9-1.15, random rotation).  Default path: the mixed-precision
solve -- FP64 return map, eigen log/exp, stresses, convergence test and
refined n x n solve; double-float FP32 residual; TF32 tensor-core stiffness --
with the learned Newton start (4 x 128 GELU network, BF16 weights) and its
previous-step fallback.  Each step is one CUDA-graph launch.

Beside the timed steps the line carries:
  * fp64_gpu: the plain-start all-FP64 path on the same instances and load
    steps, and vs_fp64_gpu = value / its value;
  * full_path: all 50 load steps of the paths on a fresh state, with the count
    of instance-steps that did not converge;
  * accuracy: the timed steps' Pbar and Abar and the final reduced coordinates
    and plastic strains of sampled instances against the FP64 oracle, which the
    CPU-baseline leg runs on the same instances over the same load steps
    (the line is flagged inadmissible, and the exit status is 3, if the Pbar
    error exceeds 1e-7).

usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                       [--workload c2|c3|c5] [--precision fp64|fp32|tf32|bf16] [--start plain|prev|mlp]
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 FMA pipe: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz (unit count and clock of the recipe)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12      # 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12    # 152 SMs x 128 FFMA/clk x 2 FLOP x 2.07 GHz
# executed FP64 FLOPs (2 x DFMA + DMUL + DADD, SASS thread counters of one ncu capture) per
# cubature point and evaluation of the constitutive kernel (kinematics, return map, P, pull-backs;
# the tangent runs in FP32 on the mixed paths, in FP64 on the FP64 path), taken on the first
# Newton pass of load step 10 (every instance evaluated; c2 at B = 4096, c3 at B = 2048):
#   ncu --profile-from-start off --metrics <the three counters> -k regex:k_constitutive -c 1 \
#       python bench.py [--workload c2] [--batch 2048] [--precision fp64 --start plain] --steps 1 \
#       --warmup 10 --no-graphs --no-cpu --no-e2e --no-fp64-arm --no-full-path --profile-range
# (the yield filter makes elastic points cheaper, so the count depends on the plastic fraction)
CONST_FP64_FLOP_PER_POINT = {(3, "mixed"): 1225.9, (3, "fp64"): 5828.2, (2, "mixed"): 544.7, (2, "fp64"): 1433.9}
# DRAM bytes (read + write) per evaluated point of the mixed-path constitutive kernel, from the same
# captures with dram__bytes_read.sum and dram__bytes_write.sum added: c3 1293 MB / 2048 x 600 points
# (algorithmic ~660 per point; the rest is register-spill traffic of the five-block configuration
# written back from L2), c2 105 MB / 4096 x 160 points
CONST_DRAM_BYTES_PER_POINT = {(3, "mixed"): 1052.1, (2, "mixed"): 161.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c2", "c3", "c5"])
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32", "tf32", "bf16"])
    ap.add_argument("--start", default=None, choices=["plain", "prev", "mlp"],
                    help="Newton start (default: the learned start with data/mlp_<workload>.npz where that "
                         "network exists, else the previous-step predictor)")
    ap.add_argument("--mlp", default=None, help="trained learned-start network (npz) for --start mlp "
                                                "(default data/mlp_<workload>.npz)")
    ap.add_argument("--no-graphs", action="store_true", help="time the host-driven pass loop instead of graphs")
    ap.add_argument("--batch", type=int, default=None, help="override the batch size (testing)")
    ap.add_argument("--sensitivity", action="store_true",
                    help="also compute the shape sensitivities dPbar/dmu after every step (rom_sensitivity_device)")
    ap.add_argument("--fp64-residual", action="store_true",
                    help="form the residual of the tensor-core paths in FP64 instead of double-float FP32 pairs")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg (and with it the accuracy check)")
    ap.add_argument("--no-fp64-arm", action="store_true", help="skip the plain-start FP64 GPU arm")
    ap.add_argument("--no-full-path", action="store_true", help="skip the run over all load steps of the paths")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the first timed step of the first timed region by cudaProfilerStart/Stop (for "
                         "ncu --profile-from-start off: its first constitutive launch evaluates every instance)")
    ap.add_argument("--serve-budget-gb", type=float, default=None,
                    help="ragged workload: device budget for the instances' states (default: 80%% of free memory)")
    ap.add_argument("--sample", type=int, default=None,
                    help="instances the oracle runs for the CPU baseline and the accuracy check "
                         "(default 16 for c3, 256 for c2)")
    args = ap.parse_args()
    default_mlp = os.path.join(ROOT, "data", "mlp_%s.npz" % args.workload)
    if args.start is None:
        args.start = "mlp" if os.path.exists(default_mlp) else "prev"
    if args.start == "mlp" and args.mlp is None:
        args.mlp = default_mlp
    return args


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return parse_clock_lines(self.lines)


def parse_clock_lines(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen in nvidia-smi CSV lines
    (clocks.sm, clocks.max.sm, power.draw, then the four reason columns in CLOCK_REASONS order)."""
    sm, mx, reasons = [], [], set()
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 7:
            continue
        try:
            sm.append(float(f[0]))
            mx.append(float(f[1]))
        except ValueError:
            continue
        for nm, v in zip(CLOCK_REASONS, f[3:7]):
            if v.lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": sorted(reasons), "samples": len(sm)}


CLOCK_REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
# reasons that invalidate a timing (sw_power_cap is normal under load and only noted)
INVALIDATING_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def throttled(clk):
    """True if a reason that invalidates the timing was active during the timed region."""
    return any(r in INVALIDATING_REASONS for r in clk.get("reasons", []))


def load_workload(args, first=0, B=None):
    from paper_2307_16894_gb300 import workload
    B = B or args.batch
    rom, mu, coef, paths = workload.batch(args.workload, B=B, first=first)
    return rom, mu, coef, paths


def solver_opts(args, rom):
    # default: FP64 return map, eigen log/exp, stresses and convergence test; the residual of the
    # tensor-core paths in double-float FP32 pairs (--fp64-residual: FP64); the stiffness on the
    # tensor cores: the 3D one in TF32, the 2D one FP32-accurate (TF32 hi/lo split)
    prec = args.precision or ("tf32" if args.workload == "c3" else "fp32")
    tol_rel = 1e-10 if prec == "fp64" else 1e-9
    max_iter = 25 if prec == "fp64" else 50
    return prec, dict(tol_rel=tol_rel, tol_abs=rom["tol_abs"], max_iter=max_iter, max_ls=6, precision=prec,
                      start=args.start, polar_split=True, want_abar=True, fp64_residual=args.fp64_residual)


def flush_l2(buf):
    buf.add_(1.0)


def sample_indices(B, ns):
    """ns instances spread evenly over a batch of B (first and last included)."""
    return np.unique(np.linspace(0, B - 1, max(1, min(ns, B))).round().astype(np.int64))


def default_sample(args):
    return args.sample or (16 if args.workload == "c3" else 256)


def run_ours(args, rank, world):
    import torch
    from paper_2307_16894_gb300 import binding
    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    from paper_2307_16894_gb300 import workload
    B_total = args.batch or workload.WORKLOADS[args.workload]["B"]
    # weak scaling: every rank solves its own B instances (seeds offset by rank)
    rom, mu, coef, paths = workload.shard(args.workload, B_total, rank)
    B = len(coef)
    d = rom["d"]
    nsteps = paths.shape[1]
    W, K = args.warmup, args.steps
    if W + K > nsteps:
        raise SystemExit("warmup + steps must be <= %d load steps" % nsteps)
    prec, kw = solver_opts(args, rom)
    stream = torch.cuda.current_stream()
    ctx = binding.Context(d, dev, stream.cuda_stream)
    ctx.load_basis(rom["G"])
    ctx.load_cubature(rom["w"], rom["phase"], rom["phases"], rom["omega"])
    ctx.set_geometry(rom["Gmu"], coef)
    if args.start == "mlp":
        from paper_2307_16894_gb300 import warmstart
        warmstart.load_into(ctx, args.mlp, B)
    opts = binding.make_opts(**kw)
    Fd = torch.from_numpy(np.ascontiguousarray(paths.transpose(1, 0, 2, 3))).to("cuda")    # [steps, B, d, d]
    # one output slice per timed step, so that the timed steps' Pbar and Abar can be checked afterwards
    Pk = torch.empty((K, B, d, d), dtype=torch.float64, device="cuda")
    Ak = torch.empty((K, B, d * d, d * d), dtype=torch.float64, device="cuda")
    Pd, Ad = Pk[0], Ak[0]
    Id = torch.empty((B, binding.INFO_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > 129 MB L2
    # CUDA-core assembly tiles picked by rom_autotune on the tangents of the first load step
    # (the tensor-core tiles are fixed; the call then returns tile 0)
    st0 = ctx.state_create(B)
    ctx.step_device(st0, opts, Fd[0], Pd, Ad, Id)
    tile = ctx.autotune(st0, opts)
    st0.close()

    # shape sensitivities dPbar/dmu after every step (optional, inside the timed region)
    Sd = torch.empty(B * rom["d"] ** 2 * coef.shape[1], dtype=torch.float64, device="cuda") if args.sensitivity else None

    def max_over_ranks(ms):
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms

    ranged = [False]

    def timed_region(graphs, profile, o=opts, keep_state=False):
        st = ctx.state_create(B)
        ctx.use_graphs(graphs)
        for k in range(W):
            ctx.step_device(st, o, Fd[k], Pd, Ad, Id)
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        clocks = Clocks(dev)
        clocks.start()
        if profile:
            ctx.profile(1)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        infos = []
        torch.cuda.synchronize()
        for k in range(K):
            flush_l2(flush)
            mark = args.profile_range and k == 0 and not ranged[0]
            if mark:
                torch.cuda.cudart().cudaProfilerStart()
            ev[k][0].record(stream)
            ctx.step_device(st, o, Fd[W + k], Pk[k], Ak[k], Id)
            if Sd is not None:
                ctx.sensitivity_device(st, Sd)
            ev[k][1].record(stream)
            if mark:
                torch.cuda.synchronize()
                torch.cuda.cudart().cudaProfilerStop()
                ranged[0] = True
            infos.append(Id.clone())
        torch.cuda.synchronize()
        prof = ctx.profile_read() if profile else None
        if profile:
            ctx.profile(0)
        clk = clocks.stop()
        ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev))
        info = np.frombuffer(torch.cat(infos).cpu().numpy().tobytes(), dtype=binding.INFO_DTYPE)
        if keep_state:
            return ms, info, prof, clk, st
        st.close()
        return ms, info, prof, clk

    graphs = not args.no_graphs
    ms, info, prof_main, clk, st_main = timed_region(graphs, profile=not graphs, keep_state=True)
    # a timing taken under a hardware or thermal slowdown is discarded and taken once more
    # (the decision is the same on every rank, so the collectives inside stay matched)
    again = throttled(clk)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([1 if again else 0], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        again = bool(t.item())
    if again:
        first = clk["reasons"]
        st_main.close()
        ms, info, prof_main, clk, st_main = timed_region(graphs, profile=not graphs, keep_state=True)
        clk = dict(clk, remeasured=True, first_reasons=first)
    # the timed steps' outputs and final state of the sampled instances (accuracy check)
    samp = sample_indices(B, default_sample(args))
    si = torch.from_numpy(samp).cuda()
    a_fin, _, xi_fin = st_main.export()
    check = dict(idx=samp, Pbar=Pk.index_select(1, si).cpu().numpy(), Abar=Ak.index_select(1, si).cpu().numpy(),
                 status=info["status"].reshape(K, B)[:, samp], a=a_fin[samp], xi=xi_fin[samp])
    st_main.close()
    if graphs:
        # kernel times and FLOPs of the same K steps through the per-launch path (events per launch)
        ms_prof, _, prof, clk_prof = timed_region(False, profile=True)
    else:
        ms_prof, prof, clk_prof = ms, prof_main, clk
    n_ok = int((info["status"] == 0).sum())
    value = B * world * K / (ms / 1e3)
    groups = {k: v for k, v in prof.items()}
    dom = max(groups, key=lambda g: groups[g][0])
    launches = sum(v[1] for v in groups.values())
    res = dict(value=value, ms=ms, n_ok=n_ok, n_total=len(info), iters_mean=float(info["iters"].mean()),
               evals_mean=float(info["evals"].mean()), prof=groups, dom=dom, launches=launches, clocks=clk,
               prec=prec, fp64_residual=bool(args.fp64_residual), B=B, W=W, K=K, graphs=graphs, ms_profiled=ms_prof,
               clocks_profiled=clk_prof, workload=args.workload, tile=tile, check=check)
    # all load steps of the paths on a fresh state (graphs), with the instance-steps that did not converge
    if not args.no_full_path:
        ctx.use_graphs(graphs)
        st = ctx.state_create(B)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stats = []
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(nsteps):
            ctx.step_device(st, opts, Fd[k], Pd, Ad, Id)
            stats.append(Id.clone())
        e1.record(stream)
        torch.cuda.synchronize()
        msf = max_over_ranks(e0.elapsed_time(e1))
        fi = np.frombuffer(torch.cat(stats).cpu().numpy().tobytes(), dtype=binding.INFO_DTYPE).reshape(nsteps, B)
        bad = fi["status"] != 0
        st.close()
        res["full_path"] = dict(value=B * world * nsteps / (msf / 1e3), unit="macro-point load-steps/s",
                                load_steps=nsteps, ms=msf, not_converged=int(bad.sum()), instance_steps=int(bad.size),
                                first_failure_step=int(np.argmax(bad.any(1))) if bad.any() else None,
                                newton_iters_mean=float(fi["iters"].mean()),
                                note="every load step of the 50-step paths from the initial state; instances that "
                                     "do not converge keep their last converged history")
    # end-to-end through the public host-buffer call (H2D of Fbar, D2H of Pbar, Abar, info each step)
    if not args.no_e2e:
        ctx.use_graphs(False)
        st2 = ctx.state_create(B)
        ctx.sync()
        for k in range(W):
            ctx.step(st2, opts, paths[:, k])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(K):
            ctx.step(st2, opts, paths[:, W + k])
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        res["e2e"] = dict(value=B * world * K / te, unit="macro-point load-steps/s",
                          h2d_bytes_per_step=B * d * d * 8,
                          d2h_bytes_per_step=B * (d * d + d ** 4) * 8 + B * binding.INFO_DTYPE.itemsize)
        st2.close()
    # the plain-start all-FP64 path on the same instances and load steps (the method without the
    # mixed precision and the learned start)
    if not args.no_fp64_arm and prec != "fp64":
        o64 = binding.make_opts(tol_rel=1e-10, tol_abs=rom["tol_abs"], max_iter=25, max_ls=6, precision="fp64",
                                start="plain", polar_split=True, want_abar=True)
        ms64, info64, _, clk64 = timed_region(graphs, profile=False, o=o64)
        res["fp64_gpu"] = dict(value=B * world * K / (ms64 / 1e3), unit="macro-point load-steps/s",
                               ms_per_step=ms64 / K, newton_iters_mean=float(info64["iters"].mean()),
                               converged=int((info64["status"] == 0).sum()), total=len(info64),
                               precision="fp64", start="plain", clocks=clk64)
    ctx.close()
    return res


def run_serving(args, rank, world):
    """Ragged batch of 2D and 3D models of different n and m served together (rom_serve)."""
    import torch
    from paper_2307_16894_gb300 import serving
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    B_total = args.batch or 65536
    W, K = args.warmup, args.steps
    groups = serving.make_groups(B_total, share_2d=0.75, steps=W + K, seed0=40_000 + rank * B_total)
    budget = int(args.serve_budget_gb * 2 ** 30) if args.serve_budget_gb else None
    srv = serving.Server(groups, precision=args.precision or "fp32", start=args.start, budget_bytes=budget)
    for k in range(W):
        srv.step(k)
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", 0)))
    clocks.start()
    walls, lats, its, ok = [], [], [], 0
    for k in range(K):
        wall, lat, info = srv.step(W + k)
        walls.append(wall)
        lats.append(lat)
        its.append(info["iters"].mean())
        ok += int((info["status"] == 0).sum())
    clk = clocks.stop()
    ms = float(np.sum(walls))
    lat = np.concatenate(lats)
    desc = ["%s:B=%d,n=%d,m=%d" % (g["name"], g["B"], g["rom"]["n"], g["rom"]["m"]) for g in groups]
    chunks = ["%s[%d:%d]@wave%d" % (groups[c["group"]]["name"], c["start"], c["start"] + c["count"], c["wave"])
              for c in srv.chunks]
    waves = len(srv.waves)
    srv.close()
    return dict(value=B_total * world * K / (ms / 1e3), ms=ms, lat_p50=float(np.percentile(lat, 50)),
                lat_p99=float(np.percentile(lat, 99)), iters=float(np.mean(its)), ok=ok, total=B_total * K,
                groups=desc, chunks=chunks, waves=waves, budget=srv.budget, clocks=clk)


def cpu_baseline(args, n_inst=None, n_steps=None, budget_s=20.0, idx=None, keep=False):
    """The FP64 oracle (as it stands) on the host cores, on a bounded sample of the workload:
    instances idx (default: the first n_inst) over the first n_steps load steps (or until
    budget_s has passed), each started from the previous-step predictor.  keep: also return
    the oracle's Pbar and Abar of every step and its final reduced coordinates and plastic
    strains (the accuracy check of the timed steps)."""
    import oracle
    from paper_2307_16894_gb300 import workload
    if idx is None:
        rom, mu, coef, paths = load_workload(args, B=n_inst or (512 if args.workload == "c2" else 16))
    else:
        parts = [workload.batch(args.workload, B=1, first=int(i)) for i in idx]
        rom = parts[0][0]
        coef = np.concatenate([p[2] for p in parts])
        paths = np.concatenate([p[3] for p in parts])
    B = len(coef)
    d, n, m = rom["d"], rom["n"], rom["m"]
    Gmu = rom["Gmu"].reshape(m, d, d, -1)
    Fm = np.eye(d)[None, None] + np.einsum("iack,bk->biac", Gmu, coef)
    Finv, J = np.linalg.inv(Fm), np.abs(np.linalg.det(Fm))
    q = np.zeros((B, n))
    dq_prev = np.zeros((B, n))
    Fp = np.tile(np.eye(3), (B, m, 1, 1)).copy()
    xi = np.zeros((B, m))
    nthreads = os.cpu_count() or 1
    steps = paths.shape[1] if n_steps is None else min(n_steps, paths.shape[1])
    P_all, A_all, S_all = [], [], []
    t0 = time.perf_counter()
    done = 0
    for k in range(steps):
        qs = q + dq_prev
        o = oracle.rom_batch(rom, Finv, J, paths[:, k], qs, Fp, xi, 1e-10, rom["tol_abs"], 25, max_ls=6,
                             nthreads=nthreads)
        ok = o["status"] == 0
        dq_prev[ok] = qs[ok] - q[ok]
        q[ok] = qs[ok]
        if keep:
            P_all.append(o["Pbar"].copy())
            A_all.append(o["Abar"].copy())
            S_all.append(o["status"].copy())
        done += 1
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    t = time.perf_counter() - t0
    which = ("instances %s" % ",".join(str(int(i)) for i in idx)) if idx is not None else "the first %d instances" % B
    res = dict(value=B * done / t, unit="macro-point load-steps/s", cores=nthreads, kind="oracle",
               sample="%s (%d) x first %d load steps of the %s workload (%.1f s)" % (which, B, done, args.workload, t))
    if keep:
        res["_out"] = dict(Pbar=np.stack(P_all), Abar=np.stack(A_all), status=np.stack(S_all), q=q.copy(),
                           xi=xi.copy(), steps=done)
    return res


def accuracy(check, ref, W, K, tol=1e-7):
    """Errors of the timed steps' outputs on the sampled instances against the oracle: Pbar and
    Abar per instance and step (max |difference| / max |oracle value| of that instance-step),
    the reduced coordinates and plastic strains after the last timed step (over the sample).
    An instance is compared while both sides agree on convergence; from the first step where one
    side converges and the other does not, its histories differ and it is counted in `split`."""
    if ref["steps"] < W + K:
        return dict(checked=False, reason="the oracle ran %d of %d load steps" % (ref["steps"], W + K))
    gs, os_ = check["status"], ref["status"][W:W + K]
    # instances whose oracle run already stalled during the warm-up steps carry another history
    alive = (ref["status"][:W] == 0).all(0) if W else np.ones(gs.shape[1], bool)
    ep = ea = 0.0
    compared = 0
    for k in range(K):
        alive &= gs[k] == os_[k]
        for j in np.nonzero(alive & (os_[k] == 0))[0]:
            P0, A0 = ref["Pbar"][W + k, j], ref["Abar"][W + k, j]
            ep = max(ep, float(np.abs(check["Pbar"][k, j] - P0).max() / max(np.abs(P0).max(), 1e-300)))
            ea = max(ea, float(np.abs(check["Abar"][k, j] - A0).max() / max(np.abs(A0).max(), 1e-300)))
            compared += 1
    fin = alive & (gs[-1] == 0)
    eq = float(np.abs(check["a"][fin] - ref["q"][fin]).max() / max(np.abs(ref["q"][fin]).max(), 1e-300)) if fin.any() else None
    exi = float(np.abs(check["xi"][fin] - ref["xi"][fin]).max() / max(np.abs(ref["xi"][fin]).max(), 1e-300)) if fin.any() else None
    split = [int(i) for i in check["idx"][~alive]]
    return dict(checked=True, instances=[int(i) for i in check["idx"]], load_steps=[W, W + K - 1],
                pbar_rel_err=ep, abar_rel_err=ea, q_rel_err=eq, xi_rel_err=exi, instance_steps_compared=compared,
                instance_steps=int(gs.size), split=split, tol_pbar=tol, admissible=bool(ep <= tol and compared > 0),
                oracle="FP64, Newton tolerance 1e-10 relative, max 25 iterations, previous-step start")


def kernel_rooflines(r, peaks):
    """Achieved rate of each timed kernel group against the peak of the unit that bounds it (the
    FLOP counts are the library's per-launch algorithmic counts; the constitutive group's FP64
    FLOPs are points evaluated x CONST_FP64_FLOP_PER_POINT)."""
    from paper_2307_16894_gb300 import workload
    rom = workload.load_model(workload.WORKLOADS[r["workload"]]["model"])
    d, n, m = rom["d"], rom["n"], rom["m"]
    prof, prec = r["prof"], r["prec"]
    tot = sum(v[0] for v in prof.values())
    bf16 = peaks.get("bf16_tflops", 1900.0)
    src = "MEASURED_PEAKS.json" if "bf16_tflops" in peaks else "fallback 1.9 PFLOP/s"
    out = {}

    def add(name, bound, flops, peak, peak_source, traffic=None):
        ms = prof[name][0]
        if ms <= 0 or flops <= 0:
            return
        a = flops / (ms / 1e3) / 1e12
        out[name] = dict(kernel=name, bound=bound, achieved=a, peak=peak, unit="TFLOP/s", frac=a / peak,
                         traffic=traffic, share=ms / tot, peak_source=peak_source)

    kin = 2.0 * m * d * d * n
    points = prof["constitutive"][2] / kin * m
    key = (d, "fp64" if prec == "fp64" else "mixed")
    if key in CONST_FP64_FLOP_PER_POINT:
        nl = max(prof["constitutive"][1], 1)
        traffic = (points / nl * CONST_DRAM_BYTES_PER_POINT[key]) if key in CONST_DRAM_BYTES_PER_POINT else None
        add("constitutive", "alu", points * CONST_FP64_FLOP_PER_POINT[key], FP64_PEAK_TFLOPS,
            "FP64 pipe: 152 SM x 2 DFMA/clk x 2 FLOP x 2.07 GHz", traffic)
    if n <= 64 and prec != "fp64":   # the stiffness runs on the tensor cores
        pk = bf16 * (1.0 if prec == "bf16" else 0.5)
        add("assemble", "tensor", prof["assemble"][2], pk,
            src + " bf16_tflops" + ("" if prec == "bf16" else " x 0.5 (TF32 rate)") +
            ("; FP32 as a TF32 hi/lo split: 3 MMAs per algorithmic product" if prec == "fp32" else ""))
    elif prec == "fp64":
        add("assemble", "alu", prof["assemble"][2], FP64_PEAK_TFLOPS, "FP64 pipe")
    else:
        add("assemble", "alu", prof["assemble"][2], FP32_PEAK_TFLOPS, "FP32 pipe: 152 SM x 128 FFMA/clk x 2 x 2.07 GHz")
    if prof.get("force", (0, 0, 0))[2] > 0:
        if r.get("fp64_residual"):
            add("force", "alu", prof["force"][2], FP64_PEAK_TFLOPS, "FP64 pipe")
        else:   # double-float residual: 12 FP32 pipe operations per multiply-add
            add("force", "alu", prof["force"][2], FP32_PEAK_TFLOPS / 12,
                "FP32 pipe / 12: double-float multiply-add of 12 FP32 operations")
    # the LU runs in FP64 on the FP64 path and in FP32 (with FP64 refinement) on the mixed paths
    if prec == "fp64":
        add("solve", "alu", prof["solve"][2], FP64_PEAK_TFLOPS, "FP64 pipe")
    else:
        add("solve", "alu", prof["solve"][2], FP32_PEAK_TFLOPS, "FP32 pipe: FP32 LU with FP64 refinement")
    return out

WORKLOAD_TEXT = {"c2": "2D porous RVE 64x64 Q4, n=24, m=160, B=4096, 50-step paths",
                 "c3": "3D inclusion RVE 24^3 hex8, n=64, m=600, B=16384, 50-step paths"}


def workload_name(args):
    w = WORKLOAD_TEXT[args.workload]
    if args.start == "mlp":
        w += "; learned Newton start (MLP 4 x 128 GELU, BF16 weights)"
    return w


def main():
    args = parse()
    rank, world, local = dist_env()
    metric = "macro-point ROM load-steps/s"
    unit = "macro-point load-steps/s"
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        if rank != 0:
            return
        cb = cpu_baseline(args, budget_s=max(5.0, 60.0 / max(args.steps + args.warmup, 1)))
        line = dict(metric=metric, value=cb["value"], unit=unit, n_gpus=args.gpus, steps=args.steps,
                    warmup=args.warmup, impl="reference", higher_is_better=True, scaling="weak",
                    vs_baseline=None, dtype="f64", data="synthetic",
                    config=dict(workload=workload_name(args)), cpu_baseline=cb,
                    e2e=dict(value=cb["value"], unit=unit, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
        print(json.dumps(line))
        return
    if args.workload == "c5":
        r = run_serving(args, rank, world)
        if rank == 0:
            line = dict(metric=metric, value=r["value"], unit=unit, n_gpus=world, steps=args.steps,
                        warmup=args.warmup, ms_per_step=r["ms"] / args.steps, higher_is_better=True,
                        scaling="weak", vs_baseline=None, dtype="f64+f32", data="synthetic",
                        config=dict(workload="ragged: 2D n 16/24/32 m 100/150/200 + 3D n 48/64/95 m 400/650/900",
                                    groups=r["groups"], chunks=r["chunks"], waves=r["waves"],
                                    state_budget_bytes=r["budget"], graph_launches_per_step=r["waves"],
                                    converged=r["ok"], total=r["total"],
                                    newton_iters_mean=r["iters"], l2="working set >> L2"),
                        latency_ms=dict(p50=r["lat_p50"], p99=r["lat_p99"]), roofline=None, clocks=r["clocks"])
            print(json.dumps(line))
        return
    r = run_ours(args, rank, world)
    if rank != 0:
        return
    peaks = {}
    if os.path.exists(PEAKS_FILE):
        peaks = json.load(open(PEAKS_FILE))
    rooflines = kernel_rooflines(r, peaks)
    roof = rooflines.get(r["dom"]) or dict(kernel=r["dom"], bound="alu", achieved=None, peak=FP64_PEAK_TFLOPS,
                                            unit="TFLOP/s", frac=None, traffic=None)
    line = dict(metric=metric, value=r["value"], unit=unit, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=r["ms"] / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype={"fp64": "f64", "fp32": "f64+f32", "tf32": "f64+tf32", "bf16": "f64+bf16"}[r["prec"]],
                data="synthetic",
                config=dict(workload=workload_name(args), B_per_gpu=r["B"], precision=r["prec"], start=args.start,
                            load_steps_timed=[r["W"], r["W"] + r["K"] - 1],
                            sensitivity=bool(args.sensitivity),
                            residual=("fp64" if r["prec"] == "fp64" or args.fp64_residual else "double-float FP32 pairs"),
                            step_driver="CUDA graph, device-driven Newton loop" if r["graphs"] else "host-driven passes",
                            l2="flushed between timed steps (256 MB write)", converged=r["n_ok"],
                            assembly_tile=dict(edge=r["tile"][0], chunk=r["tile"][1]),
                            total=r["n_total"], newton_iters_mean=r["iters_mean"], evals_mean=r["evals_mean"]),
                roofline=roof, rooflines=rooflines, clocks=r["clocks"], gpu_launches=int(r["launches"]),
                profiled_ms_per_step=r["ms_profiled"] / args.steps,
                kernels={k: dict(ms=v[0], launches=v[1], gflop=v[2] / 1e9) for k, v in r["prof"].items()})
    if "e2e" in r:
        line["e2e"] = r["e2e"]
    if "fp64_gpu" in r:
        line["fp64_gpu"] = r["fp64_gpu"]
        line["vs_fp64_gpu"] = r["value"] / r["fp64_gpu"]["value"]
    if "full_path" in r:
        line["full_path"] = r["full_path"]
    admissible = True
    if not args.no_cpu:
        # the oracle on the sampled instances over the warm-up and timed load steps: timed as the
        # CPU baseline, and its outputs are the reference of the accuracy check
        cb = cpu_baseline(args, idx=r["check"]["idx"], n_steps=r["W"] + r["K"], budget_s=None, keep=True)
        ref = cb.pop("_out")
        line["cpu_baseline"] = cb
        line["accuracy"] = accuracy(r["check"], ref, r["W"], r["K"])
        admissible = line["accuracy"].get("admissible", True)
    else:
        line["accuracy"] = dict(checked=False, reason="--no-cpu")
    print(json.dumps(line))
    if not admissible:
        sys.exit(3)


if __name__ == "__main__":
    main()
