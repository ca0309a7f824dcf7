"""Throughput of the hyper-reduced RVE load step on GB300.

One bench "step" = one load step of the whole hot path for every instance of
the batch: geometry, kinematics, FP64 return map, tangent, force and
stiffness assembly, Newton with line search, effective stress and stiffness,
history commit (all Newton iterations included).  Metric: macro-point ROM
load-steps/s = instances x load steps / time.

Default workload: 4096 macro points of the 2D plane-strain porous RVE family
(64x64 Q4 parent mesh, POD n = 24, ECM m = 160), each with its own seeded
geometry mu in [0.2, 0.35] and its own seeded 50-step load path (principal
stretches 0.9-1.15, random axes and rotation).  Default precision: FP64
residual, kinematics, return map, eigen log/exp and n x n solve with an FP32
tangent and stiffness (--precision fp64 for the all-FP64 path); previous-step
Newton predictor.  Each step is one CUDA-graph launch.

usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                       [--workload c2|c3] [--precision fp64|fp32|tf32|bf16] [--start plain|prev|mlp]
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
# the tangent runs in FP32 on the mixed paths, in FP64 on the FP64 path)
CONST_FP64_FLOP_PER_POINT = {(3, "mixed"): 1590.0, (3, "fp64"): 5917.0, (2, "mixed"): 881.0, (2, "fp64"): 2288.0}
# DRAM bytes (read + write) per evaluated cubature point of the constitutive kernel, from one ncu
# capture of its first (all instances active) launch: --metrics dram__bytes_read.sum,
# dram__bytes_write.sum -k regex:k_constitutive -s 0 -c 1 on `bench.py --workload c3 --batch 2048
# --steps 2 --warmup 3 --no-cpu --no-e2e --no-graphs` (1.168 GB / 2048 x 600 points) and on
# `bench.py --steps 2 --warmup 3 --no-cpu --no-e2e --no-graphs` (81.9 MB / 4096 x 160 points; the
# 2D outputs stay in L2 during the kernel, so DRAM sees less than the algorithmic bytes)
CONST_DRAM_BYTES_PER_POINT = {(3, "mixed"): 950.5, (2, "mixed"): 125.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c5"])
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32", "tf32", "bf16"])
    ap.add_argument("--start", default=None, choices=["plain", "prev", "mlp"],
                    help="Newton start (default: the learned start with data/mlp_<workload>.npz on the 2D workload, "
                         "where it beats the previous-step predictor, else the previous-step predictor)")
    ap.add_argument("--mlp", default=None, help="trained learned-start network (npz) for --start mlp "
                                                "(default data/mlp_<workload>.npz)")
    ap.add_argument("--no-graphs", action="store_true", help="time the host-driven pass loop instead of graphs")
    ap.add_argument("--batch", type=int, default=None, help="override the batch size (testing)")
    ap.add_argument("--sensitivity", action="store_true",
                    help="also compute the shape sensitivities dPbar/dmu after every step (rom_sensitivity_device)")
    ap.add_argument("--fp64-residual", action="store_true",
                    help="form the residual of the tensor-core paths in FP64 instead of double-float FP32 pairs")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    default_mlp = os.path.join(ROOT, "data", "mlp_%s.npz" % args.workload)
    if args.start is None:
        args.start = "mlp" if (args.workload == "c2" and os.path.exists(default_mlp)) else "prev"
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
    # tensor-core paths in double-float FP32 pairs (--fp64-residual: FP64); the 3D stiffness in
    # TF32 on the tensor cores, the 2D stiffness in FP32 on the CUDA cores
    prec = args.precision or ("tf32" if args.workload == "c3" else "fp32")
    tol_rel = 1e-10 if prec == "fp64" else 1e-9
    max_iter = 25 if prec == "fp64" else 50
    return prec, dict(tol_rel=tol_rel, tol_abs=rom["tol_abs"], max_iter=max_iter, max_ls=6, precision=prec,
                      start=args.start, polar_split=True, want_abar=True, fp64_residual=args.fp64_residual)


def flush_l2(buf):
    buf.add_(1.0)


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
    Pd = torch.empty((B, d, d), dtype=torch.float64, device="cuda")
    Ad = torch.empty((B, d * d, d * d), dtype=torch.float64, device="cuda")
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

    def timed_region(graphs, profile):
        st = ctx.state_create(B)
        ctx.use_graphs(graphs)
        for k in range(W):
            ctx.step_device(st, opts, Fd[k], Pd, Ad, Id)
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
            ev[k][0].record(stream)
            ctx.step_device(st, opts, Fd[W + k], Pd, Ad, Id)
            if Sd is not None:
                ctx.sensitivity_device(st, Sd)
            ev[k][1].record(stream)
            infos.append(Id.clone())
        torch.cuda.synchronize()
        prof = ctx.profile_read() if profile else None
        if profile:
            ctx.profile(0)
        clk = clocks.stop()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        info = np.frombuffer(torch.cat(infos).cpu().numpy().tobytes(), dtype=binding.INFO_DTYPE)
        st.close()
        return ms, info, prof, clk

    graphs = not args.no_graphs
    ms, info, prof_main, clk = timed_region(graphs, profile=not graphs)
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
        ms, info, prof_main, clk = timed_region(graphs, profile=not graphs)
        clk = dict(clk, remeasured=True, first_reasons=first)
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
               prec=prec, fp64_residual=bool(args.fp64_residual), B=B, W=W, K=K, graphs=graphs, ms_profiled=ms_prof, clocks_profiled=clk_prof,
               workload=args.workload, tile=tile)
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
    srv = serving.Server(groups, precision=args.precision or "fp32", start=args.start)
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
    desc = ["%s:B=%d,n=%d,m=%d,wave=%d" % (g["name"], g["B"], g["rom"]["n"], g["rom"]["m"], g["wave"]) for g in groups]
    srv.close()
    return dict(value=B_total * world * K / (ms / 1e3), ms=ms, lat_p50=float(np.percentile(lat, 50)),
                lat_p99=float(np.percentile(lat, 99)), iters=float(np.mean(its)), ok=ok, total=B_total * K,
                groups=desc, clocks=clk)


def cpu_baseline(args, n_inst=None, n_steps=None, budget_s=20.0):
    """The FP64 oracle (as it stands) on the host cores, on a bounded sample of the workload:
    the first n_inst instances over the first n_steps load steps."""
    import oracle
    from paper_2307_16894_gb300 import workload  # noqa: F401
    rom, mu, coef, paths = load_workload(args, B=n_inst or (512 if args.workload == "c2" else 16))
    B = len(coef)
    d, n, m = rom["d"], rom["n"], rom["m"]
    Gmu = rom["Gmu"].reshape(m, d, d, -1)
    Fm = np.eye(d)[None, None] + np.einsum("iack,bk->biac", Gmu, coef)
    Finv, J = np.linalg.inv(Fm), np.abs(np.linalg.det(Fm))
    q = np.zeros((B, n))
    Fp = np.tile(np.eye(3), (B, m, 1, 1)).copy()
    xi = np.zeros((B, m))
    prec, kw = solver_opts(args, rom)
    nthreads = os.cpu_count() or 1
    t0 = time.perf_counter()
    done = 0
    for k in range(paths.shape[1]):
        oracle.rom_batch(rom, Finv, J, paths[:, k], q, Fp, xi, 1e-10, rom["tol_abs"], 25, max_ls=6,
                         nthreads=nthreads)
        done += 1
        if (n_steps and done >= n_steps) or time.perf_counter() - t0 > budget_s:
            break
    t = time.perf_counter() - t0
    return dict(value=B * done / t, unit="macro-point load-steps/s", cores=nthreads, kind="oracle",
                sample="%d instances x first %d load steps of the %s workload (%.1f s)" % (B, done, args.workload, t))



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
    tc = (d == 3 and n <= 64 and prec != "fp64") or prec in ("tf32", "bf16")
    if tc:
        pk = bf16 * (1.0 if prec == "bf16" else 0.5)
        add("assemble", "tensor", prof["assemble"][2], pk,
            src + " bf16_tflops" + ("" if prec == "bf16" else " x 0.5 (TF32 rate)"))
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
    add("solve", "alu", prof["solve"][2], FP64_PEAK_TFLOPS, "FP64 pipe")
    return out

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
                    config=dict(workload=args.workload), cpu_baseline=cb,
                    e2e=dict(value=cb["value"], unit=unit, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
        print(json.dumps(line))
        return
    if args.workload == "c5":
        r = run_serving(args, rank, world)
        if rank == 0:
            line = dict(metric=metric, value=r["value"], unit=unit, n_gpus=world, steps=args.steps,
                        warmup=args.warmup, ms_per_step=r["ms"] / args.steps, higher_is_better=True,
                        scaling="weak", vs_baseline=None, dtype="f64+f32", data="synthetic",
                        config=dict(workload="ragged: 2D n 16/24/32 m 100/150/200 + 3D n 48/64/96 m 400/650/900",
                                    groups=r["groups"], converged=r["ok"], total=r["total"],
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
    wl = {"c2": "2D porous RVE 64x64 Q4, n=24, m=160, B=4096, 50-step paths",
          "c3": "3D inclusion RVE 24^3 hex8, n=64, m=600, B=16384, 50-step paths"}[args.workload]
    line = dict(metric=metric, value=r["value"], unit=unit, n_gpus=world, steps=args.steps, warmup=args.warmup,
                ms_per_step=r["ms"] / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype={"fp64": "f64", "fp32": "f64+f32", "tf32": "f64+tf32", "bf16": "f64+bf16"}[r["prec"]],
                data="synthetic",
                config=dict(workload=wl, B_per_gpu=r["B"], precision=r["prec"], start=args.start,
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
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
