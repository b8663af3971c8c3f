"""Benchmark: phi_l(hJ)v actions/s of EXPRB43 time steps on 2D Gray-Scott.

Workload (one "step" = one EXPRB43 step = the whole Leja hot path: power
iteration for the spectral interval, divided differences, the Newton-Leja
passes phi_1(h/2 J) f h and phi_1(h J) f h (vertical), phi_1(h J) R(a) h,
phi_3(h J)(16 R(a) - 2 R(b)) h, phi_4(h J)(-48 R(a) + 12 R(b)) h, and the
stage assembly): Gray-Scott, 1024 x 1024 periodic grid, 2 species
(N = 2,097,152), D_u = 2e-5, D_v = 1e-5, F = 0.04, k = 0.06, h = 100x the
explicit limit, tol 1e-8, double-float iteration arithmetic; the state
evolves over the timed steps.  5 phi-actions per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl phix|reference]

Under torchrun (N > 1) every rank integrates its own independent problem
(seed = rank) on its own GPU: weak scaling, no collective on the data path.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

ACTIONS_PER_STEP = 5
METRIC = "phi_l(hJ)v actions/s"
UNIT = "phi-actions/s"


# DRAM bytes (read + write) of one launch of the dominant kernel, from an ncu --set full capture
# of this configuration (k_iter, a K = 2 launch; k_arnf for KIOPS; cold caches); null for configurations without a
# capture of the current kernel.  Keyed by (method, n, precision, Newton kernel).
TRAFFIC = {("leja", 1024, "DF64", "single"): 67.16e6 + 3.71e6,
           ("leja", 2048, "DF64", "tma"): 270.30e6 + 146.65e6,
           ("kiops", 1024, "DF64", "single"): 86.58e6 + 8.34e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="phix", choices=["phix", "reference"])
    ap.add_argument("--prec", default="DF64", choices=["DF64", "FP64", "FP32_JV", "FP32"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--clock-ms", type=int, default=20, help="nvidia-smi sampling period (0 = off)")
    ap.add_argument("--method", default="leja", choices=["leja", "kiops"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "single", "tma", "fused2"],
                    help="Newton-step kernel of the Leja path (auto: TMA-staged once an iteration exceeds L2; "
                         "fused2: two iterations per launch)")
    ap.add_argument("--chain", default="auto", choices=["auto", "persistent", "graph"],
                    help="Newton passes as one cooperative launch (auto, persistent) or one launch per "
                         "iteration in a conditional graph")
    ap.add_argument("--direct-launch", action="store_true",
                    help="launch every iteration kernel on its own (for ncu, which does not see into "
                         "conditional graphs); not a bench measurement")
    ap.add_argument("--workload", default="grayscott", choices=["grayscott", "burgers", "batched", "learned",
                                                                "advdiff"],
                    help="grayscott: EXPRB43 steps (headline, with every other workload as a leg); the others "
                         "run one leg on its own")
    ap.add_argument("--no-legs", action="store_true", help="headline line only (no other workloads)")
    ap.add_argument("--full", action="store_true",
                    help="--workload learned at its stated scale: 200k labelled states of sides 128..1024 "
                         "(drawn on the GPU), 10k phi_1 actions on held-out states")
    ap.add_argument("--labels", type=int, default=200000, help="--full: labelled states")
    ap.add_argument("--actions", type=int, default=10000, help="--full: timed phi_1 actions per interval")
    ap.add_argument("--ckpt", default=None, help="--full: directory of the label checkpoint shards (resumable)")
    return ap.parse_args()


def max_over_ranks(x, world, device="cpu"):
    """The largest value of x over all ranks (x itself when world == 1)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, ms_max, world):
    """Throughput of the whole job: every rank's units over the slowest rank's time."""
    return units_per_rank * world / (ms_max * 1e-3)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, period_ms=200):
        self.index = index
        self.period = period_ms
        self.lines = []
        self.proc = None

    def start(self):
        """Start sampling and wait for the first sample, so that nvidia-smi's
        own start-up does not fall inside the timed region."""
        if self.period <= 0:
            return
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", str(self.period)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 10.0:
                time.sleep(0.05)
            self.n0 = len(self.lines)
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def roofline(kernel, stats, peak, peak_src, traffic):
    """Roofline object of the dominant kernel from the library's per-call
    profile: algorithmic bytes of the iteration launches over their CUDA-event
    time (events on the context's stream around each loop of iterations)."""
    it_ms = sum(s["iter_ms"] for s in stats)
    it_b = sum(s["iter_bytes"] for s in stats)
    it_l = sum(s["iter_launches"] for s in stats)
    achieved = it_b / (it_ms * 1e-3) / 1e9 if it_ms > 0 else None
    return {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None, "traffic": traffic, "launches": it_l,
            "avg_launch_us": 1e3 * it_ms / max(1, it_l), "peak_source": peak_src}


class GrayScottRun:
    """EXPRB43 steps of the Gray-Scott workload on one context: timed runs
    with the L2 flushed before every step inside the timed region."""

    def __init__(self, torch, phix, synth, ctx, stream, n, seed, flush):
        self.torch, self.phix, self.ctx, self.stream, self.flush = torch, phix, ctx, stream, flush
        self.n = n
        self.chain = "auto"
        self.prm = synth.grayscott_params(n)
        self.u0 = synth.grayscott_state(n, seed=seed)
        self.N = self.u0.size
        self.op = phix.make_jop(phix.PHIX_OP_GRAYSCOTT, n, n,
                                [self.prm["Du"], self.prm["Dv"], self.prm["F"], self.prm["k"]])

    def opts(self, prec, profile=1, kernel="auto"):
        ph = self.phix
        return ph.phix_opts_default(prec=getattr(ph, "PHIX_" + prec), profile=profile,
                                    kernel={"auto": ph.PHIX_KERNEL_AUTO, "single": ph.PHIX_KERNEL_SINGLE,
                                            "tma": ph.PHIX_KERNEL_TMA, "fused2": ph.PHIX_KERNEL_FUSED2}[kernel],
                                    chain={"auto": ph.PHIX_CHAIN_AUTO, "persistent": ph.PHIX_CHAIN_PERSISTENT,
                                           "graph": ph.PHIX_CHAIN_GRAPH}[self.chain])

    def run(self, steps, warmup, prec="DF64", method="leja", profile=1, kernel="auto", dist=None,
            sampler=None):
        """(ms of the timed steps, per-step stats, final state)."""
        torch, ph = self.torch, self.phix
        meth = ph.PHIX_KIOPS if method == "kiops" else ph.PHIX_LEJA
        o = self.opts(prec, profile, kernel)
        h, tol = self.prm["h"], 1e-8
        u = torch.tensor(self.u0, dtype=torch.float64, device="cuda")
        for _ in range(warmup):
            self.flush.fill_(1.0)
            ph.phix_exprb43_step(self.ctx, self.op, u, h, tol, meth, o)
        u.copy_(torch.tensor(self.u0, dtype=torch.float64, device="cuda"))
        if sampler:
            sampler.start()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        stats = []
        e0.record(self.stream)
        for _ in range(steps):
            self.flush.fill_(1.0)  # L2 flush between steps
            stats.append(ph.phix_exprb43_step(self.ctx, self.op, u, h, tol, meth, o).as_dict())
        e1.record(self.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), stats, u.cpu().numpy()


def rel_err(a, b, ref0=None):
    """||a - b|| / ||b|| (or / ||b - ref0||: the error of the increment)."""
    d = np.linalg.norm(a - b)
    return float(d / max(np.linalg.norm(b if ref0 is None else b - ref0), 1e-300))


def leg_grayscott(run, args, prec, method, kernel="auto", fp64_final=None):
    """One Gray-Scott EXPRB43 leg: phi-actions/s, ms/step, the roofline of the
    iteration kernel, and the error against the float64 path's state after
    the same steps (run here unless given)."""
    peaks = load_peaks()
    ms, st, u = run.run(args.steps, args.warmup, prec=prec, method=method, kernel=kernel)
    if fp64_final is None and prec != "FP64":
        _, _, fp64_final = run.run(args.steps, 0, prec="FP64", method=method, profile=0)
    tma = sum(s.get("tma_passes", 0) for s in st) > 0
    kname = ("k_iter_tma (TMA-staged Newton-Leja step)" if tma else "k_iter (Newton-Leja step)") \
        if method == "leja" else "k_arnf (fused Arnoldi step)"
    out = {"workload": "Gray-Scott %dx%dx2, EXPRB43, h=100x explicit, %s, tol 1e-8, %s" % (
               run.n, run.n, "Leja" if method == "leja" else "KIOPS", prec),
           "value": ACTIONS_PER_STEP * args.steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / args.steps,
           "iters_per_step": statistics.mean(s["iters"] for s in st),
           "roofline": roofline(kname, st, peaks.get("hbm_gbs", 6800.0),
                                "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback",
                                TRAFFIC.get((method, run.n, prec, "tma" if tma else "single")))}
    if fp64_final is not None and prec != "FP64":
        out["rel_err_vs_fp64"] = rel_err(u, fp64_final)
        out["rel_err_of_increment_vs_fp64"] = rel_err(u, fp64_final, run.u0)
    return out, u


def run_phix(args, world, rank, local):
    import torch
    import synth
    from paper_2211_08948_gb300 import build, phix

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    phix.load()
    stream = torch.cuda.current_stream()
    ctx = phix.phix_create(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 129 MB L2
    n = args.n
    run = GrayScottRun(torch, phix, synth, ctx, stream, n, rank, flush)
    run.chain = args.chain
    meth = phix.PHIX_KIOPS if args.method == "kiops" else phix.PHIX_LEJA
    profile = 2 if args.direct_launch else 1

    # ---- device-resident run (the headline) ----------------------------------
    sampler = ClockSampler(local, args.clock_ms)
    ms, stats, u_fast = run.run(args.steps, args.warmup, prec=args.prec, method=args.method, profile=profile,
                                kernel=args.kernel, dist=dist, sampler=sampler)
    clocks = sampler.stop()
    ms = max_over_ranks(ms, world, "cuda")
    if world > 1:
        dist.barrier()

    # ---- the plain float64 path: same steps, timed (also the error reference) --
    ms64, st64, u64 = run.run(args.steps, min(args.warmup, 3), prec="FP64", method=args.method)
    rel = rel_err(u_fast, u64)
    rel_incr = rel_err(u_fast, u64, run.u0)

    # ---- end to end through the C-ABI with HOST buffers -------------------------
    # phix_step_host copies the state in, steps, and copies it back before it
    # returns: every step moves N doubles each way inside the timed region
    e2e = None
    if not args.no_e2e:
        o = run.opts(args.prec, profile=0, kernel=args.kernel)
        hbuf = torch.tensor(run.u0, dtype=torch.float64).pin_memory()
        for _ in range(min(args.warmup, 3)):
            phix.phix_step_host(ctx, phix.PHIX_EXPRB43, run.op, hbuf, run.prm["h"], 1e-8, meth, o)
        hbuf.copy_(torch.tensor(run.u0, dtype=torch.float64))
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(args.steps):
            flush.fill_(1.0)
            phix.phix_step_host(ctx, phix.PHIX_EXPRB43, run.op, hbuf, run.prm["h"], 1e-8, meth, o)
        f1.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(f0.elapsed_time(f1), world, "cuda")
        e2e = {"value": whole_job_rate(ACTIONS_PER_STEP * args.steps, ems, world), "unit": UNIT,
               "h2d_bytes_per_step": run.N * 8, "d2h_bytes_per_step": run.N * 8,
               "api": "phix_step_host (host buffer in, host buffer out, per step)",
               "rel_err_vs_device_run": rel_err(hbuf.numpy(), u_fast)}

    peaks = load_peaks()
    peak = peaks.get("hbm_gbs", 6800.0)
    tma = sum(s.get("tma_passes", 0) for s in stats) > 0
    kname = (("k_iter_tma (TMA-staged Newton-Leja step" if tma else "k_iter (Newton-Leja step")
             + "; CUDA events around each pass's chain)") if args.method == "leja" else \
        "k_arnf (fused Arnoldi step; k_arn1 + k_arn2 on grids of partial tiles; CUDA events around each run of steps)"
    rf = roofline(kname, stats, peak, "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks
                  else "fallback", TRAFFIC.get((args.method, n, args.prec, "tma" if tma else "single")))
    if n <= 1024:
        rf["note"] = ("one iteration's operands (~117 MB at K = 2) fit in the 126 MB L2: the fraction is "
                      "algorithmic bandwidth with L2 assistance; legs.grayscott_2048 is the HBM-bound case")
    result = {
        "metric": METRIC,
        "value": whole_job_rate(ACTIONS_PER_STEP * args.steps, ms, world),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32x2 (double-float)" if args.prec == "DF64" else args.prec.lower(),
        "data": "synthetic (seeded Gray-Scott initial state, seed = rank)",
        "config": bench_config(args, world),
        "time_steps_per_s": args.steps * world / (ms * 1e-3),
        "hbm_gbs_iteration_algorithmic": rf["achieved"],
        "rel_err_vs_fp64": rel,
        "rel_err_of_increment_vs_fp64": rel_incr,
        "fp64_path": {"value": ACTIONS_PER_STEP * args.steps / (ms64 * 1e-3), "unit": UNIT,
                      "ms_per_step": ms64 / args.steps, "speedup_of_headline": ms64 / ms},
        "newton_iters_per_step": statistics.mean(s["iters"] for s in stats),
        "power_mv_per_step": statistics.mean(s["power_mv"] for s in stats),
        "gpu_launches": int(sum(s["launches"] for s in stats)),
        "e2e": e2e,
        "roofline": rf,
        "clocks": clocks,
    }
    if world == 1 and not args.no_legs:
        legs = {}
        t0 = time.perf_counter()
        legs["kiops"], _ = leg_grayscott(run, args, args.prec, "kiops")
        run2 = GrayScottRun(torch, phix, synth, ctx, stream, 2048, rank, flush)
        legs["grayscott_2048"], _ = leg_grayscott(run2, args, args.prec, "leja")
        del run2
        legs["advdiff_64"] = leg_advdiff(torch, phix, synth, ctx, stream, args)
        legs["burgers_2048"] = leg_burgers(torch, phix, synth, ctx, stream, args)
        legs["batched_4096"] = leg_batched(torch, phix, synth, ctx, stream, args)
        legs["learned"] = leg_learned(torch, phix, synth, ctx, stream, args)
        legs["wall_s"] = time.perf_counter() - t0
        result["legs"] = legs
    phix.phix_destroy(ctx)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(n, run.u0, run.prm, 1e-8)
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


def bench_config(args, world):
    """The workload the line is quoted on (shared by both arms)."""
    n = args.n
    return {"workload": workload_name(n, args.method, args.prec),
            "grid": [n, n], "species": 2, "unknowns": 2 * n * n, "h": 100.0 / (4.0 * 2e-5 * n * n), "tol": 1e-8,
            "method": args.method, "prec": args.prec, "kernel": args.kernel, "chain": args.chain,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "flushed between steps (256 MB write, inside the timed region)"}


def workload_name(n, method, prec):
    return "Gray-Scott %dx%dx2, EXPRB43 steps, h=100x explicit limit, %s, tol 1e-8" % (
        n, n, "Leja" if method == "leja" else "KIOPS")


def timed(torch, stream, fn, reps, warmup):
    """CUDA-event ms of `reps` calls of fn() after `warmup` untimed calls; fn's results."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    res = []
    e0.record(stream)
    for _ in range(reps):
        res.append(fn())
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), res


def leg_advdiff(torch, phix, synth, ctx, stream, args):
    """Advection-diffusion 64^2 (u_t = lap u + 10 (u_x + u_y)), phi_0..phi_3 of the
    Gaussian v at h = 50x the explicit diffusive step, tol 1e-10, Leja (vertical,
    one basis) and KIOPS, float64 and double-float.  1 call = 4 phi-actions."""
    n = 64
    p = synth.advdiff_params(n)
    v = torch.tensor(synth.advdiff_gaussian(n), dtype=torch.float64, device="cuda")
    op = phix.make_jop(phix.PHIX_OP_ADVDIFF, n, n, [p["D"], p["ax"], p["ay"]])
    rho = 8.0 * p["D"] * n * n
    outs = {}
    res = {}
    reps = max(args.steps, 20)
    for meth in ["leja", "kiops"]:
        for prec in ["FP64", "DF64"]:
            o = phix.phix_opts_default(prec=getattr(phix, "PHIX_" + prec), rho_re=rho)
            out = [torch.empty_like(v) for _ in range(4)]
            mid = phix.PHIX_LEJA if meth == "leja" else phix.PHIX_KIOPS
            ms, st = timed(torch, stream, lambda: phix.phix_phi_action(ctx, op, p["h"], v, [0, 1, 2, 3], [1.0] * 4,
                                                                      out, 1e-10, mid, o), reps, args.warmup)
            outs[(meth, prec)] = [t.clone() for t in out]
            res["%s_%s" % (meth, prec)] = {"value": 4 * reps / (ms * 1e-3), "unit": UNIT,
                                          "us_per_call": 1e3 * ms / reps, "iters": st[-1].iters}
    for meth in ["leja", "kiops"]:
        ref = outs[(meth, "FP64")]
        res["%s_DF64" % meth]["rel_err_vs_fp64"] = max(
            float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) for a, b in zip(outs[(meth, "DF64")], ref))
    res["max_rel_diff_leja_vs_kiops_fp64"] = max(
        float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) for a, b in zip(outs[("leja", "FP64")],
                                                                                outs[("kiops", "FP64")]))
    res["workload"] = "advection-diffusion 64x64, phi_0..phi_3, h=50x explicit, tol 1e-10"
    return res


def leg_burgers(torch, phix, synth, ctx, stream, args, n=2048):
    """phi_1(h J) f(u) h on the Burgers state (nu = 1e-3, h = 50x explicit), one
    action per call, interval by power iteration, imaginary bound from the
    state; every precision's result against the float64 path's."""
    prm = synth.burgers_params(n)
    u0 = torch.tensor(synth.burgers_state(n, seed=0), dtype=torch.float64, device="cuda")
    op = phix.make_jop(phix.PHIX_OP_BURGERS, n, n, [prm["nu"]], u0)
    h = prm["h"]
    v = torch.empty_like(u0)
    phix.phix_rhs(ctx, op, u0, v)
    v.mul_(h)
    rho_im = 2.0 * n * float(torch.max(torch.abs(u0)))
    peaks = load_peaks()
    res, outs = {}, {}
    for pr in ["FP64", "DF64", "FP32_JV", "FP32"]:
        o = phix.phix_opts_default(prec=getattr(phix, "PHIX_" + pr), profile=1, rho_im=rho_im)
        out = torch.empty_like(v)
        ms, st = timed(torch, stream, lambda: phix.phix_phi_action(ctx, op, h, v, [1], [1.0], [out], 1e-8,
                                                                  phix.PHIX_LEJA, o).as_dict(),
                       args.steps, args.warmup)
        outs[pr] = out.clone()
        res[pr] = {"value": args.steps / (ms * 1e-3), "unit": UNIT, "ms_per_action": ms / args.steps,
                   "newton_iters": st[-1]["iters"], "substeps": st[-1]["substeps"], "power_mv": st[-1]["power_mv"],
                   "roofline": roofline("k_iter / k_iter_tma", st, peaks.get("hbm_gbs", 6800.0),
                                        "MEASURED_PEAKS.json hbm_gbs (of measured)", None)}
    for pr in res:
        res[pr]["rel_err_vs_fp64"] = float(torch.linalg.norm(outs[pr] - outs["FP64"]) / torch.linalg.norm(outs["FP64"]))
        res[pr]["speedup_vs_fp64"] = res[pr]["value"] / res["FP64"]["value"]
    res["workload"] = "Burgers %dx%d, nu=1e-3, phi_1(hJ) f h, h=50x explicit, tol 1e-8, Leja" % (n, n)
    return res


def batched_setup(torch, synth, count, seed):
    spec = synth.batched_problems(count, seed=seed)
    probs, unknowns = [], 0
    for q in spec:
        n = q["n"]
        v = torch.tensor(synth.random_vector(n * n, q["seed_v"]), dtype=torch.float64, device="cuda")
        probs.append(dict(nx=n, ny=n, D=q["D"], ax=q["ax"], ay=q["ay"], h=q["h"],
                          rho_re=8.0 * q["D"] * n * n, rho_im=(abs(q["ax"]) + abs(q["ay"])) * n, v=v,
                          out=[torch.empty_like(v) for _ in range(3)]))
        unknowns += n * n
    return probs, unknowns


def leg_batched(torch, phix, synth, ctx, stream, args, count=4096):
    """4096 independent periodic advection-diffusion problems (sides log-uniform
    32..512, D ~ U(0.1, 1), a ~ U(0, 50)^2, h = 10..200x explicit, Gaussian v),
    phi_0, phi_1, phi_2 of each, tol 1e-8, one persistent launch per batch."""
    probs, unknowns = batched_setup(torch, synth, count, 0)
    res, outs = {}, {}
    reps = max(1, min(args.steps, 3))
    for pr in ["FP64", "DF64", "FP32_JV"]:
        o = phix.phix_opts_default(prec=getattr(phix, "PHIX_" + pr), profile=1)
        ms, rr = timed(torch, stream, lambda: phix.phix_phi_action_batched(ctx, probs, [0, 1, 2], 1e-8, o),
                       reps, 1)
        st, per = rr[-1]
        outs[pr] = [[t.clone() for t in q["out"]] for q in probs[:256]]
        bt, smem, per_sm = phix.phix_batched_config(ctx)
        res[pr] = {"value": 3 * len(probs) * reps / (ms * 1e-3), "unit": UNIT, "ms_per_batch": ms / reps,
                   "launch_ms": st.iter_ms, "tuned": {"threads_per_cta": bt, "smem_bytes": smem,
                                                      "ctas_per_sm": per_sm},
                   "newton_iters": st.iters, "failed": int(sum(1 for s in per if s != 0))}
        # the untuned launch (512 threads, no shared-memory passes, 2 CTAs per SM) on a fresh context
        ctx0 = phix.phix_create(stream)
        o0 = phix.phix_opts_default(prec=getattr(phix, "PHIX_" + pr))
        ms0, _ = timed(torch, stream, lambda: phix.phix_phi_action_batched(ctx0, probs, [0, 1, 2], 1e-8, o0), reps, 1)
        phix.phix_destroy(ctx0)
        res[pr]["untuned_value"] = 3 * len(probs) * reps / (ms0 * 1e-3)
    for pr in res:
        num = sum(float(torch.linalg.norm(a - b) ** 2) for x, y in zip(outs[pr], outs["FP64"]) for a, b in zip(x, y))
        den = sum(float(torch.linalg.norm(b) ** 2) for y in outs["FP64"] for b in y)
        res[pr]["rel_err_vs_fp64_first256"] = (num / den) ** 0.5
        res[pr]["speedup_vs_fp64"] = res[pr]["value"] / res["FP64"]["value"]
    res["workload"] = ("batched: %d periodic advection-diffusion problems (%d unknowns), sides 32..512, "
                       "phi_0..phi_2, tol 1e-8, one persistent launch per batch, %d batches timed" % (
                           count, unknowns, reps))
    return res


def leg_learned(torch, phix, synth, ctx, stream, args, nlabel=1024, nact=200):
    """Learned spectral interval: label Gray-Scott / Burgers states (sides
    32..128) with the method's power iteration, train the MLP on the GPU, then
    phi_1 actions on held-out states with the learned interval and with power
    iteration; matvecs saved and the error against the float64 power-iteration
    path."""
    from paper_2211_08948_gb300 import learned
    specs = synth.learned_state_specs(nlabel + 256, seed=0)
    probs = []
    for sp in specs:
        st = torch.tensor(synth.learned_state(sp), dtype=torch.float64, device="cuda")
        kind = phix.PHIX_OP_GRAYSCOTT if sp["kind"] == 1 else phix.PHIX_OP_BURGERS
        probs.append((phix.make_jop(kind, sp["n"], sp["n"], sp["params"], st), sp["h"], st))
    t0 = time.perf_counter()
    X, T, mv_labels = learned.make_dataset(ctx, probs[:nlabel], torch)
    t1 = time.perf_counter()
    params, loss = learned.train(ctx, X, T, torch)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    evalp = probs[nlabel:]
    # two Leja approximants at tolerance tau (different intervals, different stopping
    # points) differ by a few tau: tol 1e-9 keeps both within 1e-8 of the float64 result
    tol = 1e-9
    vs = []
    for a in range(min(nact, len(evalp))):
        gen = torch.Generator(device="cuda").manual_seed(a)
        vs.append(torch.randn(evalp[a][2].numel(), dtype=torch.float64, device="cuda", generator=gen))

    def act(mode, a, out):
        op, h, st = evalp[a % len(evalp)]
        v = vs[a % len(vs)]
        rho_im = 0.0 if op.kind == phix.PHIX_OP_GRAYSCOTT else float(op._keepalive.abs().max()) * 2 * op.nx
        o = phix.phix_opts_default(rho_im=rho_im)
        if mode == "fp64":
            o.prec = phix.PHIX_FP64
        if mode == "learned":
            return phix.phix_phi_action_learned(ctx, op, h, v, [1], [1.0], [out], tol, params, o)
        return phix.phix_phi_action(ctx, op, h, v, [1], [1.0], [out], tol, phix.PHIX_LEJA, o)

    outs = {m: [torch.empty_like(vs[a % len(vs)]) for a in range(nact)] for m in ["learned", "power", "fp64"]}
    res = {}
    for mode in ["learned", "power"]:
        for a in range(nact):  # warm-up: tables, graphs, workspace
            act(mode, a, outs[mode][a])
        cnt = {"mv": 0, "fb": 0}

        def one_pass():
            for a in range(nact):
                s = act(mode, a, outs[mode][a])
                cnt["mv"] += s.power_mv
                cnt["fb"] += s.rejections
        ms, _ = timed(torch, stream, one_pass, 1, 0)
        res[mode] = {"value": nact / (ms * 1e-3), "unit": UNIT, "power_matvecs": cnt["mv"], "fallbacks": cnt["fb"]}
    for a in range(nact):
        act("fp64", a, outs["fp64"][a])
    err = {m: max(float(torch.linalg.norm(x - r) / torch.linalg.norm(r)) for x, r in zip(outs[m], outs["fp64"]))
           for m in ["learned", "power"]}
    return {"workload": "learned spectral interval: phi_1(hJ)v on %d held-out Gray-Scott/Burgers states "
                        "(sides 32..128), tol 1e-9; labels from %d states" % (nact, nlabel),
            "by_interval": res, "speedup_vs_power": res["learned"]["value"] / res["power"]["value"],
            "matvecs_saved": res["power"]["power_matvecs"] - res["learned"]["power_matvecs"],
            "rel_err_vs_fp64_power_path": err, "label_power_matvecs": mv_labels, "label_s": t1 - t0,
            "train_s": t2 - t1, "train_loss": loss}


def leg_learned_full(torch, phix, synth, ctx, stream, args):
    """The learned spectral interval at its stated scale: args.labels
    Gray-Scott / Burgers states of sides log-uniform 128..1024 drawn on the
    GPU, each labelled by the library's power iteration and label targets
    (checkpointed in shards under args.ckpt: a stopped run resumes), the MLP
    trained on the GPU, then args.actions phi_1 actions (tol 1e-9) on
    held-out states with the learned interval and with power iteration; every
    action timed by CUDA events on the stream, states drawn outside the timed
    calls; errors against the float64 power-iteration path on every 20th
    state.  States are visited in order of size (the chain graphs are cached
    per grid shape); the first action of each size runs once untimed in both
    modes."""
    from paper_2211_08948_gb300 import learned
    nl, na = args.labels, args.actions
    specs = synth.learned_state_specs(nl + na, seed=5, n_lo=128, n_hi=1024)
    lab = sorted(range(nl), key=lambda i: (specs[i]["n"], i))
    ev = sorted(range(nl, nl + na), key=lambda i: (specs[i]["n"], i))

    def problem(j):
        sp = specs[lab[j]]
        st = synth.learned_state_torch(sp, torch)
        kind = phix.PHIX_OP_GRAYSCOTT if sp["kind"] == 1 else phix.PHIX_OP_BURGERS
        return phix.make_jop(kind, sp["n"], sp["n"], sp["params"], st), sp["h"], st

    t0 = time.perf_counter()
    X, T, mv_labels = learned.make_dataset(ctx, problem, torch, n=nl, ckpt_dir=args.ckpt,
                                           tag="learned_state_specs(seed=5, 128..1024)[:%d] by side" % nl)
    t1 = time.perf_counter()
    perm = np.random.default_rng(0).permutation(nl)  # batches mixing sizes and kinds
    params, loss = learned.train(ctx, X[perm], T[perm], torch)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    tol = 1e-9
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    modes = ("learned", "power")
    tot, mv, fb, err = ({m: 0 for m in modes} for _ in range(4))
    iters, subs = {m: 0 for m in modes}, {m: 0 for m in modes}
    nerr, last_n, sizes, ratio = 0, None, [], []

    def act(mode, op, h, v, out, rho_im):
        o = phix.phix_opts_default(rho_im=rho_im, prec=phix.PHIX_FP64 if mode == "fp64" else phix.PHIX_DF64)
        if mode == "learned":
            return phix.phix_phi_action_learned(ctx, op, h, v, [1], [1.0], [out], tol, params, o)
        return phix.phix_phi_action(ctx, op, h, v, [1], [1.0], [out], tol, phix.PHIX_LEJA, o)

    for a, i in enumerate(ev):
        sp = specs[i]
        st = synth.learned_state_torch(sp, torch)
        kind = phix.PHIX_OP_GRAYSCOTT if sp["kind"] == 1 else phix.PHIX_OP_BURGERS
        op = phix.make_jop(kind, sp["n"], sp["n"], sp["params"], st)
        gen = torch.Generator(device="cuda").manual_seed(i)
        v = torch.randn(st.numel(), dtype=torch.float64, device="cuda", generator=gen)
        rho_im = 0.0 if kind == phix.PHIX_OP_GRAYSCOTT else float(st.abs().max()) * 2 * sp["n"]
        outs = {m: torch.empty_like(v) for m in modes}
        if sp["n"] != last_n:  # graphs and tables of a new size, untimed
            for m in modes:
                act(m, op, sp["h"], v, outs[m], rho_im)
            last_n = sp["n"]
        sizes.append(sp["n"])
        rho = {}
        for m in modes:
            torch.cuda.synchronize()
            e0.record(stream)
            s = act(m, op, sp["h"], v, outs[m], rho_im)
            e1.record(stream)
            torch.cuda.synchronize()
            tot[m] += e0.elapsed_time(e1)
            mv[m] += s.power_mv
            fb[m] += s.rejections
            iters[m] += s.iters
            subs[m] += s.substeps
            rho[m] = s.rho
        ratio.append(rho["learned"] / rho["power"])
        if a % 20 == 0:
            ref = torch.empty_like(v)
            act("fp64", op, sp["h"], v, ref, rho_im)
            nr = float(torch.linalg.norm(ref))
            for m in modes:
                err[m] = max(err[m], float(torch.linalg.norm(outs[m] - ref)) / nr)
            nerr += 1
    res = {m: {"value": na / (tot[m] * 1e-3), "unit": UNIT, "ms": tot[m], "power_matvecs": mv[m],
               "fallbacks": fb[m]} for m in modes}
    return {"workload": "learned spectral interval at scale: %d labelled Gray-Scott/Burgers states (sides "
                        "128..1024, drawn on the GPU), phi_1(hJ)v on %d held-out states, tol 1e-9, double-float"
                        % (nl, na),
            "by_interval": res, "speedup_vs_power": res["learned"]["value"] / res["power"]["value"],
            "matvecs_saved": mv["power"] - mv["learned"],
            "rel_err_vs_fp64_power_path": {"max": err, "states": nerr},
            "label_power_matvecs": mv_labels, "label_s": t1 - t0, "train_s": t2 - t1, "train_loss": loss,
            "eval_sides": {"min": min(sizes), "median": int(np.median(sizes)), "max": max(sizes)},
            "newton_iters_per_action": {m: iters[m] / na for m in modes},
            "substeps_per_action": {m: subs[m] / na for m in modes},
            "rho_learned_over_power": {q: float(np.quantile(ratio, x)) for q, x in
                                       (("min", 0.0), ("p01", 0.01), ("median", 0.5), ("p99", 0.99), ("max", 1.0))}}


def run_leg(args, world, rank, local):
    """One leg on its own (--workload), printed as its own JSON object."""
    import torch
    import synth
    from paper_2211_08948_gb300 import build, phix
    torch.cuda.set_device(local)
    build.build()
    stream = torch.cuda.current_stream()
    ctx = phix.phix_create(stream)
    if args.workload == "burgers":
        out = leg_burgers(torch, phix, synth, ctx, stream, args, n=2048 if args.n == 1024 else args.n)
    elif args.workload == "batched":
        out = leg_batched(torch, phix, synth, ctx, stream, args)
    elif args.workload == "advdiff":
        out = leg_advdiff(torch, phix, synth, ctx, stream, args)
    elif args.full:
        out = leg_learned_full(torch, phix, synth, ctx, stream, args)
    else:
        out = leg_learned(torch, phix, synth, ctx, stream, args)
    phix.phix_destroy(ctx)
    out.update({"metric": METRIC, "steps": args.steps, "warmup": args.warmup})
    print(json.dumps(out), flush=True)


def cpu_baseline(n, u0, prm, tol):
    """The oracle as it stands, one full EXPRB43 step of the same workload."""
    from oracle import integrators, leja
    from oracle.operators import GrayScott
    leja.leja_points(501)
    op = GrayScott(n, prm["Du"], prm["Dv"], prm["F"], prm["k"])
    t = time.perf_counter()
    integrators.exprb43_step(op, u0, prm["h"], tol=tol)
    dt = time.perf_counter() - t
    return {"value": ACTIONS_PER_STEP / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "one EXPRB43 step (5 phi-actions) of the same 1024^2 Gray-Scott workload, "
                      "NumPy float64, single thread (%.1f s)" % dt}


def run_reference(args, world, rank):
    """Reference arm: the CPU oracle, each step a bounded sample of the same
    workload (the vertical Leja pass phi_1(h/2 J) f h, phi_1(h J) f h of one
    EXPRB43 step: 2 phi-actions)."""
    if rank != 0:
        return
    import synth
    from oracle import leja, integrators
    from oracle.operators import GrayScott, with_state
    n = args.n
    prm = synth.grayscott_params(n)
    u0 = synth.grayscott_state(n, seed=0)
    op = with_state(GrayScott(n, prm["Du"], prm["Dv"], prm["F"], prm["k"]), u0)
    leja.leja_points(501)
    spec, _ = integrators.spectrum(op)
    v = op.f(u0) * prm["h"]

    def sample():
        leja.leja_phi(op.jv, v, prm["h"], spec[0], spec[1], [(1, 0.5), (1, 1.0)], 1e-8)

    for _ in range(args.warmup):
        sample()
    t = time.perf_counter()
    for _ in range(args.steps):
        sample()
    dt = time.perf_counter() - t
    val = 2 * args.steps / dt
    desc = ("per step: the vertical Leja pass (2 phi-actions) of one EXPRB43 step on the 1024^2 "
            "Gray-Scott state, NumPy float64 oracle, single thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": bench_config(args, world),
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload != "grayscott":
        run_leg(args, world, rank, local)
    else:
        run_phix(args, world, rank, local)


if __name__ == "__main__":
    main()
