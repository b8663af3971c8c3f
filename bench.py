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
WORKLOAD = "Gray-Scott 1024x1024x2, EXPRB43 steps, h=100x explicit limit, Leja, tol 1e-8"


# DRAM bytes (read + write) of one launch of the dominant kernel, from an ncu --set full capture
# of this configuration (k_iter, a K = 2 launch; k_arnf for KIOPS; cold caches); null for configurations without a
# capture of the current kernel.  Keyed by (method, n, precision, Newton kernel).
TRAFFIC = {("leja", 1024, "DF64", "single"): 67.17e6 + 8.82e6,
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
    ap.add_argument("--clock-ms", type=int, default=100, help="nvidia-smi sampling period (0 = off)")
    ap.add_argument("--method", default="leja", choices=["leja", "kiops"])
    ap.add_argument("--kernel", default="auto", choices=["auto", "single", "tma"],
                    help="Newton-step kernel of the Leja path (auto: TMA-staged once an iteration exceeds L2)")
    ap.add_argument("--direct-launch", action="store_true",
                    help="launch every iteration kernel on its own (for ncu, which does not see into "
                         "conditional graphs); not a bench measurement")
    ap.add_argument("--workload", default="grayscott", choices=["grayscott", "burgers", "batched", "learned"],
                    help="grayscott: EXPRB43 steps (headline); burgers: phi_1(hJ) f h actions on the "
                         "2048^2 Burgers state (mixed-precision workload)")
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


def run_phix(args, world, rank, local):
    import torch
    import synth
    from paper_2211_08948_gb300 import build, phix

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
    n = args.n
    prm = synth.grayscott_params(n)
    u0 = synth.grayscott_state(n, seed=rank)
    N = u0.size
    op = phix.make_jop(phix.PHIX_OP_GRAYSCOTT, n, n, [prm["Du"], prm["Dv"], prm["F"], prm["k"]])
    prec = getattr(phix, "PHIX_" + args.prec)
    opts = phix.phix_opts_default(prec=prec, profile=2 if args.direct_launch else 1,
                                  kernel={"auto": phix.PHIX_KERNEL_AUTO, "single": phix.PHIX_KERNEL_SINGLE,
                                          "tma": phix.PHIX_KERNEL_TMA}[args.kernel])
    meth = phix.PHIX_KIOPS if args.method == "kiops" else phix.PHIX_LEJA
    tol = 1e-8
    h = prm["h"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 135 MB L2

    # ---- device-resident run -------------------------------------------------
    u = torch.tensor(u0, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        flush.fill_(1.0)  # the warm-up also loads the flush kernel
        phix.phix_exprb43_step(ctx, op, u, h, tol, meth, opts)
    u.copy_(torch.tensor(u0, dtype=torch.float64, device="cuda"))
    stats = []
    sampler = ClockSampler(local, args.clock_ms)
    sampler.start()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        flush.fill_(1.0)  # L2 flush between steps
        stats.append(phix.phix_exprb43_step(ctx, op, u, h, tol, meth, opts).as_dict())
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
    if world > 1:
        dist.barrier()
    u_fast = u.cpu().numpy()

    # ---- accuracy against the plain float64 path (same steps, untimed) -------
    uref = torch.tensor(u0, dtype=torch.float64, device="cuda")
    o64 = phix.phix_opts_default(prec=phix.PHIX_FP64)
    for _ in range(args.steps):
        phix.phix_exprb43_step(ctx, op, uref, h, tol, meth, o64)
    ur = uref.cpu().numpy()
    rel_err = float(np.linalg.norm(u_fast - ur) / np.linalg.norm(ur))
    rel_err_incr = float(np.linalg.norm(u_fast - ur) / max(np.linalg.norm(ur - u0), 1e-300))

    # ---- end to end: pinned host buffers, H2D + step + D2H every step ---------
    e2e = None
    if not args.no_e2e:
        hbuf = torch.tensor(u0, dtype=torch.float64).pin_memory()
        hout = torch.empty_like(hbuf).pin_memory()
        ud = torch.empty(N, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        # the two pinned buffers alternate: each step's input is the previous
        # step's result as read back to the host
        bufs = (hbuf, hout)
        f0.record(stream)
        for k in range(args.steps):
            flush.fill_(1.0)
            ud.copy_(bufs[k & 1], non_blocking=True)
            phix.phix_exprb43_step(ctx, op, ud, h, tol, meth, opts)
            bufs[(k + 1) & 1].copy_(ud, non_blocking=True)
            torch.cuda.current_stream().synchronize()  # the step's result is on the host
        f1.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(f0.elapsed_time(f1), world, "cuda")
        e2e = {"value": whole_job_rate(ACTIONS_PER_STEP * args.steps, ems, world), "unit": UNIT,
               "h2d_bytes_per_step": N * 8, "d2h_bytes_per_step": N * 8}

    phix.phix_destroy(ctx)

    iter_ms = sum(s["iter_ms"] for s in stats)
    iter_bytes = sum(s["iter_bytes"] for s in stats)
    iter_launches = sum(s["iter_launches"] for s in stats)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = iter_bytes / (iter_ms * 1e-3) / 1e9 if iter_ms > 0 else None
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
        "config": {"workload": WORKLOAD if args.method == "leja" else WORKLOAD.replace("Leja", "KIOPS"),
                   "grid": [n, n], "species": 2, "unknowns": N, "h": h, "tol": tol,
                   "method": args.method, "prec": args.prec, "kernel": args.kernel,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed between steps (256 MB write, inside the timed region)"},
        "time_steps_per_s": args.steps * world / (ms * 1e-3),
        "hbm_gbs_iteration_algorithmic": achieved,
        "rel_err_vs_fp64": rel_err,
        "rel_err_of_increment_vs_fp64": rel_err_incr,
        "newton_iters_per_step": statistics.mean(s["iters"] for s in stats),
        "power_mv_per_step": statistics.mean(s["power_mv"] for s in stats),
        "gpu_launches": int(sum(s["launches"] for s in stats)),
        "e2e": e2e,
        "roofline": {
            "bound": "hbm",
            "kernel": (("k_iter_tma (TMA-staged Newton-Leja step" if sum(s.get("tma_passes", 0) for s in stats) > 0
                        else "k_iter (Newton-Leja step") + "; CUDA events around each pass's WHILE loop)"
                       if args.method == "leja"
                       else "k_arnf (fused Arnoldi step; k_arn1 + k_arn2 on grids of partial tiles; CUDA events around each run of steps)"),
            "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": TRAFFIC.get((args.method, n, args.prec, "tma" if sum(s.get("tma_passes", 0) for s in stats) > 0
                                    else "single")),
            "launches": iter_launches,
            "avg_launch_us": 1e3 * iter_ms / max(1, iter_launches),
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else "fallback",
        },
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(n, u0, prm, tol)
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


def run_burgers(args, world, rank, local):
    """phi_1(h J) f(u) h on the Burgers 2048^2 state: one action per step, with
    the interval from power iteration; every precision's result is compared
    with the float64 path's."""
    import torch
    import synth
    from paper_2211_08948_gb300 import build, phix
    torch.cuda.set_device(local)
    build.build()
    stream = torch.cuda.current_stream()
    ctx = phix.phix_create(stream)
    n = 2048 if args.n == 1024 else args.n
    prm = synth.burgers_params(n)
    u0 = torch.tensor(synth.burgers_state(n, seed=rank), dtype=torch.float64, device="cuda")
    op = phix.make_jop(phix.PHIX_OP_BURGERS, n, n, [prm["nu"]], u0)
    h = prm["h"]
    # v = f(u0) h (the expensive term of the step), by the library's RHS kernel
    v = torch.empty_like(u0)
    phix.phix_rhs(ctx, op, u0, v)
    v.mul_(h)
    meth = phix.PHIX_KIOPS if args.method == "kiops" else phix.PHIX_LEJA
    tol = 1e-8
    res = {}
    outs = {}
    for pr in ["FP64", "DF64", "FP32_JV", "FP32"]:
        o = phix.phix_opts_default(prec=getattr(phix, "PHIX_" + pr), profile=1)
        out = torch.empty_like(v)
        for _ in range(args.warmup):
            phix.phix_phi_action(ctx, op, h, v, [1], [1.0], [out], tol, meth, o)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        st = []
        e0.record(stream)
        for _ in range(args.steps):
            st.append(phix.phix_phi_action(ctx, op, h, v, [1], [1.0], [out], tol, meth, o).as_dict())
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        outs[pr] = out.clone()
        it_ms = sum(s["iter_ms"] for s in st)
        it_b = sum(s["iter_bytes"] for s in st)
        res[pr] = {"actions_per_s": args.steps / (ms * 1e-3), "ms_per_action": ms / args.steps,
                   "newton_iters": st[-1]["iters"], "power_mv": st[-1]["power_mv"],
                   "iter_gbs": it_b / (it_ms * 1e-3) / 1e9 if it_ms > 0 else None}
    ref = outs["FP64"]
    for pr in res:
        res[pr]["rel_err_vs_fp64"] = float(torch.linalg.norm(outs[pr] - ref) / torch.linalg.norm(ref))
    phix.phix_destroy(ctx)
    print(json.dumps({"metric": METRIC, "workload": "Burgers %dx%d, nu=1e-3, phi_1(hJ) f h, h=50x explicit, "
                      "tol 1e-8, %s" % (n, n, args.method), "unit": UNIT, "steps": args.steps,
                      "warmup": args.warmup, "by_precision": res}), flush=True)


def run_batched(args, world, rank, local):
    """4096 independent periodic advection-diffusion problems (sides log-uniform
    32..512, D ~ U(0.1, 1), a ~ U(0, 50)^2, h = 10..200x explicit, Gaussian v),
    phi_0, phi_1, phi_2 of each, tol 1e-8, in one persistent launch per step."""
    import torch
    import synth
    from paper_2211_08948_gb300 import build, phix
    torch.cuda.set_device(local)
    build.build()
    stream = torch.cuda.current_stream()
    ctx = phix.phix_create(stream)
    spec = synth.batched_problems(4096, seed=rank)
    probs = []
    unknowns = 0
    for q in spec:
        n = q["n"]
        v = torch.tensor(synth.random_vector(n * n, q["seed_v"]), dtype=torch.float64, device="cuda")
        probs.append(dict(nx=n, ny=n, D=q["D"], ax=q["ax"], ay=q["ay"], h=q["h"],
                          rho_re=8.0 * q["D"] * n * n, rho_im=(abs(q["ax"]) + abs(q["ay"])) * n, v=v,
                          out=[torch.empty_like(v) for _ in range(3)]))
        unknowns += n * n
    res = {}
    outs = {}
    for pr in ["FP64", "DF64", "FP32_JV"]:
        o = phix.phix_opts_default(prec=getattr(phix, "PHIX_" + pr), profile=1)
        for _ in range(args.warmup):
            st, _ = phix.phix_phi_action_batched(ctx, probs, [0, 1, 2], 1e-8, o)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        launch_ms = 0.0
        for _ in range(args.steps):
            st, per = phix.phix_phi_action_batched(ctx, probs, [0, 1, 2], 1e-8, o)
            launch_ms += st.iter_ms
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        outs[pr] = [[t.clone() for t in q["out"]] for q in probs[:256]]
        res[pr] = {"actions_per_s": 3 * len(probs) * args.steps / (ms * 1e-3), "ms_per_batch": ms / args.steps,
                   "launch_ms": launch_ms / args.steps, "ctas_per_sm": st.substeps,
                   "newton_iters": st.iters, "failed": int(sum(1 for s in per if s != 0))}
    for pr in res:
        num = sum(float(torch.linalg.norm(a - b) ** 2) for x, y in zip(outs[pr], outs["FP64"]) for a, b in zip(x, y))
        den = sum(float(torch.linalg.norm(b) ** 2) for y in outs["FP64"] for b in y)
        res[pr]["rel_err_vs_fp64_first256"] = (num / den) ** 0.5
    phix.phix_destroy(ctx)
    print(json.dumps({"metric": METRIC, "workload": "batched: 4096 periodic advection-diffusion problems, "
                      "sides 32..512, phi_0..phi_2, tol 1e-8, one persistent launch", "unit": UNIT,
                      "unknowns": unknowns, "steps": args.steps, "warmup": args.warmup, "by_precision": res}),
          flush=True)


def run_learned(args, world, rank, local):
    """Learned spectral interval: label 1024 Gray-Scott / Burgers states (sides
    32..128) with the method's power iteration, train the MLP on the GPU, then
    run phi_1 actions on 256 held-out states (cycled, fresh v each time) with
    the learned interval and with power iteration; report actions/s, matvecs
    saved, fallbacks and the largest difference between the two results."""
    import torch
    import synth
    from paper_2211_08948_gb300 import build, phix, learned
    torch.cuda.set_device(local)
    build.build()
    stream = torch.cuda.current_stream()
    ctx = phix.phix_create(stream)
    specs = synth.learned_state_specs(1280, seed=rank)
    probs = []
    for sp in specs:
        st = torch.tensor(synth.learned_state(sp), dtype=torch.float64, device="cuda")
        kind = phix.PHIX_OP_GRAYSCOTT if sp["kind"] == 1 else phix.PHIX_OP_BURGERS
        probs.append((phix.make_jop(kind, sp["n"], sp["n"], sp["params"], st), sp["h"], st))
    t0 = time.perf_counter()
    X, T, mv_labels = learned.make_dataset(ctx, probs[:1024], torch)
    t1 = time.perf_counter()
    params, loss = learned.train(ctx, X, T, torch)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    nact = max(1, args.steps)
    evalp = probs[1024:]
    res = {}
    outs = {}
    # two Leja approximants at tolerance tau (different intervals, different stopping
    # points) differ by a few tau: tol 1e-9 keeps both within 1e-8 of the float64 result
    tol = 1e-9

    def act(mode, a):
        op, h, st = evalp[a % len(evalp)]
        gen = torch.Generator(device="cuda").manual_seed(a)
        v = torch.randn(st.numel(), dtype=torch.float64, device="cuda", generator=gen)
        out = torch.empty_like(v)
        rho_im = 0.0 if op.kind == phix.PHIX_OP_GRAYSCOTT else float(torch.max(torch.abs(st))) * 2 * op.nx
        o = phix.phix_opts_default(rho_im=rho_im)
        if mode == "fp64":
            o.prec = phix.PHIX_FP64
        if mode == "learned":
            s = phix.phix_phi_action_learned(ctx, op, h, v, [1], [1.0], [out], tol, params, o)
        else:
            s = phix.phix_phi_action(ctx, op, h, v, [1], [1.0], [out], tol, phix.PHIX_LEJA, o)
        return out, s

    # warm-up: both arms see every timed problem once (tables, graphs, workspace)
    for mode in ["learned", "power"]:
        for a in range(min(nact, len(evalp))):
            act(mode, a)
    for mode in ["learned", "power"]:
        mv, fb, worst = 0, 0, 0.0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for a in range(nact):
            out, s = act(mode, a)
            if mode == "learned":
                fb += s.rejections
            mv += s.power_mv
            if a < 256:
                outs.setdefault(mode, []).append(out)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        res[mode] = {"actions_per_s": nact / (ms * 1e-3), "power_matvecs": mv, "fallbacks": fb}
    worst = max(float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) for a, b in zip(outs["learned"], outs["power"]))
    # the plain float64 path (power iteration, float64 arithmetic), untimed, on the first 64 problems
    nref = min(64, len(outs["learned"]))
    err = {"learned": 0.0, "power": 0.0}
    for a in range(nref):
        ref, _ = act("fp64", a)
        for mode in err:
            err[mode] = max(err[mode], float(torch.linalg.norm(outs[mode][a] - ref) / torch.linalg.norm(ref)))
    phix.phix_destroy(ctx)
    print(json.dumps({"metric": METRIC, "workload": "learned spectral interval: phi_1(hJ)v on 256 held-out Gray-Scott/"
                      "Burgers states (sides 32..128), tol 1e-9", "unit": UNIT, "actions": nact,
                      "rel_err_vs_fp64_power": err, "fp64_reference_problems": nref,
                      "label_states": 1024, "label_power_matvecs": mv_labels, "label_s": t1 - t0, "train_s": t2 - t1,
                      "train_loss": loss, "by_interval": res,
                      "matvecs_saved": res["power"]["power_matvecs"] - res["learned"]["power_matvecs"],
                      "max_rel_diff_learned_vs_power": worst}), flush=True)


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
        "data": "synthetic", "config": {"workload": WORKLOAD, "grid": [n, n]},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "burgers":
        run_burgers(args, world, rank, local)
    elif args.workload == "batched":
        run_batched(args, world, rank, local)
    elif args.workload == "learned":
        run_learned(args, world, rank, local)
    else:
        run_phix(args, world, rank, local)


if __name__ == "__main__":
    main()
