"""Benchmark of the Hubbard HMC path on GB300.

A step is one HMC trajectory (Sec. 4.1 of arXiv:1007.3432): momentum and
pseudofermion heatbath, n_md + 1 CG solves of Q x = chi for two pseudofermion
components, n_md + 1 force evaluations with momentum updates, the sigma steps,
both Hamiltonians and the Metropolis test.  The default workload is the d = 1,
N_x = 1024, N_tau = 512 lattice (524,288 sites) with 20 leapfrog steps, CG to a
true relative residual of 1e-10, in FP64.

value: M^T M applies per second inside the CG solves of the timed
trajectories (every CG step and every FP64 true-residual recomputation applies
Q = M^T M once per right-hand side), with sigma resident on the device when a
step's timed region starts.  e2e: the same count over wall time of the public
calls hh_set_field(host) -> hh_trajectory -> hh_get_field(host) per step.

After the timed trajectories the default line also carries, measured in the
same run on the same GPU (--no-extras skips them): the FP32 M^T M apply on the
d = 3, 32^3 x 128 lattice with 16 vectors per launch and with one
(c2_apply_fp32_*), two-right-hand-side CG solves to 1e-10 on that lattice in
FP64 and in mixed precision (c2_solves), and the 64-chain d = 3 batch in FP64
and in mixed precision (batch64_d3), each with its own roofline.

Further modes measure parts of the path (they print the same JSON line):
  --mode solve : a step is one CG solve of Q x = b for two right-hand sides
                 (value in solves/s), to compare FP64 with mixed precision;
  --mode apply : a step is one M^T M apply of --nvec vectors with L2 flushed
                 before it (value in applies/s), the HBM roofline of the
                 stencil;
  --mode batch : a step solves two right-hand sides for each of 64 d=3 chains of
                 uneven volume in the batched engine (autotuned), in solves/s;
  --mode serve : a Poisson stream of solve and trajectory requests at each rate
                 of --rates, served by the continuous-batching worker; reports
                 p50/p99 latency and solves/s per rate.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload c0|c1|c2] [--precision fp64|mixed]
                       [--mode trajectory|solve|apply|batch|serve] [--cg-maxit M]
                       [--nvec K] [--no-extras] [--no-cpu]
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "M\u1d40M applies/s & HBM GB/s; CG solves/s @1e-10, mixed vs FP64; p50/p99 ms"
UNIT = "MTM applies/s"
WORKLOADS = {"c0": workloads.C0, "c1": workloads.C1, "c2": workloads.C2}

# Algorithmic work per site (see the design notes): FP64 flops of one CG step
# (p update, M p with |Mp|^2, M^T t, x and r updates, |r|^2) and of one FP64
# true-residual step (M x, M^T t, b - Q x, |r|^2; + x accumulate when mixed).
def flops_per_site(d, kind, precision):
    m = 2 * d + 3
    if kind == "cg":
        return 2 * m + 10
    return 2 * m + 3 + (1 if precision == "mixed" else 0)


# Algorithmic bytes per site of a CG step: the minimum traffic of the step as
# the method states it, 11 words: p = r + beta p with q = Q p and <p, q> reads
# r, p and the links and writes p, q; x += alpha p, r -= alpha q with <r, r>
# reads x, p, r, q and writes x, r (88 B in FP64, 44 B in FP32; the 16-bit link
# precisions read 2 bytes of link instead of 4).  The engine's kernel moves 13
# words (t = M p is stored between the two sweeps of Q and the links are read
# by both sweeps); the roofline fractions use the 11 algorithmic words.  A true-
# residual step r = b - Q x reads x, the links and b and writes r (4 FP64
# words), plus, in mixed precision, x32 read and written and r32 written.
def bytes_per_site(kind, precision):
    """Algorithmic bytes per site of a CG step or of an FP64 true-residual step."""
    if kind == "cg":
        if precision == "fp64":
            return 11 * 8
        return 11 * 4 - (2 if precision.endswith("16link") else 0)
    return 4 * 8 + (12 if precision != "fp64" else 0)


# DRAM bytes per engine iteration (two right-hand sides) of the engine kernel
# as it stands, from one ncu --set full capture each (dram__bytes_read.sum +
# dram__bytes_write.sum over a 202-iteration launch; profiles/engine_kernel_*).
# A launch's traffic scales with its iterations.
ENGINE_DRAM_PER_ITER = {("d1_nx1024_nt512", "fp64"): (12724992 + 70935296) / 202.0,
                        ("d3_nx32_nt128", "mixed"): (35195983000 + 27069706000) / 202.0}

# DRAM bytes (read + write) per launch of the Q apply from one ncu capture each
# (profiles/mtm_*): (workload, dtype, vectors per launch) -> bytes.
APPLY_DRAM_PER_LAUNCH = {("d3_nx32_nt128", "fp32", 1): 33557760 + 344320 + 88320 + 6871040,
                         ("d3_nx32_nt128", "fp32", 16): 300300288 + 229754880}


def engine_traffic(wl, precision, cheb, cnt):
    """Estimated DRAM bytes per engine launch, or None without a capture."""
    per_iter = ENGINE_DRAM_PER_ITER.get((wl.name, precision))
    if per_iter is None or cheb or cnt["engine_launches"] == 0:
        return None
    # both right-hand sides advance together: one INIT iteration, then the CG
    # steps and true-residual checks of one system
    iters = (cnt["cg_steps"] + cnt["ru_steps"]) / 2.0 / cnt["engine_launches"] + 1.0
    return per_iter * iters


def us_per_engine_iteration(cnt, n_rhs=2):
    """Engine time per iteration in microseconds: the n_rhs systems of a
    launch advance together, one INIT iteration per launch, then their CG
    steps and true-residual checks (summed over systems in the counters)."""
    iters = (cnt["cg_steps"] + cnt["ru_steps"]) / float(n_rhs) + cnt["engine_launches"]
    return 1000.0 * cnt["engine_ms"] / iters if iters > 0 else None


def fp64_peak_tflops():
    """FP64 peak of GB300 from unit counts and clocks: 152 SMs x 2 DFMA per
    clock per SM x 2 flops x 2.07 GHz (maximum SM clock) = 1.26 TFLOP/s, the
    nominal 1.25 TFLOP/s of the part."""
    return 152 * 2 * 2 * 2.07e9 / 1e12


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, value):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def _oracle_cg_rate(name, seconds):
    """M^T M applies per second of the oracle's FP64 CG on workload `name`,
    run for about `seconds` (one thread); returns (applies/s, iterations,
    applies, seconds)."""
    import oracle
    wl = {w.name: w for w in WORKLOADS.values()}[name]
    lat = oracle.lattice(wl.d, wl.nx, wl.ntau)
    n = wl.nsites
    sigma = workloads.sigma_field(n, seed=wl.seed)
    L = oracle.links(lat, workloads.A_HS, sigma)
    b = workloads.source(n, seed=wl.seed)
    h = workloads.T_HOP * workloads.DTAU
    t0 = time.perf_counter()
    oracle.cg(lat, h, L, b, 1e-10, 2)
    per_it = max((time.perf_counter() - t0) / 3.0, 1e-6)
    iters = max(3, int(seconds / per_it))
    t0 = time.perf_counter()
    _, st, it, rr = oracle.cg(lat, h, L, b, 1e-10, iters)
    dt = time.perf_counter() - t0
    applies = it + 1  # it CG steps + one final true-residual apply
    return applies / dt, it, applies, dt


def cpu_baseline(wl, seconds=15.0, all_cores=True):
    """The oracle, as it stands, on this host: CG iterations on the same
    lattice and field for about `seconds`, as M^T M applies per second, on
    one thread; with all_cores, also one copy of that run per host core at
    once (spawned processes, the oracle unchanged) and their summed rate."""
    rate, it, applies, dt = _oracle_cg_rate(wl.name, seconds)
    out = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "oracle FP64 CG on the %s lattice (seed %d): %d CG iterations (%d M^T M applies) in %.1f s, single thread"
                     % (wl.name, wl.seed, it, applies, dt)}
    if all_cores:
        import multiprocessing as mp
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        ctx = mp.get_context("spawn")   # the parent has used the GPU: no fork
        with ctx.Pool(cores) as pool:
            res = pool.starmap(_oracle_cg_rate, [(wl.name, seconds)] * cores)
        out["all_cores"] = {"value": float(sum(r[0] for r in res)), "unit": UNIT, "cores": cores,
                            "kind": "oracle",
                            "sample": "%d concurrent copies of the single-thread run, one per host core, rates summed"
                                      % cores}
    return out


def run_reference(args, wl, world, rank):
    """The oracle timed as the reference arm (rank 0 only)."""
    if rank != 0:
        return
    per_step = max(2.0, 40.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_baseline(wl, seconds=min(per_step, 3.0), all_cores=False)
    vals, samples = [], []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = cpu_baseline(wl, seconds=per_step, all_cores=False)
        vals.append(r["value"])
        samples.append(r["sample"])
    wall = time.perf_counter() - t0
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": dict(config_of(args, wl),
                           step="about %.0f s of the oracle's FP64 CG iterations (Q applies) on a Gaussian b, "
                                "same lattice and field" % per_step),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": samples[-1] if samples else ""},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(args, wl):
    return {"workload": wl.name, "d": wl.d, "nx": wl.nx, "ntau": wl.ntau, "sites": wl.nsites,
            "t": workloads.T_HOP, "dtau": workloads.DTAU, "A": workloads.A_HS, "seed": wl.seed,
            "n_md": args.n_md, "dt": args.dt, "n_pf": 2, "cg_tol": 1e-10,
            "precision": args.precision, "step": "one HMC trajectory", "integrator": args.integrator,
            "cg": ("Chebyshev-preconditioned, n=%d eps=%g" % (args.cheb, args.cheb_eps)) if args.cheb else "plain",
            "l2": "flushed between steps (512 MiB write, then 512 MiB read)", "parallelism": "replicas%d" % args.gpus}


class L2Flush:
    """Evicts L2 between timed steps: writes a buffer larger than L2 (129 MB on
    GB300), then reads another one, so that the lines left in L2 are clean and
    the next step does not pay the write-back of the flush."""

    def __init__(self, dev, mbytes=512):
        import torch
        self.w = torch.empty(mbytes * (1 << 20) // 4, dtype=torch.float32, device=dev)
        self.r = torch.ones(mbytes * (1 << 20) // 4, dtype=torch.float32, device=dev)

    def __call__(self, v=1.0):
        self.w.fill_(v)
        self.r.sum()


def measure_solve(wl, precision, rank, dev, stream, steps, warmup, flush, cg_maxit=1000000, cheb=0,
                  cheb_eps=1e-4):
    """CG solves of Q x = b for two right-hand sides b ~ N(0, 1) on workload wl,
    each CUDA-event timed on the context stream with L2 flushed before it, the
    host -> device copy of b before and the device -> host copy of x after the
    timed call (counted in e2e).  Returns the rates, the engine roofline and the
    per-step device and wall times."""
    import torch
    from paper_1007_3432_gb300 import Context
    from paper_1007_3432_gb300.binding import HH_ENOCONV
    n = wl.nsites
    ctx = Context(wl.d, wl.nx, wl.ntau, seed=wl.seed, chain_id=rank, precision=precision,
                  cg_maxit=cg_maxit, stream=stream, cheb_degree=cheb, cheb_eps=cheb_eps)
    ctx.set_field(torch.from_numpy(workloads.sigma_field(n, seed=wl.seed, chain=rank)).to(dev))
    b_h = np.stack([workloads.source(n, seed=wl.seed, chain=rank, rhs=a) for a in range(2)])
    b = torch.from_numpy(b_h).to(dev)
    x = torch.zeros_like(b)
    x_h = torch.empty(b.shape, dtype=torch.float64).pin_memory()
    b_pin = torch.from_numpy(b_h).pin_memory()
    infos = []

    def one():
        flush()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0 = time.perf_counter()
        b.copy_(b_pin, non_blocking=True)      # host -> device input
        e0.record(stream)
        # an iteration cap below convergence (--cg-maxit, as the profiling
        # commands use) returns HH_ENOCONV with the last iterate
        rc, inf = ctx.solve(b, x, 2, info=True, allow=(HH_ENOCONV,))
        e1.record(stream)
        x_h.copy_(x, non_blocking=True)        # device -> host result
        torch.cuda.synchronize(dev)
        infos.append(inf)
        return e0.elapsed_time(e1), (time.perf_counter() - w0) * 1000.0

    for _ in range(warmup):
        one()
    infos.clear()
    ctx.counters_reset(profile_engine=True)
    dev_ms, wall_ms = [], []
    for _ in range(steps):
        a, w = one()
        dev_ms.append(a)
        wall_ms.append(w)
    cnt = ctx.counters()
    ctx.close()
    peaks, src = measured_peaks()
    eng_s = cnt["engine_ms"] / 1000.0
    # With the Chebyshev preconditioner every CG step and true-residual check
    # is followed by 2n sub-steps, each one Q apply with its vector update
    # (counted at the flops of a CG step).
    q_per_step = 2 * cheb + 1
    if precision == "fp64":
        flops = n * (cnt["cg_steps"] * flops_per_site(wl.d, "cg", "fp64") + cnt["ru_steps"] * flops_per_site(wl.d, "ru", "fp64"))
        flops += n * (cnt["cg_steps"] + cnt["ru_steps"]) * (q_per_step - 1) * flops_per_site(wl.d, "cg", "fp64")
        ach = flops / eng_s / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": fp64_peak_tflops(), "unit": "TFLOP/s",
                "frac": ach / fp64_peak_tflops(), "traffic": engine_traffic(wl, precision, cheb, cnt),
                "kernel": "engine_kernel (FP64 CG)",
                "peak_source": "FP64 from unit counts and clocks (152 SMs x 2 DFMA/clk x 2.07 GHz)"}
    else:
        byts = n * (cnt["cg_steps"] * bytes_per_site("cg", precision)
                    + cnt["ru_steps"] * bytes_per_site("ru", precision))
        ach = byts / eng_s / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": engine_traffic(wl, precision, cheb, cnt),
                "kernel": "engine_kernel (FP32-inner CG)",
                "peak_source": "%s MEASURED_PEAKS.json hbm_gbs" % src,
                "algorithmic_bytes_per_site_cg_step": bytes_per_site("cg", precision)}
    t_dev = sum(dev_ms) / 1000.0
    t_wall = sum(wall_ms) / 1000.0
    return {"workload": wl.name, "precision": precision, "solves": cnt["solves"],
            "solves_per_s": cnt["solves"] / t_dev, "e2e_solves_per_s": cnt["solves"] / t_wall,
            "ms_per_step": 1000.0 * t_dev / steps, "dev_s": t_dev, "wall_s": t_wall,
            "cg_steps_per_solve": cnt["cg_steps"] / max(1, cnt["solves"]),
            "q_applies_per_solve": (cnt["cg_steps"] + cnt["ru_steps"]) * q_per_step / max(1, cnt["solves"]),
            "ru_steps": cnt["ru_steps"], "fp64_steps": cnt["fp64_steps"], "cheb_degree": cheb,
            "max_true_relres": max(i["true_relres"] for i in infos), "all_converged": all(i["converged"] for i in infos),
            "gpu_launches": int(cnt["kernel_launches"]), "roofline": roof,
            "e2e_bytes": (n * 16, n * 16)}


def measure_apply(wl, precision, nvec, rank, dev, stream, steps, warmup, flush):
    """One M^T M apply of nvec vectors per step (hh_apply for one vector,
    hh_apply_multi for more), CUDA-event timed with L2 flushed before it."""
    import torch
    from paper_1007_3432_gb300 import HH_OP_MTM, Context
    n = wl.nsites
    ctx = Context(wl.d, wl.nx, wl.ntau, seed=wl.seed, chain_id=rank, precision=precision, stream=stream)
    ctx.set_field(torch.from_numpy(workloads.sigma_field(n, seed=wl.seed, chain=rank)).to(dev))
    dt = torch.float64 if precision == "fp64" else torch.float32
    xs = torch.from_numpy(np.concatenate([workloads.source(n, seed=wl.seed, chain=rank, rhs=a)
                                          for a in range(nvec)])).to(dev).to(dt)
    ys = torch.empty_like(xs)

    def one():
        flush()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if nvec == 1:
            ctx.apply(HH_OP_MTM, xs, ys)
        else:
            ctx.apply_multi(HH_OP_MTM, xs, ys, nvec)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1)

    for _ in range(warmup):
        one()
    ctx.counters_reset()
    dev_ms = [one() for _ in range(steps)]
    cnt = ctx.counters()     # raises if a bounded device-side wait ran out
    ctx.close()
    peaks, src = measured_peaks()
    # x_v and y_v once per vector, the links once per launch (multi-vector
    # kernel, FP32 d = 3); separate applies read the links per vector.
    multi = nvec > 1 and precision != "fp64" and wl.d == 3
    bps = 24 * nvec if precision == "fp64" else (8 * nvec + 4 if multi else 12 * nvec)
    t_dev = sum(dev_ms) / 1000.0
    ach = steps * n * bps / t_dev / 1e9
    traffic = APPLY_DRAM_PER_LAUNCH.get((wl.name, "fp64" if precision == "fp64" else "fp32", nvec))
    roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": ach / peaks["hbm_gbs"], "traffic": traffic,
            "kernel": ("multi-vector Q apply (FP32, %d vectors per launch; k_mtm_multi_rp_d3 for N_x = 32)" % nvec)
                      if multi else
                      "M^T M apply (%s, %d vector%s)" % ("FP64" if precision == "fp64" else "FP32", nvec,
                                                        "s" if nvec > 1 else ""),
            "peak_source": "%s MEASURED_PEAKS.json hbm_gbs" % src,
            "algorithmic_bytes_per_launch_site": bps}
    return {"workload": wl.name, "precision": "fp64" if precision == "fp64" else "fp32", "vectors_per_launch": nvec,
            "applies_per_s": steps * nvec / t_dev, "median_launch_us": 1000.0 * float(np.median(dev_ms)),
            "dev_s": t_dev, "gpu_launches": int(cnt["kernel_launches"]), "roofline": roof,
            "l2": "flushed before every launch (512 MiB write, then 512 MiB read)"}


def run_part(args, wl, world, rank, local, dev, stream):
    """--mode solve / --mode apply: one CG solve (2 right-hand sides) or one
    M^T M apply of --nvec vectors per step, each bracketed by CUDA events on the
    context stream, L2 flushed before every step."""
    flush = L2Flush(dev)
    clocks = ClockSampler(local)
    if args.mode == "solve":
        clocks.start()
        r = measure_solve(wl, args.precision, rank, dev, stream, args.steps, args.warmup, flush, args.cg_maxit,
                          args.cheb, args.cheb_eps)
        clk = clocks.stop()
        t_dev = max_over_ranks(world, r["dev_s"])
        t_wall = max_over_ranks(world, r["wall_s"])
        units = sum_over_ranks(world, float(r["solves"]))
        unit = "CG solves/s"
        extra = {k: r[k] for k in ("cg_steps_per_solve", "q_applies_per_solve", "ru_steps", "fp64_steps",
                                   "cheb_degree", "max_true_relres", "all_converged")}
        e2e_bytes = r["e2e_bytes"]
        e2e = {"value": units / t_wall, "unit": unit, "h2d_bytes_per_step": e2e_bytes[0],
               "d2h_bytes_per_step": e2e_bytes[1]}
    else:
        clocks.start()
        r = measure_apply(wl, args.precision, args.nvec, rank, dev, stream, args.steps, args.warmup, flush)
        clk = clocks.stop()
        t_dev = max_over_ranks(world, r["dev_s"])
        units = float(world * args.steps * args.nvec)
        unit = "MTM applies/s"
        extra = {"median_apply_us": r["median_launch_us"], "vectors_per_launch": args.nvec}
        # inputs resident on the device: no host copies in this mode
        e2e = {"value": units / t_dev, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    line = {"metric": METRIC, "value": units / t_dev, "unit": unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t_dev / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else ("f32" if args.mode == "apply" else "f32+f64"),
            "data": "synthetic", "config": dict(config_of(args, wl), mode=args.mode,
                                                step=("one CG solve, 2 right-hand sides" if args.mode == "solve"
                                                      else "one M^T M apply of %d vector(s)" % args.nvec),
                                                **({"cheb_degree": args.cheb, "cheb_eps": args.cheb_eps}
                                                   if args.cheb else {})),
            "e2e": e2e, "gpu_launches": r["gpu_launches"], "clocks": clk, "roofline": r["roofline"]}
    line.update(extra)
    if rank == 0:
        print(json.dumps(line), flush=True)


def _batch_requests(B, chains, precision, rank, keep):
    from paper_1007_3432_gb300.binding import HH_REQ_SOLVE
    reqs = []
    for c in chains:
        n = c.nsites
        sigma = workloads.sigma_field(n, seed=workloads.BATCH_SEED, chain=c.chain + 1000 * rank)
        b = np.stack([workloads.source(n, seed=workloads.BATCH_SEED, chain=c.chain, rhs=a) for a in range(2)])
        keep.append((sigma, b))
        reqs.append(B.make_request(HH_REQ_SOLVE, 3, c.nx, c.ntau, sigma=sigma, b=b, out=None,
                                   precision=precision, n_pf=2))
    return reqs


def measure_batch(precision, rank, dev, stream, steps, warmup, budget_gb, autotune_rounds=6):
    """64 independent d=3 chains of uneven volume; one step solves both
    right-hand sides of every chain in the batched engine.  The engine
    configuration comes from the library's autotuner on this request mix."""
    import torch
    from paper_1007_3432_gb300 import binding as B
    chains = workloads.batch_chains(64)
    sites = sum(c.nsites for c in chains)
    keep = []
    reqs = _batch_requests(B, chains, precision, rank, keep)
    budget = int(min(budget_gb, 120.0) * (1 << 30))
    t0 = time.perf_counter()
    tuned = B.autotune(reqs, hbm_budget_bytes=budget, rounds=autotune_rounds,
                       cache_path=os.path.join(ROOT, "paper_1007_3432_gb300", "lib", "autotune.jsonl"),
                       stream=stream)
    tune_s = time.perf_counter() - t0
    batch = B.Batch(max_slots=64, hbm_budget_bytes=budget, chunk_iters=tuned["chunk_iters"],
                    tile_sites=tuned["tile_sites"], max_active_sites=tuned["max_active_sites"], stream=stream)

    def one():
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for r in reqs:
            batch.submit(r)
        res = batch.run_until_idle()
        torch.cuda.synchronize(dev)
        return time.perf_counter() - t0, res

    for _ in range(warmup):
        one()
    times, allres = [], []
    for _ in range(steps):
        t, res = one()
        times.append(t)
        allres += res
    batch.close()
    solves = float(sum(r["n_solves"] for r in allres))
    its = sum(r["cg_iterations"] for r in allres)
    bad = sum(1 for r in allres if r["status"] != 0 or r["max_true_relres"] > 1e-10)
    peaks, src = measured_peaks()
    per_site = bytes_per_site("cg", precision)
    size_of = {j: c.nsites for j, c in enumerate(chains)}
    site_its = sum(r["cg_iterations"] * size_of[(r["ticket"] - 1) % len(chains)] for r in allres)
    ach = site_its * per_site / sum(times) / 1e9
    if precision == "fp64":
        flops = sum(r["cg_iterations"] * size_of[(r["ticket"] - 1) % len(chains)] for r in allres) \
            * flops_per_site(3, "cg", "fp64")
        fl = flops / sum(times) / 1e12
        roof = {"bound": "alu", "achieved": fl, "peak": fp64_peak_tflops(), "unit": "TFLOP/s",
                "frac": fl / fp64_peak_tflops(), "traffic": None, "kernel": "engine_kernel (batched, fp64)",
                "note": "algorithmic CG flops over the whole step wall time"}
    else:
        roof = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": None,
                "kernel": "engine_kernel (batched, %s)" % precision,
                "note": "algorithmic CG bytes (11 words per site and step) over the whole step wall time"}
    return {"workload": "batch64_d3", "precision": precision, "chains": len(chains), "sites_total": sites,
            "solves": solves, "solves_per_s": solves / sum(times), "s_per_step": sum(times) / steps,
            "wall_s": sum(times), "autotuned": tuned, "autotune_s": tune_s,
            "cg_iterations_per_solve": its / max(1, solves), "failed_solves": bad, "roofline": roof,
            "h2d_bytes_per_step": int(sum(3 * 8 * c.nsites for c in chains))}


def run_batch(args, world, rank, local, dev, stream):
    """--mode batch: the 64-chain batch in the precision of --precision."""
    clocks = ClockSampler(local)
    clocks.start()
    r = measure_batch(args.precision, rank, dev, stream, args.steps, args.warmup, args.budget_gb)
    clk = clocks.stop()
    t_tot = max_over_ranks(world, r["wall_s"])
    solves = sum_over_ranks(world, r["solves"])
    line = {"metric": METRIC, "value": solves / t_tot, "unit": "CG solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": "batch64_d3", "chains": r["chains"], "sites_total": r["sites_total"],
                       "nx_choices": list(workloads.BATCH_NX), "ntau_choices": list(workloads.BATCH_NTAU),
                       "seed": workloads.BATCH_SEED, "precision": args.precision, "n_rhs": 2,
                       "autotuned": r["autotuned"], "mode": "batch", "parallelism": "replicas%d" % world},
            "cg_iterations_per_solve": r["cg_iterations_per_solve"], "failed_solves": r["failed_solves"],
            "e2e": {"value": solves / t_tot, "unit": "CG solves/s",
                    "h2d_bytes_per_step": r["h2d_bytes_per_step"], "d2h_bytes_per_step": 0},
            "gpu_launches": None, "clocks": clk, "roofline": r["roofline"]}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_slab(args, wl, world, rank, local, dev, stream):
    """--mode slab: the time-slab decomposition of one lattice over the ranks
    (hh_slab_*), FP64 CG on one right-hand side, capped at --cg-maxit
    iterations (default 2000 here), with both forms of the torch.distributed
    callbacks: host (halos and sums staged through host memory, gloo) and,
    with one rank or NCCL, device (enqueued on the slab's stream).  Reports
    the wall time per CG iteration of each, max over ranks, beside the
    context solver's on the same lattice (rank 0, one GPU)."""
    import torch
    from paper_1007_3432_gb300 import Context
    from paper_1007_3432_gb300.binding import HH_ENOCONV, Slab, TorchDistComm
    group = None
    if world > 1:
        import torch.distributed as dist
        group = dist.new_group(backend="gloo")
    maxit = args.cg_maxit if args.cg_maxit < 1000000 else 2000
    V, n = wl.nx ** wl.d, wl.nsites
    t0, t1 = rank * wl.ntau // world, (rank + 1) * wl.ntau // world
    sigma = workloads.sigma_field(n, seed=wl.seed)
    b = workloads.source(n, seed=wl.seed, rhs=0)
    sig_d = torch.from_numpy(sigma[t0 * V:t1 * V].copy()).to(dev)
    b_d = torch.from_numpy(b[t0 * V:t1 * V].copy()).to(dev)
    x_d = torch.zeros_like(b_d)
    forms = {}
    side = torch.cuda.Stream(dev)   # a stream of its own (the device form replays its iterations as a graph)
    for form in ("host", "device"):
        comm = TorchDistComm(group)
        if form == "device" and not comm.device_capable():
            continue
        per_it = []
        with Slab(wl.d, wl.nx, wl.ntau, t0, t1, comm=comm, stream=side, cg_maxit=maxit,
                  device_comm=form == "device") as sl:
            sl.set_field(sig_d)
            for k in range(args.warmup + args.steps):
                barrier(world)
                torch.cuda.synchronize(dev)
                w0 = time.perf_counter()
                rc, info = sl.solve(b_d, x_d, allow=(HH_ENOCONV,))
                torch.cuda.synchronize(dev)
                w = time.perf_counter() - w0
                if k >= args.warmup:
                    per_it.append(w / max(1, info["iterations"]))
        forms[form] = {"us_per_iteration": 1e6 * max_over_ranks(world, statistics.median(per_it)),
                       "iterations": info["iterations"]}
    us_slab = min(f["us_per_iteration"] for f in forms.values())
    us_ctx = None
    if rank == 0:
        with Context(wl.d, wl.nx, wl.ntau, cg_maxit=maxit, stream=stream) as ctx:
            ctx.set_field(torch.from_numpy(sigma).to(dev))
            bb = torch.from_numpy(b).to(dev).reshape(1, -1)
            xx = torch.zeros_like(bb)
            ctx.solve(bb, xx, 1, allow=(HH_ENOCONV,))
            torch.cuda.synchronize(dev)
            w0 = time.perf_counter()
            rc, cinfo = ctx.solve(bb, xx, 1, allow=(HH_ENOCONV,))
            torch.cuda.synchronize(dev)
            us_ctx = 1e6 * (time.perf_counter() - w0) / max(1, cinfo["iterations"])
    line = {"metric": METRIC, "value": us_slab, "unit": "us per CG iteration (wall)", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": us_slab * maxit / 1000.0,
            "higher_is_better": False, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": dict(config_of(args, wl), mode="slab", step="FP64 CG, one right-hand side, %d iterations" % maxit,
                           parallelism="tau-slabs%d" % world,
                           halo="one slice per exchange; host form: staged through pinned host memory, "
                                "gloo between ranks; device form: enqueued on the slab's stream"),
            "context_solver_us_per_iteration": us_ctx, "callback_forms": forms,
            "e2e": None, "gpu_launches": None}
    if rank == 0:
        print(json.dumps(line), flush=True)


def default_extras(rank, dev, stream, budget_gb):
    """The spec comparisons, measured in the same run as the headline
    trajectory line: the C2 FP32 M^T M apply (16 vectors per launch, and one),
    C2 solves in FP64 and in mixed precision, and the 64-chain batch in FP64
    and mixed precision, each with its roofline."""
    flush = L2Flush(dev)
    c2 = workloads.C2
    out = {}
    out["c2_apply_fp32_16vec"] = measure_apply(c2, "mixed", 16, rank, dev, stream, 20, 3, flush)
    out["c2_apply_fp32_1vec"] = measure_apply(c2, "mixed", 1, rank, dev, stream, 20, 3, flush)
    sol = {p: measure_solve(c2, p, rank, dev, stream, 2, 1, flush) for p in ("fp64", "mixed")}
    for r in sol.values():
        r.pop("e2e_bytes", None)
    out["c2_solves"] = dict(sol, mixed_over_fp64=sol["mixed"]["solves_per_s"] / sol["fp64"]["solves_per_s"])
    del flush
    bat = {p: measure_batch(p, rank, dev, stream, 1, 1, budget_gb, autotune_rounds=4) for p in ("fp64", "mixed")}
    out["batch64_d3"] = dict(bat, mixed_over_fp64=bat["mixed"]["solves_per_s"] / bat["fp64"]["solves_per_s"])
    return out


def solver_for(r, arm="mixed"):
    """Solver of a served request.  Arm "mixed": d = 1 lattices with N_tau >=
    256 (beta >= 12.8) use FP64 CG with the Chebyshev preconditioner of Sec.
    4.2 (n = 8, eps = 1e-4): on some of them plain CG, FP64 or mixed, stalls
    near a relative residual of 1e-7 (1255 x 504, seed 101103049: 400k FP64 CG
    steps reach 1.4e-7; the preconditioned solve converges in 4.2k steps); the
    others use mixed precision.  Arm "fp64": the same with FP64 CG in place of
    mixed precision."""
    if r.d == 1 and r.ntau >= 256:
        return {"precision": "fp64", "cheb_degree": 8, "cheb_eps": 1e-4}
    return {"precision": "mixed" if arm == "mixed" else "fp64"}


def _percentiles(vals):
    if not vals:
        return {"p50": None, "p99": None, "max": None}
    a = np.array(vals)
    return {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99)), "max": float(a.max())}


def serve_one(args, rate, arm, rank, dev, stream, n_req, cap_s, n_check):
    """One Poisson stream of n_req requests at `rate` served by the continuous-
    batching worker, for at most cap_s seconds of wall time (arrivals and
    service); latencies of the completed requests split into queueing (submit
    -> admitted into a slot) and service (admitted -> result).  The first
    n_check solve requests keep their solutions, and are then solved alone in
    a fresh batch: the results must be bitwise the same."""
    import torch
    from paper_1007_3432_gb300 import binding as B
    from paper_1007_3432_gb300.binding import HH_REQ_SOLVE, HH_REQ_TRAJECTORY
    budget = int(args.budget_gb * (1 << 30))
    reqs = workloads.poisson_requests(rate, n_req, seed=workloads.SERVE_SEED + 17 * rank)

    def make(r, out=None):
        sigma = workloads.sigma_field(r.nsites, seed=r.seed)
        prm = solver_for(r, arm)
        if r.kind == "solve":
            return B.make_request(HH_REQ_SOLVE, r.d, r.nx, r.ntau, sigma=sigma, seed=r.seed, n_pf=2,
                                  traj_index=r.rid, out=out, **prm), sigma
        return B.make_request(HH_REQ_TRAJECTORY, r.d, r.nx, r.ntau, sigma=sigma, seed=r.seed, n_pf=2,
                              n_md=args.serve_n_md, dt=args.serve_dt, traj_index=r.rid, **prm), sigma

    checks = {}
    batch = B.Batch(max_slots=64, hbm_budget_bytes=budget, chunk_iters=32, tile_sites=4096, stream=stream)
    batch.start()
    keep, got, tickets = [], [], {}
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    submitted = 0
    for r in reqs:
        while time.perf_counter() - t0 < r.arrival_s:
            time.sleep(0.0002)
        if time.perf_counter() - t0 > cap_s:
            break
        out = None
        if r.kind == "solve" and len(checks) < n_check:
            out = np.zeros((2, r.nsites))
        req, sigma = make(r, out)
        keep.append((sigma, out))
        _, t = batch.submit(req)
        tickets[t] = r
        if out is not None:
            checks[t] = (r, out)
        submitted += 1
        got += batch.poll()
    while len(got) < submitted and time.perf_counter() - t0 < cap_s:
        got += batch.poll()
        time.sleep(0.001)
    wall = time.perf_counter() - t0
    batch.stop()
    got += batch.poll()
    batch.close()
    done = [g for g in got]
    ok = [g for g in done if g["status"] == 0]
    lat = [g["latency_ms"] for g in ok]
    que = [g["queue_ms"] for g in ok]
    svc = [g["latency_ms"] - g["queue_ms"] for g in ok]
    # alone-vs-mix: the sampled solves, each alone in a fresh batch
    same, compared = True, 0
    done_tickets = {g["ticket"] for g in ok}
    for t, (r, out) in checks.items():
        if t not in done_tickets:
            continue
        ref = np.zeros_like(out)
        with B.Batch(max_slots=4, hbm_budget_bytes=budget, chunk_iters=32, tile_sites=4096, stream=stream) as solo:
            req, sigma = make(r, ref)
            solo.submit(req, keep=(sigma, ref))
            solo.run_until_idle()
        same = same and bool(np.array_equal(out, ref))
        compared += 1
    return {"rate_hz": rate, "arm": arm, "requests_offered": n_req, "submitted": submitted,
            "completed": len(done), "failed": sum(1 for g in done if g["status"] != 0),
            "unfinished_at_cap": submitted - len(done), "wall_s": wall, "cap_s": cap_s,
            "solves_per_s": sum(g["n_solves"] for g in ok) / wall, "requests_per_s": len(ok) / wall,
            "latency_ms": _percentiles(lat), "queue_ms": _percentiles(que), "service_ms": _percentiles(svc),
            "alone_vs_mix": {"compared": compared, "bitwise_equal": same if compared else None},
            "failed_detail": [[tickets[g["ticket"]].rid, tickets[g["ticket"]].kind, tickets[g["ticket"]].d,
                               tickets[g["ticket"]].nx, tickets[g["ticket"]].ntau, g["status"], g["cg_iterations"],
                               g["dH"]] for g in done if g["status"] != 0],
            "status_counts": {str(k): int(v) for k, v in zip(*np.unique([g["status"] for g in done],
                                                                       return_counts=True))} if done else {}}


def run_serve(args, world, rank, local, dev, stream):
    """Poisson arrivals of solve and trajectory requests, served by the
    continuous-batching worker; per rate and arm: solves/s, end-to-end,
    queueing and service latency percentiles, completion within the cap, and
    the alone-vs-mix check."""
    per = []
    clocks = ClockSampler(local)
    clocks.start()
    for arm in args.serve_arms.split(","):
        rates = [float(x) for x in (args.rates if arm == "mixed" else args.fp64_rates).split(",")]
        for rate in rates:
            below = rate < 1.0
            n_req = (args.requests_low if arm == "mixed" else args.fp64_requests_low) if below else args.requests
            # below capacity: long enough for every arrival plus a minute of service
            cap = n_req / rate + 60.0 if below else args.serve_cap_s
            r = serve_one(args, rate, arm, rank, dev, stream, n_req, cap, args.serve_checks)
            per.append(r)
            if rank == 0:
                print("# serve %s %.2f/s: %d/%d done, %.2f solves/s, p50 %.0f ms, p99 %.0f ms"
                      % (arm, rate, r["completed"], r["submitted"], r["solves_per_s"],
                         r["latency_ms"]["p50"] or -1, r["latency_ms"]["p99"] or -1), file=sys.stderr, flush=True)
    clk = clocks.stop()
    mixed = [r for r in per if r["arm"] == "mixed"]
    best = max(mixed or per, key=lambda d: d["solves_per_s"])
    line = {"metric": METRIC, "value": best["solves_per_s"], "unit": "CG solves/s", "n_gpus": world,
            "steps": len(per), "warmup": 0, "ms_per_step": 1000.0 * sum(d["wall_s"] for d in per) / len(per),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": "serve_poisson", "seed": workloads.SERVE_SEED,
                       "requests_per_rate": args.requests, "requests_below_capacity": args.requests_low,
                       "requests_below_capacity_fp64": args.fp64_requests_low,
                       "cap_s_per_rate": args.serve_cap_s,
                       "d1": {"nx": [64, 2048], "ntau": [64, 512]}, "d3": {"nx": [8, 24], "ntau": [40, 256]},
                       "trajectory_n_md": args.serve_n_md, "trajectory_dt": args.serve_dt,
                       "hbm_budget_gb": args.budget_gb,
                       "arms": {"mixed": "mixed; FP64 + Chebyshev n=8 eps=1e-4 for d=1 with N_tau >= 256",
                                "fp64": "FP64; FP64 + Chebyshev n=8 eps=1e-4 for d=1 with N_tau >= 256"},
                       "mode": "serve", "parallelism": "replicas%d" % world},
            "per_rate": per, "clocks": clk, "e2e": None, "gpu_launches": None}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c1", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "mixed-bf16link", "mixed-fix16link"],
                    help="mixed-*16link: 16-bit links in the FP32 steps (solve and trajectory modes)")
    ap.add_argument("--n-md", type=int, default=None)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--mode", default="trajectory", choices=["trajectory", "solve", "apply", "batch", "serve", "slab"])
    ap.add_argument("--cg-maxit", type=int, default=1000000)
    ap.add_argument("--cheb", type=int, default=0, help="Chebyshev preconditioner degree n (FP64; solve and trajectory)")
    ap.add_argument("--integrator", default="leapfrog", choices=["leapfrog", "omelyan"])
    ap.add_argument("--cheb-eps", type=float, default=1e-4)
    ap.add_argument("--rates", default="0.25,10,30,100,300,1000",
                    help="serve: arrival rates (req/s) of the mixed arm; rates below 1 are below capacity")
    ap.add_argument("--fp64-rates", default="10,1000", help="serve: arrival rates of the FP64 arm")
    ap.add_argument("--serve-arms", default="mixed,fp64")
    ap.add_argument("--requests", type=int, default=200, help="serve: requests per rate")
    ap.add_argument("--requests-low", type=int, default=30, help="serve: requests at rates below 1/s (mixed arm)")
    ap.add_argument("--fp64-requests-low", type=int, default=30, help="serve: requests at rates below 1/s (FP64 arm)")
    ap.add_argument("--serve-cap-s", type=float, default=100.0, help="serve: wall-time cap per rate")
    ap.add_argument("--serve-checks", type=int, default=2, help="serve: alone-vs-mix checks per rate")
    ap.add_argument("--serve-n-md", type=int, default=4)
    ap.add_argument("--serve-dt", type=float, default=0.002)
    ap.add_argument("--dt", type=float, default=None, help="MD step (default: the workload's)")
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--nvec", type=int, default=1, help="--mode apply: vectors per launch (hh_apply_multi)")
    ap.add_argument("--no-extras", action="store_true",
                    help="trajectory mode: skip the C2 apply, C2 solve and batch comparisons after the timed region")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    if args.n_md is None:
        args.n_md = wl.n_md
    if args.dt is None:
        args.dt = wl.dt if wl.dt > 0 else 1.0 / args.n_md
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, wl, world, rank)
        return

    import torch
    from __graft_entry__ import build
    from paper_1007_3432_gb300 import Context

    if rank == 0:
        build()
    barrier(world)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    if args.mode == "batch":
        return run_batch(args, world, rank, local, dev, stream)
    if args.mode == "serve":
        return run_serve(args, world, rank, local, dev, stream)
    if args.mode == "slab":
        return run_slab(args, wl, world, rank, local, dev, stream)
    if args.mode != "trajectory":
        return run_part(args, wl, world, rank, local, dev, stream)
    n = wl.nsites
    sigma_h = workloads.sigma_field(n, seed=wl.seed, chain=rank)
    ctx = Context(wl.d, wl.nx, wl.ntau, seed=wl.seed, n_pf=2, chain_id=rank, precision=args.precision,
                  cg_maxit=args.cg_maxit, stream=stream, integrator=args.integrator,
                  cheb_degree=args.cheb, cheb_eps=args.cheb_eps)
    flush = L2Flush(dev)
    dt = args.dt

    def step(traj, timed):
        flush(float(traj))
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e2 = torch.cuda.Event(enable_timing=True)
        w0 = time.perf_counter()
        e0.record(stream)
        ctx.set_field(sigma_h)              # host -> device (the step's input)
        e1.record(stream)
        info = ctx.trajectory(args.n_md, dt, traj)
        e2.record(stream)
        ctx.get_field(sigma_h)              # device -> host (the step's output)
        w1 = time.perf_counter()
        torch.cuda.synchronize(dev)
        return e1.elapsed_time(e2), (w1 - w0) * 1000.0, info

    for w in range(args.warmup):
        step(w, False)
    barrier(world)
    torch.cuda.synchronize(dev)
    ctx.counters_reset(profile_engine=True)
    clocks = ClockSampler(local)
    clocks.start()
    dev_ms, wall_ms, infos = [], [], []
    for k in range(args.steps):
        a, b, inf = step(args.warmup + k, True)
        dev_ms.append(a)
        wall_ms.append(b)
        infos.append(inf)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    barrier(world)
    cnt = ctx.counters()

    # Every CG step and true-residual check applies Q once per right-hand
    # side; with the Chebyshev preconditioner each is followed by 2n more.
    q_per_step = 2 * args.cheb + 1
    applies = (cnt["cg_steps"] + cnt["ru_steps"]) * q_per_step
    t_dev = max_over_ranks(world, sum(dev_ms) / 1000.0)
    t_wall = max_over_ranks(world, sum(wall_ms) / 1000.0)
    tot_applies = sum_over_ranks(world, float(applies))
    tot_solves = sum_over_ranks(world, float(cnt["solves"]))
    value = tot_applies / t_dev
    e2e = tot_applies / t_wall

    # Roofline of the dominant kernel: the persistent CG engine.
    f_cg = flops_per_site(wl.d, "cg", args.precision)
    f_ru = flops_per_site(wl.d, "ru", args.precision)
    peaks, src = measured_peaks()
    eng_s = cnt["engine_ms"] / 1000.0
    per_launch = eng_s / max(1, cnt["engine_launches"])
    if args.precision == "fp64":
        flops = n * (cnt["cg_steps"] * f_cg + cnt["ru_steps"] * f_ru)
        # preconditioner sub-steps: one Q apply with its vector update each,
        # counted at the flops of a CG step
        flops += n * (cnt["cg_steps"] + cnt["ru_steps"]) * (q_per_step - 1) * f_cg
        achieved = flops / eng_s / 1e12 if eng_s > 0 else 0.0
        peak = fp64_peak_tflops()
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": engine_traffic(wl, args.precision, args.cheb, cnt),
                "kernel": "engine_kernel (persistent FP64 CG)",
                "peak_source": "FP64 from unit counts and clocks (152 SMs x 2 DFMA/clk x 2.07 GHz)",
                "launch_ms": per_launch * 1000.0}
    else:
        byts = n * (cnt["cg_steps"] * bytes_per_site("cg", args.precision)
                    + cnt["ru_steps"] * bytes_per_site("ru", args.precision))
        achieved = byts / eng_s / 1e9 if eng_s > 0 else 0.0
        peak = peaks["hbm_gbs"]
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": "engine_kernel (persistent FP32-inner CG)",
                "peak_source": "%s MEASURED_PEAKS.json hbm_gbs" % src, "launch_ms": per_launch * 1000.0}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic", "config": config_of(args, wl),
        "solves_per_s": tot_solves / t_dev, "trajectories_per_s": world * args.steps / t_dev,
        "cg_steps_per_solve": cnt["cg_steps"] / max(1, cnt["solves"]),
        "q_applies_per_solve": applies / max(1, cnt["solves"]),
        "acceptance": float(np.mean([i["accepted"] for i in infos])),
        "dH": [i["dH"] for i in infos],
        "exp_minus_dH_mean": float(np.mean([np.exp(-i["dH"]) for i in infos])),
        "max_true_relres": max(i["max_true_relres"] for i in infos),
        "us_per_cg_iteration": us_per_engine_iteration(cnt),
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8},
        "gpu_launches": int(cnt["kernel_launches"]),
        "clocks": clk, "roofline": roof,
    }
    ctx.close()
    if not args.no_extras:
        # After the timed region: the spec comparisons on this GPU.
        extras = default_extras(rank, dev, stream, args.budget_gb)
        line.update(extras)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
    elif rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = None
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
