"""Benchmark of the GB300 ASDSM solver: unknowns/s to a 1e-10 relative residual.

Workload (the 2D random-coefficient configuration): unit square, uniform
4097 x 4097 grid, alpha_i log-uniform in [1e-2, 1], beta_i uniform in
[-10, 10], s a seeded sum of 16 random sine modes, zero Dirichlet data;
mc = 256 coarse intervals (hole size 16); FP32 submesh solves, merge and
fill, exact (64-bit fixed-point / FP32-pair) residual and accumulation;
GCR(8) refinement; tol 1e-10.

A step is one complete solve (Algorithm 1 + Algorithm 4 sweeps until the
relative residual reaches 1e-10) of that problem with s and u resident in HBM.
    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Prints one JSON line (rank 0).  Under torchrun each rank solves its own
instance (seed = rank; weak scaling, no collective on the data path).

The CPU legs time the FP64 oracle as it stands: complete solves to 1e-10 of
the 1025 x 1025 instance of the same workload (seed 0, mc 64), one per
worker process, on one core and on every host core (cpu_baseline), and on
every host core per step for --impl reference.  The final iterate of the
GPU solves is judged by the FP64 residual (rel_res_fp64).
"""
import os

# The CPU legs (oracle) run single-threaded so their core count is exact.
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import platform
import signal
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "unknowns/s to 1e-10 rel. residual"
UNIT = "unknowns/s"
N_GRID = 4097
MC = 256
TOL = 1e-10
ACCEL_M = 8
ACCEL_M_BATCH = 16
STAG_WINDOW_BATCH = 30
MAX_SWEEPS = 1000
FP32_LANES_PER_SM = 128


def workload_config(N=N_GRID, mc=MC, seed=0):
    return {"workload": f"2D advection-diffusion, random coefficients + random-Fourier source, {N}x{N} grid",
            "grid": N, "unknowns": (N - 2) ** 2, "mc": mc, "hole": (N - 1) // mc, "tol": TOL,
            "accel_m": ACCEL_M, "seed": seed, "precision": "FP32 solves/merge/fill, exact residual + int64 accumulation",
            "l2": "inputs larger than L2 (s and u are 134 MB each; L2 is 129 MB), no flush",
            "data": "synthetic"}


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            pk = json.load(f)
        return pk, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        top = max(sm)
        loaded = [v for v in sm if v >= 0.5 * top] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle, timed as it stands on the host cores
# ---------------------------------------------------------------------------
ORACLE_N = 1025          # the sample instance: same workload family, sized for ~10 s of CPU per solve
ORACLE_MC = 64


def _oracle_solve(job):
    """One complete oracle solve (setup, Algorithm 1, sweeps to TOL) of the
    random-Fourier instance (N, mc, seed).  Runs in a spawned worker."""
    N, mc, seed = job
    from oracle import asdsm2d as orc
    from paper_2303_01163_gb300 import workloads as wl
    p = wl.random_fourier_2d(N, seed)
    t0 = time.perf_counter()
    _, info, _, _ = orc.solve_problem(N, mc, p.alpha, p.beta, p.s, p.g, tol=TOL, max_sweeps=MAX_SWEEPS,
                                      accel_m=ACCEL_M)
    return time.perf_counter() - t0, info["sweeps"], float(info["hist"][-1]), info["status"]


class OracleBaseline:
    """The oracle timed on `procs` host cores: a pool of spawned worker
    processes, each limited to one BLAS thread, each solving the instance of
    the workload family completely; throughput = unknowns solved / wall time.
    Spawned (not forked) so that it is safe after CUDA has been initialised."""

    def __init__(self, procs, N=ORACLE_N, mc=ORACLE_MC):
        import multiprocessing as mp
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"            # inherited by the spawned workers
        self.procs, self.N, self.mc = procs, N, mc
        self.pool = mp.get_context("spawn").Pool(procs)

    def run(self, seed=0):
        jobs = [(self.N, self.mc, seed)] * self.procs
        t0 = time.perf_counter()
        out = self.pool.map(_oracle_solve, jobs, chunksize=1)
        wall = time.perf_counter() - t0
        unknowns = self.procs * (self.N - 2) ** 2
        return {"value": unknowns / wall, "unit": UNIT, "cores": self.procs, "kind": "oracle",
                "seconds": wall, "sweeps": [o[1] for o in out], "rel_res": max(o[2] for o in out),
                "converged": all(o[3] == "converged" for o in out),
                "sample": (f"FP64 oracle (scipy splu + CubicSpline), {self.procs} worker process(es) x 1 thread, "
                           f"each one complete solve to {TOL:g} (GCR({ACCEL_M})) of a {self.N}x{self.N} instance "
                           f"of the same workload family (mc {self.mc}, seed {seed}, the GPU arm's instance at this size); "
                           f"measured, not extrapolated")}

    def close(self):
        self.pool.close()
        self.pool.join()


def host_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def host_cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline_line():
    """cpu_baseline of the GPU arm: the oracle on one core and on every host core."""
    cores = host_cores()
    one = OracleBaseline(1)
    r1 = one.run()
    one.close()
    allc = OracleBaseline(cores)
    ra = allc.run()
    allc.close()
    ra["single_thread"] = {"value": r1["value"], "seconds": r1["seconds"], "sweeps": r1["sweeps"]}
    ra["host"] = {"nproc": cores, "cpu": host_cpu_model(), "machine": platform.machine()}
    return ra


# ---------------------------------------------------------------------------
# Multi-rank host logic (one process per GPU under torchrun; weak scaling:
# every rank solves its own instance, seed = rank, with no collective on the
# data path).  The timing of a region is the maximum over ranks and the
# job's throughput counts every rank's unknowns.
# ---------------------------------------------------------------------------
def rank_env():
    """(world, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def instance_seed(rank: int) -> int:
    return rank


def max_over_ranks(ms: float, dist=None, device=None) -> float:
    """The slowest rank's time (an all-reduce of one scalar), ms itself on one rank."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, unknowns_per_rank: int, steps: int, ms: float) -> float:
    """Unknowns solved by all ranks per second of the (max-over-ranks) time."""
    return world * unknowns_per_rank * steps / (ms * 1e-3)


def family_roofline(fname, frec, peaks, peak_src, num_sms, sm_max):
    """Roofline entry of one kernel family from its profile record (launches, ms,
    algorithmic bytes and flops): the block cyclic reductions and the reduction
    Filler against the derived FP32 FMA peak, every other family - the
    tensor-core Filler included - against the measured HBM bandwidth.  The
    tensor-core Filler moves 4 (225 + 60) bytes per hole for 2 x 225 x 60 flops,
    about 24 flop/byte, far below the TF32 ridge (~140 flop/byte): HBM bounds it;
    its tensor rate is given beside."""
    avg_ms = frec["ms"] / max(1, frec["launches"])
    if frec["flops"] > 0 and fname in ("bcr_aniso", "fill_holes"):
        achieved = frec["flops"] / (frec["ms"] * 1e-3) / 1e12
        peak = num_sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        return {"kernel": fname, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "peak_source": f"derived: {num_sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {sm_max:.0f} MHz",
                "avg_launch_us": avg_ms * 1e3, "launches": frec["launches"]}
    achieved = frec["bytes"] / (frec["ms"] * 1e-3) / 1e9
    peak = float(peaks["hbm_gbs"])
    out = {"kernel": fname, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "traffic": None, "peak_source": f"{peak_src} hbm_gbs",
           "avg_launch_us": avg_ms * 1e3, "launches": frec["launches"]}
    if fname == "fill_tc" and frec["flops"] > 0:
        tf = frec["flops"] / (frec["ms"] * 1e-3) / 1e12
        tpeak = float(peaks["bf16_tflops"]) * 1.1 / 2.25
        out["tensor"] = {"achieved_tflops": tf, "peak_tflops": tpeak, "frac": tf / tpeak,
                         "peak_source": f"{peak_src} bf16_tflops x 1.1/2.25 (nominal TF32/BF16 dense)"}
    return out


def run_reference(args):
    """--impl reference: the oracle on every host core, one measured batch of
    complete solves per step (OracleBaseline); rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    base = OracleBaseline(host_cores())
    vals = []
    for k in range(args.warmup + args.steps):
        r = base.run()
        if k >= args.warmup:
            vals.append(r)
    base.close()
    secs = [v["seconds"] for v in vals]
    value = base.procs * (base.N - 2) ** 2 * len(vals) / sum(secs)
    cfg = workload_config()
    cfg.update({"timed_instance": f"{base.N}x{base.N}, mc {base.mc}", "instances_per_step": base.procs})
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / len(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": base.procs, "kind": "oracle",
                             "sample": vals[-1]["sample"],
                             "host": {"nproc": host_cores(), "cpu": host_cpu_model(), "machine": platform.machine()}},
            "sweeps": vals[-1]["sweeps"], "converged": all(v["converged"] for v in vals),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_01163_gb300 import asdsm, workloads as wl

    world, rank, local = rank_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)

    N, mc = args.grid, args.mc
    p = wl.random_fourier_2d(N, instance_seed(rank))
    s = torch.tensor(p.s, dtype=torch.float64, device=dev)
    g = torch.tensor(p.g, dtype=torch.float64, device=dev)
    u = g.clone()
    solver = asdsm.Solver(N, mc, p.alpha, p.beta, precision=asdsm.MIXED, tol=TOL, max_sweeps=MAX_SWEEPS,
                          accel_m=ACCEL_M, sweep_graph=0 if args.host_sweeps else 1)
    stream = torch.cuda.current_stream()
    # Per-handle setup outside the timed region: launch shapes tuned for both
    # precisions (the initial guess runs in FP64).
    t_tune = time.time()
    if args.tune_cache and os.path.exists(args.tune_cache):
        with open(args.tune_cache) as f:
            solver.set_tune_state(json.load(f))     # shapes tuned by an earlier run (e.g. one timed without a profiler)
    else:
        solver.autotune(asdsm.MIXED)
        solver.autotune(asdsm.FP64)
        if args.tune_cache:
            with open(args.tune_cache, "w") as f:
                json.dump(solver.tune_state(), f)
    tune_ms = (time.time() - t_tune) * 1e3

    def step():
        u.copy_(g)
        return solver.solve(s, u)

    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    launches = 0
    sweeps = []
    rels = []
    rels64 = []                # every solve's returned iterate, judged in FP64 by the library at its end
    torch.cuda.nvtx.range_push("timed")       # lets a profiler select the timed launches
    for _ in range(args.steps):
        res = step()
        launches += res.stats["launches"]
        sweeps.append(res.stats["sweeps"])
        rels.append(res.stats["rel_res"])
        rels64.append(res.stats["rel_res_fp64"])
        if res.status != asdsm.OK:
            raise RuntimeError(f"solve did not converge: {res.stats}")
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
    # The last timed iterate judged by the FP64 fine residual (asdsm_residual,
    # FP64 arithmetic, pinned to the oracle's stencil): the tolerance must hold
    # in FP64, not only by the solver's own fixed-point residual.
    rel_res_fp64 = max(rels64 + [solver.residual(s, u)])
    if not rel_res_fp64 <= TOL:
        raise RuntimeError(f"FP64 residual of a returned iterate {rel_res_fp64:.3e} is above {TOL:g}")
    # Per-kernel-family times from separate profiled solves (event pairs around
    # each family on the handle's stream; the profiled loop is host-driven, the
    # kernels are the ones the timed solves ran).
    solver.profile(True)
    for _ in range(2):
        step()
    torch.cuda.synchronize()
    prof = solver.profile_read()
    solver.profile(False)
    unknowns = (N - 2) ** 2
    value = job_throughput(world, unknowns, args.steps, ms)

    # End to end through the public API with host buffers (pinned), per step:
    # H2D of s and of u's initial grid (ring = g), the solve, D2H of u.
    s_host = torch.tensor(p.s, dtype=torch.float64).pin_memory()
    g_host = torch.tensor(p.g, dtype=torch.float64).pin_memory()
    u_host = torch.empty_like(g_host).pin_memory()
    s_e = torch.empty_like(s)
    u_e = torch.empty_like(u)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        s_e.copy_(s_host, non_blocking=True)
        u_e.copy_(g_host, non_blocking=True)
        r2 = solver.solve(s_e, u_e)
        u_host.copy_(u_e, non_blocking=True)
        if r2.status != asdsm.OK:
            raise RuntimeError(f"e2e solve did not converge: {r2.stats}")
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    e2e = {"value": job_throughput(world, unknowns, args.steps, ms_e2e), "unit": UNIT,
           "h2d_bytes_per_step": 2 * N * N * 8, "d2h_bytes_per_step": N * N * 8}

    # Plain FP64 GPU ASDSM on the same problem (the comparison the metric names).
    fp64 = None
    if args.fp64_compare and rank == 0:
        sv64 = asdsm.Solver(N, mc, p.alpha, p.beta, precision=asdsm.FP64, tol=TOL, max_sweeps=MAX_SWEEPS,
                            accel_m=ACCEL_M)
        sv64.autotune(asdsm.FP64)
        u64 = g.clone()
        sv64.solve(s, u64)
        u64.copy_(g)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        r64 = sv64.solve(s, u64)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1)
        fp64 = {"value": unknowns / (ms64 * 1e-3), "unit": UNIT, "sweeps": r64.stats["sweeps"],
                "rel_res": r64.stats["rel_res"], "status": r64.status,
                "speedup_mixed_over_fp64": (value / world) / (unknowns / (ms64 * 1e-3))}
        sv64.close()

    # Uneven batch of 64 problems (N in {129, ..., 2049}) through asdsm_solve_batch.
    batch = None
    if args.batch and rank == 0:
        probs, mcs = wl.batch_problems(64, 0)
        b_unknowns = sum((q.N - 2) ** 2 for q in probs)
        # The slowest instance (N = 257, alpha = (0.0100, 0.0182), beta = (-7.23, -2.39), cell Peclet
        # 1.41 along x) needs about 730 sweeps in FP64 and mixed alike and progresses slowly near the
        # end: the stagnation test looks 30 sweeps back instead of 10.
        bsv = asdsm.BatchSolver([(q.N, mc, q.alpha, q.beta) for q, mc in zip(probs, mcs)], precision=asdsm.MIXED,
                                tol=TOL, max_sweeps=MAX_SWEEPS, accel_m=ACCEL_M_BATCH,
                                stagnation_window=STAG_WINDOW_BATCH)
        bsv.autotune(asdsm.MIXED)
        bsv.autotune(asdsm.FP64)
        bs_s = [torch.tensor(q.s, dtype=torch.float64, device=dev) for q in probs]
        bs_g = [torch.tensor(q.g, dtype=torch.float64, device=dev) for q in probs]
        bs_u = [x.clone() for x in bs_g]
        bsv.solve(bs_s, bs_u)                      # warm-up (captures the sweep graphs)
        torch.cuda.synchronize()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 2
        b0.record(stream)
        for _ in range(reps):
            for x, y in zip(bs_u, bs_g):
                x.copy_(y)
            brc, bst = bsv.solve(bs_s, bs_u)
        b1.record(stream)
        torch.cuda.synchronize()
        bms = b0.elapsed_time(b1) / reps
        batch = {"value": b_unknowns / (bms * 1e-3), "unit": UNIT, "instances": len(probs), "unknowns": b_unknowns,
                 "ms_per_solve": bms, "status": brc, "max_sweeps": max(x["sweeps"] for x in bst),
                 "worst_rel_res": max(x["rel_res"] for x in bst),
                 "accel_m": ACCEL_M_BATCH, "stagnation_window": STAG_WINDOW_BATCH,
                 "workload": "64 random-Fourier problems, N drawn from {129,257,513,1025,2049} (seed 0), "
                             "hole n = min(32, (N-1)/16), per-instance alpha/beta as the 2D workload"}
        bsv.close()

    # The 3D extension (Section 3.5) on its configuration: 257^3, mc = 16.
    leg3d = bench_3d(asdsm, wl, dev, stream) if (args.bench3d and rank == 0) else None

    if rank != 0:
        return

    peaks, peak_src = read_peaks()
    # Dominant kernel family by measured time.
    fam = max(prof.items(), key=lambda kv: kv[1]["ms"])
    name, f = fam
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count

    def roofline_of(fname, frec):
        return family_roofline(fname, frec, peaks, peak_src, num_sms, sm_max)

    roof = roofline_of(name, f)
    roof_resid = roofline_of("residual", prof["residual"])
    roof_fill = roofline_of("fill_tc", prof["fill_tc"]) if prof.get("fill_tc", {}).get("launches") else None
    roof_merge = roofline_of("merge", prof["merge"]) if prof.get("merge", {}).get("launches") else None
    # DRAM traffic per launch from the committed ncu capture (profiles/), where one exists.
    tpath = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles", "ncu_traffic_4097_mixed.json")
    if N == N_GRID and mc == MC and os.path.exists(tpath):
        with open(tpath) as tf:
            traffic = json.load(tf)
        for rl in (roof, roof_resid, roof_fill):
            if rl is not None and rl["kernel"] in traffic:
                rl["traffic"] = traffic[rl["kernel"]]["traffic_bytes_per_launch"]
    total_prof_ms = sum(v["ms"] for v in prof.values())
    shares = {k: round(v["ms"] / total_prof_ms, 4) for k, v in prof.items() if v["ms"] > 0}

    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline_line()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+i64", "data": "synthetic",
            "config": workload_config(N, mc, 0), "roofline": roof, "roofline_residual": roof_resid,
            "roofline_fill": roof_fill, "roofline_merge": roof_merge,
            "kernel_shares": shares, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "sweeps_per_solve": sweeps, "rel_res": max(rels), "rel_res_fp64": rel_res_fp64, "fp64_gpu": fp64,
            "setup_excluded": {"autotune_ms": tune_ms}, "batch": batch, "solve_3d": leg3d}
    print(json.dumps(line), flush=True)
    solver.close()
    if dist is not None:
        dist.destroy_process_group()


N3D, MC3D, ACCEL_M3D = 257, 16, 256


def bench_3d(asdsm, wl, dev, stream, N=N3D, mc=MC3D, reps=2):
    """The 3D leg: u = prod sin(pi x_i) on the unit cube, alpha_i log-uniform in
    [1e-2, 1], beta_i in [-5, 5] (seed 0), N^3 grid, mc coarse intervals,
    mixed precision, GCR with up to ACCEL_M3D directions, tol 1e-10; CUDA
    events around `reps` complete solves (setup excluded), one more solve
    with per-family timing for the shares."""
    import torch
    p = wl.random_sine_3d(N, 0)
    t0 = time.time()
    sv = asdsm.Solver(N, mc, p.alpha, p.beta, precision=asdsm.MIXED, tol=TOL, max_sweeps=3000, accel_m=ACCEL_M3D)
    setup_s = time.time() - t0
    s = torch.tensor(p.s, dtype=torch.float64, device=dev)
    g = torch.tensor(p.g, dtype=torch.float64, device=dev)
    u = g.clone()
    sv.solve(s, u)                                  # warm-up (allocates the direction store)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    results = []
    for _ in range(reps):
        u.copy_(g)
        results.append(sv.solve(s, u))
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    for r in results:
        if r.status != asdsm.OK or not r.stats["rel_res_fp64"] <= TOL:
            raise RuntimeError(f"3D solve did not reach {TOL:g}: {r.stats}")
    err = float((u - torch.tensor(p.u_exact, device=dev)).abs().max())
    sv.profile(True)
    u.copy_(g)
    sv.solve(s, u)
    torch.cuda.synchronize()
    prof = sv.profile_read()
    sv.profile(False)
    sv.close()
    total = sum(v["ms"] for v in prof.values()) or 1.0
    unknowns = (N - 2) ** 3
    return {"value": unknowns / (ms * 1e-3), "unit": UNIT, "ms_per_solve": ms, "unknowns": unknowns,
            "sweeps": results[-1].stats["sweeps"], "rel_res_fp64": max(r.stats["rel_res_fp64"] for r in results),
            "hole_fixes": results[-1].stats["hole_fixes"], "max_error_vs_manufactured": err,
            "launches_per_solve": results[-1].stats["launches"], "setup_s": setup_s,
            "kernel_shares": {k: round(v["ms"] / total, 4) for k, v in prof.items() if v["ms"] > 0},
            "families": {k: {"ms": v["ms"], "launches": v["launches"], "GB/s": v["bytes"] / (v["ms"] * 1e-3) / 1e9,
                             "TFLOP/s": v["flops"] / (v["ms"] * 1e-3) / 1e12} for k, v in prof.items() if v["ms"] > 0},
            "workload": f"3D extension: {N}^3 grid, mc {mc} (holes 15^3), alpha_i log-uniform [1e-2,1], "
                        f"beta_i in [-5,5], u = prod sin(pi x_i), seed 0; FP32 solves/merge/fill, FP64 residual "
                        f"and accumulation, GCR with up to {ACCEL_M3D} directions"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--grid", type=int, default=N_GRID)
    ap.add_argument("--mc", type=int, default=MC)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", dest="fp64_compare", action="store_false")
    ap.add_argument("--no-batch", dest="batch", action="store_false", help="skip the 64-problem batch measurement")
    ap.add_argument("--no-3d", dest="bench3d", action="store_false", help="skip the 3D leg (257^3)")
    ap.add_argument("--tune-cache", default=None,
                    help="JSON file of tuned launch shapes: written after autotuning, read instead of tuning if present")
    ap.add_argument("--host-sweeps", action="store_true",
                    help="host-driven sweep loop instead of CUDA graphs (same kernels; lets ncu list every launch)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
