#!/usr/bin/env python
"""Benchmark of the Darcy-Boussinesq state solve + adjoint on GB300.

One step = one pass of the whole path on one synthetic design: design pipeline (PDE filter,
RAMP) -> damped Newton state solve to relative residual 1e-8 -> adjoint solve -> sensitivities.
Workload (default): 128 x 128 x 128 Q1 elements (unit cube, h = 1/128), filtered-random density
at volume fraction 0.2, buoyancy factor alpha = 1e4, mixed-precision multigrid with 6 levels,
FP64 outer Newton. Metric: state solves per second (each including its adjoint and
sensitivities), whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the FP64 CPU oracle (the reference arm of this method) on the host cores,
on a bounded sample of the same workload. N > 1 runs one independent replica per GPU (the path
does not shard across GPUs here) with max-over-ranks timing.
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

# the oracle legs run on one host core: BLAS / OpenMP pools are pinned to one thread before NumPy loads
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from synthetic import filtered_random  # noqa: E402

METRIC = "state solves/s at 128^3 (mixed precision, rel. res 1e-8, with adjoint + sensitivities)"
UNIT = "solves/s"
CPU_SAMPLE_N = 16


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--alpha", type=float, default=1e4)
    ap.add_argument("--volfrac", type=float, default=0.2)
    ap.add_argument("--levels", type=int, default=6)
    ap.add_argument("--mg-op0", default="picard", choices=["exact", "picard"],
                    help="finest-level multigrid operator of the mixed path: the exact Jacobian or the "
                         "frozen-coefficient (Picard) operator")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--fast-steps", type=int, default=2)
    ap.add_argument("--concurrent-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--cavity-steps", type=int, default=2)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=300)
    ap.add_argument("--detail-out", default=None,
                    help="write the full record (per-class rooflines, kernel-time breakdown, solver histories) "
                         "to this JSON file; the printed line stays short")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, dist, device):
    """The maximum of a per-rank number over all ranks (the identity on one rank)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_design_seeds(rank, count):
    """Seeds of the designs one rank solves: every replica works on its own designs (weak scaling)."""
    return [100 * rank + i for i in range(count)]


def whole_job_rate(world, steps, seconds):
    """Solves per second of the whole job: every rank ran `steps` steps in at most `seconds`."""
    return world * steps / seconds


# ------------------------------------------------------------------------------- clocks ------
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region. Sampling starts
    before the region (start() waits for the first sample, so the tool's start-up is not inside it),
    every line is stamped with its arrival time, and stop(window) keeps the samples that arrived
    within the region's host-time window."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        t_end = time.perf_counter() + 5.0
        while not self.lines and time.perf_counter() < t_end and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self, window=None):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, util, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        lines = self.lines
        if window is not None:
            # a sample reports the state at its arrival, up to one period late: keep one period more
            inside = [(t, ln) for t, ln in lines if window[0] <= t <= window[1] + 0.05]
            lines = inside or lines
        for _, ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 10:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                util.append(float(parts[4]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[6:10]):
                if v.lower() == "active":
                    reasons.add(nm)
        loaded = [s for s, u in zip(sm, util) if u > 0] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------- CPU oracle --
def oracle_steps(seconds, n=CPU_SAMPLE_N, alpha=1e4, volfrac=0.2, max_steps=None):
    """Time the FP64 oracle's whole path (design, state, adjoint, sensitivities) on n^3 designs."""
    try:
        from threadpoolctl import threadpool_limits
        limiter = threadpool_limits(limits=1)
    except ImportError:  # the GPU machine has no threadpoolctl; NumPy/SciPy work here is single-threaded
        limiter = None
    import oracle
    times = []
    t_end = time.perf_counter() + seconds
    k = 0
    while True:
        rho = filtered_random(n, n, n, seed=1000 + k, volfrac=volfrac)
        t0 = time.perf_counter()
        op = oracle.Problem(oracle.Mesh(n, n, n, 1.0 / n), oracle.Params(alpha=alpha, newton_rtol=1e-8))
        op.set_design(rho)
        op.solve_state()
        op.solve_adjoint()
        op.sensitivities()
        times.append(time.perf_counter() - t0)
        k += 1
        if (max_steps is not None and k >= max_steps) or (max_steps is None and time.perf_counter() > t_end):
            break
    if limiter is not None:
        limiter.unregister() if hasattr(limiter, "unregister") else None
    return times


def scale_to_workload(sec_per_solve, n_sample, n_work, exponent=1.0):
    """Solves/s at the workload size assuming the oracle's cost grows as (node count)^exponent; the
    default 1 is optimistic for the oracle, whose sparse direct solves grow faster than linearly."""
    ratio = (((n_work + 1) ** 3) / ((n_sample + 1) ** 3)) ** exponent
    return 1.0 / (sec_per_solve * ratio)


def cpu_baseline_entry(seconds, n_work, alpha, volfrac):
    """The oracle on one host core: 16^3 solves for about `seconds`, then one 20^3 solve; the value is the
    16^3 time scaled to the workload by node count, with the growth exponent measured between the two
    sizes (and the value it implies) beside it."""
    t16 = oracle_steps(seconds, n=CPU_SAMPLE_N, alpha=alpha, volfrac=volfrac)
    t20 = oracle_steps(0, n=20, alpha=alpha, volfrac=volfrac, max_steps=1)
    a, b = float(np.mean(t16)), float(np.mean(t20))
    expo = np.log(b / a) / np.log((21.0 / 17.0) ** 3)
    return {"value": scale_to_workload(a, CPU_SAMPLE_N, n_work), "unit": UNIT, "cores": 1,
            "cores_available": os.cpu_count(), "kind": "oracle",
            "sample": "%d oracle whole-path solves (filter, Newton to 1e-8, adjoint, sensitivities) on %d^3 designs, "
                      "%.2f s each, scaled to %d^3 by node count; one 20^3 solve %.2f s"
                      % (len(t16), CPU_SAMPLE_N, a, n_work, b),
            "growth_exponent_16_20": _r(expo, 3),
            "value_at_measured_growth": scale_to_workload(a, CPU_SAMPLE_N, n_work, max(1.0, expo))}


# ------------------------------------------------------------------------------- reference ---
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        oracle_steps(0, max_steps=1, alpha=args.alpha, volfrac=args.volfrac)
    t0 = time.perf_counter()
    times = oracle_steps(0, max_steps=args.steps, alpha=args.alpha, volfrac=args.volfrac)
    wall = time.perf_counter() - t0
    per = wall / args.steps
    value = scale_to_workload(per, CPU_SAMPLE_N, args.n)
    sample = ("oracle whole path (filter, Newton to 1e-8, adjoint, sensitivities) on %d^3 designs, "
              "scaled to %d^3 by node count" % (CPU_SAMPLE_N, args.n))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "cores_available": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args, dev):
    """The 300-request stream (Poisson arrivals at 20/s, grids {32,48,64,96,128}^3, alpha log-uniform in
    [1e3, 1e5], half state-only and half state+adjoint) through the continuous-batching server. Every
    request has its own seeded filtered-random design, drawn on the device before the stream starts
    (inputs resident in HBM)."""
    import torch
    from synthetic import filtered_random_torch, request_stream
    from paper_1904_00182_gb300.serving import Request, Server, summarize
    stream = request_stream(n=args.serve_requests)
    designs = [filtered_random_torch(r["n"], r["n"], r["n"], seed=r["design_seed"], volfrac=args.volfrac, device=dev)
               for r in stream]
    torch.cuda.synchronize(dev)
    reqs = [Request(i, r["t_arrival"], r["n"], r["alpha"], r["adjoint"], designs[i]) for i, r in enumerate(stream)]
    srv = Server(slots=6, hbm_budget_bytes=48 << 30, device=dev,
                 mg_op0=1 if args.mg_op0 == "picard" else 0)
    # warm the pools with one request per grid size (problem creation is not part of serving)
    sizes = sorted({r.n for r in reqs})
    warm = [Request(-1 - k, 0.0, n, 1e4, True,
                    filtered_random_torch(n, n, n, seed=k, volfrac=args.volfrac, device=dev)) for k, n in enumerate(sizes)]
    torch.cuda.synchronize(dev)
    srv.run(warm)
    srv.done = []
    done = srv.run(reqs)
    out = summarize(done, srv.t_total)
    out.update({"slots": srv.slots, "hbm_budget_gb": srv.budget / 2 ** 30, "peak_pool_gb": srv.peak_bytes / 2 ** 30,
                "stream": "%d requests, Poisson 20/s, grids {32,48,64,96,128}^3, alpha log-uniform [1e3,1e5], "
                          "half with adjoint, one seeded design each, mixed precision to 1e-8" % len(reqs)})
    srv.close()
    return out


def workload_config(args):
    return {"workload": "%dx%dx%d Q1 Darcy-Boussinesq, filtered-random density V=%.1f, alpha=%g, "
                        "mixed GMG (%d levels), Newton to 1e-8 + adjoint + sensitivities"
                        % (args.n, args.n, args.n, args.volfrac, args.alpha, args.levels),
            "grid": [args.n, args.n, args.n], "alpha": args.alpha, "volfrac": args.volfrac,
            "mg_levels": args.levels, "newton_rtol": 1e-8, "mg_op0": args.mg_op0,
            "precision": "mixed: FP32 multigrid and Krylov operator; IEEE FP64 Newton residual, Krylov basis, "
                         "accepting adjoint residual, sensitivities, coarse residual",
            "l2": "inputs larger than L2 (Krylov basis ~1 GB, multigrid hierarchy ~0.4 GB per solve)",
            "parallelism": "replicas (one independent problem per GPU)"}


# ------------------------------------------------------------------------------- GPU arm -----
# Bound of each kernel class: "alu" classes are arithmetic-bound element kernels (their roofline is
# the plain FP32 or FP64 ALU peak derived from 152 SMs x lanes x 2 flops x 2.07 GHz: FP32 128 FMA
# lanes per SM -> 80.5 TFLOP/s, FP64 2 FMA units per SM -> 1.26 TFLOP/s); the rest stream vectors
# or stencils and are bound by HBM (measured copy bandwidth).
ALU_CLASSES = {"mg_op0": "fp32", "outer_op32": "fp32", "mg_setup_fine": "fp32",
               "residual": "fp64", "outer_op64": "fp64", "sens": "fp64", "adjoint_df64": "fp32"}
# On the mixed-precision path the outer residual classes run in double-float on the FP32 units; the
# library then counts their FP32 operations (a double-float add 11, a multiply 10 flops).
DF64_CLASSES = ("residual", "outer_op64", "sens")
ALU_PEAK_TFLOPS = {"fp32": 152 * 128 * 2 * 2.07e9 / 1e12, "fp64": 152 * 2 * 2 * 2.07e9 / 1e12}
# classes that time one kernel (with its output clear): candidates for the dominant-kernel roofline
SINGLE_KERNEL_CLASSES = ("residual", "outer_op64", "mg_op0", "mg_op0_picard", "mg_setup_fine", "adjoint_df64",
                         "coarse_factor", "mg_stencil_l1", "sens")


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the kernel behind a class at
# 128^3, from one ncu capture of the current kernel in the benchmark command (summaries under
# profiles/); a class whose kernel changes after its capture must leave this table.
NCU_TRAFFIC_128 = {
    "residual": (110.47e6, "profiles/k_residual_fp64_128cubed.md"),
    "outer_op64": (171.59e6, "profiles/k_jprod_transpose_fp64_128cubed.md"),
    "mg_op0": (69.80e6, "profiles/k_level0_apply_float_128cubed.md"),
    "mg_op0_picard": (86.72e6, "profiles/k_level0_picard_float_128cubed.md"),
}


def roofline_entry(name, v, peaks, df64=False):
    ms, n, nbytes, flops = v
    per_launch_s = ms * 1e-3 / n
    if name in ALU_CLASSES:
        kind = ALU_CLASSES[name]
        if df64 and name in DF64_CLASSES:
            kind = "fp32"
        achieved = flops / n / per_launch_s / 1e12
        peak = ALU_PEAK_TFLOPS[kind]
        return {"bound": "alu", "kernel_class": name,
                "arith": "df64 on fp32" if ((df64 and name in DF64_CLASSES) or name == "adjoint_df64") else kind,
                "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None, "per_launch_us": per_launch_s * 1e6,
                "launches": n, "alg_flops_per_launch": flops / n, "alg_bytes_per_launch": nbytes / n,
                "hbm_frac": nbytes / n / per_launch_s / 1e9 / peaks["hbm_gbs"],
                "peak_source": "derived from unit counts and the 2.07 GHz maximum SM clock"}
    achieved = nbytes / n / per_launch_s / 1e9
    return {"bound": "hbm", "kernel_class": name, "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": None, "per_launch_us": per_launch_s * 1e6,
            "launches": n, "alg_bytes_per_launch": nbytes / n,
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}


def run_gpu(args, rank, world, local):
    import torch
    import paper_1904_00182_gb300 as nc
    from paper_1904_00182_gb300 import build as ncbuild
    from paper_1904_00182_gb300.presets import solver_settings

    ncbuild.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=dev)
        dist = tdist
    n = args.n
    E = n ** 3
    ndes = max(1, min(3, args.steps + args.warmup))
    designs = [filtered_random(n, n, n, seed=sd, volfrac=args.volfrac) for sd in replica_design_seeds(rank, ndes)]
    rho_dev = [torch.from_numpy(d).to(dev) for d in designs]
    rho_host = [torch.from_numpy(d).pin_memory() for d in designs]
    grad_dev = torch.empty(E, dtype=torch.float64, device=dev)
    grad_host = torch.empty(E, dtype=torch.float64).pin_memory()
    stream = torch.cuda.Stream(device=dev)
    mg_op0 = nc.NC_MGOP_PICARD if args.mg_op0 == "picard" else nc.NC_MGOP_EXACT
    pb = nc.Problem(n, n, n, 1.0 / n, stream=stream.cuda_stream, device=dev, alpha=args.alpha,
                    mg_levels=args.levels, precision=nc.NC_PREC_MIXED, mg_op0=mg_op0)
    pb_params = pb.params.as_dict()
    stats_log = []

    def step(i, host=False):
        if host:
            pb.set_design(rho_host[i % ndes])
        else:
            pb.set_design(rho_dev[i % ndes])
        st = pb.solve_state()
        f, ast = pb.solve_adjoint()
        pb.sensitivities(out=grad_host if host else grad_dev)
        stats_log.append((st, ast))
        return f

    # warm-up: every kernel class timed (the breakdown and the choice of the dominant class);
    # timed region: only the dominant class is timed, so the events do not slow the other launches
    pb.set_profiling(True)
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize(dev)
    warm_prof = pb.profile()
    # the dominant kernel: the single-kernel class with the most device time (classes that group
    # several kernels of many small launches are left out; timing their every launch would also
    # perturb the timed region)
    dom = max((k for k in warm_prof if k in SINGLE_KERNEL_CLASSES), key=lambda k: warm_prof[k][0])
    if dist:
        dist.barrier()
    pb.set_profiling(classes=[dom])
    l0, _ = pb.counters()
    clocks = ClockSampler(local)
    clocks.start()
    stats_log.clear()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    th0 = time.perf_counter()
    ev0.record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize(dev)
    th1 = time.perf_counter()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop((th0, th1))
    l1, _ = pb.counters()
    prof = pb.profile()
    pb.set_profiling(False)
    ms = max_over_ranks(ms, dist, dev)
    if dist:
        dist.barrier()
    timed_stats = list(stats_log)
    value = whole_job_rate(world, args.steps, ms * 1e-3)

    # end to end through the C ABI with host buffers (H2D of the design, D2H of f and the gradient)
    e2e = None
    if not args.no_e2e:
        step(0, host=True)
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for i in range(args.steps):
            step(i, host=True)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        wall = max_over_ranks(wall, dist, dev)
        e2e = {"value": whole_job_rate(world, args.steps, wall), "unit": UNIT, "h2d_bytes_per_step": 8 * E,
               "d2h_bytes_per_step": 8 * E + 8}

    # the finest-level multigrid operator (the matrix-free operator of the preconditioner) timed on its
    # own over two more steps: every launch of its class bracketed by CUDA events on the library stream
    l0cls = "mg_op0_picard" if args.mg_op0 == "picard" else "mg_op0"
    pb.set_profiling(classes=[l0cls])
    for i in range(2):
        step(args.warmup + args.steps + i)
    torch.cuda.synchronize(dev)
    l0prof = pb.profile()[l0cls]
    pb.set_profiling(False)

    # the same workload on the all-FP64 path (the mixed-vs-FP64 comparison) and on the fast mixed
    # variant (double-float outer residuals, FP32 Krylov basis); each on its own problem
    pb.close()

    def time_variant(steps, **kw):
        if steps <= 0:
            return None
        pv = nc.Problem(n, n, n, 1.0 / n, stream=stream.cuda_stream, device=dev, alpha=args.alpha,
                        mg_levels=args.levels, **kw)

        def stepv(i):
            pv.set_design(rho_dev[i % ndes])
            st = pv.solve_state()
            _, ast = pv.solve_adjoint()
            pv.sensitivities(out=grad_dev)
            return st, ast
        stepv(0)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sts = [stepv(args.warmup + i) for i in range(steps)]
        e1.record(stream)
        e1.synchronize()
        msv = e0.elapsed_time(e1)
        pv.close()
        return {"value": steps / (msv * 1e-3), "unit": UNIT, "ms_per_step": msv / steps, "steps": steps,
                "newton_its": [x[0]["newton_its"] for x in sts], "krylov_its": [x[0]["krylov_its"] for x in sts],
                "adjoint_krylov_its": [x[1]["krylov_its"] for x in sts],
                "rel_residual": [x[0]["rel_residual"] for x in sts]}

    fp64 = time_variant(args.fp64_steps, precision=nc.NC_PREC_FP64)
    if fp64:
        fp64["precision"] = "IEEE FP64 throughout (multigrid, Krylov, residuals, coarse solve)"
    fast = time_variant(args.fast_steps, precision=nc.NC_PREC_MIXED, outer_arith=nc.NC_ARITH_DF64,
                        krylov_basis=nc.NC_BASIS_FP32, mg_op0=mg_op0)
    if fast:
        fast["precision"] = ("mixed, further reduced: double-float (48-bit significand) Newton residual, adjoint "
                             "residual and sensitivities; FP32 Krylov basis with FP64 cross-thread sums; "
                             "convergence still judged on the FP64 residual norm")

    # two independent problems in flight on two streams (the serving pattern at one grid size): FP64-
    # and FP32-bound phases of the two solves overlap on the device
    concurrent = None
    if args.concurrent_steps > 0:
        streams = [torch.cuda.Stream(device=dev) for _ in range(2)]
        pcs = [nc.Problem(n, n, n, 1.0 / n, stream=streams[i].cuda_stream, device=dev, alpha=args.alpha,
                          mg_levels=args.levels, mg_op0=mg_op0) for i in range(2)]

        def worker(i, steps):
            for j in range(steps):
                pcs[i].set_design(rho_dev[(i + j) % ndes])
                pcs[i].solve_state()
                pcs[i].solve_adjoint()
                pcs[i].sensitivities()

        def run_both(steps):
            ths = [threading.Thread(target=worker, args=(i, steps)) for i in range(2)]
            for t in ths:
                t.start()
            for t in ths:
                t.join()
            torch.cuda.synchronize(dev)

        run_both(1)
        t0 = time.perf_counter()
        run_both(args.concurrent_steps)
        wall_c = time.perf_counter() - t0
        for pc in pcs:
            pc.close()
        concurrent = {"in_flight": 2, "value": 2 * args.concurrent_steps / wall_c, "unit": UNIT,
                      "ms_per_solve_per_problem": wall_c / args.concurrent_steps * 1e3,
                      "timed": "host wall clock around both threads, device synchronised"}

    # the paper's benchmark geometry (Sec. 6.1): quarter of the closed 1 m cavity on 80 x 80 x 160 elements
    # (h = 1/160 m), heat source 0.05^3 m (quarter) with Q = 1e4 W/m^3, design box 0.375 x 0.375 x 0.75 m
    # on top of it with the initial design gamma = 0.05, passive fluid elsewhere; state solve from zero
    cavity = None
    if args.cavity_steps > 0 and rank == 0:
        cavity = []
        for alpha_c in (1e3, 1e6):
            pcv = nc.Problem(80, 80, 160, 1.0 / 160, stream=stream.cuda_stream, device=dev, alpha=alpha_c,
                             Q=1e4, bc=nc.NC_BC_CAVITY, heat_nx=8, heat_ny=8, heated_layers=8, design_nx=60,
                             design_ny=60, design_nz=120, timeout_s=60.0, mg_op0=mg_op0,
                             **solver_settings(alpha_c))
            rho_c = torch.full((80 * 80 * 160,), 0.05, dtype=torch.float64, device=dev)
            entry = {"alpha": alpha_c, "grid": [80, 80, 160], "settings": solver_settings(alpha_c)}
            try:
                pcv.set_design(rho_c)
                pcv.solve_state()
                torch.cuda.synchronize(dev)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sts = []
                for _ in range(args.cavity_steps):
                    pcv.set_design(rho_c)
                    sts.append(pcv.solve_state())
                e1.record(stream)
                e1.synchronize()
                msc = e0.elapsed_time(e1) / args.cavity_steps
                entry.update({"ms_per_state_solve": msc, "steps": args.cavity_steps,
                              "newton_its": [x["newton_its"] for x in sts], "krylov_its": [x["krylov_its"] for x in sts],
                              "ramped": [x["ramped"] for x in sts], "rel_residual": [x["rel_residual"] for x in sts]})
                # the adjoint of the mean heated-box temperature and the sensitivities at that state
                e0.record(stream)
                _, ast = pcv.solve_adjoint()
                pcv.sensitivities()
                e1.record(stream)
                e1.synchronize()
                entry.update({"ms_adjoint": e0.elapsed_time(e1), "adjoint_krylov_its": ast["krylov_its"]})
            except nc.NatConvError as e:
                entry["error"] = str(e)
            pcv.close()
            cavity.append(entry)

    serving = None
    if not args.no_serve and rank == 0:
        serving = run_serving(args, dev)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel class, from the live CUDA-event timing of the timed region
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
        peaks = json.load(fh)
    df64 = pb_params["precision"] == nc.NC_PREC_MIXED and pb_params["outer_arith"] == nc.NC_ARITH_DF64
    roof = roofline_entry(dom, prof[dom], peaks, df64) if prof[dom][1] > 0 else None
    def add_traffic(entry, cls):
        if entry and n == 128 and not df64 and cls in NCU_TRAFFIC_128:
            entry["traffic"], entry["traffic_source"] = NCU_TRAFFIC_128[cls]
    add_traffic(roof, dom)
    if roof:
        roof["timed"] = "live, CUDA events on the library stream around every launch of this class in the timed region"
    roof_l0 = roofline_entry(l0cls, l0prof, peaks, df64) if l0prof[1] > 0 else None
    add_traffic(roof_l0, l0cls)
    if roof_l0:
        roof_l0["timed"] = "CUDA events on the library stream around every launch of this class, two steps after the timed region"
    # breakdown and per-class rooflines from the profiled warm-up steps (all classes timed)
    warm_ms = sum(v[0] for v in warm_prof.values())
    rooflines = {k: roofline_entry(k, v, peaks, df64) for k, v in warm_prof.items() if v[1] > 0}
    breakdown = {k: {"ms_per_step": v[0] / args.warmup, "launches_per_step": v[1] / args.warmup,
                     "share_of_kernel_time": v[0] / warm_ms} for k, v in warm_prof.items() if v[1] > 0}

    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline_entry(args.cpu_seconds, n, args.alpha, args.volfrac)

    st_last = timed_stats[-1][0] if timed_stats else {}
    solver = {"newton_its": [s[0]["newton_its"] for s in timed_stats],
              "krylov_its": [s[0]["krylov_its"] for s in timed_stats],
              "adjoint_krylov_its": [s[1]["krylov_its"] for s in timed_stats],
              "rel_residual": [s[0]["rel_residual"] for s in timed_stats],
              "state_ms": [s[0]["t_total_ms"] for s in timed_stats],
              "adjoint_ms": [s[1]["t_total_ms"] for s in timed_stats],
              "krylov_hist_last": st_last.get("krylov_hist"),
              "newton_res_hist_last": st_last.get("res_hist"),
              "adjoint_res_hist_last": timed_stats[-1][1].get("res_hist") if timed_stats else None,
              "adjoint_krylov_hist_last": timed_stats[-1][1].get("krylov_hist") if timed_stats else None}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
            "config": workload_config(args), "clocks": clk, "e2e": e2e,
            "gpu_launches": int(l1 - l0), "roofline": roof, "roofline_level0": roof_l0, "cpu_baseline": cpu,
            "fp64_path": fp64, "mixed_fast": fast, "concurrent": concurrent, "cavity": cavity, "serving": serving,
            "solver": solver, "kernel_time_share_warmup": breakdown, "rooflines_warmup": rooflines}
    if args.detail_out:
        with open(args.detail_out, "w") as fh:
            json.dump(line, fh, indent=1)
    print(json.dumps(compact_line(line)), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def _r(x, d=4):
    """Round for the printed line (significant digits)."""
    return None if x is None else float("%.*g" % (d, x))


def compact_line(line):
    """The printed JSON line: the contract keys, the dominant kernel's roofline, a short kernel-time
    breakdown, and (last, so that a tail of the output still holds them) the comparison numbers: the
    all-FP64 path at equal final residual, the fast mixed variant, two problems in flight, the paper's
    cavity geometry and the serving stream's latency percentiles."""
    out = {k: line[k] for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                                "clocks", "e2e", "gpu_launches")}
    roof = line["roofline"]
    if roof:
        roof = {k: (_r(v) if isinstance(v, float) else v) for k, v in roof.items() if k != "timed"}
        roof["timed"] = "live CUDA events on the library stream, every launch of the class in the timed region"
    out["roofline"] = roof
    r0 = line.get("roofline_level0")
    if r0:
        out["roofline_level0"] = {k: (_r(v) if isinstance(v, float) else v) for k, v in r0.items()
                                  if k in ("bound", "kernel_class", "achieved", "peak", "unit", "frac", "traffic",
                                           "per_launch_us", "alg_bytes_per_launch", "alg_flops_per_launch",
                                           "hbm_frac")}
    out["cpu_baseline"] = line["cpu_baseline"]
    sv = line["solver"]
    out["solver"] = {"newton_its": sv["newton_its"], "krylov_its": sv["krylov_its"],
                     "adjoint_krylov_its": sv["adjoint_krylov_its"],
                     "max_rel_residual": _r(max(sv["rel_residual"])) if sv["rel_residual"] else None}
    bd = sorted(line["kernel_time_share_warmup"].items(), key=lambda kv: -kv[1]["ms_per_step"])[:8]
    out["breakdown_ms_per_step"] = {k: _r(v["ms_per_step"], 3) for k, v in bd}
    hb = {k: _r(v["frac"], 3) for k, v in line["rooflines_warmup"].items() if v["bound"] == "hbm"}
    out["hbm_frac_by_class"] = dict(sorted(hb.items(), key=lambda kv: -(kv[1] or 0))[:5])
    fp64, fast = line["fp64_path"], line["mixed_fast"]
    if fp64:
        out["fp64_path"] = {"value": _r(fp64["value"]), "ms_per_step": _r(fp64["ms_per_step"]),
                            "newton_its": fp64["newton_its"], "krylov_its": fp64["krylov_its"],
                            "max_rel_residual": _r(max(fp64["rel_residual"]))}
        out["mixed_over_fp64"] = _r(line["value"] / fp64["value"], 3)
    if fast:
        out["mixed_fast"] = {"value": _r(fast["value"]), "ms_per_step": _r(fast["ms_per_step"]),
                             "krylov_its": fast["krylov_its"]}
    c = line["concurrent"]
    if c:
        out["concurrent"] = {"in_flight": c["in_flight"], "value": _r(c["value"])}
    if line["cavity"]:
        out["cavity"] = [{"alpha": e["alpha"], "smoother": "zline" if e.get("settings") else "jacobi",
                          "ms": _r(e.get("ms_per_state_solve")),
                          "newton": (e.get("newton_its") or [None])[-1], "krylov": (e.get("krylov_its") or [None])[-1],
                          "adjoint_ms": _r(e.get("ms_adjoint")), "adjoint_krylov": e.get("adjoint_krylov_its"),
                          "error": e.get("error")} for e in line["cavity"]]
    sv = line["serving"]
    if sv:
        out["serving"] = {k: (_r(v) if isinstance(v, float) else v) for k, v in sv.items()
                          if k in ("requests", "errors", "p50_ms", "p99_ms", "requests_per_s", "state_solves_per_s",
                                   "adjoint_solves_per_s", "slots", "peak_pool_gb")}
    return out


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_gpu(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
