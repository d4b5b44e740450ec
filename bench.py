#!/usr/bin/env python
"""Benchmark of the FETI interface solve: backward-Euler time steps per second.

One step = the whole per-step hot path: right-hand side, d = B K^+ f, lambda_0, the PCG
loop of Algorithm 1 (F p, coarse projection, Dirichlet preconditioner, reductions) to a
relative projected residual of `tol`, and the recovery of (u, xi, eta, p).

Arms
  native (default)   the CUDA library, one independent replica per GPU ("replicas only":
                     the library solves one problem on one GPU).  The mixed-precision arm
                     (FP32 local operators, FP64 outer PCG, learned lambda_0) is the value;
                     the plain FP64 arm of the same workload runs beside it (fp64_arm).
  --impl reference   the CPU oracle (plain FP64 scipy FETI) on all host cores, on bounded
                     samples of the same workload (4 x 4 blocks of the same subdomains, one
                     block per core), scaled to the full workload by the subdomain count.

Accuracy (the oracle leg, rank 0): a 4 x 4 block of the workload is solved by the oracle's
monolithic sparse LU, and by the library under each arm's exact settings (tolerance,
refinement stop, explicit operators, graph, the learned lambda_0 trained on the block's own
recorded steps), over the same step numbers as the timed steps.  The line states the maximum
relative error of lambda, u, xi, eta and p for each arm, and the loosest tolerance of the
ladder 1e-8 .. 1e-14 at which each arm meets its bar (1e-8 mixed, 1e-10 FP64); both arms are
then also timed on the full workload at those tolerances (``at_accuracy``).

Output: one JSON line on rank 0.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time steps/s at lambda rel. residual 1e-8"
TOL_LADDER = (1e-8, 1e-9, 1e-10, 1e-11, 1e-12, 1e-13, 1e-14)
BARS = {"mixed": 1e-8, "fp64": 1e-10}


def job_rate(local_s, steps, world, device="cuda"):
    """Whole-job rate of `world` independent replicas that each ran `steps` steps in
    `local_s` seconds: the slowest rank bounds the job (MAX over ranks with
    torch.distributed when world > 1).  Returns (steps per second of the job, job seconds)."""
    job_s = float(local_s)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([job_s], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        job_s = float(t.item())
    return world * steps / job_s, job_s


def config5s():
    """Profiling case: the subdomains and physics of config 5 on a 16 x 16 partition
    (256 subdomains, about 3 GB of FP32 factors: larger than L2, small enough for ncu)."""
    from paper_2509_06673_gb300 import workloads as W
    c = W.config5().with_(perm=None)
    c = W.grid_case("config5s: 16x16 subdomains of config 5 (24x24 cells, P2, nu=0.499, log-normal K)",
                    16, 16, 24, 24, order_k=2, lame_lambda=c.lame_lambda, tau=c.tau, tol=c.tol,
                    precision="mixed", source="manufactured_t")
    return c.with_(perm=W.lognormal_perm(c, sigma=1.0, seed=0))


def coarse64():
    """Profiling case for the coarse projection: a 64 x 64 partition of 2 x 2-cell P1 subdomains
    (3844 floating subdomains, coarse order 11 532 as in config 5) with small local factors."""
    from paper_2509_06673_gb300 import workloads as W
    return W.grid_case("coarse64: 64x64 subdomains of 2x2 P1 cells, nu=0.499 (config 5's coarse order)",
                       64, 64, 2, 2, order_k=1, lame_lambda=W.lame_from_nu(0.499), tau=1e-3,
                       precision="mixed", source="manufactured_t")


def workload(name, precision=None):
    from paper_2509_06673_gb300 import workloads as W
    cfg = {"config2": W.config2, "config3": W.config3, "config5": W.config5, "config5s": config5s,
           "coarse64": coarse64}[name]()
    cfg = cfg.with_(tol=1e-8, max_it=2000)
    if precision:
        cfg = cfg.with_(precision=precision)
    return cfg


def block_of(case, bi, bj, n=4):
    """Bounded sample: the n x n block (bi, bj) of the partition, as a problem of its own on the
    unit square (same subdomain sizes, physics and permeabilities; bottom half poroelastic)."""
    from paper_2509_06673_gb300 import workloads as W
    cx = case.cells_x[n * bj: n * bj + n]
    cy = case.cells_y[n * bi: n * bi + n]
    s = W.grid_case("sample", n, n, list(cx), list(cy), order_k=case.order_k,
                    lame_lambda=case.lame_lambda, mu=case.mu, alpha=case.alpha, c0=case.c0,
                    perm_k=case.perm_k, mu_f=case.mu_f, tau=case.tau, tol=case.tol, max_it=case.max_it,
                    source=case.source, precision=case.precision, precond=case.precond)
    if case.perm is not None:
        s = s.with_(perm=[case.perm[(n * bi + r) * case.nsub_x + n * bj + q] for r in range(n) for q in range(n)])
    return s


def sample_of(case):
    """The 4 x 4 block at the origin of the partition (the accuracy sample)."""
    return block_of(case, 0, 0)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        rows = [l.split(",") for l in open(self.path) if l.strip()]
        os.unlink(self.path)
        sm = sorted(float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit())
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            for nm, v in zip(names, r[5:9]):
                if "Active" in v and "Not" not in v:
                    reasons.add(nm)
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": sorted(reasons)}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def fp64_peak():
    """FP64 arithmetic rate of this GPU, measured: cuBLAS FP64 GEMM through torch.matmul
    (float64, 4096^3, 2 N^3 flops, best of 5 after a warm-up).  Used only as the
    denominator of the FP64 arm's ALU roofline."""
    import torch
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    best = None
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b
    torch.cuda.empty_cache()
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12, "measured: cuBLAS FP64 GEMM (torch.matmul float64, 4096^3, best of 5)"


def host_cpu():
    """(CPU model, logical cores) of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return model, os.cpu_count() or 1


# DRAM traffic of the dominant kernel (dram__bytes_read.sum + dram__bytes_write.sum per launch) from
# one ncu capture on config5s (the same 24 x 24-cell subdomains on a 16 x 16 partition, with config 5's
# solve launch shape pinned: 8 warps per CTA, 4 KB stages, 2 CTAs per SM): 2.983 GB per full solve
# against 2.8856 GB algorithmic.  For config 5 it is scaled by the algorithmic bytes (46.416 GB / 2.8856
# GB: traffic grows with the band bytes, every subdomain being the same size), see
# profiles/k_band_solve_float_config5s_traffic.md.  A record holds only while the solve's source and
# the launch shape are the ones captured.
_BAND_SHA = "8c14320b1e3b5f3502f593809244d00ac85bdbba2310c570180f3b85427b785e"
TRAFFIC_RECORDS = [
    {"workload": "config5s", "precision": "mixed", "kernel": "k_band_solve_blk<float>", "shape": [8, 4096, 2],
     "band_cu_sha256": _BAND_SHA, "bytes_per_launch": 2.9578e9 + 0.0256e9},
    {"workload": "config5", "precision": "mixed", "kernel": "k_band_solve_blk<float>", "shape": [8, 4096, 2],
     "band_cu_sha256": _BAND_SHA, "bytes_per_launch": (2.9578e9 + 0.0256e9) * 46.4158e9 / 2.8856e9},
]


# the record is keyed on the source of the band solve: band.cu from its TMA ring helpers to the end
# (the solve kernels and their launchers; the factorisation above them does not affect the traffic)
_SOLVE_MARK = b"// ============================ TMA ring helpers"


def traffic_of(workload, precision, shape):
    import hashlib
    src = open(os.path.join(ROOT, "paper_2509_06673_gb300", "csrc", "band.cu"), "rb").read()
    i = src.find(_SOLVE_MARK)
    digest = hashlib.sha256(src[i:] if i >= 0 else src).hexdigest()
    for r in TRAFFIC_RECORDS:
        if (r["workload"] == workload and r["precision"] == precision and r["band_cu_sha256"] == digest
                and r["shape"] == shape and r["bytes_per_launch"]):
            return r["bytes_per_launch"]
    return None


# ------------------------------- the oracle leg --------------------------------------------
def _oracle_block(arg):
    """Pool worker: the oracle FETI on one 4 x 4 block of the workload; per-step wall times of
    the steps after `warmup` and the PCG iterations of every step."""
    config, precision, bi, bj, warmup, steps = arg
    from oracle.monolithic import Discretization
    from oracle.feti import FETI
    smp = block_of(workload(config, precision), bi, bj)
    f = FETI(smp, Discretization(smp))
    marks = []
    st = f.run(n_steps=warmup + steps, callback=lambda _: marks.append(time.perf_counter()))
    # marks[k] ends step k + 1; the timed steps are warmup + 1 .. warmup + steps (warmup >= 1)
    times = [marks[k] - marks[k - 1] for k in range(warmup, warmup + steps)]
    return times, [s["iterations"] for s in st], smp.nsub


def oracle_throughput(config, precision, warmup, steps, nsub_full, its_full=None, workers=None):
    """The oracle FETI on all host cores: one 4 x 4 block of the workload per core (a process
    pool started with spawn), `warmup` untimed steps then `steps` timed steps per block.
    Throughput of the full workload = (subdomain-steps per second over all blocks) / subdomains.
    With its_full (the full workload's PCG iterations per step, same Krylov and warm start),
    value_iteration_adjusted also scales it by (iterations per step of the blocks) / its_full: a
    4 x 4 partition has a coarser mesh and needs fewer iterations than the full one."""
    import multiprocessing as mp
    model, cores = host_cpu()
    workers = workers or cores
    full = workload(config, precision)
    nbx, nby = max(1, full.nsub_x // 4), max(1, full.nsub_y // 4)
    blocks = [((i // nbx) % nby, i % nbx) for i in range(workers)]
    warmup = max(1, warmup)
    args = [(config, precision, bi, bj, warmup, steps) for bi, bj in blocks]
    # one BLAS thread per process: the pool already uses every core
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    os.environ.update({k: "1" for k in saved})
    try:
        t0 = time.perf_counter()
        with mp.get_context("spawn").Pool(workers) as pool:
            res = pool.map(_oracle_block, args)
        wall = time.perf_counter() - t0
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    rate = sum(nsub / (sum(times) / len(times)) for times, _, nsub in res)   # subdomain-steps / s
    its_blk = [i for _, its, _ in res for i in its[warmup:]]
    its_mean = sum(its_blk) / len(its_blk)
    value = rate / nsub_full
    step_s = max(sum(times) / len(times) for times, _, _ in res)
    return {"value": value, "unit": "steps/s", "cores": workers, "kind": "oracle", "cpu_model": model,
            "host_cores": cores,
            "value_iteration_adjusted": value * its_mean / its_full if its_full else None,
            "block_iterations_mean": its_mean, "full_iterations_mean": its_full,
            "block_step_s": step_s, "wall_s": wall,
            "sample": "%d processes (spawn), one 4x4 block of the workload's subdomains each (blocks %s ...), "
                      "%d warm-up + %d timed oracle FETI steps per block (one BLAS thread each), setup "
                      "excluded; subdomain-steps/s over all blocks / %d subdomains"
                      % (workers, blocks[:3], warmup, steps, nsub_full)}


def oracle_reference(smp, n_steps):
    """The oracle's monolithic sparse-LU solution of the sample for steps 1..n_steps:
    per step (lambda, per-subdomain (u, xi, eta, p))."""
    from oracle.monolithic import Discretization, solve_monolithic
    mono = solve_monolithic(smp, Discretization(smp), n_steps=n_steps)
    return [(m["lambda"], m["fields"]) for m in mono]


# ------------------------------- accuracy on the sample ------------------------------------
def _errors(F, smp, sol, ref):
    """Max relative errors (max |gpu - oracle| / max |oracle| over the sample) per field."""
    import numpy as np
    lam, fields_ref = ref
    out = {"lambda": float(np.abs(sol.get_lambda() - lam).max() / np.abs(lam).max())}
    got = F.split_fields(smp, *sol.get_fields())
    for k, name in enumerate(("u", "xi", "eta", "p")):
        num = max((np.abs(g[k] - r[k]).max() for g, r in zip(got, fields_ref) if r[k] is not None), default=0.0)
        den = max((np.abs(r[k]).max() for r in fields_ref if r[k] is not None), default=1.0)
        out[name] = float(num / den)
    return out


def arm_options(args, precision):
    """The library options an arm runs with (the same on the full workload and on the sample)."""
    if precision == "fp64":
        opts = (("explicit", args.fp64_explicit), ("graph", args.graph))
    else:
        opts = (("solve_kernel", args.solve_kernel), ("solve_wpc", args.wpc), ("solve_chunk", args.chunk),
                ("solve_cps", args.cps),
                ("factor_fp64", args.factor_fp64), ("graph", args.graph), ("factor_nb", args.factor_nb),
                ("explicit", args.explicit), ("precond_bf16", args.precond_bf16),
                ("explicit_df", args.explicit_df))
    return [(k, v) for k, v in opts if v is not None]


def sample_errors(F, smp, mono, precision, tol, args, stream):
    """The library on the sample under one arm's bench settings at tolerance `tol`: the same
    options, learned-guess recording and training, warm-up and step count as the timed run on
    the full workload.  Returns the max relative error per field over the timed step numbers."""
    case = smp.with_(precision=precision, tol=tol)
    sol = F.Solver(case, stream=stream.cuda_stream)
    for key, val in arm_options(args, precision):
        sol.set_option(key, val)
    sol.assemble()
    sol.factor()
    learned = bool(args.learned) and precision == "mixed"
    if learned:
        sol.learned_record(True, max_samples=4_000_000)
        for _ in range(args.learned_record_steps):
            sol.step()
        sol.learned_train(epochs=args.learned_epochs, batch=4096, lr=2e-3, seed=1)
        sol.learned_record(False)
        sol.learned_use(True)
    for _ in range(args.warmup):
        sol.step()
    worst, its, first, failed = {}, [], None, None
    for _ in range(args.steps):
        st = sol.step(allow_failure=True)
        if st["status"] != F.FP_OK:
            failed = "step %d: %s" % (st["step"], F.STATUS_NAMES.get(st["status"], st["status"]))
            break
        first = first or st["step"]
        its.append(st["iterations"])
        e = _errors(F, case, sol, mono[st["step"] - 1])
        worst = {k: max(v, worst.get(k, 0.0)) for k, v in e.items()}
    sol.close()
    worst["max"] = max(worst.values()) if worst and not failed else None
    out = {"tol": tol, "errors": worst, "steps": [first, first + args.steps - 1] if first else None,
           "iterations": its}
    if failed:
        out["failed"] = failed
    return out


def accuracy(F, smp, mono, precision, args, stream):
    """Errors at the metric's tolerance, then down the ladder until the arm's bar is met."""
    bar = BARS[precision]
    ladder, at_bar = [], None
    for tol in TOL_LADDER:
        r = sample_errors(F, smp, mono, precision, tol, args, stream)
        ladder.append({"tol": tol, "max_error": r["errors"]["max"], "iterations_mean":
                       sum(r["iterations"]) / max(len(r["iterations"]), 1), "failed": r.get("failed")})
        if tol == TOL_LADDER[0]:
            at_metric = r
        if r["errors"]["max"] is not None and r["errors"]["max"] <= bar:
            at_bar = tol
            break
    return {"bar": bar, "error_vs_oracle": at_metric["errors"], "steps_compared": at_metric["steps"],
            "tol_for_bar": at_bar, "ladder": ladder}


# ------------------------------- timing helpers --------------------------------------------
def timed_steps(sol, steps, stream, barrier, world):
    """CUDA-event time of `steps` steps on the library stream (barrier + sync on both sides).
    Each step's statistics carry its phase times (fp_get_step_timing: prologue, Algorithm 1,
    recovery; events recorded inside the step)."""
    import torch
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sts = []
    for _ in range(steps):
        st = sol.step()
        st["phase_ms"] = [float(x) for x in sol.step_timing()[:3]]
        sts.append(st)
    e1.record(stream)
    barrier()
    value, job_s = job_rate(e0.elapsed_time(e1) / 1000.0, steps, world)
    return value, job_s * 1000.0 / steps, sts


def run_reference(args):
    """The oracle arm: the CPU oracle on all host cores (rank 0 only under torchrun)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    case = workload(args.config, args.precision)
    cb = oracle_throughput(args.config, "fp64", args.warmup, args.steps, case.nsub)
    value = cb["value"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            # the wall time of one timed step of the slowest block (what was timed); value is the
            # full-workload throughput derived from all blocks
            "ms_per_step": cb["block_step_s"] * 1000.0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": case.name, "tol": case.tol},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_native(args):
    import numpy as np
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2509_06673_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2509_06673_gb300 import fetipe as F
    case = workload(args.config, args.precision)
    if args.precond:
        case = case.with_(precond=args.precond)
    stream = torch.cuda.current_stream()
    fp64_steps = args.fp64_steps or args.steps
    run_fp64 = not args.no_fp64_arm and case.precision != "fp64"

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- the oracle leg (rank 0): reference solution of the sample, accuracy of both arms --
    acc = {}
    if rank == 0 and not args.no_cpu_baseline:
        smp = sample_of(case)
        n_ref = (args.learned_record_steps if args.learned else 0) + args.warmup + args.steps
        n_ref = max(n_ref, args.warmup + fp64_steps)
        t0 = time.perf_counter()
        mono = oracle_reference(smp, n_ref)
        ref_s = time.perf_counter() - t0
        arms = [case.precision] + (["fp64"] if run_fp64 else [])
        for arm in arms:
            a = argparse.Namespace(**vars(args))
            if arm == "fp64" and arm != case.precision:
                a.steps = fp64_steps
            acc[arm] = accuracy(F, smp, mono, arm, a, stream)
        acc["oracle_reference_s"] = ref_s
        acc["sample"] = "%s: 4x4 block of the workload's subdomains (%dx%d cells), oracle monolithic " \
                        "sparse LU, steps 1..%d" % (smp.name, smp.cells_x[0], smp.cells_y[0], n_ref)
    if world > 1:
        torch.distributed.barrier()

    # ---- the headline arm ---------------------------------------------------------------
    sol = F.Solver(case, stream=stream.cuda_stream)
    for key, val in arm_options(args, case.precision):
        sol.set_option(key, val)
    t0 = time.perf_counter()
    sol.assemble()
    sol.factor()
    setup_s = time.perf_counter() - t0
    tuning = sol.tuning()
    learned = bool(args.learned) and case.precision == "mixed"
    train_s, train_loss, record_s = None, None, None
    if learned:
        # setup of the learned lambda_0 (outside the timed region): the solver records
        # (features, lambda increment) samples over its first steps, then the network is
        # trained on them with the library's own kernels
        t0 = time.perf_counter()
        sol.learned_record(True, max_samples=4_000_000)
        for _ in range(args.learned_record_steps):
            sol.step()
        record_s = time.perf_counter() - t0
        t0 = time.perf_counter()
        train_loss = sol.learned_train(epochs=args.learned_epochs, batch=4096, lr=2e-3, seed=1)
        train_s = time.perf_counter() - t0
        sol.learned_record(False)
        sol.learned_use(True)
    for _ in range(args.warmup):
        sol.step()

    # ---- device-timed region: inputs resident in HBM ----------------------------------
    sol.set_profiling(True)
    clocks = Clocks(local)
    torch.cuda.nvtx.range_push("timed_region")  # lets ncu select the timed launches
    value, ms, sts = timed_steps(sol, args.steps, stream, barrier, world)
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    kN, kD = sol.kernel_stats(0), sol.kernel_stats(1)
    sol.set_profiling(False)
    its = [s["iterations"] for s in sts]
    phase_ms = {k: float(np.mean([x["phase_ms"][i] for x in sts]))
                for i, k in enumerate(("prologue", "algorithm1", "recovery"))}

    # ---- the same arm at the tolerance its accuracy bar needs (when tighter) -------------
    at_acc = {}
    tol_bar = acc.get(case.precision, {}).get("tol_for_bar")
    if tol_bar is not None:
        try:
            if tol_bar != case.tol:
                sol.set_option("tol", tol_bar)
                for _ in range(2):
                    sol.step()
                v2, ms2, st2 = timed_steps(sol, args.steps, stream, barrier, world)
                sol.set_option("tol", case.tol)
                for _ in range(2):
                    sol.step()
            else:
                v2, ms2, st2 = value, ms, sts
            at_acc[case.precision] = {"tol": tol_bar, "value": v2, "ms_per_step": ms2,
                                      "pcg_iterations": [s["iterations"] for s in st2]}
        except F.FetipeError as ex:
            at_acc[case.precision] = {"tol": tol_bar, "failed": str(ex)}
            sol.set_option("tol", case.tol)

    # ---- end to end through the public API, host buffers ------------------------------
    s = sol.sizes
    lam_h = torch.empty(s.n_lambda, dtype=torch.float64).pin_memory().numpy()
    u_h = torch.empty(2 * s.n_unode_total, dtype=torch.float64).pin_memory().numpy()
    f_h = [torch.empty(s.n_pnode_total, dtype=torch.float64).pin_memory().numpy() for _ in range(3)]
    xfer = [0, 0]
    e2e_its = []
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st = sol.step()
        sol.get_lambda(lam_h)
        F._lib.fp_get_fields(sol._h, u_h.ctypes.data, f_h[0].ctypes.data, f_h[1].ctypes.data,
                             f_h[2].ctypes.data, 0)
        xfer[0] += st["h2d_bytes"]
        xfer[1] += st["d2h_bytes"]
        e2e_its.append(st["iterations"])
    barrier()
    e2e_rate, e2e_s = job_rate(time.perf_counter() - t0, args.steps, world)
    # per step: the library's own scalar and flag copies (reported by fp_step) plus the
    # caller's read of lambda and all fields
    h2d = xfer[0] // args.steps
    d2h = xfer[1] // args.steps + 8 * (s.n_lambda + 2 * s.n_unode_total + 3 * s.n_pnode_total)

    # ---- roofline of the dominant kernel (banded local solves) -------------------------
    nl = kN["launches"] + kD["launches"]
    avg_ms = (kN["total_ms"] + kD["total_ms"]) / max(nl, 1)
    hbm, src = peaks()
    if case.precision == "fp64":
        p64, p64_src = fp64_peak()
        ach = kN["flops_per_launch"] / (avg_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": p64, "unit": "TFLOP/s", "frac": ach / p64,
                "traffic": None, "kernel": "k_band_solve_blk<double>" if args.solve_kernel != 0 else
                "k_band_solve<double>", "peak_source": p64_src,
                "achieved_gbs": kN["bytes_per_launch"] / (avg_ms * 1e-3) / 1e9}
    else:
        ach = kN["bytes_per_launch"] / (avg_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": None, "kernel": "k_band_solve_blk<float>" if args.solve_kernel != 0 else
                "k_band_solve<float>", "peak_source": src + " (burst copy)"}
    shape = [tuning["solve_wpc"], tuning["solve_chunk"], tuning["solve_ctas_per_sm"]]
    roof["traffic"] = traffic_of(args.config, case.precision, shape)
    roof.update({"launch_shape": {"warps_per_cta": shape[0], "stage_bytes": shape[1], "ctas_per_sm": shape[2]},
                 "algorithmic_bytes_per_launch": kN["bytes_per_launch"],
                 "launches_timed": nl, "avg_launch_ms": avg_ms,
                 "timed_launches": "CUDA events around every local solve outside the device-side "
                                   "PCG loop (a conditional graph body holds no events): the "
                                   "right-hand side, reference, initial and learned-guess solves "
                                   "with their refinement sweeps" if args.graph != 0 else
                                   "CUDA events around every local solve launch"})
    line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if case.precision == "fp64" else "f32 local / f64 outer",
            "data": "synthetic",
            "config": {"workload": case.name, "precision": case.precision, "tol": case.tol,
                       "subdomains": case.nsub, "n_lambda": s.n_lambda, "dofs": s.n_dofs,
                       "factor_gb": s.factor_bytes / 1e9, "l2": "inputs larger than L2 (factors %.1f GB)"
                       % (s.factor_bytes / 1e9), "setup_s": setup_s,
                       "explicit_build_s": tuning["explicit_ms"] / 1000.0,
                       "pcg_iterations": its, "pcg_restarts": [x["restarts"] for x in sts],
                       "pcg_stagnation_stops": [x["stagnations"] for x in sts], "autotuned": tuning,
                       "graph": args.graph != 0, "explicit_operators": bool(args.explicit),
                       "preconditioner": {0: "dirichlet", 1: "lumped", 2: "none"}.get(tuning["precond"]),
                       "learned_lambda0": learned,
                       "learned_guess_chosen": [x["lambda0_learned"] for x in sts] if learned else None,
                       "guess_rel_residual_prev_learned": [[x["guess_res_prev"], x["guess_res_learned"]]
                                                           for x in sts] if learned else None,
                       "learned_record_steps": args.learned_record_steps if learned else 0,
                       "learned_record_s": record_s, "learned_train_s": train_s,
                       "learned_train_loss": train_loss,
                       "first_timed_step": sts[0]["step"],
                       "parallelism": "replicas (one independent problem per GPU)"},
            "roofline": roof, "clocks": clk,
            "e2e": {"value": e2e_rate, "unit": "steps/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "pcg_iterations": e2e_its,
                    "inputs": "per-step inputs are the time level and the loop settings copied from "
                              "pinned host memory; the sources are closed-form functions of (x, t) "
                              "evaluated by the library on the device"},
            "gpu_launches": int(sum(x["kernel_launches"] for x in sts)),
            "gpu_launches_detail": "kernels of the library launched in the timed steps, as fp_step reports them: "
                                   "the step graph's kernel nodes, its outer loop body's per round and its inner "
                                   "loop body's per execution (executions counted on the device)",
            "step_phase_ms": phase_ms}
    if case.precision in acc:
        line["error_vs_oracle"] = dict(acc[case.precision], sample=acc["sample"])
    sol.close()
    del sol
    if run_fp64:
        # the comparison arm of the metric: plain FP64 FETI on the same workload, same steps,
        # warm-up and tolerance policy
        c64 = case.with_(precision="fp64")
        s64 = F.Solver(c64, stream=stream.cuda_stream)
        for key, val in arm_options(args, "fp64"):
            s64.set_option(key, val)
        t0 = time.perf_counter()
        s64.assemble()
        s64.factor()
        setup64 = time.perf_counter() - t0
        for _ in range(args.warmup):
            s64.step()
        v64, ms64, st64 = timed_steps(s64, fp64_steps, stream, barrier, world)
        t64 = s64.tuning()
        line["fp64_arm"] = {"value": v64, "unit": "steps/s", "steps": fp64_steps, "warmup": args.warmup,
                            "ms_per_step": ms64, "pcg_iterations": [x["iterations"] for x in st64],
                            "setup_s": setup64, "explicit_build_s": t64["explicit_ms"] / 1000.0,
                            "autotuned": t64, "explicit_operators": bool(args.fp64_explicit),
                            "speedup_of_value": value / v64}
        if "fp64" in acc:
            line["fp64_arm"]["error_vs_oracle"] = acc["fp64"]
            tb = acc["fp64"]["tol_for_bar"]
            if tb is not None:
                try:
                    if tb != c64.tol:
                        s64.set_option("tol", tb)
                        for _ in range(2):
                            s64.step()
                        v2, ms2, st2 = timed_steps(s64, fp64_steps, stream, barrier, world)
                    else:
                        v2, ms2, st2 = v64, ms64, st64
                    at_acc["fp64"] = {"tol": tb, "value": v2, "ms_per_step": ms2,
                                      "pcg_iterations": [x["iterations"] for x in st2]}
                except F.FetipeError as ex:
                    at_acc["fp64"] = {"tol": tb, "failed": str(ex)}
        s64.close()
    if at_acc:
        if "value" in at_acc.get(case.precision, {}) and "value" in at_acc.get("fp64", {}) \
                and case.precision != "fp64":
            at_acc["speedup"] = at_acc[case.precision]["value"] / at_acc["fp64"]["value"]
        at_acc["how"] = ("each arm timed on the full workload at the loosest tolerance of the ladder "
                         "%s at which its error against the oracle on the sample meets its bar %s"
                         % (list(TOL_LADDER), BARS))
        line["at_accuracy"] = at_acc
    if rank == 0 and not args.no_cpu_baseline:
        its_full = None
        if "fp64_arm" in line:
            its_full = float(np.mean(line["fp64_arm"]["pcg_iterations"]))
        line["cpu_baseline"] = oracle_throughput(args.config, "fp64", 1, args.cpu_steps, case.nsub,
                                                 its_full=its_full)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_config4(args):
    """Learned lambda_0 on its own workload (config 4: config-3 geometry, point source): the
    network is trained on the steps the solver records at the training source location
    (seed 0, 400 steps), then 200 steps at an unseen location (seed 1) are run twice, with
    the previous-step guess and with the learned guess; iterations and device time per step
    at the metric's tolerance are compared.  Training is setup, outside the timed runs."""
    import numpy as np
    import torch
    from paper_2509_06673_gb300 import build
    build.build()
    from paper_2509_06673_gb300 import fetipe as F
    from paper_2509_06673_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    n_train, n_eval = args.config4_train, args.config4_eval

    def solver(seed):
        c = W.config4(seed=seed).with_(tol=1e-8, max_it=2000)
        if args.precond:
            c = c.with_(precond=args.precond)
        sol = F.Solver(c, stream=stream.cuda_stream)
        sol.set_option("explicit", args.explicit)
        sol.assemble()
        sol.factor()
        return sol

    t0 = time.perf_counter()
    tr = solver(0)
    tr.learned_record(True, max_samples=4_000_000)
    for _ in range(n_train):
        tr.step()
    record_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    loss = tr.learned_train(epochs=args.learned_epochs, batch=4096, lr=2e-3, seed=1)
    train_s = time.perf_counter() - t0
    theta = tr.mlp_get_params()
    tr.close()

    def evaluate(learned):
        sol = solver(1)
        if learned:
            sol.mlp_set_params(theta)
            sol.learned_use(True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its, wins, gres = [], 0, []
        for _ in range(n_eval):
            st = sol.step()
            its.append(st["iterations"])
            wins += st["lambda0_learned"]
            if learned and st["guess_res_prev"] > 0:
                gres.append(st["guess_res_learned"] / st["guess_res_prev"])
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        lam = sol.get_lambda()
        sol.close()
        return its, wins, ms, lam, gres

    its0, _, ms0, lam0, _ = evaluate(False)
    its1, wins, ms1, lam1, gres = evaluate(True)
    line = {"metric": METRIC, "value": n_eval / (ms1 / 1000.0), "unit": "steps/s", "n_gpus": 1,
            "steps": n_eval, "warmup": 0, "ms_per_step": ms1 / n_eval, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 local / f64 outer", "data": "synthetic",
            "config": {"workload": "config4: config-3 geometry (32x32 subdomains, uneven 16..48 cells, P2, "
                                   "nu=0.49), point source; train seed 0, evaluate seed 1",
                       "train_steps": n_train, "eval_steps": n_eval, "tol": 1e-8,
                       "explicit_operators": bool(args.explicit), "record_s": record_s, "train_s": train_s,
                       "train_loss": loss},
            "learned_gain": {"its_prev_guess": int(np.sum(its0)), "its_learned": int(np.sum(its1)),
                             "iteration_ratio": float(np.sum(its1) / np.sum(its0)),
                             "steps_per_s_prev_guess": n_eval / (ms0 / 1000.0),
                             "steps_per_s_learned": n_eval / (ms1 / 1000.0),
                             "time_ratio": ms1 / ms0, "learned_guess_chosen": int(wins),
                             "median_start_residual_ratio": float(np.median(gres)) if gres else None,
                             "lambda_rel_diff": float(np.abs(lam1 - lam0).max() / np.abs(lam0).max())}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--config", default="config5",
                    choices=["config2", "config3", "config4", "config5", "config5s", "coarse64"])
    ap.add_argument("--config4-train", type=int, default=400, help="config4: recorded training steps")
    ap.add_argument("--config4-eval", type=int, default=200, help="config4: evaluation steps")
    ap.add_argument("--no-fp64-arm", action="store_true", help="skip the FP64 comparison arm")
    ap.add_argument("--fp64-steps", type=int, default=None, help="FP64 arm timed steps (default: --steps)")
    ap.add_argument("--cpu-steps", type=int, default=2, help="timed oracle steps per block (cpu_baseline)")
    ap.add_argument("--precision", default=None, choices=[None, "fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--solve-kernel", type=int, default=None, help="1 blocked sweeps, 0 row-step sweeps")
    ap.add_argument("--wpc", type=int, default=None, help="warps per CTA of the local solves")
    ap.add_argument("--chunk", type=int, default=None, help="bytes per shared-memory stage of the solves")
    ap.add_argument("--cps", type=int, default=None, help="CTAs per SM of the local solves")
    ap.add_argument("--factor-fp64", type=int, default=None, help="mixed: factor in FP64, round to FP32")
    ap.add_argument("--factor-nb", type=int, default=None, help="panel width of the factorisation")
    ap.add_argument("--explicit", type=int, default=1, help="1: explicit local interface operators")
    ap.add_argument("--precond", default=None, choices=[None, "dirichlet", "lumped", "auto"],
                    help="preconditioner (both arms); default: the workload's (Dirichlet)")
    ap.add_argument("--fp64-explicit", type=int, default=1, help="explicit operators in the FP64 arm")
    ap.add_argument("--precond-bf16", type=int, default=None, help="mixed arm: S_s tiles in BF16")
    ap.add_argument("--explicit-df", type=int, default=None,
                    help="mixed arm: 1 build the FP64 F_s in two-float arithmetic, 0 in FP64")
    ap.add_argument("--graph", type=int, default=None, help="1: one CUDA graph launch per time step")
    ap.add_argument("--learned", type=int, default=1, help="mixed arm: learned lambda_0 (trained in warm-up)")
    ap.add_argument("--learned-epochs", type=int, default=8)
    ap.add_argument("--learned-record-steps", type=int, default=10,
                    help="steps the solver records for training the lambda_0 network (setup)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "config4":
        return run_config4(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
