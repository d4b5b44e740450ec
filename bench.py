#!/usr/bin/env python
"""Benchmark of the FETI interface solve: backward-Euler time steps per second.

One step = the whole per-step hot path: right-hand side, d = B K^+ f, lambda_0, the PCG
loop of Algorithm 1 (F p, coarse projection, Dirichlet preconditioner, reductions) to a
relative projected residual of `tol`, and the recovery of (u, xi, eta, p).

Arms
  native (default)   the CUDA library, one independent replica per GPU ("replicas only":
                     the library solves one problem on one GPU).
  --impl reference   the CPU oracle (plain FP64 scipy FETI) on the host cores, on a bounded
                     sample of the same workload (a smaller partition of the same
                     subdomains), scaled to the full workload by the subdomain count.

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


def workload(name, precision=None):
    from paper_2509_06673_gb300 import workloads as W
    cfg = {"config2": W.config2, "config3": W.config3, "config5": W.config5, "config5s": config5s}[name]()
    cfg = cfg.with_(tol=1e-8, max_it=2000)
    if precision:
        cfg = cfg.with_(precision=precision)
    return cfg


def sample_of(case):
    """Bounded CPU sample: a 4 x 4 partition of subdomains of the same size and physics."""
    from paper_2509_06673_gb300 import workloads as W
    cx = case.cells_x[:4]
    cy = case.cells_y[:4]
    s = W.grid_case("sample", 4, 4, list(cx), list(cy), order_k=case.order_k,
                    lame_lambda=case.lame_lambda, mu=case.mu, alpha=case.alpha, c0=case.c0,
                    perm_k=case.perm_k, mu_f=case.mu_f, tau=case.tau, tol=case.tol, max_it=case.max_it)
    if case.perm is not None:
        s = s.with_(perm=[case.perm[(r * case.nsub_x) + c] for r in range(4) for c in range(4)])
    return s


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


FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 rate of the profiling recipe's table

# DRAM traffic of the dominant kernel from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum per launch, profiles/k_band_solve_float_config5_launches.md).  The
# record holds only while the kernel source and its launch shape are the ones captured.
TRAFFIC_RECORDS = [
    {"workload": "config5", "precision": "mixed", "kernel": "k_band_solve_blk<float>",
     "shape": [8, 4096, 2], "band_cu_sha256": "14f2dc3e7b85ed1cfc01ae558464fa0c1bc73c0fc89f173be89354b81be1ae27",
     "bytes_per_launch": 54.394e9 + 0.378e9},
]


def traffic_of(workload, precision, shape):
    import hashlib
    src = os.path.join(ROOT, "paper_2509_06673_gb300", "csrc", "band.cu")
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()
    for r in TRAFFIC_RECORDS:
        if (r["workload"] == workload and r["precision"] == precision and r["band_cu_sha256"] == digest
                and r["shape"] == shape and r["bytes_per_launch"]):
            return r["bytes_per_launch"]
    return None


def cpu_baseline(case, n_steps=1):
    """Oracle FETI on the bounded sample; returns (steps/s scaled to the full workload, info)."""
    from oracle.monolithic import Discretization
    from oracle.feti import FETI
    smp = sample_of(case)
    d = Discretization(smp)
    f = FETI(smp, d)
    t0 = time.perf_counter()
    st = f.run(n_steps=n_steps)
    dt = (time.perf_counter() - t0) / n_steps
    scale = smp.nsub / case.nsub
    return 1.0 / dt * scale, {
        "sample": "%d step(s) of a 4x4 partition of the same subdomains (%dx%d cells, same physics), "
                  "oracle setup excluded; steps/s scaled by %d/%d subdomains; %d PCG iterations"
                  % (n_steps, smp.cells_x[0], smp.cells_y[0], smp.nsub, case.nsub, st[-1]["iterations"]),
        "cores": 1,
    }


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    case = workload(args.config, args.precision)
    from oracle.monolithic import Discretization
    from oracle.feti import FETI
    smp = sample_of(case)
    d = Discretization(smp)
    f = FETI(smp, d)
    f.run(n_steps=args.warmup)
    t0 = time.perf_counter()
    f.run(n_steps=args.steps)
    dt = time.perf_counter() - t0
    scale = smp.nsub / case.nsub
    value = args.steps / dt * scale
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": case.name, "tol": case.tol},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "value": value, "unit": "steps/s",
                             "sample": "4x4 partition of the same subdomains, %d steps after %d warm-up, "
                                       "scaled by %d/%d subdomains" % (args.steps, args.warmup, smp.nsub, case.nsub)},
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
    sol = F.Solver(case, stream=stream.cuda_stream)
    for key, val in (("solve_kernel", args.solve_kernel), ("solve_wpc", args.wpc), ("solve_chunk", args.chunk),
                     ("factor_fp64", args.factor_fp64), ("graph", args.graph), ("factor_nb", args.factor_nb),
                     ("explicit", args.explicit)):
        if val is not None:
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
    warmup = args.warmup

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # ---- device-timed region: inputs resident in HBM ----------------------------------
    sol.set_profiling(True)
    clocks = Clocks(local)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    torch.cuda.nvtx.range_push("timed_region")  # lets ncu select the timed launches
    its, restarts, wins, stags, gres = [], [], [], [], []
    for _ in range(args.steps):
        st = sol.step()
        its.append(st["iterations"])
        wins.append(st["lambda0_learned"])
        restarts.append(st["restarts"])
        stags.append(st["stagnations"])
        gres.append([st["guess_res_prev"], st["guess_res_learned"]])
    torch.cuda.nvtx.range_pop()
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    kN, kD = sol.kernel_stats(0), sol.kernel_stats(1)
    sol.set_profiling(False)
    value, job_s = job_rate(ms / 1000.0, args.steps, world)
    ms = job_s * 1000.0
    # ---- end to end through the public API, host buffers ------------------------------
    s = sol.sizes
    lam_h = torch.empty(s.n_lambda, dtype=torch.float64).pin_memory().numpy()
    u_h = torch.empty(2 * s.n_unode_total, dtype=torch.float64).pin_memory().numpy()
    f_h = [torch.empty(s.n_pnode_total, dtype=torch.float64).pin_memory().numpy() for _ in range(3)]
    xfer = [0, 0]
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st = sol.step()
        sol.get_lambda(lam_h)
        F._lib.fp_get_fields(sol._h, u_h.ctypes.data, f_h[0].ctypes.data, f_h[1].ctypes.data,
                             f_h[2].ctypes.data, 0)
        xfer[0] += st["h2d_bytes"]
        xfer[1] += st["d2h_bytes"]
    barrier()
    e2e_rate, e2e_s = job_rate(time.perf_counter() - t0, args.steps, world)
    # per step: the library's own scalar and flag copies (reported by fp_step) plus the
    # caller's read of lambda and all fields
    h2d = xfer[0] // args.steps
    d2h = xfer[1] // args.steps + 8 * (s.n_lambda + 2 * s.n_unode_total + 3 * s.n_pnode_total)
    # ---- roofline of the dominant kernel (banded local solves) -------------------------
    launches = kN["launches"] + kD["launches"]
    avg_ms = (kN["total_ms"] + kD["total_ms"]) / max(launches, 1)
    hbm, src = peaks()
    if case.precision == "fp64":
        ach = kN["flops_per_launch"] / (avg_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                "kernel": "k_band_solve_blk<double>" if args.solve_kernel != 0 else "k_band_solve<double>", "peak_source": "nominal FP64 rate (derived)",
                "achieved_gbs": kN["bytes_per_launch"] / (avg_ms * 1e-3) / 1e9}
    else:
        ach = kN["bytes_per_launch"] / (avg_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "traffic": None, "kernel": "k_band_solve_blk<float>" if args.solve_kernel != 0 else "k_band_solve<float>", "peak_source": src + " (burst copy)"}
    shape = [tuning["solve_wpc"], tuning["solve_chunk"], tuning["solve_ctas_per_sm"]]
    roof["traffic"] = traffic_of(args.config, case.precision, shape)
    roof.update({"launch_shape": {"warps_per_cta": shape[0], "stage_bytes": shape[1], "ctas_per_sm": shape[2]},
                 "algorithmic_bytes_per_launch": kN["bytes_per_launch"],
                 "launches_timed": launches, "avg_launch_ms": avg_ms,
                 "timed_launches": "CUDA events around every local solve outside the device-side "
                                   "PCG loop (a conditional graph body holds no events): the "
                                   "right-hand side, reference, initial and learned-guess solves "
                                   "with their refinement sweeps" if args.graph != 0 else
                                   "CUDA events around every local solve launch"})
    line = {"metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if case.precision == "fp64" else "f32 local / f64 outer",
            "data": "synthetic",
            "config": {"workload": case.name, "precision": case.precision, "tol": case.tol,
                       "subdomains": case.nsub, "n_lambda": s.n_lambda, "dofs": s.n_dofs,
                       "factor_gb": s.factor_bytes / 1e9, "l2": "inputs larger than L2 (factors %.1f GB)"
                       % (s.factor_bytes / 1e9), "setup_s": setup_s, "pcg_iterations": its, "pcg_restarts": restarts,
                       "pcg_stagnation_stops": stags, "autotuned": tuning,
                       "graph": args.graph != 0, "explicit_operators": bool(args.explicit),
                       "preconditioner": {0: "dirichlet", 1: "lumped", 2: "none"}.get(tuning["precond"]),
                       "learned_lambda0": learned,
                       "learned_guess_chosen": wins if learned else None,
                       "guess_rel_residual_prev_learned": gres if learned else None,
                       "learned_record_steps": args.learned_record_steps if learned else 0,
                       "learned_record_s": record_s, "learned_train_s": train_s,
                       "learned_train_loss": train_loss,
                       "first_timed_step": (args.learned_record_steps if learned else 0) + args.warmup + 1,
                       "parallelism": "replicas (one independent problem per GPU)"},
            "roofline": roof, "clocks": clk,
            "e2e": {"value": e2e_rate, "unit": "steps/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "inputs": "per-step inputs are the time level and the loop settings copied from "
                              "pinned host memory; the sources are closed-form functions of (x, t) "
                              "evaluated by the library on the device"},
            "gpu_launches": None}
    # kernel launches of the library in the timed region, from the loop structure (the ncu launch
    # list of the explicit-operator step: about 21 per PCG iteration and 155 per step outside it)
    line["gpu_launches"] = int(sum(its) * 21 + args.steps * 155)
    if rank == 0 and not args.no_cpu_baseline:
        v, info = cpu_baseline(case)
        line["cpu_baseline"] = {"value": v, "unit": "steps/s", "cores": info["cores"], "kind": "oracle",
                                "sample": info["sample"]}
    sol.close()
    del sol
    if not args.no_fp64_arm and case.precision != "fp64":
        # the comparison arm of the metric: plain FP64 FETI on the same workload
        c64 = case.with_(precision="fp64")
        s64 = F.Solver(c64, stream=stream.cuda_stream)
        if args.fp64_explicit is not None:
            s64.set_option("explicit", args.fp64_explicit)
        t0 = time.perf_counter()
        s64.assemble()
        s64.factor()
        setup64 = time.perf_counter() - t0
        for _ in range(args.warmup):
            s64.step()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        its64 = [s64.step()["iterations"] for _ in range(args.fp64_steps)]
        e1.record(stream)
        barrier()
        ms64 = e0.elapsed_time(e1)
        line["fp64_arm"] = {"value": world * args.fp64_steps / (ms64 / 1000.0), "unit": "steps/s",
                            "steps": args.fp64_steps, "ms_per_step": ms64 / args.fp64_steps,
                            "pcg_iterations": its64, "setup_s": setup64, "autotuned": s64.tuning(),
                            "explicit_operators": bool(args.fp64_explicit),
                            "speedup_of_value": value / (world * args.fp64_steps / (ms64 / 1000.0))}
        s64.close()
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
    ap.add_argument("--config", default="config5", choices=["config2", "config3", "config4", "config5", "config5s"])
    ap.add_argument("--config4-train", type=int, default=400, help="config4: recorded training steps")
    ap.add_argument("--config4-eval", type=int, default=200, help="config4: evaluation steps")
    ap.add_argument("--no-fp64-arm", action="store_true", help="skip the FP64 comparison arm")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--precision", default=None, choices=[None, "fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--solve-kernel", type=int, default=None, help="1 blocked sweeps, 0 row-step sweeps")
    ap.add_argument("--wpc", type=int, default=None, help="warps per CTA of the local solves")
    ap.add_argument("--chunk", type=int, default=None, help="bytes per shared-memory stage of the solves")
    ap.add_argument("--factor-fp64", type=int, default=None, help="mixed: factor in FP64, round to FP32")
    ap.add_argument("--factor-nb", type=int, default=None, help="panel width of the factorisation")
    ap.add_argument("--explicit", type=int, default=1, help="1: explicit local interface operators")
    ap.add_argument("--precond", default=None, choices=[None, "dirichlet", "lumped", "auto"],
                    help="preconditioner (both arms); default: the workload's (Dirichlet)")
    ap.add_argument("--fp64-explicit", type=int, default=1, help="explicit operators in the FP64 arm")
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
