#!/usr/bin/env python3
"""Benchmark: seconds to a 1e-8 relative residual for flexible PCG preconditioned by SMG with
post-smoothing off (-v 1 0) on the 128^3 7-point Dirichlet Laplacian, with the V-cycle in FP32
(outer Krylov recurrences, inner products and norms in FP64), on one GB300.

One step = one complete solve (x0 = 0, seeded U[-1,1) right-hand side) through the C ABI:
every kernel of the path (plane relaxation with the 2D plane cycle and x-line solves,
residual + restriction, prolongation, the FP64 Krylov kernels) runs in the timed region.
The same solve with an FP64 cycle and with a BF16-storage cycle is timed beside it.

Prints one JSON line.  `--impl reference` times the plain FP64 CPU oracle on the same
workload instead (the reference arm; rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "s to 1e-8 rel. residual, 3D Laplacian FPCG-SMG: mixed/learned vs FP64"
NX = NY = NZ = 128
TOL = 1e-8
WORKLOAD = "FPCG-SMG(1,0) 128^3 7-point Dirichlet Laplacian, V-cycle FP32, Krylov FP64, tol 1e-8"
HBM_FALLBACK_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the 256^3 learned-correction comparison")
    ap.add_argument("--workload", choices=["fpcg128", "batched64", "lobpcg128", "learned256", "bricks", "cg128",
                                           "lobpcg_bricks"],
                    default="fpcg128",
                    help="fpcg128: one 128^3 system (default); batched64: 64 uneven systems, sides in {32..96}; "
                         "lobpcg128: 16 smallest eigenpairs at 128^3; learned256: learned post-correction at 256^3; "
                         "bricks: the paper's 16n x n x n bricks, n = 10..32, every Krylov variant and cycle; "
                         "cg128: no preconditioner at 128^3 (CG by eq. (1) and eq. (2), steepest descent); "
                         "lobpcg_bricks: LOBPCG, one eigenpair, 4n x 2n x 2n bricks, (1,1) against (1,0)")
    return ap.parse_args()


def measured_bf16_peak():
    """Measured dense BF16 tensor throughput (TFLOP/s, burst) from MEASURED_PEAKS.json, else the
    fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return 1900.0


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def source_hash():
    import hashlib

    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1212_6680_gb300", "csrc")
    for f in ("plane_lean.cuh", "plane_relax.cuh", "plane_relax_inst.cu"):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic():
    """DRAM bytes per level-0 launch of the plane-relaxation kernel from the committed ncu
    summary, if it was captured from the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "plane_lean_traffic_level0_128cube.txt")
    try:
        d = json.load(open(p))
        if d.get("source_hash") == source_hash():
            return d
    except Exception:
        pass
    return None


NSYS = 64
BATCH_WORKLOAD = ("64 independent FPCG-SMG(1,0) solves, 7-point Dirichlet Laplacian, sides i.i.d. uniform in "
                  "{32..96} per axis, V-cycle FP32, Krylov FP64, tol 1e-8 each")


def batched_inputs():
    """Grid sides (seed 1000 + i for system i) and right-hand sides (same seeds) of the 64 systems."""
    from paper_1212_6680_gb300 import inputs

    dims = inputs.uneven_dims(NSYS, 32, 96, seed=1000)
    bs = [inputs.rhs(int(nx), int(ny), int(nz), seed=1000 + i) for i, (nx, ny, nz) in enumerate(dims)]
    return dims, bs


def oracle_batched_sample(nsample):
    """Oracle FPCG-SMG(1,0) solves of the first `nsample` systems on every host core; seconds
    scaled to all 64 by the unknowns they hold (no scaling when nsample = 64)."""
    import oracle

    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    dims, bs = batched_inputs()
    t0 = time.perf_counter()
    its = []
    for i in range(nsample):
        nx, ny, nz = map(int, dims[i])
        out = oracle.krylov(bs[i], "fpcg", oracle.SMG(nx, ny, nz, 1, 0), tol=TOL, maxit=100)
        assert out["status"] == 0 and out["relres"] <= TOL
        its.append(out["iters"])
    t = time.perf_counter() - t0
    n_all = float(sum(int(np.prod(d)) for d in dims))
    n_s = float(sum(int(np.prod(d)) for d in dims[:nsample]))
    return t * n_all / n_s, its, t


def oracle_solve_baseline():
    """The oracle's full FPCG-SMG(1,0) solve at 128^3 timed on every host core (OpenMP) and on one."""
    import oracle
    from paper_1212_6680_gb300 import inputs

    oracle.build()
    bo = inputs.rhs(NX, NY, NZ, seed=0)
    T = oracle.SMG(NX, NY, NZ, 1, 0)
    cores = os.cpu_count() or 1
    out_t = {}
    for nt in (cores, 1):
        oracle.set_threads(nt)
        t0 = time.perf_counter()
        out = oracle.krylov(bo, "fpcg", T, tol=TOL, maxit=100)
        out_t[nt] = time.perf_counter() - t0
        assert out["status"] == 0 and out["relres"] <= TOL
    oracle.set_threads(cores)
    return {"value": out_t[cores], "unit": "s", "cores": cores, "kind": "oracle",
            "single_thread_s": out_t[1],
            "sample": f"one full FPCG-SMG(1,0) solve at 128^3 in FP64 ({out['iters']} iterations) on {cores} "
                      f"host cores (OpenMP over planes, lines and transfer points; bitwise the single-thread "
                      f"result), and on one thread"}


def run_reference(args):
    import oracle
    from paper_1212_6680_gb300 import inputs

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload in ("lobpcg128", "learned256"):
        from paper_1212_6680_gb300 import inputs as _in

        times, sample = [], ""
        for _ in range(args.steps):
            if args.workload == "lobpcg128":
                from oracle import lobpcg as olob

                oracle.build()
                oracle.set_threads(os.cpu_count() or 1)
                X0 = _in.initial_block(NX, NY, NZ, LOB_M, seed=7)
                t0 = time.perf_counter()
                olob.lobpcg((NZ, NY, NX), np.ascontiguousarray(X0.T), oracle.SMG(NX, NY, NZ, 1, 0), tol=TOL, maxit=1)
                t1 = time.perf_counter() - t0
                times.append(t1 * 37)
                sample = (f"extrapolated: oracle LOBPCG set-up + 1 iteration at 128^3, m=16 ({t1:.1f} s) x 37 "
                          f"iterations, {os.cpu_count() or 1} host cores")
            else:
                v, t1 = oracle_learned_sample(_in.net_init_weights(seed=77), 9)
                times.append(v)
                sample = (f"extrapolated: one oracle application of the learned preconditioner at 64^3 ({t1:.1f} s) "
                          f"x 64 points x 9 iterations, {os.cpu_count() or 1} host cores (OpenMP in the SMG cycle; "
                          f"the network's convolutions on one core)")
        v = statistics.mean(times)
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": (LOB_WORKLOAD if args.workload == "lobpcg128" else LEARNED_WORKLOAD)
                           + " (FP64 CPU oracle, bounded sample)"},
                "cpu_baseline": {"value": v, "unit": "s", "cores": os.cpu_count() or 1, "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    if args.workload == "batched64":
        times = []
        for _ in range(args.steps):
            v, its, raw = oracle_batched_sample(NSYS)
            times.append(v)
        v = statistics.mean(times)
        sample = (f"oracle FPCG-SMG(1,0) solves of all 64 systems one after another ({raw:.1f} s), "
                  f"{os.cpu_count() or 1} host cores (OpenMP)")
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": BATCH_WORKLOAD.replace("V-cycle FP32, Krylov FP64", "FP64 CPU oracle")},
                "cpu_baseline": {"value": v, "unit": "s", "cores": os.cpu_count() or 1, "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    oracle.build()
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    b = inputs.rhs(NX, NY, NZ, seed=0)
    T = oracle.SMG(NX, NY, NZ, 1, 0)
    for _ in range(args.warmup):  # warm-up: one full solve each
        oracle.krylov(b, "fpcg", T, tol=TOL, maxit=100)
    times, iters = [], None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        out = oracle.krylov(b, "fpcg", T, tol=TOL, maxit=100)
        times.append(time.perf_counter() - t0)
        iters = out["iters"]
        assert out["status"] == 0 and out["relres"] <= TOL
    v = statistics.mean(times)
    sample = (f"full FPCG-SMG(1,0) solve, 128^3, FP64, {iters} iterations, {cores} host cores (OpenMP over planes, "
              f"lines and transfer points; bitwise the single-thread result)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.replace("V-cycle FP32", "V-cycle FP64 (CPU oracle)"),
                       "grid": [NX, NY, NZ], "iters": iters},
            "cpu_baseline": {"value": v, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    from paper_1212_6680_gb300 import build as _build
    from paper_1212_6680_gb300 import inputs

    world, rank, local, dist = _dist_init()
    _build.build()
    from paper_1212_6680_gb300 import smg

    b_np = inputs.rhs(NX, NY, NZ, seed=0).ravel().copy()
    n = b_np.size
    b = torch.from_numpy(b_np).cuda()
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def timed_solves(h, steps, warmup, host=False):
        """Per-step device time (events) of `steps` solves, L2 flushed before each."""
        bh = torch.from_numpy(b_np).pin_memory() if host else None
        xh = torch.zeros(n, dtype=torch.float64).pin_memory() if host else None
        for _ in range(warmup):
            x.zero_()
            smg.krylov_solve(h, "fpcg", b, x, TOL, 100)
        times, its, res = [], None, None
        for _ in range(steps):
            flush.zero_()
            if host:
                xh.zero_()
            else:
                x.zero_()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if host:
                rc, its, res = smg.krylov_solve(h, "fpcg", bh.numpy(), xh.numpy(), TOL, 100)
            else:
                rc, its, res = smg.krylov_solve(h, "fpcg", b, x, TOL, 100)
            e1.record(stream)
            barrier()
            assert rc == smg.SMG_OK and res <= TOL, (rc, res)
            times.append(e0.elapsed_time(e1) / 1e3)
        return times, its, res

    handles = {}
    for prec in ("fp32", "fp64", "bf16"):
        h = smg.smg_setup(NX, NY, NZ, 1, 0)
        smg.smg_set_precision(h, prec)
        handles[prec] = h
    h32 = handles["fp32"]

    # ---- main arm: FP32 cycle, device buffers, the device-side solve loop (one CUDA graph) ----
    for _ in range(args.warmup):
        x.zero_()
        smg.krylov_solve(h32, "fpcg", b, x, TOL, 100)
    l0 = smg.smg_launch_count(h32)
    barrier()
    wall0 = time.perf_counter()
    with ClockSampler(local) as clk:
        times, iters, relres = timed_solves(h32, args.steps, 0)
    wall = time.perf_counter() - wall0
    launches = smg.smg_launch_count(h32) - l0
    t_step = statistics.median(times)  # median of the timed steps
    t_max = max_over_ranks(t_step, dist, "cuda")
    # ---- the finest level's plane-relaxation launches timed with CUDA events on the launching
    # stream, in solves run right after the timed region (per-launch events cannot sit inside the
    # graph, so these solves take the host loop) ----
    kp = max(1, min(args.steps, 3))
    smg.smg_set_option(h32, smg.SMG_OPT_PROFILE, 1)
    smg.smg_profile_read(h32, 0)
    tprof, _, _ = timed_solves(h32, kp, 0)
    pl, pms, pbytes = smg.smg_profile_read(h32, 0)
    smg.smg_set_option(h32, smg.SMG_OPT_PROFILE, 0)
    # ---- host loop without profiling, for comparison with the device-side loop ----
    smg.smg_set_option(h32, smg.SMG_OPT_GRAPH, 0)
    thost, _, _ = timed_solves(h32, kp, 1)
    smg.smg_set_option(h32, smg.SMG_OPT_GRAPH, 1)

    # ---- every plane-relaxation launch of one solve timed (all z-levels, the FP64 coarsest plane) ----
    smg.smg_set_option(h32, smg.SMG_OPT_PROFILE, 2)
    for c in range(6):
        smg.smg_profile_read(h32, c)
    x.zero_()
    smg.krylov_solve(h32, "fpcg", b, x, TOL, 100)
    prof_all = {c: smg.smg_profile_read(h32, c) for c in range(5)}
    smg.smg_set_option(h32, smg.SMG_OPT_PROFILE, 0)
    # ---- comparison arms on the same GPU: FP64 and BF16 cycles ----
    k2 = max(1, min(args.steps, 3))
    t64, it64, _ = timed_solves(handles["fp64"], k2, 1)
    t16, it16, _ = timed_solves(handles["bf16"], k2, 1)
    # ---- end to end: host buffers, copies inside the call ----
    te, _, _ = timed_solves(h32, max(1, min(args.steps, 3)), 1, host=True)

    for h in handles.values():
        smg.smg_destroy(h)
    # ---- the learned post-correction at 256^3 against the plain cycles (stored, GPU-trained weights) ----
    learned256 = None if args.no_learned else learned_comparison(smg, inputs, barrier, flush, stream, k2)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    peak, peak_kind = measured_peaks()
    achieved = (pbytes / 1e9) / (pms / 1e3) if pms > 0 else None
    tr = ncu_traffic()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": (tr["dram_bytes_per_launch"] if tr else None),
                "kernel": "plane_lean_kernel<float,float,4,false> (finest level)",
                "launches": pl, "avg_launch_us": (pms * 1e3 / pl) if pl else None,
                "algorithmic_bytes_per_launch": (pbytes / pl) if pl else None,
                "duration_source": f"CUDA events around every finest-level launch on the launching stream, in {kp} "
                                   f"solves right after the timed region (the timed solves run as one CUDA graph, "
                                   f"which cannot hold the events)",
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else
                "fallback 6.8 TB/s"}
    # the same ratio over every plane-relaxation launch of a solve (all z-levels, FP32, and the FP64
    # coarsest plane), and each class of the cycle (CUDA events around every launch: the profiled
    # solve's launches lose their programmatic-dependent-launch overlap)
    names = {0: "plane relaxation, finest level", 1: "plane relaxation, other levels", 2: "coarsest plane (FP64)",
             3: "restriction + prolongation", 4: "Krylov kernels"}
    classes = {}
    for c, (nl, ms, by) in prof_all.items():
        classes[names[c]] = {"launches": nl, "us_per_launch": (ms * 1e3 / nl) if nl else None,
                             "ms_per_solve": ms, "GB_per_s": ((by / 1e9) / (ms / 1e3)) if (ms > 0 and by > 0) else None}
    rl_ms = sum(prof_all[c][1] for c in (0, 1, 2))
    rl_by = sum(prof_all[c][2] for c in (0, 1, 2))
    if rl_ms > 0:
        roofline["all_levels"] = {"achieved": (rl_by / 1e9) / (rl_ms / 1e3), "frac": ((rl_by / 1e9) / (rl_ms / 1e3)) / peak,
                                  "unit": "GB/s", "note": "every plane-relaxation launch of one solve"}
    cpu = None
    if not args.no_cpu_baseline:
        cpu = oracle_solve_baseline()
    line = {
        "metric": METRIC, "value": t_max, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [NX, NY, NZ], "variant": "fpcg", "npre": 1, "npost": 0,
                   "value_is": f"median of the {args.steps} timed solves (mean {statistics.mean(times):.6f} s)",
                   "cycle_precision": "fp32", "iters": iters, "true_relres": relres,
                   "l2": "256 MB buffer written before every timed solve", "parallelism": "replicas" if world > 1 else "single GPU",
                   "fp64_cycle_s": statistics.mean(t64), "fp64_cycle_iters": it64,
                   "bf16_cycle_s": statistics.mean(t16), "bf16_cycle_iters": it16,
                   "speedup_fp32_vs_fp64": statistics.mean(t64) / t_step,
                   "host_loop_s": statistics.mean(thost), "profiled_solve_s": statistics.mean(tprof),
                   "cycle_classes_profiled_solve": classes,
                   "learned256": learned256},
        "roofline": roofline, "cpu_baseline": cpu,
        "e2e": {"value": statistics.mean(te), "unit": "s", "h2d_bytes_per_step": 2 * n * 8, "d2h_bytes_per_step": n * 8},
        "gpu_launches": launches, "clocks": clk.summary(), "wall_s_timed_region": wall,
    }
    print(json.dumps(line), flush=True)


LEARNED_WEIGHTS = os.path.join(ROOT, "paper_1212_6680_gb300", "weights", "learned_fpcg_seed5000.npz")


def learned_comparison(smg, inputs, barrier, flush, stream, steps):
    """FPCG at 256^3 with the learned post-correction (weights written by learned.train, recipe stored
    beside them) against the plain FP32 (1,0) and (1,1) cycles and the FP64 (1,0) cycle."""
    import torch

    from paper_1212_6680_gb300 import learned

    w, recipe = learned.load_weights(LEARNED_WEIGHTS)
    b = torch.from_numpy(inputs.rhs(LN, LN, LN, seed=0).ravel().copy()).cuda()
    x = torch.zeros_like(b)
    out = {"workload": "FPCG to 1e-8 at 256^3 (7-point Dirichlet Laplacian, rhs seed 0), L2 flushed before every "
                       "timed solve",
           "weights": {"file": os.path.relpath(LEARNED_WEIGHTS, ROOT),
                       **{k: recipe.get(k) for k in ("nsys", "sides", "seed", "init_seed", "epochs", "lr", "act", "pairs")}}}
    for name, npost, prec, use_w in (("learned_10_fp32", 0, "fp32", True), ("plain_10_fp32", 0, "fp32", False),
                                     ("balanced_11_fp32", 1, "fp32", False), ("plain_10_fp64", 0, "fp64", False)):
        h = smg.smg_setup(LN, LN, LN, 1, npost)
        smg.smg_set_precision(h, prec)
        if use_w:
            smg.smg_set_learned(h, w)

        def once():
            x.zero_()
            rc, it, res = smg.krylov_solve(h, "fpcg", b, x, TOL, 100)
            assert rc == smg.SMG_OK and res <= TOL, (rc, res)
            return it
        times, it = _timed(once, steps, 1, barrier, flush, stream)
        out[name] = {"s": statistics.mean(times), "iters": it}
        smg.smg_destroy(h)
    out["speedup_learned_vs_plain_10"] = out["plain_10_fp32"]["s"] / out["learned_10_fp32"]["s"]
    out["speedup_learned_vs_fp64"] = out["plain_10_fp64"]["s"] / out["learned_10_fp32"]["s"]
    return out


def run_batched(args):
    """64 uneven systems through one batched handle (setup outside the timed region)."""
    import torch

    from paper_1212_6680_gb300 import build as _build

    world, rank, local, dist = _dist_init()
    _build.build()
    from paper_1212_6680_gb300 import smg

    dims, b_np = batched_inputs()
    n_all = sum(b.size for b in b_np)
    bs = [torch.from_numpy(b.ravel().copy()).cuda() for b in b_np]
    xs = [torch.zeros_like(b) for b in bs]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    t0 = time.perf_counter()
    h = smg.smg_batched_setup(dims, npre=1, npost=0, prec="fp32")
    setup_s = time.perf_counter() - t0
    info0 = smg.smg_batched_info(h)

    def solve(host=None):
        for x in xs:
            x.zero_()
        if host is not None:
            bh, xh = host
            for d, hsrc in zip(bs, bh):
                d.copy_(hsrc, non_blocking=True)
        rc, its, rel = smg.smg_batched_solve(h, "fpcg", bs, xs, TOL, 100)
        if host is not None:
            for hdst, d in zip(xh, xs):
                hdst.copy_(d, non_blocking=True)
        return rc, its, rel

    for _ in range(args.warmup):
        solve()
    smg.smg_batched_set_profile(h, 1)
    smg.smg_batched_profile_read(h, 0)
    smg.smg_batched_profile_read(h, 1)
    la0 = smg.smg_batched_info(h)["launches"]
    times = []
    barrier()
    wall0 = time.perf_counter()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc, its, rel = solve()
            e1.record(stream)
            barrier()
            assert rc == smg.SMG_OK and (rel <= TOL).all(), (rc, rel.max())
            times.append(e0.elapsed_time(e1) / 1e3)
    wall = time.perf_counter() - wall0
    launches = smg.smg_batched_info(h)["launches"] - la0
    pl, pms, pbytes = smg.smg_batched_profile_read(h, 0)
    kl, kms, _ = smg.smg_batched_profile_read(h, 1)
    smg.smg_batched_set_profile(h, 0)
    t_step = statistics.mean(times)
    t_max = max_over_ranks(t_step, dist, "cuda")

    # end to end: pinned host inputs and outputs, copies inside the timed region
    bh = [torch.from_numpy(b.ravel().copy()).pin_memory() for b in b_np]
    xh = [torch.zeros(b.size, dtype=torch.float64).pin_memory() for b in b_np]
    te = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc, _, _ = solve(host=(bh, xh))
        e1.record(stream)
        barrier()
        assert rc == smg.SMG_OK
        te.append(e0.elapsed_time(e1) / 1e3)

    # the same 64 systems one after another through the single-system path (FP32 and FP64 cycles)
    seq = {}
    for prec in ("fp32", "fp64"):
        hs_ = []
        for i, (nx, ny, nz) in enumerate(dims):
            hh = smg.smg_setup(int(nx), int(ny), int(nz), 1, 0)
            smg.smg_set_precision(hh, prec)
            hs_.append(hh)
        for i, hh in enumerate(hs_):  # warm-up (first-use costs)
            xs[i].zero_()
            smg.krylov_solve(hh, "fpcg", bs[i], xs[i], TOL, 100)
        flush.zero_()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i, hh in enumerate(hs_):
            xs[i].zero_()
            rc1, _, r1 = smg.krylov_solve(hh, "fpcg", bs[i], xs[i], TOL, 100)
            assert rc1 == smg.SMG_OK and r1 <= TOL
        e1.record(stream)
        barrier()
        seq[prec] = e0.elapsed_time(e1) / 1e3
        for hh in hs_:
            smg.smg_destroy(hh)
    smg.smg_batched_destroy(h)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    peak, peak_kind = measured_peaks()
    achieved = (pbytes / 1e9) / (pms / 1e3) if pms > 0 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": None,
                "kernel": "persistent_vcycle_kernel<float,4> (every V-cycle step of every active system)",
                "launches": pl, "avg_launch_us": (pms * 1e3 / pl) if pl else None,
                "algorithmic_bytes_per_launch": (pbytes / pl) if pl else None,
                "krylov_avg_us_per_iteration": (kms * 1e3 / kl) if kl else None,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else
                "fallback 6.8 TB/s"}
    cpu = None
    if not args.no_cpu_baseline:
        v, its_o, raw = oracle_batched_sample(NSYS)
        cpu = {"value": v, "unit": "s", "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": f"oracle FPCG-SMG(1,0) solves of all 64 systems one after another (iterations "
                         f"{min(its_o)}-{max(its_o)}), {os.cpu_count() or 1} host cores (OpenMP)"}
    line = {
        "metric": METRIC, "value": t_max, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "nsys": NSYS, "unknowns": int(n_all), "variant": "fpcg",
                   "npre": 1, "npost": 0, "cycle_precision": "fp32", "iters_max": int(its.max()),
                   "iters_mean": float(its.mean()), "true_relres_max": float(rel.max()),
                   "unknowns_per_s": n_all / t_max, "setup_s": setup_s,
                   "schedule": {k: info0[k] for k in ("rows_per_lane", "threads", "blocks", "order", "tasks")},
                   "sequential_fp32_s": seq["fp32"], "sequential_fp64_s": seq["fp64"],
                   "speedup_vs_sequential_fp32": seq["fp32"] / t_step,
                   "speedup_vs_sequential_fp64": seq["fp64"] / t_step,
                   "l2": "256 MB buffer written before every timed solve",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline, "cpu_baseline": cpu,
        "e2e": {"value": statistics.mean(te), "unit": "s", "h2d_bytes_per_step": int(n_all) * 8,
                "d2h_bytes_per_step": int(n_all) * 8},
        "gpu_launches": launches, "clocks": clk.summary(), "wall_s_timed_region": wall,
    }
    print(json.dumps(line), flush=True)


def _dist_init(backend="nccl"):
    """(world, rank, local rank, torch.distributed or None) from the torchrun environment.  One
    process per GPU; the replicas share nothing but the barriers around the timed region and the
    max-over-ranks reduction of its duration."""
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        if backend == "nccl":
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    return world, rank, local, dist


def max_over_ranks(value, dist, device):
    """The largest of every rank's value: the job takes as long as its slowest replica."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _timed(fn, steps, warmup, barrier, flush, stream):
    """Per-step device seconds of fn() (L2 flushed before each), after `warmup` untimed calls."""
    import torch

    for _ in range(warmup):
        fn()
    out, times = None, []
    for _ in range(steps):
        flush.zero_()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        barrier()
        times.append(e0.elapsed_time(e1) / 1e3)
    return times, out


def closed_form_smallest(nx, ny, nz, m):
    """The m smallest eigenvalues of the 7-point Dirichlet Laplacian with unit spacing."""
    ev = [4 * np.sin(np.pi * np.arange(1, n + 1) / (2 * (n + 1))) ** 2 for n in (nx, ny, nz)]
    lam = (ev[2][:, None, None] + ev[1][None, :, None] + ev[0][None, None, :]).ravel()
    return np.sort(lam)[:m]


LOB_M = 16
LOB_WORKLOAD = ("LOBPCG-SMG(1,0): 16 smallest eigenpairs, 128^3 7-point Dirichlet Laplacian, Gaussian initial "
                "block, V-cycle FP32 applied to all 16 vectors per launch, FP64 Rayleigh-Ritz, tol 1e-8")


def run_lobpcg(args):
    import torch

    from paper_1212_6680_gb300 import build as _build
    from paper_1212_6680_gb300 import inputs

    world, rank, local, dist = _dist_init()
    _build.build()
    from paper_1212_6680_gb300 import smg

    n = NX * NY * NZ
    X0 = inputs.initial_block(NX, NY, NZ, LOB_M, seed=7)
    X0d = torch.from_numpy(np.ascontiguousarray(X0).ravel().copy()).cuda()
    X = torch.empty_like(X0d)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    ref = closed_form_smallest(NX, NY, NZ, LOB_M)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def arm(npost, prec, steps, warmup, profile=False):
        h = smg.smg_setup(NX, NY, NZ, 1, npost)
        smg.smg_set_precision(h, prec)
        res = {}

        def once():
            X.copy_(X0d)
            rc, it, lam = smg.lobpcg_solve(h, LOB_M, X, tol=TOL, maxit=200)
            assert rc == smg.SMG_OK, smg.smg_last_error()
            return it, lam
        if profile:
            for _ in range(warmup):
                once()
            smg.smg_set_option(h, smg.SMG_OPT_PROFILE, 1)
            smg.smg_profile_read(h, 0)
            l0 = smg.smg_launch_count(h)
            with ClockSampler(local) as clk:
                times, (it, lam) = _timed(once, steps, 0, barrier, flush, stream)
            res["launches"] = smg.smg_launch_count(h) - l0
            res["prof"] = smg.smg_profile_read(h, 0)
            res["clocks"] = clk.summary()
        else:
            times, (it, lam) = _timed(once, steps, warmup, barrier, flush, stream)
        smg.smg_destroy(h)
        err = float(np.max(np.abs(lam - ref) / ref))
        assert err <= 1e-10, err
        res.update({"s": statistics.mean(times), "iters": it, "max_rel_eig_err": err})
        return res

    main = arm(0, "fp32", args.steps, args.warmup, profile=True)
    k2 = max(1, min(args.steps, 2))
    a64 = arm(0, "fp64", k2, 1)
    a11 = arm(1, "fp32", k2, 1)
    # end to end: the initial block from pinned host memory, eigenvectors and values back
    Xh = torch.from_numpy(np.ascontiguousarray(X0).ravel().copy()).pin_memory()
    Xo = torch.empty(Xh.numel(), dtype=torch.float64).pin_memory()
    h = smg.smg_setup(NX, NY, NZ, 1, 0)
    smg.smg_set_precision(h, "fp32")

    def e2e_once():
        X.copy_(Xh, non_blocking=True)
        rc, it, lam = smg.lobpcg_solve(h, LOB_M, X, tol=TOL, maxit=200)
        Xo.copy_(X, non_blocking=True)
        return rc
    te, _ = _timed(e2e_once, max(1, min(args.steps, 2)), 1, barrier, flush, stream)
    smg.smg_destroy(h)
    t_step = main["s"]
    t_max = max_over_ranks(t_step, dist, "cuda")
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    peak, peak_kind = measured_peaks()
    pl, pms, pbytes = main["prof"]
    achieved = (pbytes / 1e9) / (pms / 1e3) if pms > 0 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": None,
                "kernel": "plane_lean_kernel<float,float,4,false> (finest level, 16 vectors per launch)",
                "launches": pl, "avg_launch_us": (pms * 1e3 / pl) if pl else None,
                "algorithmic_bytes_per_launch": (pbytes / pl) if pl else None,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"}
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        from oracle import lobpcg as olob

        oracle.build()
        oracle.set_threads(os.cpu_count() or 1)
        T = oracle.SMG(NX, NY, NZ, 1, 0)
        t0 = time.perf_counter()
        olob.lobpcg((NZ, NY, NX), np.ascontiguousarray(X0.T), T, tol=TOL, maxit=1)
        t1 = time.perf_counter() - t0
        cpu = {"value": t1 * max(main["iters"], 1), "unit": "s", "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": f"extrapolated: oracle LOBPCG set-up + 1 iteration at 128^3, m=16 ({t1:.1f} s), scaled by "
                         f"the GPU's {main['iters']} iterations, {os.cpu_count() or 1} host cores (OpenMP)"}
    line = {
        "metric": METRIC, "value": t_max, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": LOB_WORKLOAD, "grid": [NX, NY, NZ], "m": LOB_M, "npre": 1, "npost": 0,
                   "cycle_precision": "fp32", "iters": main["iters"],
                   "max_rel_eig_err_vs_closed_form": main["max_rel_eig_err"],
                   "fp64_cycle_s": a64["s"], "fp64_cycle_iters": a64["iters"],
                   "balanced_11_s": a11["s"], "balanced_11_iters": a11["iters"],
                   "l2": "256 MB buffer written before every timed solve",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline, "cpu_baseline": cpu,
        "e2e": {"value": statistics.mean(te), "unit": "s", "h2d_bytes_per_step": n * LOB_M * 8,
                "d2h_bytes_per_step": n * LOB_M * 8 + LOB_M * 8},
        "gpu_launches": main["launches"], "clocks": main["clocks"],
    }
    print(json.dumps(line), flush=True)


LN = 256
LEARNED_WORKLOAD = ("FPCG-SMG(1,0) with the learned post-correction, 256^3 7-point Dirichlet Laplacian, V-cycle "
                    "FP32, network BF16/FP32-accumulate, Krylov FP64, tol 1e-8; network trained on GPU on pairs "
                    "from 200 seeded solves with sides in {64..128}")


def oracle_learned_sample(w, iters):
    """Seconds of one oracle application of the learned preconditioner at 64^3, scaled to 256^3
    (x64 points) and to `iters` iterations; returns (scaled value, raw seconds)."""
    import oracle
    from paper_1212_6680_gb300 import inputs

    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    T = oracle.SMG(64, 64, 64, 1, 0)
    T.set_learned(np.asarray(w, dtype=np.float64))
    r = inputs.rhs(64, 64, 64, seed=0)
    t0 = time.perf_counter()
    T.apply(r)
    t1 = time.perf_counter() - t0
    return t1 * 64 * iters, t1


def run_learned(args):
    import torch

    from paper_1212_6680_gb300 import build as _build
    from paper_1212_6680_gb300 import inputs

    world, rank, local, dist = _dist_init()
    _build.build()
    from paper_1212_6680_gb300 import learned, smg

    w, tinfo = learned.train(nsys=200, lo=64, hi=128, epochs=4, lr=1e-3)
    n = LN ** 3
    b_np = inputs.rhs(LN, LN, LN, seed=0).ravel().copy()
    b = torch.from_numpy(b_np).cuda()
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def arm(npost, prec, use_w, steps, warmup, profile=False):
        h = smg.smg_setup(LN, LN, LN, 1, npost)
        smg.smg_set_precision(h, prec)
        if use_w:
            smg.smg_set_learned(h, w)

        def once():
            x.zero_()
            rc, it, res = smg.krylov_solve(h, "fpcg", b, x, TOL, 100)
            assert rc == smg.SMG_OK and res <= TOL, (rc, res)
            return it, res
        out = {}
        if profile:
            for _ in range(warmup):
                once()
            smg.smg_set_option(h, smg.SMG_OPT_PROFILE, 1)
            smg.smg_profile_read(h, 0)
            smg.smg_profile_read(h, 5)
            l0 = smg.smg_launch_count(h)
            with ClockSampler(local) as clk:
                times, (it, res) = _timed(once, steps, 0, barrier, flush, stream)
            out["launches"] = smg.smg_launch_count(h) - l0
            out["prof0"] = smg.smg_profile_read(h, 0)
            out["prof5"] = smg.smg_profile_read(h, 5)
            out["clocks"] = clk.summary()
        else:
            times, (it, res) = _timed(once, steps, warmup, barrier, flush, stream)
        if use_w:
            out["judge"] = smg.smg_learned_stats(h)
        smg.smg_destroy(h)
        out.update({"s": statistics.mean(times), "iters": it, "relres": res})
        return out

    main = arm(0, "fp32", True, args.steps, args.warmup, profile=True)
    k2 = max(1, min(args.steps, 3))
    plain = arm(0, "fp32", False, k2, 1)
    bal = arm(1, "fp32", False, k2, 1)
    f64 = arm(0, "fp64", False, k2, 1)
    # end to end through the C ABI with host buffers
    h = smg.smg_setup(LN, LN, LN, 1, 0)
    smg.smg_set_precision(h, "fp32")
    smg.smg_set_learned(h, w)
    bh = torch.from_numpy(b_np).pin_memory()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory()

    def e2e_once():
        xh.zero_()
        return smg.krylov_solve(h, "fpcg", bh.numpy(), xh.numpy(), TOL, 100)
    te, _ = _timed(e2e_once, k2, 1, barrier, flush, stream)
    smg.smg_destroy(h)
    t_max = max_over_ranks(main["s"], dist, "cuda")
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    peak, peak_kind = measured_peaks()
    l0n, l0ms, l0b = main["prof0"]
    achieved = (l0b / 1e9) / (l0ms / 1e3) if l0ms > 0 else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "traffic": None,
                "kernel": "plane_relax_kernel<float,float,8> (finest level of the 256^3 cycle)",
                "launches": l0n, "avg_launch_us": (l0ms * 1e3 / l0n) if l0n else None,
                "algorithmic_bytes_per_launch": (l0b / l0n) if l0n else None,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"}
    pl, pms, pflops = main["prof5"]
    bf16_peak = measured_bf16_peak()
    learned_region = {"launches": pl, "avg_us": (pms * 1e3 / pl) if pl else None,
                      "flops": (pflops / pl) if pl else None,
                      "achieved_tflops": ((pflops / 1e12) / (pms / 1e3)) if pms > 0 else None,
                      "bf16_tensor_peak_tflops": bf16_peak,
                      "note": "the whole correction: residual, layer 1 (CUDA cores), layer 2 (tcgen05), layer 3 "
                              "(CUDA cores), judge, update; flops of the three convolutions"}
    cpu = None
    if not args.no_cpu_baseline:
        v, t1 = oracle_learned_sample(w, main["iters"])
        cpu = {"value": v, "unit": "s", "cores": os.cpu_count() or 1, "kind": "oracle",
               "sample": f"extrapolated: one oracle application of the learned preconditioner at 64^3 ({t1:.1f} s), "
                         f"scaled by 64x the points and the GPU's {main['iters']} iterations (Krylov work not "
                         f"included), {os.cpu_count() or 1} host cores (OpenMP in the SMG cycle; the network's "
                         f"convolutions on one core)"}
    line = {
        "metric": METRIC, "value": t_max, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16+f32+f64", "data": "synthetic",
        "config": {"workload": LEARNED_WORKLOAD, "grid": [LN, LN, LN], "variant": "fpcg", "npre": 1, "npost": 0,
                   "iters": main["iters"], "true_relres": main["relres"], "judge_calls_accepted": main["judge"],
                   "plain_10_fp32_s": plain["s"], "plain_10_fp32_iters": plain["iters"],
                   "balanced_11_fp32_s": bal["s"], "balanced_11_fp32_iters": bal["iters"],
                   "plain_10_fp64_s": f64["s"], "plain_10_fp64_iters": f64["iters"],
                   "speedup_vs_fp64": f64["s"] / main["s"], "speedup_vs_plain_10": plain["s"] / main["s"],
                   "speedup_vs_balanced_11": bal["s"] / main["s"],
                   "learned_correction": learned_region,
                   "training": tinfo, "l2": "256 MB buffer written before every timed solve",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": roofline, "cpu_baseline": cpu,
        "e2e": {"value": statistics.mean(te), "unit": "s", "h2d_bytes_per_step": 2 * n * 8, "d2h_bytes_per_step": n * 8},
        "gpu_launches": main["launches"], "clocks": main["clocks"],
    }
    print(json.dumps(line), flush=True)


BRICK_NS = (10, 16, 20, 32, 48, 64, 80)
BRICK_WORKLOAD = ("the paper's 16n x n x n bricks (long in x), n = 10, 16, 20, 32, 48, 64, 80, 7-point Dirichlet "
                  "Laplacian; FPCG-SMG(1,0) with the FP32 and the FP64 cycle timed, iteration counts of PCG eq. (1), "
                  "FPCG eq. (2) and PSD with the (1,1) and (1,0) FP64 cycles, and figure 5's residual histories "
                  "((1,0) FP64 cycle) at n = 80; tol 1e-8")


def run_bricks(args):
    """The brick sweep of the paper's figures 4, 5 and 7 up to n = 80 (x-lines of 1280 rows, split
    over three warps from n = 33 on): the timed value is the FP32-cycle FPCG-SMG(1,0) solve of the
    largest brick."""
    import torch

    from paper_1212_6680_gb300 import build as _build
    from paper_1212_6680_gb300 import inputs

    world, rank, local, dist = _dist_init()
    _build.build()
    from paper_1212_6680_gb300 import smg

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    table = []
    main_t, main_launches, main_clk = None, 0, None
    for nb in BRICK_NS:
        nx, ny, nz = 16 * nb, nb, nb
        b = torch.from_numpy(inputs.rhs(nx, ny, nz, seed=0).ravel().copy()).cuda()
        x = torch.zeros_like(b)
        row = {"n": nb, "grid": [nx, ny, nz], "unknowns": nx * ny * nz}
        for npost in (1, 0):
            h = smg.smg_setup(nx, ny, nz, 1, npost)
            for v in ("pcg", "fpcg", "psd"):
                x.zero_()
                rc, it, rr = smg.krylov_solve(h, v, b, x, TOL, 40, check=False)
                row[f"{v}_{1}{npost}_iters"] = it if rc == smg.SMG_OK else f">40 (relres {rr:.1e})"
                if npost == 0 and nb == BRICK_NS[-1]:
                    row[f"{v}_10_history"] = [float(f"{v_:.3e}") for v_ in smg.smg_krylov_history(h)]
            smg.smg_destroy(h)
        for prec in ("fp32", "fp64"):
            h = smg.smg_setup(nx, ny, nz, 1, 0)
            smg.smg_set_precision(h, prec)
            last = prec == "fp32" and nb == BRICK_NS[-1]

            def once():
                x.zero_()
                rc, it, rr = smg.krylov_solve(h, "fpcg", b, x, TOL, 100)
                assert rc == smg.SMG_OK and rr <= TOL, (rc, rr)
                return it
            l0 = smg.smg_launch_count(h)
            if last:
                for _ in range(args.warmup):
                    once()
                l0 = smg.smg_launch_count(h)
                with ClockSampler(local) as clk:
                    times, it = _timed(once, args.steps, 0, barrier, flush, stream)
                main_t, main_launches, main_clk = statistics.mean(times), smg.smg_launch_count(h) - l0, clk.summary()
            else:
                times, it = _timed(once, max(1, min(args.steps, 3)), 1, barrier, flush, stream)
            row[f"fpcg_10_{prec}_s"] = statistics.mean(times)
            row[f"fpcg_10_{prec}_iters"] = it
            smg.smg_destroy(h)
        table.append(row)
    t_max = max_over_ranks(main_t, dist, "cuda")
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        import oracle

        oracle.build()
        nb = BRICK_NS[-1]
        cores = os.cpu_count() or 1
        oracle.set_threads(cores)
        bo = inputs.rhs(16 * nb, nb, nb, seed=0)
        t0 = time.perf_counter()
        out = oracle.krylov(bo, "fpcg", oracle.SMG(16 * nb, nb, nb, 1, 0), tol=TOL, maxit=100)
        tc = time.perf_counter() - t0
        assert out["status"] == 0
        cpu = {"value": tc, "unit": "s", "cores": cores, "kind": "oracle",
               "sample": f"one full FPCG-SMG(1,0) solve of the n = {nb} brick in FP64 ({out['iters']} iterations, "
                         f"set-up included) on {cores} host cores (OpenMP)"}
    line = {
        "metric": METRIC, "value": t_max, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": BRICK_WORKLOAD, "timed": f"FPCG-SMG(1,0), FP32 cycle, brick n = {BRICK_NS[-1]}",
                   "bricks": table, "l2": "256 MB buffer written before every timed solve",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": None, "cpu_baseline": cpu, "e2e": None,
        "gpu_launches": main_launches, "clocks": main_clk,
    }
    print(json.dumps(line), flush=True)


CG_WORKLOAD = ("no preconditioner (T = I) at 128^3, 7-point Dirichlet Laplacian: CG by eq. (1), CG by eq. (2) "
               "(the flexible form's extra vector r_k - r_(k-1)) and steepest descent; FP64; tol 1e-8")


def run_cg(args):
    """Section 2 / figures 1-2 on the GPU path: the cost per iteration of the flexible form's extra
    vector without preconditioning, and steepest descent against CG.  The timed value is the
    eq. (2) CG solve to 1e-8."""
    import torch

    from paper_1212_6680_gb300 import build as _build
    from paper_1212_6680_gb300 import inputs

    world, rank, local, dist = _dist_init()
    _build.build()
    from paper_1212_6680_gb300 import smg

    b = torch.from_numpy(inputs.rhs(NX, NY, NZ, seed=0).ravel().copy()).cuda()
    x = torch.zeros_like(b)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    h = smg.smg_setup(NX, NY, NZ, 1, 0)
    smg.smg_set_option(h, smg.SMG_OPT_PRECOND, 0)
    res = {}
    main_t, main_launches, main_clk = None, 0, None
    for v, maxit in (("fpcg", 5000), ("pcg", 5000), ("psd", 0)):
        if v == "psd":
            maxit = res["fpcg"]["iters"]  # steepest descent given CG's iteration count

        def once():
            x.zero_()
            rc, it, rr = smg.krylov_solve(h, v, b, x, TOL, maxit, check=False)
            assert rc in (smg.SMG_OK, smg.SMG_ERR_NOCONV), rc
            return rc, it, rr
        if v == "fpcg":
            for _ in range(args.warmup):
                once()
            l0 = smg.smg_launch_count(h)
            with ClockSampler(local) as clk:
                times, (rc, it, rr) = _timed(once, args.steps, 0, barrier, flush, stream)
            main_t, main_launches, main_clk = statistics.mean(times), smg.smg_launch_count(h) - l0, clk.summary()
            assert rc == smg.SMG_OK and rr <= TOL
        else:
            times, (rc, it, rr) = _timed(once, max(1, min(args.steps, 3)), 1, barrier, flush, stream)
        t = statistics.mean(times)
        res[v] = {"s": t, "iters": it, "relres": rr, "converged": rc == smg.SMG_OK, "ms_per_iter": t * 1e3 / max(it, 1)}
    smg.smg_destroy(h)
    t_max = max_over_ranks(main_t, dist, "cuda")
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": t_max, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": CG_WORKLOAD, "grid": [NX, NY, NZ], "timed": "CG by eq. (2), no preconditioner",
                   "cg_eq2": res["fpcg"], "cg_eq1": res["pcg"], "steepest_descent": res["psd"],
                   "extra_vector_cost": res["fpcg"]["ms_per_iter"] / res["pcg"]["ms_per_iter"] - 1.0,
                   "l2": "256 MB buffer written before every timed solve",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": None, "cpu_baseline": None, "e2e": None,
        "gpu_launches": main_launches, "clocks": main_clk,
    }
    print(json.dumps(line), flush=True)


LB_NS = (10, 20, 40, 60, 80, 100, 120)
LB_WORKLOAD = ("LOBPCG-SMG, one eigenpair, the paper's 4n x 2n x 2n bricks (n = 10..120), FP32 V-cycle with (1,1) "
               "and (1,0), Gaussian initial vector, tol 1e-8, eigenvalue against the closed form")


def run_lobpcg_bricks(args):
    """Figures 8-9 on the GPU path: iterations and time of one-eigenpair LOBPCG with and without
    post-smoothing.  The timed value is the (1,0) solve of the largest brick."""
    import torch

    from paper_1212_6680_gb300 import build as _build
    from paper_1212_6680_gb300 import inputs

    world, rank, local, dist = _dist_init()
    _build.build()
    from paper_1212_6680_gb300 import smg

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    table = []
    main_t, main_launches, main_clk = None, 0, None
    for nb in LB_NS:
        nx, ny, nz = 4 * nb, 2 * nb, 2 * nb
        X0 = torch.from_numpy(np.ascontiguousarray(inputs.initial_block(nx, ny, nz, 1, seed=7)).ravel().copy()).cuda()
        X = torch.empty_like(X0)
        ref = float(closed_form_smallest(nx, ny, nz, 1)[0])
        row = {"n": nb, "grid": [nx, ny, nz], "unknowns": nx * ny * nz}
        for npost in (1, 0):
            h = smg.smg_setup(nx, ny, nz, 1, npost)
            smg.smg_set_precision(h, "fp32")
            last = npost == 0 and nb == LB_NS[-1]

            def once():
                X.copy_(X0)
                rc, it, lam = smg.lobpcg_solve(h, 1, X, tol=TOL, maxit=200)
                assert rc == smg.SMG_OK, smg.smg_last_error()
                return it, float(lam[0])
            if last:
                for _ in range(args.warmup):
                    once()
                l0 = smg.smg_launch_count(h)
                with ClockSampler(local) as clk:
                    times, (it, lam) = _timed(once, args.steps, 0, barrier, flush, stream)
                main_t, main_launches, main_clk = statistics.mean(times), smg.smg_launch_count(h) - l0, clk.summary()
            else:
                times, (it, lam) = _timed(once, max(1, min(args.steps, 3)), 1, barrier, flush, stream)
            assert abs(lam - ref) <= 1e-10 * ref, (lam, ref)
            smg.smg_destroy(h)
            row[f"v1{npost}_s"] = statistics.mean(times)
            row[f"v1{npost}_iters"] = it
        row["iters_ratio_10_over_11"] = row["v10_iters"] / row["v11_iters"]
        row["time_ratio_10_over_11"] = row["v10_s"] / row["v11_s"]
        table.append(row)
    t_max = max_over_ranks(main_t, dist, "cuda")
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": t_max, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": LB_WORKLOAD, "timed": f"(1,0) solve, brick n = {LB_NS[-1]}", "bricks": table,
                   "l2": "256 MB buffer written before every timed solve",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": None, "cpu_baseline": None, "e2e": None,
        "gpu_launches": main_launches, "clocks": main_clk,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched64":
        run_batched(args)
    elif args.workload == "lobpcg128":
        run_lobpcg(args)
    elif args.workload == "learned256":
        run_learned(args)
    elif args.workload == "bricks":
        run_bricks(args)
    elif args.workload == "cg128":
        run_cg(args)
    elif args.workload == "lobpcg_bricks":
        run_lobpcg_bricks(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
