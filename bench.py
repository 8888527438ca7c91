#!/usr/bin/env python
"""Throughput of the open-boundary RPY mobility hot path on one GB300.

One step = one pass of the hot path over one suspension:
  lm_set_positions -> lm_mdot (M [F; T], all four blocks) -> lm_sqrt_mdot
  (Lanczos M^{1/2} W at the workload's tolerance).
Metric: RPY pair-interactions per second, counting N^2 ordered pairs for
every application of M (the product and each Lanczos iteration), inputs
resident in HBM, L2 flushed (256 MB write) before every step.

Default workload: N = 32768 spheres uniform in a cube at volume fraction
0.2, a = 1, eta = 1, translation + rotation, FP32 pair arithmetic with
compensated sums, FP64 Lanczos at tol 1e-5 (seeded synthetic inputs).
"--workload melt" runs 1024 chains x 512 beads (N = 524288), tol 1e-3.

--impl reference times the FP64 CPU oracle (the only reference that exists:
the paper ships no code) on the same metric over a bounded row sample.
Multi-GPU: replicas only (the product does not shard); one process per GPU
under torchrun, value = pairs of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "RPY pair-interactions/s (N^2 ordered pairs per application of M, incl. Lanczos)"
UNIT = "pair-interactions/s"
FP32_LANES_PER_SM = 128
RECIPE_MAX_SM_MHZ = 2070.0
PAIR_KERNEL_SRCS = [os.path.join(ROOT, "paper_2510_02135_gb300", "csrc", f)
                    for f in ("pair_kernels.cu", "pair_common.cuh")]


def pair_kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in PAIR_KERNEL_SRCS:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def workload_spec(name: str):
    from paper_2510_02135_gb300 import inputs as I

    if name == "rpy6":
        c = I.RPY6_FP32_N32768
        s = I.cube_suspension(c["seed"], c["n"], c["phi"], c["a"], angular=True, fp32=True)
        desc = (f"rpy6_fp32_n32768: N={c['n']} spheres uniform in a cube, phi={c['phi']}, a={c['a']}, "
                f"eta={c['eta']}, forces+torques, FP32 compensated pairs, FP64 Lanczos tol {c['tol']}")
        return s, c["eta"], c["a"], c["tol"], desc
    if name == "melt":
        c = I.MELT_N524288
        s = I.polymer_melt(c["seed"], c["n_chains"], c["beads"], c["bond"], c["sigma"], c["phi"], c["a"])
        desc = (f"melt_n524288: {c['n_chains']} chains x {c['beads']} beads, bond {c['bond']}a, "
                f"angle jitter {c['sigma']} rad, phi={c['phi']}, forces+torques, FP32 compensated pairs, "
                f"FP64 Lanczos tol {c['tol']}")
        return s, c["eta"], c["a"], c["tol"], desc
    raise SystemExit(f"unknown workload {name}")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def oracle_pairs_per_s(pos, F, T, a, eta, budget_s: float):
    """Time the FP64 oracle direct sum on a row sample sized to ~budget_s."""
    import oracle

    n = pos.shape[0]
    rng = np.random.default_rng(0)
    rows = rng.choice(n, min(n, 32), replace=False)
    t0 = time.perf_counter()
    oracle.mdot(pos, F, T, a, eta, T is not None, rows=rows)
    t = time.perf_counter() - t0
    nrows = int(min(n, max(32, len(rows) * budget_s / max(t, 1e-6))))
    rows = rng.choice(n, nrows, replace=False)
    t0 = time.perf_counter()
    oracle.mdot(pos, F, T, a, eta, T is not None, rows=rows)
    t = time.perf_counter() - t0
    return nrows * n / t, nrows, t, oracle.num_threads()


def measured_hbm_gbs():
    """Copy bandwidth measured on this GPU pool (generated file), else the
    recipe's fallback figure."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def profile_traffic():
    """DRAM bytes per pair-kernel launch from the committed ncu summary, if it
    was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "pair_kernel_rpy6_n32768.txt")
    if not os.path.exists(path):
        return None
    src_hash = pair_kernel_source_hash()
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != src_hash:
        return None
    try:
        return float(vals["dram_bytes_per_launch"].split()[0])
    except (KeyError, ValueError, IndexError):
        return None


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    s, eta, a, tol, desc = workload_spec(args.workload)
    import oracle

    oracle.build()
    n = s.pos.shape[0]
    for _ in range(args.warmup):
        oracle_pairs_per_s(s.pos, s.F, s.T, a, eta, budget_s=0.5)
    vals, rows_used, secs = [], 0, 0.0
    for _ in range(args.steps):
        v, nr, t, cores = oracle_pairs_per_s(s.pos, s.F, s.T, a, eta, budget_s=args.ref_step_s)
        vals.append(v)
        rows_used += nr
        secs += t
    value = rows_used * n / secs
    sample = (f"each step: FP64 oracle direct sum of M [F; T] (all four blocks) for a random sample of rows "
              f"(~{args.ref_step_s:.0f} s of CPU work, {rows_used // max(1, args.steps)} rows x {n} columns per step)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["rpy6", "melt", "adjoint", "bd256", "wall", "rollers"], default="rpy6")
    ap.add_argument("--jacobi", action="store_true", help="rollers: Jacobi-preconditioned Lanczos")
    ap.add_argument("--adjoint-config", default=None,
                    help="adjoint workload: threads,ilp,splits,packed of the adjoint kernel instead of autotuning")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default pair-kernel configuration")
    ap.add_argument("--pair-config", default=None,
                    help="threads,ilp,splits,packed: use this pair-kernel configuration instead of autotuning "
                         "(profiling runs: under a profiler the autotuner's timings are not representative)")
    ap.add_argument("--cpu-budget", type=float, default=12.0, help="seconds of oracle CPU work for cpu_baseline")
    ap.add_argument("--ref-step-s", type=float, default=3.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.workload == "adjoint":
        return run_adjoint(args, ws, rank, local)
    if args.workload == "bd256":
        return run_bd(args, ws, rank, local)
    if args.workload == "wall":
        return run_wall(args, ws, rank, local)
    if args.workload == "rollers":
        return run_rollers(args, ws, rank, local)

    import torch

    from paper_2510_02135_gb300 import _build, lm

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
    _build.build()
    s_, eta, a, tol, desc = workload_spec(args.workload)
    n = s_.pos.shape[0]
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    pos, F, T, W = dev(s_.pos), dev(s_.F), dev(s_.T), dev(s_.W)
    lin = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    ang = torch.empty_like(lin)
    lin2 = torch.empty_like(lin)
    ang2 = torch.empty_like(lin)
    solver = lm.lm_create(eta, a, True, lm.LM_FP32C, cuda_stream=torch.cuda.current_stream().cuda_stream)
    lm.lm_set_positions(solver, pos)
    if args.pair_config:
        t_, i_, s_p, p_ = (int(v) for v in args.pair_config.split(","))
        lm.lm_set_pair_config(solver, t_, i_, s_p, p_)
    elif not args.no_autotune:
        lm.lm_autotune(solver, reps=2)
    cfg = lm.lm_get_pair_config(solver)
    iters = []

    def step():
        lm.lm_set_positions(solver, pos)
        lm.lm_mdot(solver, F, T, lin, ang)
        _, _, it = lm.lm_sqrt_mdot(solver, W, tol=tol, max_iter=200, lin_out=lin2, ang_out=ang2)
        iters.append(it)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    iters.clear()
    sampler = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    lm.lm_profile_read(solver, reset=True)
    lm.lm_profile_enable(solver, True)
    sampler.start()
    launches0 = lm.lm_launch_count()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall0
    launches = lm.lm_launch_count() - launches0
    clocks = sampler.stop()
    lm.lm_profile_enable(solver, False)
    prof = lm.lm_profile_read(solver, reset=True)
    step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    total_ms = float(sum(step_ms))
    pairs = float(n) * float(n) * float(sum(1 + it for it in iters))
    total_ms_max, pairs_all = _reduce(dist, total_ms, pairs)
    value = pairs_all / (total_ms_max / 1e3)

    # e2e: the same step through host (pinned) buffers, copies inside the timed region
    pos_h = torch.from_numpy(s_.pos).pin_memory()
    F_h = torch.from_numpy(s_.F).pin_memory()
    T_h = torch.from_numpy(s_.T).pin_memory()
    W_h = torch.from_numpy(s_.W).pin_memory()
    outs_h = [torch.empty((n, 3), dtype=torch.float32).pin_memory() for _ in range(4)]
    e2e_steps = max(3, min(args.steps, 10))
    e2e_iters = []

    def step_host():
        lm.lm_set_positions(solver, pos_h)
        lm.lm_mdot(solver, F_h, T_h, outs_h[0], outs_h[1])
        _, _, it = lm.lm_sqrt_mdot(solver, W_h, tol=tol, max_iter=200, lin_out=outs_h[2], ang_out=outs_h[3])
        e2e_iters.append(it)

    step_host()
    e2e_iters.clear()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step_host()
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    e2e_pairs = float(n) * float(n) * float(sum(1 + it for it in e2e_iters))
    t_e2e, e2e_pairs = _reduce(dist, t_e2e, e2e_pairs)
    e2e_value = e2e_pairs / t_e2e
    h2d = n * 3 * 4 * 3 + W_h.numel() * 8
    d2h = n * 3 * 4 * 4

    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    peak = sms * FP32_LANES_PER_SM * 2 * RECIPE_MAX_SM_MHZ * 1e6 / 1e12
    achieved = prof["pair_flops"] / (prof["pair_ms"] / 1e3) / 1e12 if prof["pair_ms"] > 0 else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": profile_traffic(),
                "kernel": ("rpy_mdot_x2_kernel (forward pair kernel, packed FP32, all four blocks)" if cfg["packed"]
                           else "rpy_mdot_kernel (forward pair kernel, scalar FP32, all four blocks)"),
                "flops_per_pair": 86, "pair_launches": prof["pair_launches"],
                "pair_kernel_ms_avg": prof["pair_ms"] / max(1, prof["pair_launches"]),
                "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {RECIPE_MAX_SM_MHZ:.0f} MHz "
                              f"(recipe max SM clock; FP32 FMA peak)"}
    if clocks and achieved:
        roofline["frac_at_sampled_clock"] = achieved / (peak * clocks["sm_mhz"] / RECIPE_MAX_SM_MHZ)
    # the Lanczos vector kernels of every timed iteration (HBM-bound FP64 streams)
    hbm = measured_hbm_gbs()
    vec_gbs = prof["vector_bytes"] / (prof["vector_ms"] / 1e3) / 1e9 if prof["vector_ms"] > 0 else None
    vec_bytes_it = prof["vector_bytes"] / max(1, prof["vector_iterations"])
    lanczos_vectors = {
        "bound": "hbm", "achieved": vec_gbs, "peak": hbm, "unit": "GB/s",
        "frac": (vec_gbs / hbm) if (vec_gbs and hbm) else None,
        "iterations": prof["vector_iterations"], "ms_per_iteration": prof["vector_ms"] / max(1, prof["vector_iterations"]),
        "share_of_step": prof["vector_ms"] / max(1e-9, total_ms),
        "bytes_per_iteration_mean": vec_bytes_it,
        "bytes_rule": "FP64 vectors of n=6N: alpha 2, three-term update 4, each Gram-Schmidt pass 2k+5 at iteration k",
        "note": (f"basis of {n * 6 * 8 / 2**20:.1f} MB per vector; it stays in the 129 MB L2 for the first "
                 f"{int(126e6 // (n * 6 * 8))} iterations of a step, so early iterations can read faster than HBM"),
        "peak_basis": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "dtype_detail": "FP32 pair arithmetic with compensated (TwoSum) accumulation; FP64 Lanczos vectors",
            "data": "synthetic (seeded; shapes of the paper's random-cube benchmark)",
            "config": {"workload": desc, "N": n, "lanczos_iterations_mean": float(np.mean(iters)),
                       "sqrt_per_s": args.steps / (total_ms_max / 1e3),
                       "l2": "flushed by a 256 MB device write before every step (outside the step events)",
                       "pair_config": cfg, "parallelism": f"replicas x{ws}", "wall_s_timed": t_wall},
            "roofline": roofline, "lanczos_vectors": lanczos_vectors,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps, "api": "lm_set_positions/lm_mdot/lm_sqrt_mdot with pinned host buffers"},
            "gpu_launches": launches, "clocks": clocks}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, nrows, t, cores = oracle_pairs_per_s(s_.pos, s_.F, s_.T, a, eta, budget_s=args.cpu_budget)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"FP64 oracle direct sum of M [F; T] for {nrows} random rows x {n} "
                                          f"columns ({t:.1f} s); the Lanczos cost per pair is the same product"}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _dist_init(ws, local):
    import torch

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
        return dist
    return None


def _reduce(dist, t_ms, units):
    """(max time over ranks, sum of units over ranks): the job's time is the
    slowest rank's and its work is every rank's (replicas, weak scaling).
    Runs on the GPU with NCCL and on the CPU with gloo."""
    if dist is None:
        return t_ms, units
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([t_ms, units], dtype=torch.float64, device=dev)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


def run_adjoint(args, ws, rank, local):
    """Forward product and fused adjoint (L = <G, M(X) F>) at N = 65536,
    translation only, FP32: one step = lm_set_positions + lm_mdot +
    lm_mdot_backward (dL/dX and dL/dF); pairs counted N^2 per launch."""
    import torch

    from paper_2510_02135_gb300 import _build, inputs as I, lm

    dist = _dist_init(ws, local)
    _build.build()
    c = I.ADJOINT_N65536
    s_ = I.cube_suspension(c["seed"], c["n"], c["phi"], c["a"], angular=False, fp32=True)
    n = c["n"]
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    pos, F, G = dev(s_.pos), dev(s_.F), dev(s_.G)
    u = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    solver = lm.lm_create(c["eta"], c["a"], False, lm.LM_FP32C, cuda_stream=torch.cuda.current_stream().cuda_stream)
    lm.lm_set_positions(solver, pos)
    if args.pair_config:
        t_, i_, s_p, p_ = (int(v) for v in args.pair_config.split(","))
        lm.lm_set_pair_config(solver, t_, i_, s_p, p_)
    elif not args.no_autotune:
        lm.lm_autotune(solver, reps=2)
    if args.adjoint_config:
        t_, i_, s_p, p_ = (int(v) for v in args.adjoint_config.split(","))
        lm.lm_set_adjoint_config(solver, t_, i_, s_p, p_)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]

    def step(e=None):
        lm.lm_set_positions(solver, pos)
        if e:
            e[0].record(stream)
        lm.lm_mdot(solver, F, None, u, None)
        if e:
            e[1].record(stream)
        lm.lm_mdot_backward(solver, F, None, G, None)
        if e:
            e[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = lm.lm_launch_count()
    for k in range(args.steps):
        flush.zero_()
        step(ev[k])
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    launches = lm.lm_launch_count() - launches0
    fwd = [e[0].elapsed_time(e[1]) for e in ev]
    bwd = [e[1].elapsed_time(e[2]) for e in ev]
    total = float(sum(fwd) + sum(bwd))
    tmax, pairs = _reduce(dist, total, 2.0 * n * n * args.steps)
    props = torch.cuda.get_device_properties(local)
    peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * RECIPE_MAX_SM_MHZ * 1e6 / 1e12
    fwd_ms = float(np.mean(fwd))
    achieved = 35.0 * n * n / (fwd_ms / 1e3) / 1e12
    line = {"metric": METRIC, "value": pairs / (tmax / 1e3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
            "config": {"workload": f"adjoint_n65536: N={n}, phi={c['phi']}, translation only, FP32 compensated; "
                                   f"step = lm_mdot + lm_mdot_backward (dX, dF)",
                       "forward_ms": fwd_ms, "backward_ms": float(np.mean(bwd)),
                       "backward_over_forward": float(np.mean(bwd)) / fwd_ms,
                       "pair_config": lm.lm_get_pair_config(solver),
                       "adjoint_config": lm.lm_get_adjoint_config(solver),
                       "l2": "flushed by a 256 MB device write before every step"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "forward pair kernel (%s, translation, 35 flops/pair)"
                                   % ("packed" if lm.lm_get_pair_config(solver)["packed"] else "scalar")},
            "gpu_launches": launches, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# Algorithmic flops of one ordered pair above a single wall, translation
# blocks (FMA = 2, counted from the formulas as the kernel evaluates them):
# the free-space far-field pair (35) plus the wall part (96); the library's
# profile counters use the same figure.
WALL_FLOPS_PER_PAIR_TT = 131


def run_wall(args, ws, rank, local):
    """Mobility product above a single no-slip wall (the paper's "bottom
    wall" benchmark shape): N = 32768 spheres uniform in a cube on the wall at
    number density 0.1 / a^3, forces only, FP32.  One step = lm_set_positions
    + lm_mdot; pairs counted N^2 per product."""
    import torch

    from paper_2510_02135_gb300 import _build, inputs as I, lm

    dist = _dist_init(ws, local)
    _build.build()
    c = I.WALL_N32768
    s_ = I.wall_suspension(c["seed"], c["n"], c["rho"], c["a"], angular=False, fp32=True)
    n = c["n"]
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    pos, F = dev(s_.pos), dev(s_.F)
    u = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    solver = lm.lm_create(c["eta"], c["a"], False, lm.LM_FP32C, periodicity=("open", "open", "single_wall"),
                          cuda_stream=torch.cuda.current_stream().cuda_stream)
    lm.lm_set_positions(solver, pos)
    if args.pair_config:
        t_, i_, s_p, p_ = (int(v) for v in args.pair_config.split(","))
        lm.lm_set_pair_config(solver, t_, i_, s_p, p_)
    elif not args.no_autotune:
        lm.lm_autotune(solver, reps=2)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]

    def step():
        lm.lm_set_positions(solver, pos)
        lm.lm_mdot(solver, F, None, u, None)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    lm.lm_profile_read(solver, reset=True)
    lm.lm_profile_enable(solver, True)
    sampler.start()
    launches0 = lm.lm_launch_count()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    launches = lm.lm_launch_count() - launches0
    lm.lm_profile_enable(solver, False)
    prof = lm.lm_profile_read(solver, reset=True)
    total = float(sum(e0.elapsed_time(e1) for e0, e1 in ev))
    tmax, pairs = _reduce(dist, total, float(n) * n * args.steps)
    props = torch.cuda.get_device_properties(local)
    peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * RECIPE_MAX_SM_MHZ * 1e6 / 1e12
    kern_ms = prof["pair_ms"] / max(1, prof["pair_launches"])
    achieved = prof["pair_flops"] / (prof["pair_ms"] / 1e3) / 1e12
    line = {"metric": METRIC, "value": pairs / (tmax / 1e3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
            "config": {"workload": f"wall_n32768: N={n} spheres uniform in a cube resting on a no-slip wall, "
                                   f"number density {c['rho']}/a^3, forces only, FP32 compensated; "
                                   f"step = lm_set_positions + lm_mdot",
                       "pair_config": lm.lm_get_pair_config(solver),
                       "l2": "flushed by a 256 MB device write before every step"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "single-wall pair kernel (%s, translation, %d flops/pair)"
                                   % ("packed" if lm.lm_get_pair_config(solver)["packed"] else "scalar",
                                      WALL_FLOPS_PER_PAIR_TT),
                         "pair_kernel_ms_avg": kern_ms},
            "gpu_launches": launches, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_rollers(args, ws, rank, local):
    """The active-roller example (Sec. 5.1) as a step of the library: soft
    steric forces (pairs and wall) + gravity, a constant torque about y, and
    one stochastic Adams-Bashforth step (mobility product, one RFD sample of
    the thermal drift = two products, Lanczos square root at tol 1e-3) for
    N = 32768 spheres above a no-slip wall, FP32, all blocks.  Pairs counted:
    N^2 per application of M (the product, the two RFD products and every
    Lanczos iteration)."""
    import torch

    from paper_2510_02135_gb300 import _build, inputs as I, lm

    dist = _dist_init(ws, local)
    _build.build()
    c = I.ROLLERS_N32768
    n, a, eta, kT = c["n"], c["a"], c["eta"], c["kT"]
    pos0 = torch.from_numpy(I.roller_monolayer(c["seed"], n, a, c["area_fraction"])).cuda()
    solver = lm.lm_create(eta, a, True, lm.LM_FP32C, periodicity=("open", "open", "single_wall"),
                          cuda_stream=torch.cuda.current_stream().cuda_stream)
    lm.lm_set_positions(solver, pos0)
    if args.pair_config:
        t_, i_, s_p, p_ = (int(v) for v in args.pair_config.split(","))
        lm.lm_set_pair_config(solver, t_, i_, s_p, p_)
    elif not args.no_autotune:
        lm.lm_autotune(solver, reps=2)
    if args.jacobi:
        lm.lm_set_sqrt_preconditioner(solver, 1)
    mg = kT / ((c["h_g"] - 1.0) * a)
    T = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    T[:, 1] = 8 * np.pi * eta * a ** 3 * c["omega"]
    hist = torch.zeros(6 * n, dtype=torch.float64, device="cuda")
    X = pos0.clone()
    stream = torch.cuda.current_stream()
    state = {"k": 0}
    iters = []

    def step(timed=False):
        F = lm.lm_soft_repulsion(solver, 4 * kT, 0.1 * a, 2 * a, a, like=X)
        F[:, 2] -= mg
        Xn, it = lm.lm_ab_step(solver, F, T, hist, state["k"] == 0, kT, c["dt"], seed=state["k"], tol=c["tol"],
                               max_iter=200, pos_out=X)
        state["k"] += 1
        if timed:
            iters.append(it)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler.start()
    launches0 = lm.lm_launch_count()
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        step(timed=True)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    launches = lm.lm_launch_count() - launches0
    total = float(sum(e0.elapsed_time(e1) for e0, e1 in evs))
    pairs = float(n) * n * float(sum(3 + it for it in iters))
    tmax, pairs_all = _reduce(dist, total, pairs)
    line = {"metric": METRIC, "value": pairs_all / (tmax / 1e3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
            "config": {"workload": f"rollers_n32768: N={n} spheres of radius {a} above a no-slip wall, soft steric "
                                   f"repulsion + gravity + torque, one stochastic Adams-Bashforth step per bench step "
                                   f"(product, RFD drift, Lanczos tol {c['tol']}), FP32 pairs, all blocks",
                       "lanczos_iterations_mean": float(np.mean(iters)),
                       "preconditioner": "jacobi" if args.jacobi else "none",
                       "pair_config": lm.lm_get_pair_config(solver),
                       "l2": "flushed by a 256 MB device write before every step (outside the step events)"},
            "gpu_launches": launches, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_bd(args, ws, rank, local):
    """Batched Brownian dynamics: 256 suspensions (N log-uniform in [64, 4096],
    phi uniform in [0.05, 0.3]), 10 Euler-Maruyama steps per bench step in one
    persistent cooperative launch captured in a CUDA graph, Lanczos tol 1e-4.
    Pairs counted: sum_s N_s^2 per Lanczos iteration of system s.  Also times
    one BD step done with per-system library calls, for the speed-up factor."""
    import torch

    from paper_2510_02135_gb300 import _build, inputs as I, lm

    dist = _dist_init(ws, local)
    _build.build()
    c = I.BATCH_BD_256
    b_ = I.batch_suspensions(c["seed"], c["S"], c["nmin"], c["nmax"], c["phi_lo"], c["phi_hi"], c["a"])
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    b = lm.lm_batch_create(b_.offsets, c["eta"], c["a"], max_iter=64,
                           cuda_stream=torch.cuda.current_stream().cuda_stream)
    lm.lm_batch_set_positions(b, dev(b_.pos))
    tiling = lm.lm_batch_autotune(b) if not args.no_autotune else {"threads": 128, "ilp": 1}
    nsub = 10
    sizes2 = b_.sizes.astype(np.float64) ** 2
    step_no = [0]

    def step():
        its = lm.lm_batch_bd_run(b, c["kT"], c["dt"], c["k_trap"], nsub, step0=step_no[0], seed=c["seed"],
                                 tol=c["tol"], use_graph=True)
        step_no[0] += nsub
        return its

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = lm.lm_launch_count()
    t0 = time.perf_counter()
    pairs = 0.0
    iters = []
    for _ in range(args.steps):
        its = step()
        pairs += float((sizes2 * its).sum())
        iters.append(its.sum() / (b.S * nsub))
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t = (time.perf_counter() - t0) * 1e3
    clocks = sampler.stop()
    launches = lm.lm_launch_count() - launches0
    tmax, pairs_all = _reduce(dist, t, pairs)
    # one BD step with per-system calls (same noise streams and tolerance): one
    # solver per system with its buffers created beforehand and warmed up by
    # one untimed step, so the timed step holds only the per-system calls
    t_loop = None
    if rank == 0:
        x = lm.lm_batch_get_positions(b, like=dev(b_.pos))
        sq = float(np.sqrt(2 * c["kT"] * c["dt"]))
        solvers, bufs = [], []
        for s in range(b.S):
            o0, o1 = int(b_.offsets[s]), int(b_.offsets[s + 1])
            solvers.append(lm.lm_create(c["eta"], c["a"], False, lm.LM_FP32C))
            ns = o1 - o0
            bufs.append((torch.empty(3 * ns, dtype=torch.float64, device="cuda"),
                         torch.empty((ns, 3), dtype=torch.float32, device="cuda"),
                         torch.empty((ns, 3), dtype=torch.float32, device="cuda"),
                         torch.empty((ns, 3), dtype=torch.float32, device="cuda")))

        def per_system_step(xx, step):
            for s in range(b.S):
                o0, o1 = int(b_.offsets[s]), int(b_.offsets[s + 1])
                sv = solvers[s]
                W, Fs, uu, y = bufs[s]
                xs = xx[o0:o1]
                lm.lm_set_positions(sv, xs)
                torch.mul(xs, -c["k_trap"], out=Fs)
                lm.lm_mdot(sv, Fs, None, uu, None)
                lm.lm_philox_normals(c["seed"], (step << 32) | s, W)
                lm.lm_sqrt_mdot(sv, W, tol=c["tol"], max_iter=64, prefactor=sq, lin_out=y)
                xx[o0:o1] = xs + c["dt"] * uu + y

        per_system_step(x.clone(), step_no[0])      # warm-up: allocations, autotuning-free defaults
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        per_system_step(x, step_no[0])
        torch.cuda.synchronize()
        t_loop = time.perf_counter() - t1
    ms_bd_step = tmax / (args.steps * nsub)
    line = {"metric": METRIC, "value": pairs_all / (tmax / 1e3), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "dtype_detail": "FP32 pairs (compensated), FP64 Lanczos",
            "data": "synthetic (seeded)",
            "config": {"workload": "bd256: 256 systems, N log-uniform [64, 4096], phi U(0.05, 0.3), a=1, eta=1, "
                                   "kT=1, dt=1e-3, k=1, tol 1e-4; one bench step = 10 EM steps in one graph launch",
                       "N_total": int(b.Ntot), "ms_per_bd_step": ms_bd_step,
                       "lanczos_iterations_mean": float(np.mean(iters)), "tiling": tiling,
                       "per_system_calls_ms_per_bd_step": None if t_loop is None else 1e3 * t_loop,
                       "speedup_vs_per_system_calls": None if t_loop is None else 1e3 * t_loop / ms_bd_step},
            "gpu_launches": launches, "clocks": clocks}
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
