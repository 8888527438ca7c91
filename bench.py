#!/usr/bin/env python
"""Throughput of the open-boundary RPY mobility hot path on one GB300.

One step = one pass of the hot path over one suspension:
  lm_set_positions -> lm_mdot (M [F; T], all four blocks) -> lm_sqrt_mdot
  (Lanczos M^{1/2} W at the workload's tolerance).
Metric: RPY pair-interactions per second, counting N^2 ordered pairs for
every application of M (the product and each Lanczos iteration), inputs
resident in HBM, L2 flushed (256 MB write) before every step.

Default workload (the largest single-GPU case, where the FP32 peak target
is set): 1024 bead-spring chains of 512 beads (N = 524288), translation +
rotation, FP32 pair arithmetic with compensated sums, FP64 Lanczos at tol
1e-3 (seeded synthetic inputs).  After the timed region the same JSON line
also reports, at one GPU:
  * "error": the relative L2 error of the timed step's M [F; T] per block
    (u from F, u from T, w from F, w from T) against the FP64 oracle on
    sampled rows (the rows of the CPU-baseline sample);
  * "rpy6_n32768": the 6N step at N = 32768 (tol 1e-5) with its own roofline and
    per-block errors;
  * "adjoint": forward and backward (dL/dX, dL/dF) times at N = 65536 and
    their ratio, and the same with angular blocks (dL/dT too);
  * "bd256": the batched Brownian-dynamics step of 256 suspensions and its
    speed-up over per-system library calls.
"--workload rpy6" makes the N = 32768 step the headline instead.

--impl reference times the FP64 CPU oracle (the only reference that exists:
the paper ships no code) on the same metric over a bounded row sample.
Multi-GPU: replicas only (the product does not shard); one process per GPU
under torchrun, value = pairs of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
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
FLOPS_PER_PAIR_6N = 86
FLOPS_PER_PAIR_TT = 35   # translation-only far-field pair (the batched and adjoint workloads)
PAIR_KERNEL_SRCS = [os.path.join(ROOT, "paper_2510_02135_gb300", "csrc", f)
                    for f in ("pair_kernels.cu", "pair_common.cuh")]
# ncu summaries of the forward pair kernel, per workload (DRAM bytes per launch)
PAIR_PROFILE = {"melt": "pair_kernel_melt_n524288.txt", "rpy6": "pair_kernel_rpy6_n32768.txt"}


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
        desc = (f"melt_n524288: {c['n_chains']} chains x {c['beads']} beads (N={c['n_chains'] * c['beads']}), "
                f"bond {c['bond']}a, angle jitter {c['sigma']} rad, phi={c['phi']}, a={c['a']}, eta={c['eta']}, "
                f"forces+torques, FP32 compensated pairs, FP64 Lanczos tol {c['tol']}")
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
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                pw.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "power_w_median": statistics.median(pw) if pw else None, "reasons": sorted(reasons)}


def measured_hbm_gbs():
    """Copy bandwidth measured on this GPU pool (generated file), else the
    recipe's fallback figure."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def profile_traffic(workload: str):
    """DRAM bytes per pair-kernel launch from the committed ncu summary of this
    workload, if it was taken on the current kernel source (else None)."""
    name = PAIR_PROFILE.get(workload)
    if name is None:
        return None
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if (vals.get("kernel_source_sha256_16", "").split() or [""])[0] != pair_kernel_source_hash():
        return None
    try:
        return float(vals["dram_bytes_per_launch"].split()[0])
    except (KeyError, ValueError, IndexError):
        return None


def fp32_peak(local: int):
    """Nominal FP32 FMA peak of this GPU: SMs x 128 lanes x 2 flop x the
    recipe's maximum SM clock."""
    import torch

    sms = torch.cuda.get_device_properties(local).multi_processor_count
    return sms * FP32_LANES_PER_SM * 2 * RECIPE_MAX_SM_MHZ * 1e6 / 1e12, sms


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


def _dist_init(ws, local):
    import torch

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group(backend="nccl", device_id=torch.device("cuda", local))
        return dist
    return None


def _rel(y, ref):
    y = np.asarray(y, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    n = float(np.linalg.norm(ref))
    return float(np.linalg.norm(y - ref) / (n if n > 0 else 1.0))


def _pair_config_arg(text):
    return tuple(int(v) for v in text.split(","))


# ---------------------------------------------------------------------------
# The hot-path step: set_positions + M [F; T] + Lanczos M^{1/2} W
# ---------------------------------------------------------------------------
def hotpath_leg(workload, steps, warmup, dist, local, *, pair_config=None, autotune=True, e2e_steps=0,
                sample_clocks=True, probe=False):
    """Times `steps` hot-path steps of `workload` after `warmup` untimed ones.
    Returns a dict of results; the solver and the device tensors of the last
    step stay in it (keys starting with "_") for the checks that follow."""
    import torch

    from paper_2510_02135_gb300 import lm

    s_, eta, a, tol, desc = workload_spec(workload)
    n = s_.pos.shape[0]
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    pos, F, T, W = dev(s_.pos), dev(s_.F), dev(s_.T), dev(s_.W)
    lin = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    ang = torch.empty_like(lin)
    lin2 = torch.empty_like(lin)
    ang2 = torch.empty_like(lin)
    solver = lm.lm_create(eta, a, True, lm.LM_FP32C, cuda_stream=torch.cuda.current_stream().cuda_stream)
    lm.lm_set_positions(solver, pos)
    t_tune = time.perf_counter()
    if pair_config:
        lm.lm_set_pair_config(solver, *pair_config)
    elif autotune:
        lm.lm_autotune(solver, reps=1 if n > 200_000 else 2)
    t_tune = time.perf_counter() - t_tune
    cfg = lm.lm_get_pair_config(solver)
    iters = []

    def step():
        lm.lm_set_positions(solver, pos)
        lm.lm_mdot(solver, F, T, lin, ang)
        _, _, it = lm.lm_sqrt_mdot(solver, W, tol=tol, max_iter=200, lin_out=lin2, ang_out=ang2)
        iters.append(it)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    iters.clear()
    sampler = ClockSampler(local) if sample_clocks else None
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    lm.lm_profile_read(solver, reset=True)
    lm.lm_profile_enable(solver, True)
    if sampler:
        sampler.start()
    launches0 = lm.lm_launch_count()
    t_wall0 = time.perf_counter()
    for k in range(steps):
        flush.zero_()
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall0
    launches = lm.lm_launch_count() - launches0
    clocks = sampler.stop() if sampler else None
    lm.lm_profile_enable(solver, False)
    prof = lm.lm_profile_read(solver, reset=True)
    stats = lm.lm_get_lanczos_stats(solver)
    step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    total_ms = float(sum(step_ms))
    pairs = float(n) * float(n) * float(sum(1 + it for it in iters))
    total_ms_max, pairs_all = _reduce(dist, total_ms, pairs)
    value = pairs_all / (total_ms_max / 1e3)

    e2e = None
    if e2e_steps > 0:
        # the same step through host (pinned) buffers, copies inside the timed region
        pos_h = torch.from_numpy(s_.pos).pin_memory()
        F_h = torch.from_numpy(s_.F).pin_memory()
        T_h = torch.from_numpy(s_.T).pin_memory()
        W_h = torch.from_numpy(s_.W).pin_memory()
        outs_h = [torch.empty((n, 3), dtype=torch.float32).pin_memory() for _ in range(4)]
        e2e_iters = []

        def step_host(tol_=tol):
            lm.lm_set_positions(solver, pos_h)
            lm.lm_mdot(solver, F_h, T_h, outs_h[0], outs_h[1])
            _, _, it = lm.lm_sqrt_mdot(solver, W_h, tol=tol_, max_iter=200, lin_out=outs_h[2], ang_out=outs_h[3])
            e2e_iters.append(it)

        step_host(tol_=0.5)   # warms the library's host staging buffers (stops after two iterations)
        e2e_iters.clear()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            step_host()
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        e2e_pairs = float(n) * float(n) * float(sum(1 + it for it in e2e_iters))
        t_e2e, e2e_pairs = _reduce(dist, t_e2e, e2e_pairs)
        e2e = {"value": e2e_pairs / t_e2e, "unit": UNIT, "h2d_bytes_per_step": n * 3 * 4 * 3 + W_h.numel() * 8,
               "d2h_bytes_per_step": n * 3 * 4 * 4, "steps": e2e_steps,
               "api": "lm_set_positions/lm_mdot/lm_sqrt_mdot with pinned host buffers"}

    peak, sms = fp32_peak(local)
    achieved = prof["pair_flops"] / (prof["pair_ms"] / 1e3) / 1e12 if prof["pair_ms"] > 0 else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": profile_traffic(workload),
                "kernel": ("rpy_mdot_x2_kernel (forward pair kernel, packed FP32, all four blocks)" if cfg["packed"]
                           else "rpy_mdot_kernel (forward pair kernel, scalar FP32, all four blocks)"),
                "flops_per_pair": FLOPS_PER_PAIR_6N, "pairs_per_launch": float(n) * n,
                "pair_launches": prof["pair_launches"],
                "pair_kernel_ms_avg": prof["pair_ms"] / max(1, prof["pair_launches"]),
                "pair_share_of_step": prof["pair_ms"] / max(1e-9, total_ms),
                "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {RECIPE_MAX_SM_MHZ:.0f} MHz "
                              f"(nominal FP32 FMA peak at the recipe's maximum SM clock)"}
    if clocks and achieved:
        roofline["frac_at_sampled_clock"] = achieved / (peak * clocks["sm_mhz"] / RECIPE_MAX_SM_MHZ)
    if probe and achieved:
        # measured FP32 FMA ceilings of this GPU (library probe, after the timed region)
        pr = {"ffma": lm.lm_fp32_probe(0), "ffma2": lm.lm_fp32_probe(1), "ffma2_distinct_operands": lm.lm_fp32_probe(2),
              "ffma2_dependent_chains": lm.lm_fp32_probe(3)}
        roofline["probe_tflops"] = pr
        roofline["frac_of_probe_ffma2"] = achieved / pr["ffma2"]
        roofline["probe_note"] = ("lm_fp32_probe on this GPU after the timed region: FMA streams on every SM; "
                                  "ffma2 = packed f32x2 FMA (the pair kernels' instruction form) with reused "
                                  "operands; distinct = three distinct register pairs per instruction; dependent "
                                  "chains = operands produced a few instructions earlier")
    hbm = measured_hbm_gbs()
    vec_gbs = prof["vector_bytes"] / (prof["vector_ms"] / 1e3) / 1e9 if prof["vector_ms"] > 0 else None
    lanczos_vectors = {
        "bound": "hbm", "achieved": vec_gbs, "peak": hbm, "unit": "GB/s",
        "frac": (vec_gbs / hbm) if (vec_gbs and hbm) else None,
        "iterations": prof["vector_iterations"],
        "ms_per_iteration": prof["vector_ms"] / max(1, prof["vector_iterations"]),
        "share_of_step": prof["vector_ms"] / max(1e-9, total_ms),
        "bytes_per_iteration_mean": prof["vector_bytes"] / max(1, prof["vector_iterations"]),
        "bytes_rule": "FP64 vectors of n=6N: alpha 2, three-term update 4, each Gram-Schmidt pass 2k+5 at iteration k",
        "peak_basis": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth), of measured"}
    # The Gram-Schmidt kernels do one FP64 FMA per 8-byte basis element: their
    # ceiling is min(HBM, 8 B x the FP64 FMA rate), measured here after the
    # timed region.  The bound time sums, per enqueued iteration k, the HBM
    # time of alpha and the three-term update and, for the dots and the
    # subtraction, the larger of their HBM time and their FP64 FMA time.
    fp64 = lm.lm_fp32_probe(4, 1 << 8)
    if hbm and fp64 > 0 and prof["vector_ms"] > 0:
        ks = []
        extra = max(0, int(prof["vector_iterations"]) - int(sum(iters)))
        for c, m in enumerate(iters):
            ks.extend(range(int(m) + (1 if c < extra else 0)))
        vec = 8.0 * (6 * n)
        bw = hbm * 1e9
        fma_rate = fp64 * 1e12 / 2.0
        bound_s = 0.0
        for k in ks:
            bound_s += (2 + (4 if k else 3)) * vec / bw
            for rows in (k + 2, k + 3):
                bound_s += max(rows * vec / bw, (k + 1) * (6 * n) / fma_rate)
        lanczos_vectors.update({
            "fp64_probe_tflops": fp64,
            "bound_ms_per_iteration": 1e3 * bound_s / max(1, len(ks)),
            "frac_of_fp64_hbm_bound": 1e3 * bound_s / prof["vector_ms"],
            "bound_rule": "per enqueued iteration k: alpha and the three-term update at the HBM copy peak; the "
                          "Gram-Schmidt dots ((k+2) vectors, (k+1) n FP64 FMAs) and subtraction ((k+3) vectors, "
                          "(k+1) n FMAs) each at max(HBM time, FMA time at the measured FP64 rate); the DGKS second "
                          "pass, rarely taken, not counted"})
    return {"workload": workload, "desc": desc, "n": n, "value": value, "ms_per_step": total_ms_max / steps,
            "steps": steps, "warmup": warmup, "iters": list(iters), "cfg": cfg, "autotune_s": t_tune,
            "roofline": roofline, "lanczos_vectors": lanczos_vectors, "e2e": e2e, "launches": launches,
            "clocks": clocks, "wall_s_timed": t_wall, "lanczos_stats": stats, "tol": tol,
            "_solver": solver, "_s": s_, "_eta": eta, "_a": a, "_lin": lin, "_ang": ang, "_F": F, "_T": T}


def cpu_baseline_and_error(leg, budget_s: float, block_rows: int):
    """The CPU-baseline leg: the FP64 oracle's direct sum of M [F; T] timed on
    a random row sample of the same workload (about budget_s of CPU work), and,
    as the checker of the timed step, the relative L2 errors of the GPU
    outputs on those rows (totals) and, on `block_rows` of them, per block
    (u from F, u from T, w from F, w from T; the GPU blocks from two more
    products with F or T alone).  Runs after the timed region, on rank 0."""
    import torch

    import oracle
    from paper_2510_02135_gb300 import lm

    oracle.build()
    s_, a, eta, n = leg["_s"], leg["_a"], leg["_eta"], leg["n"]
    rng = np.random.default_rng(0)
    probe = rng.choice(n, min(n, 32), replace=False)
    t0 = time.perf_counter()
    oracle.mdot(s_.pos, s_.F, s_.T, a, eta, True, rows=probe)
    t = time.perf_counter() - t0
    nrows = int(min(n, max(32, len(probe) * budget_s / max(t, 1e-6))))
    rows = np.sort(rng.choice(n, nrows, replace=False))
    t0 = time.perf_counter()
    ur, wr = oracle.mdot(s_.pos, s_.F, s_.T, a, eta, True, rows=rows)
    t = time.perf_counter() - t0
    cpu = {"value": nrows * n / t, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"FP64 oracle direct sum of M [F; T] (all four blocks) for {nrows} random rows x {n} columns "
                     f"({t:.1f} s); the Lanczos cost per pair is the same product"}
    lin = leg["_lin"].cpu().numpy()
    ang = leg["_ang"].cpu().numpy()
    err = {"u": _rel(lin[rows], ur), "w": _rel(ang[rows], wr)}
    brows = rows[np.sort(rng.choice(nrows, min(nrows, block_rows), replace=False))]
    solver = leg["_solver"]
    uF, wF = lm.lm_mdot(solver, leg["_F"], None)
    uT, wT = lm.lm_mdot(solver, None, leg["_T"])
    torch.cuda.synchronize()
    zero = np.zeros_like(s_.F)
    urF, wrF = oracle.mdot(s_.pos, s_.F, None, a, eta, True, rows=brows)
    urT, wrT = oracle.mdot(s_.pos, zero, s_.T, a, eta, True, rows=brows)
    err.update({"uF": _rel(uF.cpu().numpy()[brows], urF), "uT": _rel(uT.cpu().numpy()[brows], urT),
                "wF": _rel(wF.cpu().numpy()[brows], wrF), "wT": _rel(wT.cpu().numpy()[brows], wrT)})
    err["max"] = max(err.values())
    err.update({"metric": "relative L2 error |y - y_oracle| / |y_oracle| on sampled rows, FP64 oracle direct sum",
                "rows_total": int(nrows), "rows_per_block": int(len(brows)), "target": 1e-5})
    return cpu, err


def _leg_summary(leg):
    keep = ("desc", "n", "value", "ms_per_step", "steps", "warmup", "cfg", "roofline", "lanczos_vectors", "clocks")
    out = {k: leg[k] for k in keep}
    out["unit"] = UNIT
    out["lanczos_iterations_mean"] = float(np.mean(leg["iters"])) if leg["iters"] else None
    out["gpu_launches"] = leg["launches"]
    return out


# ---------------------------------------------------------------------------
# Adjoint: forward product and fused backward at N = 65536
# ---------------------------------------------------------------------------
def adjoint_leg(steps, warmup, dist, local, *, pair_config=None, adjoint_config=None, autotune=True):
    """Forward product and fused adjoint (L = <G, M(X) F>) at N = 65536,
    translation only, FP32: one step = lm_set_positions + lm_mdot +
    lm_mdot_backward (dL/dX and dL/dF); pairs counted N^2 per launch."""
    import torch

    from paper_2510_02135_gb300 import inputs as I, lm

    c = I.ADJOINT_N65536
    s_ = I.cube_suspension(c["seed"], c["n"], c["phi"], c["a"], angular=False, fp32=True)
    n = c["n"]
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    pos, F, G = dev(s_.pos), dev(s_.F), dev(s_.G)
    u = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    solver = lm.lm_create(c["eta"], c["a"], False, lm.LM_FP32C, cuda_stream=torch.cuda.current_stream().cuda_stream)
    lm.lm_set_positions(solver, pos)
    if pair_config:
        lm.lm_set_pair_config(solver, *pair_config)
    elif autotune:
        lm.lm_autotune(solver, reps=2)
    if adjoint_config:
        lm.lm_set_adjoint_config(solver, *adjoint_config)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]

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

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    launches0 = lm.lm_launch_count()
    for k in range(steps):
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
    tmax, pairs = _reduce(dist, total, 2.0 * n * n * steps)
    peak, _ = fp32_peak(local)
    fwd_ms = float(np.median(fwd))
    bwd_ms = float(np.median(bwd))
    achieved = FLOPS_PER_PAIR_TT * float(n) * n / (fwd_ms / 1e3) / 1e12

    # the same suspension with angular blocks (torques T, cotangents H): the
    # forward product M [F; T] and the adjoint (dX, dF, dT) in their default
    # (symmetric) form; reported beside the translation figures, not in value
    s6 = I.cube_suspension(c["seed"], n, c["phi"], c["a"], angular=True, fp32=True)
    T6, H6 = dev(s6.T), dev(s6.H)
    w6 = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    solver6 = lm.lm_create(c["eta"], c["a"], True, lm.LM_FP32C, cuda_stream=stream.cuda_stream)
    lm.lm_set_positions(solver6, pos)
    if autotune and not pair_config:
        lm.lm_autotune(solver6, reps=1)
    ev6 = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(3)]
    for k in range(warmup + 3):
        flush.zero_()
        e = ev6[k - warmup] if k >= warmup else None
        if e:
            e[0].record(stream)
        lm.lm_mdot(solver6, F, T6, u, w6)
        if e:
            e[1].record(stream)
        lm.lm_mdot_backward(solver6, F, T6, G, H6)
        if e:
            e[2].record(stream)
    torch.cuda.synchronize()
    fwd6 = float(np.median([e[0].elapsed_time(e[1]) for e in ev6]))
    bwd6 = float(np.median([e[1].elapsed_time(e[2]) for e in ev6]))
    angular = {"forward_ms": fwd6, "backward_ms": bwd6, "backward_over_forward": bwd6 / fwd6,
               "steps": 3, "pair_config": lm.lm_get_pair_config(solver6),
               "adjoint_config": lm.lm_get_adjoint_config(solver6),
               "desc": "same N and positions with torques; backward = dX, dF, dT (the default symmetric form)"}
    del solver6
    return {"value": pairs / (tmax / 1e3), "unit": UNIT, "ms_per_step": tmax / steps, "steps": steps,
            "warmup": warmup,
            "desc": f"adjoint_n65536: N={n}, phi={c['phi']}, translation only, FP32 compensated; "
                    f"step = lm_mdot + lm_mdot_backward (dX, dF)",
            "forward_ms": fwd_ms, "backward_ms": bwd_ms, "backward_over_forward": bwd_ms / fwd_ms,
            "target_backward_over_forward": 2.5,
            "pair_config": lm.lm_get_pair_config(solver), "adjoint_config": lm.lm_get_adjoint_config(solver),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "forward pair kernel (translation, 35 flops/pair)"},
            "gpu_launches": launches, "clocks": clocks, "angular": angular,
            "l2": "flushed by a 256 MB device write before every step"}


# ---------------------------------------------------------------------------
# Batched Brownian dynamics of 256 suspensions
# ---------------------------------------------------------------------------
def bd_leg(steps, warmup, dist, local, rank, *, autotune=True, per_system=True):
    """Batched Brownian dynamics: 256 suspensions (N log-uniform in [64, 4096],
    phi uniform in [0.05, 0.3]), 10 Euler-Maruyama steps per bench step in one
    persistent cooperative launch captured in a CUDA graph, Lanczos tol 1e-4.
    Pairs counted: sum_s N_s^2 per Lanczos iteration of system s.  Also times
    one BD step done with per-system library calls, for the speed-up factor."""
    import torch

    from paper_2510_02135_gb300 import inputs as I, lm

    c = I.BATCH_BD_256
    b_ = I.batch_suspensions(c["seed"], c["S"], c["nmin"], c["nmax"], c["phi_lo"], c["phi_hi"], c["a"])
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    b = lm.lm_batch_create(b_.offsets, c["eta"], c["a"], max_iter=64,
                           cuda_stream=torch.cuda.current_stream().cuda_stream)
    lm.lm_batch_set_positions(b, dev(b_.pos))
    tiling = lm.lm_batch_autotune(b) if autotune else {"threads": 128, "ilp": 1}
    nsub = 10
    sizes2 = b_.sizes.astype(np.float64) ** 2
    step_no = [0]

    def step():
        its = lm.lm_batch_bd_run(b, c["kT"], c["dt"], c["k_trap"], nsub, step0=step_no[0], seed=c["seed"],
                                 tol=c["tol"], use_graph=True)
        step_no[0] += nsub
        return its

    for _ in range(warmup):
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
    for _ in range(steps):
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
    if rank == 0 and per_system:
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
    ms_bd_step = tmax / (steps * nsub)
    # one more EM step with the phase timeline on (after the timed region):
    # where a BD step's time goes, the product phases' FP32 fraction and the
    # share of pair evaluations in iterations that the systems keep
    profiled = None
    if rank == 0:
        lm.lm_batch_profile_enable(b, True)
        its1 = lm.lm_batch_bd_run(b, c["kT"], c["dt"], c["k_trap"], 1, step0=step_no[0], seed=c["seed"],
                                  tol=c["tol"], use_graph=False)
        torch.cuda.synchronize()
        st = lm.lm_batch_profile_read(b).astype(np.int64)
        pairs_ev = float(lm.lm_batch_profile_pairs(b))
        lm.lm_batch_profile_enable(b, False)
        d = np.diff(st) / 1e6   # ms
        nit = (len(st) - 5) // 5
        ph = d[2:2 + 5 * nit].reshape(nit, 5) if nit > 0 else np.zeros((0, 5))
        prod_ms = float(ph[:, 0].sum())
        peak, _ = fp32_peak(local)
        kept = float((sizes2 * np.asarray(its1)).sum())
        profiled = {"iterations_run": int(nit), "step_ms": float(d.sum()),
                    "phases_ms": {"noise_forces_normalise": float(d[0] + d[1]), "products": prod_ms,
                                  "gram_schmidt": float(ph[:, 1:4].sum()), "end_of_iteration": float(ph[:, 4].sum()),
                                  "final_wait_and_update": float(d[2 + 5 * nit:].sum())},
                    "pair_evaluations": pairs_ev,
                    "product_phase_pairs_per_s": pairs_ev / (prod_ms / 1e3) if prod_ms > 0 else None,
                    "product_phase_frac_fp32": (pairs_ev / (prod_ms / 1e3) * FLOPS_PER_PAIR_TT / 1e12 / peak
                                                if prod_ms > 0 else None),
                    "kept_pair_fraction": kept / pairs_ev if pairs_ev > 0 else None,
                    "note": "lm_batch_profile_* timeline of one further EM step (direct launch); products = phase B "
                            "of every Lanczos iteration, gram_schmidt = C2 + C3 + C4, end_of_iteration = C5; FP32 "
                            "fraction at 35 flops/pair of the nominal peak; kept = pairs of the iterations the "
                            "systems keep (sum N_s^2 x iterations)"}
    return {"value": pairs_all / (tmax / 1e3), "unit": UNIT, "ms_per_step": tmax / steps, "steps": steps,
            "warmup": warmup,
            "desc": "bd256: 256 systems, N log-uniform [64, 4096], phi U(0.05, 0.3), a=1, eta=1, kT=1, dt=1e-3, "
                    "k=1, tol 1e-4; one bench step = 10 EM steps in one graph launch",
            "N_total": int(b.Ntot), "ms_per_bd_step": ms_bd_step,
            "lanczos_iterations_mean": float(np.mean(iters)), "tiling": tiling,
            "per_system_calls_ms_per_bd_step": None if t_loop is None else 1e3 * t_loop,
            "speedup_vs_per_system_calls": None if t_loop is None else 1e3 * t_loop / ms_bd_step,
            "gpu_launches": launches, "clocks": clocks, "profiled_step": profiled}


# ---------------------------------------------------------------------------
# Reference arm: the FP64 CPU oracle
# ---------------------------------------------------------------------------
def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    s, eta, a, tol, desc = workload_spec(args.workload)
    import oracle

    oracle.build()
    n = s.pos.shape[0]
    rng = np.random.default_rng(0)

    def sample(budget_s):
        rows = rng.choice(n, min(n, 32), replace=False)
        t0 = time.perf_counter()
        oracle.mdot(s.pos, s.F, s.T, a, eta, True, rows=rows)
        t = time.perf_counter() - t0
        nrows = int(min(n, max(32, len(rows) * budget_s / max(t, 1e-6))))
        rows = rng.choice(n, nrows, replace=False)
        t0 = time.perf_counter()
        oracle.mdot(s.pos, s.F, s.T, a, eta, True, rows=rows)
        return nrows, time.perf_counter() - t0

    for _ in range(args.warmup):
        sample(0.5)
    rows_used, secs = 0, 0.0
    for _ in range(args.steps):
        nr, t = sample(args.ref_step_s)
        rows_used += nr
        secs += t
    value = rows_used * n / secs
    cores = oracle.num_threads()
    smp = (f"each step: FP64 oracle direct sum of M [F; T] (all four blocks) for a random sample of rows "
           f"(~{args.ref_step_s:.0f} s of CPU work, {rows_used // max(1, args.steps)} rows x {n} columns per step)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": smp},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["melt", "rpy6", "adjoint", "bd256", "wall", "rollers"], default="melt")
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
    ap.add_argument("--no-extras", action="store_true",
                    help="headline leg only (no rpy6_n32768 / adjoint / bd256 entries)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    pcfg = _pair_config_arg(args.pair_config) if args.pair_config else None
    acfg = _pair_config_arg(args.adjoint_config) if args.adjoint_config else None
    if args.workload in ("adjoint", "bd256", "wall", "rollers"):
        return run_single(args, ws, rank, local, pcfg, acfg)

    import torch

    from paper_2510_02135_gb300 import _build

    dist = _dist_init(ws, local)
    _build.build()
    t_job0 = time.perf_counter()
    leg = hotpath_leg(args.workload, args.steps, args.warmup, dist, local, pair_config=pcfg,
                      autotune=not args.no_autotune, e2e_steps=max(1, args.e2e_steps), probe=True)
    cfg = leg["cfg"]
    line = {"metric": METRIC, "value": leg["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": leg["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "dtype_detail": "FP32 pair arithmetic with compensated (TwoSum) accumulation; FP64 Lanczos vectors",
            "data": "synthetic (seeded; shapes of the paper's benchmark workloads)",
            "config": {"workload": leg["desc"], "N": leg["n"],
                       "lanczos_iterations_mean": float(np.mean(leg["iters"])),
                       "lanczos_tol": leg["tol"], "lanczos_converged": leg["lanczos_stats"]["converged"],
                       "sqrt_per_s": args.steps / (leg["ms_per_step"] * args.steps / 1e3),
                       "l2": "flushed by a 256 MB device write before every step (outside the step events)",
                       "pair_config": cfg, "autotune_s": leg["autotune_s"], "parallelism": f"replicas x{ws}",
                       "wall_s_timed": leg["wall_s_timed"]},
            "roofline": leg["roofline"], "lanczos_vectors": leg["lanczos_vectors"], "e2e": leg["e2e"],
            "gpu_launches": leg["launches"], "clocks": leg["clocks"]}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, err = cpu_baseline_and_error(leg, args.cpu_budget, block_rows=128)
        line["cpu_baseline"] = cpu
        line["error"] = err
    for k in [k for k in leg if k.startswith("_")]:
        del leg[k]
    torch.cuda.empty_cache()
    if ws == 1 and not args.no_extras and args.workload == "melt":
        step2 = hotpath_leg("rpy6", min(args.steps, 10), 3, None, local, autotune=not args.no_autotune)
        if rank == 0 and not args.no_cpu_baseline:
            _, err2 = cpu_baseline_and_error(step2, 1.0, block_rows=256)
            step2_sum = _leg_summary(step2)
            step2_sum["error"] = err2
        else:
            step2_sum = _leg_summary(step2)
        step2_sum["roofline"]["traffic"] = profile_traffic("rpy6")
        line["rpy6_n32768"] = step2_sum
        del step2
        torch.cuda.empty_cache()
        line["adjoint"] = adjoint_leg(10, 3, None, local, autotune=not args.no_autotune)
        torch.cuda.empty_cache()
        line["bd256"] = bd_leg(5, 3, None, local, rank, autotune=not args.no_autotune)
    line["config"]["job_wall_s"] = time.perf_counter() - t_job0
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_single(args, ws, rank, local, pcfg, acfg):
    """One of the secondary workloads as the whole line."""
    from paper_2510_02135_gb300 import _build

    dist = _dist_init(ws, local)
    _build.build()
    if args.workload in ("wall", "rollers"):
        fn = run_wall if args.workload == "wall" else run_rollers
        return fn(args, ws, rank, local, dist)
    if args.workload == "adjoint":
        r = adjoint_leg(args.steps, args.warmup, dist, local, pair_config=pcfg, adjoint_config=acfg,
                        autotune=not args.no_autotune)
        extra = {"forward_ms": r["forward_ms"], "backward_ms": r["backward_ms"],
                 "backward_over_forward": r["backward_over_forward"], "pair_config": r["pair_config"],
                 "adjoint_config": r["adjoint_config"], "angular": r["angular"], "l2": r["l2"]}
    else:
        r = bd_leg(args.steps, args.warmup, dist, local, rank, autotune=not args.no_autotune)
        extra = {"N_total": r["N_total"], "ms_per_bd_step": r["ms_per_bd_step"],
                 "lanczos_iterations_mean": r["lanczos_iterations_mean"], "tiling": r["tiling"],
                 "per_system_calls_ms_per_bd_step": r["per_system_calls_ms_per_bd_step"],
                 "speedup_vs_per_system_calls": r["speedup_vs_per_system_calls"],
                 "profiled_step": r["profiled_step"]}
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
            "config": {"workload": r["desc"], **extra}, "gpu_launches": r["gpu_launches"], "clocks": r["clocks"]}
    if "roofline" in r:
        line["roofline"] = r["roofline"]
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


def run_wall(args, ws, rank, local, dist):
    """Mobility product above a single no-slip wall (the paper's "bottom
    wall" benchmark shape): N = 32768 spheres uniform in a cube on the wall at
    number density 0.1 / a^3, forces only, FP32.  One step = lm_set_positions
    + lm_mdot; pairs counted N^2 per product."""
    import torch

    from paper_2510_02135_gb300 import inputs as I, lm

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


def run_rollers(args, ws, rank, local, dist):
    """The active-roller example (Sec. 5.1) as a step of the library: soft
    steric forces (pairs and wall) + gravity, a constant torque about y, and
    one stochastic Adams-Bashforth step (mobility product, one RFD sample of
    the thermal drift = two products, Lanczos square root at tol 1e-3) for
    N = 32768 spheres above a no-slip wall, FP32, all blocks.  Pairs counted:
    N^2 per application of M (the product, the two RFD products and every
    Lanczos iteration)."""
    import torch

    from paper_2510_02135_gb300 import inputs as I, lm

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


if __name__ == "__main__":
    sys.exit(main())
