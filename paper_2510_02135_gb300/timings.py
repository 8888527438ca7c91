"""Mobility-product time against N on this GPU, in the shape of the paper's
timing figure (Sec. 5.5, Fig. timings_linear): particles uniform at random
in a cube at number density rho (0.1 and 0.001 / a^3), overlaps allowed,
forces only (linear displacements), transfers excluded; free space and a
single bottom wall (the cube resting on the wall).

    python -m paper_2510_02135_gb300.timings [--max-n 524288] [--reps 5]

prints one row per (geometry, rho, N): the best of `reps` products (CUDA
events, after the autotuner picked the launch configuration for N <= 65536
and one warm-up product), and the pair-interactions per second.

    python -m paper_2510_02135_gb300.timings --batch [--tiling 64,1] [--reps 5]

times the batched product lm_batch_mdot over the 256 suspensions of the
batched Brownian-dynamics workload instead (one cooperative launch per call).
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main() -> None:
    import torch

    from . import _build, lm

    ap = argparse.ArgumentParser()
    ap.add_argument("--max-n", type=int, default=1 << 19)
    ap.add_argument("--min-n", type=int, default=1 << 7)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--json", action="store_true", help="one JSON object per row")
    ap.add_argument("--batch", action="store_true", help="time the batched product of the 256-suspension batch")
    ap.add_argument("--tiling", default=None, help="threads,ilp of the batched launches (default: autotuned)")
    args = ap.parse_args()
    _build.build()
    if args.batch:
        return batch_product(args)
    rows = []
    for geo in ("open", "single_wall"):
        for rho in (0.1, 0.001):
            n = args.min_n
            while n <= args.max_n:
                rng = np.random.default_rng(n)
                L = (n / rho) ** (1.0 / 3.0)
                u = rng.uniform(0.0, 1.0, size=(n, 3))
                zoff = 0.0 if geo == "single_wall" else 0.5
                pos = np.column_stack([(u[:, 0] - 0.5) * L, (u[:, 1] - 0.5) * L, (u[:, 2] - zoff) * L])
                pos = torch.from_numpy(pos.astype(np.float32)).cuda()
                F = torch.from_numpy(rng.standard_normal((n, 3)).astype(np.float32)).cuda()
                out = torch.empty_like(F)
                s = lm.lm_create(1.0, 1.0, False, lm.LM_FP32C, periodicity=("open", "open", geo))
                lm.lm_set_positions(s, pos)
                if n <= 65536:
                    lm.lm_autotune(s, reps=1)
                lm.lm_mdot(s, F, None, out, None)
                best = float("inf")
                for _ in range(args.reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    lm.lm_mdot(s, F, None, out, None)
                    e1.record()
                    torch.cuda.synchronize()
                    best = min(best, e0.elapsed_time(e1))
                row = {"geometry": geo, "rho": rho, "N": n, "ms": best, "pairs_per_s": n * n / (best / 1e3),
                       "config": lm.lm_get_pair_config(s)}
                rows.append(row)
                if args.json:
                    print(json.dumps(row), flush=True)
                else:
                    print(f"{geo:12s} rho {rho:6.3f}  N {n:8d}  {best:10.4f} ms  {row['pairs_per_s']:.3e} pairs/s",
                          flush=True)
                n *= 2



def batch_product(args) -> None:
    """Best of `reps` batched products lm_batch_mdot (CUDA events, one warm-up
    call) over the batched BD workload's 256 suspensions, forces N(0, 1)."""
    import torch

    from . import inputs as I, lm

    c = I.BATCH_BD_256
    b_ = I.batch_suspensions(c["seed"], c["S"], c["nmin"], c["nmax"], c["phi_lo"], c["phi_hi"], c["a"])
    b = lm.lm_batch_create(b_.offsets, c["eta"], c["a"], max_iter=64,
                           cuda_stream=torch.cuda.current_stream().cuda_stream)
    lm.lm_batch_set_positions(b, torch.from_numpy(np.ascontiguousarray(b_.pos)).cuda())
    if args.tiling:
        t, i = (int(v) for v in args.tiling.split(","))
        lm.lm_batch_set_tiling(b, t, i)
        tiling = {"threads": t, "ilp": i}
    else:
        tiling = lm.lm_batch_autotune(b)
    F = torch.from_numpy(np.random.default_rng(1).standard_normal((b.Ntot, 3)).astype(np.float32)).cuda()
    out = torch.empty_like(F)
    lm.lm_batch_mdot(b, F, out)
    best = float("inf")
    for _ in range(args.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        lm.lm_batch_mdot(b, F, out)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    pairs = float((np.diff(b_.offsets).astype(np.float64) ** 2).sum())
    row = {"workload": "bd256 batched product", "systems": int(b.S), "N_total": int(b.Ntot), "tiling": tiling,
           "ms": best, "pairs_per_s": pairs / (best * 1e-3)}
    print(json.dumps(row) if args.json else
          f"batched product, {b.S} systems, N_total {b.Ntot}, tiling {tiling}: {best:.3f} ms, "
          f"{row['pairs_per_s']:.3e} pair-interactions/s")


if __name__ == "__main__":
    main()
