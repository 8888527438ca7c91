"""Write the expected Lanczos square root of the 6N N = 32768 workload.

Stored values for the full-size Lanczos parity test (the Krylov square root
of Sec. 3.3 applied to the workload's W).  The eigendecomposition of the
196608 x 196608 grand mobility is out of reach, so the expected vector is the
oracle's FP64 Lanczos iteration at tol 1e-10, with every product M v taken by
the oracle's FP64 direct pair sum on the FP32-rounded positions the GPU also
receives.  This script calls only ``oracle`` and the seeded input generator;
nothing here comes from the CUDA library.

Output ``lanczos_rpy6_n32768.txt``:
  * a header with the workload, the iteration count and |y|_2 of the whole
    vector y = M^{1/2} W;
  * 8 random projections g_k . y, g_k = default_rng(7000 + k).standard_normal(6N),
    which see every entry of y;
  * 4096 sampled entries (index, value), indices default_rng(4242).choice(6N, 4096).

Run: python tests/golden/make_lanczos_rpy6_n32768.py   (about 30-45 min on 8 cores)
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2510_02135_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(HERE, "lanczos_rpy6_n32768.txt")
TOL = 1e-10
MAX_ITER = 600
N_SAMPLES = 4096
N_PROJ = 8


def main():
    c = I.RPY6_FP32_N32768
    s = I.cube_suspension(c["seed"], c["n"], c["phi"], c["a"], angular=True, fp32=True)
    n, a, eta = c["n"], c["a"], c["eta"]
    calls = [0]
    t0 = time.time()

    def matvec(v):
        calls[0] += 1
        u, w = oracle.mdot(s.pos, v[: 3 * n].reshape(n, 3), v[3 * n:].reshape(n, 3), a, eta, True)
        if calls[0] % 10 == 0:
            print(f"  product {calls[0]}  {time.time() - t0:.0f} s", flush=True)
        return np.concatenate([u.ravel(), w.ravel()])

    y, it, conv = oracle.lanczos_sqrt(matvec, s.W, tol=TOL, max_iter=MAX_ITER)
    if not conv:
        raise SystemExit(f"oracle Lanczos did not converge in {MAX_ITER} iterations")
    idx = np.sort(np.random.default_rng(4242).choice(6 * n, N_SAMPLES, replace=False))
    proj = [float(np.random.default_rng(7000 + k).standard_normal(6 * n) @ y) for k in range(N_PROJ)]
    with open(OUT, "w") as f:
        f.write("# Lanczos square root y = M^{1/2} W (Sec. 3.3) of the 6N FP32 workload N = 32768\n")
        f.write(f"# (seed {c['seed']}, phi {c['phi']}, a {a}, eta {eta}; W from the same generator):\n")
        f.write(f"# oracle FP64 Lanczos, tol {TOL:g}, full reorthogonalisation, FP64 direct-sum products.\n")
        f.write("# Written by tests/golden/make_lanczos_rpy6_n32768.py (oracle only).\n")
        f.write(f"iterations {it}\n")
        f.write(f"norm_y {float(np.linalg.norm(y)):.17e}\n")
        for k, p in enumerate(proj):
            f.write(f"proj {7000 + k} {p:.17e}\n")
        for i in idx:
            f.write(f"y {int(i)} {y[i]:.17e}\n")
    print(f"wrote {OUT}: {it} iterations, {calls[0]} products, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
