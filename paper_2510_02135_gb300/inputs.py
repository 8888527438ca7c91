"""Seeded synthetic inputs shaped like the libMobility benchmark workloads.

This module only draws random inputs; it holds none of the mobility
arithmetic, and both the CUDA path and the FP64 oracle consume its arrays.

Workload shapes (libMobility paper, Sec. 5.5: particles placed uniformly at
random in a cube, overlaps allowed):
  * ``cube_suspension``  -- N spheres uniform in a cube centred at the origin,
    side L = (N (4/3) pi a^3 / phi)^(1/3); forces, torques, adjoint weights and
    Lanczos noise i.i.d. N(0, 1).
  * ``polymer_melt``     -- bead chains (random-walk conformations with a fixed
    bond length and a Gaussian bend-angle jitter), heads uniform in the cube.
  * ``batch_suspensions``-- many independent cubes with log-uniform sizes and
    uniform volume fractions.
  * ``wall_suspension``  -- N spheres uniform in a cube resting on the wall
    z = 0 (number density rho), for the single-wall geometry; centres below
    z = a overlap the wall.
  * ``roller_monolayer`` -- the active-roller setting of Sec. 5.1: centres
    uniform in a square at a given area fraction, heights uniform in [a, 2a].

Everything is drawn in FP64 with numpy's PCG64 (``default_rng(seed)``) and,
for FP32 workloads, rounded once to FP32, so the oracle and the GPU see
identical values.  The draw order is fixed and documented per function.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def box_side(n: int, phi: float, a: float = 1.0) -> float:
    """Cube side holding n spheres of radius a at volume fraction phi."""
    return float((n * (4.0 / 3.0) * np.pi * a ** 3 / phi) ** (1.0 / 3.0))


@dataclass
class Suspension:
    pos: np.ndarray                 # (N, 3)
    F: np.ndarray                   # (N, 3)
    T: np.ndarray | None            # (N, 3) or None
    W: np.ndarray                   # (3N,) or (6N,) FP64, ordering [F-part; T-part]
    G: np.ndarray                   # (N, 3) adjoint weight on u
    H: np.ndarray | None            # (N, 3) adjoint weight on w
    L: float
    a: float
    extra: dict = field(default_factory=dict)


def cube_suspension(seed: int, n: int, phi: float, a: float = 1.0, angular: bool = False,
                    fp32: bool = True) -> Suspension:
    """N spheres uniform in a centred cube.

    Draw order from default_rng(seed): pos (N,3) uniform in [-L/2, L/2);
    F (N,3); T (N,3) [always drawn, returned only if angular]; W (6N);
    G (N,3); H (N,3).  W is truncated to 3N when not angular.  pos, F, T, G, H
    are rounded to FP32 when fp32; W stays FP64."""
    rng = np.random.default_rng(seed)
    L = box_side(n, phi, a)
    pos = rng.uniform(-0.5 * L, 0.5 * L, size=(n, 3))
    F = rng.standard_normal((n, 3))
    T = rng.standard_normal((n, 3))
    W = rng.standard_normal(6 * n)
    G = rng.standard_normal((n, 3))
    H = rng.standard_normal((n, 3))
    dt = np.float32 if fp32 else np.float64
    if not angular:
        W = W[: 3 * n].copy()
    return Suspension(pos=pos.astype(dt), F=F.astype(dt), T=T.astype(dt) if angular else None,
                      W=W, G=G.astype(dt), H=H.astype(dt) if angular else None, L=L, a=a)


def polymer_melt(seed: int, n_chains: int = 1024, beads: int = 512, bond: float = 2.2,
                 sigma: float = 0.3, phi: float = 0.05, a: float = 1.0, angular: bool = True,
                 fp32: bool = True) -> Suspension:
    """Bead chains: heads uniform in the cube (side from phi over all beads);
    first bond uniform on the sphere; each later bond is the previous one
    rotated by |N(0, sigma^2)| about a uniform random axis perpendicular to
    it; bond length ``bond`` (in units of a).  Beads may leave the cube.

    Draw order (all chains at once per step): heads (n_chains, 3); first bond
    directions (n_chains, 3) normals; then for each later bond: axis normals
    (n_chains, 3) (projected perpendicular to the current bond), angle normals
    (n_chains,).  Then F, T, W, G, H as in ``cube_suspension``."""
    rng = np.random.default_rng(seed)
    n = n_chains * beads
    L = box_side(n, phi, a)
    heads = rng.uniform(-0.5 * L, 0.5 * L, size=(n_chains, 3))
    pos = np.empty((n_chains, beads, 3))
    t = rng.standard_normal((n_chains, 3))
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    p = heads.copy()
    pos[:, 0] = p
    for b in range(1, beads):
        if b > 1:
            ax = rng.standard_normal((n_chains, 3))
            ax -= np.sum(ax * t, axis=1, keepdims=True) * t
            ax /= np.linalg.norm(ax, axis=1, keepdims=True)
            ang = np.abs(rng.normal(0.0, sigma, size=(n_chains, 1)))
            t = np.cos(ang) * t + np.sin(ang) * np.cross(ax, t)
            t /= np.linalg.norm(t, axis=1, keepdims=True)
        p = p + bond * a * t
        pos[:, b] = p
    pos = pos.reshape(n, 3)
    F = rng.standard_normal((n, 3))
    T = rng.standard_normal((n, 3))
    W = rng.standard_normal(6 * n)
    G = rng.standard_normal((n, 3))
    H = rng.standard_normal((n, 3))
    dt = np.float32 if fp32 else np.float64
    if not angular:
        W = W[: 3 * n].copy()
    return Suspension(pos=pos.astype(dt), F=F.astype(dt), T=T.astype(dt) if angular else None,
                      W=W, G=G.astype(dt), H=H.astype(dt) if angular else None, L=L, a=a)


def wall_suspension(seed: int, n: int, rho: float, a: float = 1.0, angular: bool = False,
                    fp32: bool = True) -> Suspension:
    """N spheres uniform in a cube of side L = (N / rho)^(1/3) on the wall:
    x, y in [-L/2, L/2), z in [0, L).  Draw order as ``cube_suspension``
    (positions first as three uniform columns in [0, 1), scaled)."""
    rng = np.random.default_rng(seed)
    L = float((n / rho) ** (1.0 / 3.0))
    u = rng.uniform(0.0, 1.0, size=(n, 3))
    pos = np.column_stack([(u[:, 0] - 0.5) * L, (u[:, 1] - 0.5) * L, u[:, 2] * L])
    F = rng.standard_normal((n, 3))
    T = rng.standard_normal((n, 3))
    W = rng.standard_normal(6 * n)
    G = rng.standard_normal((n, 3))
    H = rng.standard_normal((n, 3))
    dt = np.float32 if fp32 else np.float64
    if not angular:
        W = W[: 3 * n].copy()
    return Suspension(pos=pos.astype(dt), F=F.astype(dt), T=T.astype(dt) if angular else None,
                      W=W, G=G.astype(dt), H=H.astype(dt) if angular else None, L=L, a=a)


@dataclass
class Batch:
    offsets: np.ndarray   # (S+1,) int64 prefix sum of sizes
    sizes: np.ndarray     # (S,) int64
    phi: np.ndarray       # (S,) FP64
    pos: np.ndarray       # (sum N, 3)
    a: float


def batch_suspensions(seed: int, S: int = 256, nmin: int = 64, nmax: int = 4096,
                      phi_lo: float = 0.05, phi_hi: float = 0.3, a: float = 1.0,
                      fp32: bool = True) -> Batch:
    """S independent cubes: N_s = round(exp(U(ln nmin, ln nmax))),
    phi_s ~ U(phi_lo, phi_hi); positions uniform in each system's centred cube.

    Draw order: log-sizes (S), phis (S), then positions system by system."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(np.log(nmin), np.log(nmax), size=S))).astype(np.int64)
    phis = rng.uniform(phi_lo, phi_hi, size=S)
    offsets = np.zeros(S + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(sizes)
    pos = np.empty((int(offsets[-1]), 3))
    for s in range(S):
        L = box_side(int(sizes[s]), float(phis[s]), a)
        pos[offsets[s]:offsets[s + 1]] = rng.uniform(-0.5 * L, 0.5 * L, size=(int(sizes[s]), 3))
    dt = np.float32 if fp32 else np.float64
    return Batch(offsets=offsets, sizes=sizes, phi=phis, pos=pos.astype(dt), a=a)


# The five workload configurations, by what they are (sizes as stated).
RPY_FP64_N1024 = dict(seed=1001, n=1024, phi=0.1, a=1.0, eta=1.0 / (6.0 * np.pi), angular=False,
                      fp32=False, tol=1e-8)
RPY6_FP32_N32768 = dict(seed=1002, n=32768, phi=0.2, a=1.0, eta=1.0, angular=True, fp32=True, tol=1e-5)
ADJOINT_N65536 = dict(seed=1003, n=65536, phi=0.1, a=1.0, eta=1.0, angular=False, fp32=True)
BATCH_BD_256 = dict(seed=1004, S=256, nmin=64, nmax=4096, phi_lo=0.05, phi_hi=0.3, a=1.0, eta=1.0,
                    kT=1.0, dt=1e-3, k_trap=1.0, nsteps=100, tol=1e-4)
MELT_N524288 = dict(seed=1005, n_chains=1024, beads=512, bond=2.2, sigma=0.3, phi=0.05, a=1.0, eta=1.0,
                    angular=True, fp32=True, tol=1e-3)
# Single wall (the paper's "bottom wall" benchmark shape: random positions at
# number density 0.1 / a^3, forces only).
WALL_N32768 = dict(seed=1006, n=32768, rho=0.1, a=1.0, eta=1.0, angular=False, fp32=True)
# The active-roller example (Sec. 5.1): N = 2^15 spheres of radius 0.656 um
# above a wall in water (eta = 1e-3 aJ s / um^3), kT = 4.11e-3 aJ, gravitational
# height 1.5 a, soft repulsion U0 = 4 kT, b = 0.1 a; a torque about y drives
# the rollers.  Initial positions: uniform in a square of area fraction 0.3,
# heights uniform in [a, 2a].
ROLLERS_N32768 = dict(seed=1007, n=32768, a=0.656, eta=1e-3, kT=4.11e-3, h_g=1.5, area_fraction=0.3, dt=1e-3,
                      tol=1e-3, omega=10.0)


def roller_monolayer(seed: int, n: int, a: float, area_fraction: float, fp32: bool = True) -> np.ndarray:
    """N centres uniform in a square of side sqrt(N pi a^2 / area_fraction)
    centred at the origin, heights uniform in [a, 2a]."""
    rng = np.random.default_rng(seed)
    L = float(np.sqrt(n * np.pi * a * a / area_fraction))
    u = rng.uniform(0.0, 1.0, size=(n, 3))
    pos = np.column_stack([(u[:, 0] - 0.5) * L, (u[:, 1] - 0.5) * L, a * (1.0 + u[:, 2])])
    return pos.astype(np.float32 if fp32 else np.float64)
