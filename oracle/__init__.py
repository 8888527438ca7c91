"""FP64 CPU oracle for the open-boundary RPY mobility and its square root.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this package; the product library
never does.  It shares no code with the CUDA path (``paper_2510_02135_gb300``)
and imports nothing from it.

Contents (libMobility paper, Sec. 2 and Sec. 3.3):
  * ``pair_blocks``   -- the four 3x3 RPY pair blocks of Eq. (block_mobility)
                         for one separation (C, ``rpy_oracle.c``);
  * ``assemble``      -- the dense 3N x 3N or 6N x 6N grand mobility;
  * ``mdot``          -- the matrix-free product M [F;T], optionally for a
                         subset of rows;
  * ``grad``          -- dL/dX of L = <[G;H], M(X) [F;T]> by the chain rule;
  * ``wall_blocks``   -- the single-wall (Swan-Brady) part of the blocks
                         (Sec. 3.5, NBody with z = "single_wall");
  * ``div_fd``        -- the divergence of M by central differences, the
                         reference of the thermal-drift test (Sec. 4);
  * ``rfd_sample``    -- one random finite difference sample of div M (Eq. rfd);
  * ``soft_repulsion``-- forces of the soft steric potential, Eq. (soft_potential);
  * ``ab_step``       -- one stochastic Adams-Bashforth step (Sec. 5.1);
  * ``langevin_velocities`` -- the terms of Eq. (bdhi) over dt (Sec. 3.2,
                         LangevinVelocities);
  * ``sqrt_jacobi_exact`` -- the square root P^{-1} (P M P)^{1/2} W that the
                         Jacobi-preconditioned Lanczos iteration approximates;
  * ``sqrt_exact``    -- the principal square root M^{1/2} W from the
                         symmetric eigendecomposition (the plain definition);
  * ``lanczos_sqrt``  -- the Krylov (Lanczos) approximation of M^{1/2} W that
                         the paper cites for solvers without their own noise
                         (Sec. 3.3), with full reorthogonalisation.
  * ``philox4x32``    -- the Philox-4x32-10 counter-based generator and the
                         Box-Muller map, for noise drawn inside the method.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(closed forms, a quadrature of Eq. (stokestomob), invariants, library
routines).  Lanczos is pinned against ``sqrt_exact`` at small sizes and, with
no eigendecomposition, by the identity M^{1/2} (M^{1/2} W) = M W and the norm
identity |M^{1/2} W|^2 = W . M W at n = 7200; at the benchmark sizes
(n >= 196608) its results are compared with the same code at a tighter
tolerance, not with an independent definition.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rpy_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lib = None
_lock = threading.Lock()

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (FP64, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.orc_pair_blocks.argtypes = [_dp, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp, _dp]
            lib.orc_pair_blocks_grad.argtypes = [_dp, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp, _dp]
            lib.orc_wall_blocks.argtypes = [_dp, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp, _dp]
            lib.orc_wall_clamp.argtypes = [_dp, ctypes.c_double, _dp]
            lib.orc_wall_clamp.restype = ctypes.c_double
            lib.orc_assemble.argtypes = [ctypes.c_int64, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_int, _dp]
            lib.orc_mdot.argtypes = [ctypes.c_int64, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int, _i64p, ctypes.c_int64, _dp, _dp]
            lib.orc_grad.argtypes = [ctypes.c_int64, _dp, _dp, _dp, _dp, _dp, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int, _i64p, ctypes.c_int64, _dp]
            lib.orc_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _ptr(x):
    return None if x is None else x.ctypes.data_as(_dp)


def num_threads() -> int:
    """OpenMP threads the C oracle runs on."""
    return int(_load().orc_num_threads())


def pair_blocks(d, a: float, eta: float):
    """(uF, uT, wF, wT) 3x3 blocks for separation d = x_i - x_j (Eq. block_mobility)."""
    lib = _load()
    d = _f64(d).reshape(3)
    out = [np.zeros((3, 3)) for _ in range(4)]
    lib.orc_pair_blocks(_ptr(d), a, eta, *[_ptr(o) for o in out])
    return tuple(out)


def pair_blocks_grad(d, a: float, eta: float):
    """d(block)/d d_k for each block: arrays of shape (3, 3, 3), index [k, p, q]."""
    lib = _load()
    d = _f64(d).reshape(3)
    out = [np.zeros((3, 3, 3)) for _ in range(4)]
    lib.orc_pair_blocks_grad(_ptr(d), a, eta, *[_ptr(o) for o in out])
    return tuple(out)


def wall_blocks(x, y, a: float, eta: float):
    """(uF, uT, wF, wT): the wall part of the Swan-Brady blocks (NBody with a
    single wall, Sec. 3.5) for field particle at x and source particle at y,
    both above the wall z = 0 (no damping); x == y gives the self term."""
    lib = _load()
    x = _f64(x).reshape(3)
    y = _f64(y).reshape(3)
    out = [np.zeros((3, 3)) for _ in range(4)]
    lib.orc_wall_blocks(_ptr(x), _ptr(y), a, eta, *[_ptr(o) for o in out])
    return tuple(out)


def wall_clamp(x, a: float):
    """(f, x_clamped): damping factor and evaluation position of a particle
    at x (the reading of the wall damping, Sec. 3.5)."""
    lib = _load()
    x = _f64(x).reshape(3)
    xc = np.zeros(3)
    f = lib.orc_wall_clamp(_ptr(x), a, _ptr(xc))
    return float(f), xc


def assemble(pos, a: float, eta: float, angular: bool, wall: bool = False) -> np.ndarray:
    """Dense grand mobility, ordering [u;w] x [F;T] (Eq. block_mobility);
    ``wall`` adds the no-slip wall at z = 0 (Swan-Brady, with damping)."""
    lib = _load()
    pos = _f64(pos).reshape(-1, 3)
    n = pos.shape[0]
    dim = 6 * n if angular else 3 * n
    M = np.zeros((dim, dim))
    lib.orc_assemble(n, _ptr(pos), a, eta, int(bool(angular)), int(bool(wall)), _ptr(M))
    return M


def mdot(pos, F, T, a: float, eta: float, angular: bool, rows=None, wall: bool = False):
    """[u, w] = M(X) [F; T] by the direct pair sum (Sec. 3.2, Mdot).

    ``T`` may be None (zero torques).  ``rows`` selects output particles.
    ``wall`` adds the no-slip wall at z = 0 (Swan-Brady, with damping).
    Returns (u, w); w is None when ``angular`` is False."""
    lib = _load()
    pos = _f64(pos).reshape(-1, 3)
    n = pos.shape[0]
    F = _f64(F).reshape(n, 3)
    Tt = None if (T is None or not angular) else _f64(T).reshape(n, 3)
    if rows is None:
        r_arr, nrows = None, n
    else:
        r_arr = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        nrows = r_arr.size
    U = np.zeros((nrows, 3))
    W = np.zeros((nrows, 3)) if angular else None
    lib.orc_mdot(n, _ptr(pos), _ptr(F), _ptr(Tt), a, eta, int(bool(angular)), int(bool(wall)),
                 None if r_arr is None else r_arr.ctypes.data_as(_i64p), nrows, _ptr(U), _ptr(W))
    return U, W


def div_fd(pos, a: float, eta: float, angular: bool, wall: bool, delta: float):
    """Deterministic divergence of the mobility by central differences, the
    reference of the thermal-drift test (Sec. 4):
        div M = sum_k [M(q + delta e_k / 2) e_k - M(q - delta e_k / 2) e_k] / delta
    over the 3N position coordinates q_k (e_k the unit vector of q_k; the
    mobility of spheres does not depend on orientation).  Returns (lin, ang):
    the rows of M_uF and, with angular blocks, of M_wF."""
    pos = _f64(pos).reshape(-1, 3)
    n = pos.shape[0]
    lin = np.zeros((n, 3))
    ang = np.zeros((n, 3)) if angular else None
    for k in range(3 * n):
        F = np.zeros((n, 3))
        F.flat[k] = 1.0
        qp = pos.copy()
        qp.flat[k] += 0.5 * delta
        qm = pos.copy()
        qm.flat[k] -= 0.5 * delta
        up, wp = mdot(qp, F, None, a, eta, angular, wall=wall)
        um, wm = mdot(qm, F, None, a, eta, angular, wall=wall)
        lin += (up - um) / delta
        if angular:
            ang += (wp - wm) / delta
    return lin, ang


def grad(pos, F, T, G, H, a: float, eta: float, angular: bool, rows=None) -> np.ndarray:
    """dL/dX for L = sum_i G_i.u_i + H_i.w_i, [u;w] = M(X)[F;T] (chain rule)."""
    lib = _load()
    pos = _f64(pos).reshape(-1, 3)
    n = pos.shape[0]
    F = _f64(F).reshape(n, 3)
    G = _f64(G).reshape(n, 3)
    Tt = None if (T is None or not angular) else _f64(T).reshape(n, 3)
    Ht = None if (H is None or not angular) else _f64(H).reshape(n, 3)
    if rows is None:
        r_arr, nrows = None, n
    else:
        r_arr = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        nrows = r_arr.size
    dX = np.zeros((nrows, 3))
    lib.orc_grad(n, _ptr(pos), _ptr(F), _ptr(Tt), _ptr(G), _ptr(Ht), a, eta, int(bool(angular)),
                 None if r_arr is None else r_arr.ctypes.data_as(_i64p), nrows, _ptr(dX))
    return dX


def sqrt_exact(M: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Principal square root applied to W: Q diag(sqrt(lambda)) Q^T W (Eq. fdt).

    Eigenvalues below zero from round-off are clamped to zero."""
    lam, Q = np.linalg.eigh(M)
    lam = np.clip(lam, 0.0, None)
    W = np.asarray(W, dtype=np.float64)
    root = np.sqrt(lam) if W.ndim == 1 else np.sqrt(lam)[:, None]
    return Q @ (root * (Q.T @ W))


def tridiag_sqrt_e1(alpha, beta) -> np.ndarray:
    """f(T) e1 with f = sqrt for the symmetric tridiagonal T (diag alpha, off beta).

    Uses LAPACK's tridiagonal eigensolver through scipy; negative eigenvalues
    from round-off are clamped to zero."""
    from scipy.linalg import eigh_tridiagonal

    alpha = np.asarray(alpha, dtype=np.float64)
    beta = np.asarray(beta, dtype=np.float64)
    if alpha.size == 1:
        return np.array([np.sqrt(max(alpha[0], 0.0))])
    lam, Q = eigh_tridiagonal(alpha, beta)
    lam = np.clip(lam, 0.0, None)
    return Q @ (np.sqrt(lam) * Q[0, :])


def lanczos_sqrt(matvec, W, tol: float, max_iter: int = 200, breakdown: float = 1e-14):
    """Krylov approximation of M^{1/2} W (Sec. 3.3; Ando, Chow, Saad & Skolnick 2012).

    Steps, in order, for k = 1, 2, ...:
      v_1 = W / |W|
      w   = M v_k
      alpha_k = v_k . w
      w  -= alpha_k v_k + beta_{k-1} v_{k-1}
      h0  = |w|;  w -= V_k (V_k^T w);  h1 = |w|     (full reorthogonalisation)
      if h1 < h0 / sqrt(2):  w -= V_k (V_k^T w)      (second pass only after
                                                       cancellation: the DGKS
                                                       criterion of Daniel,
                                                       Gragg, Kaufman & Stewart 1976)
      beta_k = |w|
      z_k = |W| f(T_k) e1 with f = sqrt,  y_k = V_k z_k
      stop when k >= 2 and |z_k - [z_{k-1}; 0]| / |z_k| < tol   (converged)
      stop when beta_k <= breakdown * max_j |alpha_j|            (invariant subspace)
      stop when k == max_iter                                     (not converged)
      v_{k+1} = w / beta_k
    Since V_k is orthonormal, |y_k - y_{k-1}| = |z_k - [z_{k-1}; 0]|.
    Returns (y, iterations, converged)."""
    W = np.asarray(W, dtype=np.float64).ravel()
    n = W.size
    normW = float(np.linalg.norm(W))
    if normW == 0.0:
        return np.zeros(n), 0, True
    max_iter = int(min(max_iter, n))
    V = np.zeros((max_iter + 1, n))
    V[0] = W / normW
    alpha, beta = [], []
    z_prev = None
    converged = False
    k = 0
    z = None
    for k in range(max_iter):
        w = np.asarray(matvec(V[k]), dtype=np.float64).ravel().copy()
        a_k = float(V[k] @ w)
        w -= a_k * V[k]
        if k > 0:
            w -= beta[k - 1] * V[k - 1]
        h0 = float(np.linalg.norm(w))
        w -= V[: k + 1].T @ (V[: k + 1] @ w)
        h1 = float(np.linalg.norm(w))
        if h1 < h0 / np.sqrt(2.0):
            w -= V[: k + 1].T @ (V[: k + 1] @ w)
        b_k = float(np.linalg.norm(w))
        alpha.append(a_k)
        z = normW * tridiag_sqrt_e1(alpha, beta)
        if k >= 1:
            diff = np.linalg.norm(z - np.concatenate([z_prev, [0.0]])) / np.linalg.norm(z)
            if diff < tol:
                converged = True
                break
        if b_k <= breakdown * max(abs(x) for x in alpha):
            converged = True
            break
        if k + 1 == max_iter:
            break
        beta.append(b_k)
        V[k + 1] = w / b_k
        z_prev = z
    y = V[: k + 1].T @ z
    return y, k + 1, converged


# --------------------------------------------------------------------------
# Philox-4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) and Box-Muller.
# --------------------------------------------------------------------------
_PHILOX_M0 = 0xD2511F53
_PHILOX_M1 = 0xCD9E8D57
_PHILOX_W0 = 0x9E3779B9
_PHILOX_W1 = 0xBB67AE85
_MASK32 = 0xFFFFFFFF


def philox4x32(counter, key):
    """Philox-4x32 with 10 rounds on arrays of counters.

    counter: uint32 array of shape (..., 4); key: uint32 array of shape (..., 2)
    (broadcast).  Returns uint32 array of shape (..., 4)."""
    c = np.array(counter, dtype=np.uint64) & _MASK32
    k = np.array(key, dtype=np.uint64) & _MASK32
    c0, c1, c2, c3 = c[..., 0].copy(), c[..., 1].copy(), c[..., 2].copy(), c[..., 3].copy()
    k0 = np.broadcast_to(k[..., 0], c0.shape).copy()
    k1 = np.broadcast_to(k[..., 1], c0.shape).copy()
    for rnd in range(10):
        p0 = c0 * np.uint64(_PHILOX_M0)
        p1 = c2 * np.uint64(_PHILOX_M1)
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(_MASK32)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(_MASK32)
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
        if rnd < 9:
            k0 = (k0 + np.uint64(_PHILOX_W0)) & np.uint64(_MASK32)
            k1 = (k1 + np.uint64(_PHILOX_W1)) & np.uint64(_MASK32)
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def box_muller(u32_pair):
    """Two standard normals from two uint32 words (FP64 Box-Muller).

    u1 = (w0 + 1) / 2^32 in (0, 1], u2 = w1 / 2^32 in [0, 1);
    n0 = sqrt(-2 ln u1) cos(2 pi u2), n1 = sqrt(-2 ln u1) sin(2 pi u2)."""
    w = np.asarray(u32_pair, dtype=np.float64)
    u1 = (w[..., 0] + 1.0) / 4294967296.0
    u2 = w[..., 1] / 4294967296.0
    rad = np.sqrt(-2.0 * np.log(u1))
    return rad * np.cos(2.0 * np.pi * u2), rad * np.sin(2.0 * np.pi * u2)


def philox_normals(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normals from Philox-4x32-10: element e is normal (e % 4) of
    block q = e // 4, counter (q low, q high, stream low, stream high), key
    (seed low, seed high); normals 0, 1 from words (0, 1), 2, 3 from (2, 3)."""
    nq = (n + 3) // 4
    q = np.arange(nq, dtype=np.uint64)
    ctr = np.zeros((nq, 4), dtype=np.uint32)
    ctr[:, 0] = (q & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    ctr[:, 1] = (q >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = np.uint32(stream & 0xFFFFFFFF)
    ctr[:, 3] = np.uint32((stream >> 32) & 0xFFFFFFFF)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    w = philox4x32(ctr, key)
    z0, z1 = box_muller(w[:, 0:2])
    z2, z3 = box_muller(w[:, 2:4])
    return np.stack([z0, z1, z2, z3], axis=1).ravel()[:n]


def bd_noise_stream(system: int, step: int) -> int:
    """Philox stream of the Brownian noise of one system at one step."""
    return (int(step) << 32) | int(system)


def em_step(pos, a: float, eta: float, kT: float, dt: float, k_trap: float, W, tol: float,
            max_iter: int = 200, exact_sqrt: bool = False):
    """One Euler-Maruyama step of Eq. (bdhi) for an open system (drift term 0):
    X' = X + dt M F + sqrt(2 kT dt) M^{1/2} W with the harmonic trap
    F = -k_trap X (centre at the origin), forces only.
    Returns (X', iterations)."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    n = pos.shape[0]
    F = -k_trap * pos
    u, _ = mdot(pos, F, None, a, eta, False)
    if exact_sqrt:
        M = assemble(pos, a, eta, False)
        y = sqrt_exact(M, W)
        it = 0
    else:
        y, it, _ = lanczos_sqrt(lambda v: mdot(pos, v.reshape(n, 3), None, a, eta, False)[0].ravel(), W, tol,
                                max_iter)
    return pos + dt * u + np.sqrt(2.0 * kT * dt) * y.reshape(n, 3), it


RFD_STREAM = 0x524644   # Philox stream of the random-finite-difference noise ("RFD")


def rfd_sample(pos, seed: int, delta: float, a: float, eta: float, angular: bool, wall: bool):
    """One random finite difference sample of div M, Eq. (rfd) of Sec. 3.4:
    (M(X + delta W/2) [W; 0] - M(X - delta W/2) [W; 0]) / delta with W the 3N
    Philox normals of (seed, RFD_STREAM).  Returns (lin, ang)."""
    pos = _f64(pos).reshape(-1, 3)
    n = pos.shape[0]
    W = philox_normals(seed, RFD_STREAM, 3 * n).reshape(n, 3)
    T0 = np.zeros((n, 3)) if angular else None
    up, wp = mdot(pos + 0.5 * delta * W, W, T0, a, eta, angular, wall=wall)
    um, wm = mdot(pos - 0.5 * delta * W, W, T0, a, eta, angular, wall=wall)
    return (up - um) / delta, ((wp - wm) / delta if angular else None)


def soft_repulsion(pos, U0: float, b: float, d_pair: float, d_wall: float, wall: bool) -> np.ndarray:
    """Forces F = -dU/dX of the soft steric potential of the roller example,
    Eq. (soft_potential) of Sec. 5.1:
        U(r) = U0 (1 + (d - r) / b)   for r < d,
        U(r) = U0 exp((d - r) / b)    for r >= d,
    over every particle pair (d = d_pair, r the centre distance) and, with a
    wall, every particle-wall pair (d = d_wall, r the height z).  A pair at
    r = 0 exerts no force (no direction)."""
    pos = _f64(pos).reshape(-1, 3)
    n = pos.shape[0]
    F = np.zeros((n, 3))
    for i in range(n):
        d = pos[i] - pos
        r = np.sqrt(np.sum(d * d, axis=1))
        m = r > 0.0
        # -dU/dr: U0 / b inside d, (U0 / b) exp((d - r) / b) outside
        mag = np.where(r[m] < d_pair, U0 / b, U0 / b * np.exp((d_pair - r[m]) / b))
        F[i] = np.sum((mag / r[m])[:, None] * d[m], axis=0)
    if wall:
        z = pos[:, 2]
        F[:, 2] += np.where(z < d_wall, U0 / b, U0 / b * np.exp((d_wall - z) / b))
    return F


def ab_step(pos, F, T, W, prev_u, prev_d, first: bool, kT: float, dt: float, a: float, eta: float,
            angular: bool, wall: bool, rfd_seed: int, rfd_delta: float):
    """One step of the stochastic Adams-Bashforth scheme of Sec. 5.1 for the
    positions X (N x 3):
      X' = X + dt [(3/2) u^n - (1/2) u^{n-1} + kT ((3/2) d^n - (1/2) d^{n-1})]
             + sqrt(2 kT dt) (M^n)^{1/2} W,
    u^n = (M^n [F; T])_lin, d^n = one RFD sample of div M^n (seed rfd_seed;
    zero in the open geometry or at kT = 0).  ``first``: the previous terms
    equal the current ones (an Euler-Maruyama step).  W: 3N (6N with angular
    blocks) normals; the linear part of (M^n)^{1/2} W moves X; the square root
    is the principal one (eigendecomposition).  Returns (X', u^n, d^n)."""
    pos = _f64(pos).reshape(-1, 3)
    n = pos.shape[0]
    u, _ = mdot(pos, F, T if angular else None, a, eta, angular, wall=wall)
    if wall and kT > 0.0:
        d, _ = rfd_sample(pos, rfd_seed, rfd_delta, a, eta, angular, wall)
    else:
        d = np.zeros((n, 3))
    if first:
        prev_u, prev_d = u, d
    M = assemble(pos, a, eta, angular, wall=wall)
    y = sqrt_exact(M, _f64(W).ravel())[: 3 * n].reshape(n, 3)
    new = pos + dt * (1.5 * u - 0.5 * np.asarray(prev_u) + kT * (1.5 * d - 0.5 * np.asarray(prev_d))) \
        + np.sqrt(2.0 * kT * dt) * y
    return new, u, d


def sqrt_jacobi_exact(M: np.ndarray, W: np.ndarray) -> np.ndarray:
    """B W with B = P^{-1} (P M P)^{1/2}, P = diag(M)^{-1/2} (P_ii = 1 where
    M_ii = 0): a square root of M (B B^T = M) that the Jacobi-preconditioned
    Lanczos iteration approximates (Sec. 3.3 notes that the Krylov method can
    be preconditioned).  The principal root of P M P is taken from its
    symmetric eigendecomposition."""
    d = np.diag(M).copy()
    p = np.where(d > 0.0, 1.0 / np.sqrt(np.where(d > 0.0, d, 1.0)), 1.0)
    Mt = p[:, None] * M * p[None, :]
    return sqrt_exact(Mt, np.asarray(W, dtype=np.float64).ravel()) / p


def langevin_velocities(pos, F, T, W, kT: float, dt: float, a: float, eta: float, angular: bool, wall: bool,
                        rfd_seed: int, rfd_delta: float):
    """LangevinVelocities of Sec. 3.2 (the terms of Eq. bdhi divided by dt):
    M [F; T] + sqrt(2 kT / dt) M^{1/2} W + kT div M, with the principal root
    (eigendecomposition) and one RFD sample of div M (zero in the open
    geometry or at kT = 0).  Returns (lin, ang)."""
    pos = _f64(pos).reshape(-1, 3)
    n = pos.shape[0]
    u, w = mdot(pos, F, T if angular else None, a, eta, angular, wall=wall)
    y = np.zeros((6 if angular else 3) * n)
    if kT > 0.0:
        y = np.sqrt(2.0 * kT / dt) * sqrt_exact(assemble(pos, a, eta, angular, wall=wall), _f64(W).ravel())
    lin = u + y[: 3 * n].reshape(n, 3)
    ang = (w + y[3 * n:].reshape(n, 3)) if angular else None
    if wall and kT > 0.0:
        dl, da = rfd_sample(pos, rfd_seed, rfd_delta, a, eta, angular, wall)
        lin = lin + kT * dl
        if angular:
            ang = ang + kT * da
    return lin, ang
