"""Python binding of the C ABI in ``include/lm.h`` (ctypes; marshalling only).

Every function keeps the name of the C entry point it calls.  Arrays may be
torch tensors (CUDA or CPU) or numpy arrays; their data pointers are passed
as they are, and the library copies host arrays to and from the GPU itself
(libMobility paper, Sec. 3.2).  Outputs are allocated with the same kind
(device tensor, host tensor or numpy array) as the first array argument.
Calls on CUDA tensors run on torch's current stream.

All arithmetic happens in the CUDA library; if the shared object is missing
this module raises instead of computing anything itself.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LM_DEBUG_BOUNDS=1 selects the bounds-checked build (``_build.build(debug_bounds=True)``)
LIB_PATH = os.path.join(_HERE, "_lib", "liblm_gb300_debug.so" if os.environ.get("LM_DEBUG_BOUNDS") == "1"
                        else "liblm_gb300.so")

LM_OK = 0
LM_ERR_INVALID_ARG = 1
LM_ERR_UNSUPPORTED_GEOMETRY = 2
LM_ERR_STATE = 3
LM_ERR_NONFINITE = 4
LM_ERR_NOT_CONVERGED = 5
LM_ERR_TIMEOUT = 6
LM_ERR_OOM = 7
LM_ERR_CUDA = 8
LM_FP32C = 0
LM_FP64 = 1

_STATUS_NAMES = {0: "LM_OK", 1: "LM_ERR_INVALID_ARG", 2: "LM_ERR_UNSUPPORTED_GEOMETRY", 3: "LM_ERR_STATE",
                 4: "LM_ERR_NONFINITE", 5: "LM_ERR_NOT_CONVERGED", 6: "LM_ERR_TIMEOUT", 7: "LM_ERR_OOM",
                 8: "LM_ERR_CUDA"}


class LmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class lm_pair_config(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int), ("ilp", ctypes.c_int), ("splits", ctypes.c_int),
                ("packed", ctypes.c_int)]


class lm_lanczos_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("rel_change", ctypes.c_double),
                ("norm_w", ctypes.c_double), ("clamped_eigs", ctypes.c_int)]


class lm_profile(ctypes.Structure):
    _fields_ = [("pair_launches", ctypes.c_int64), ("pair_ms", ctypes.c_double),
                ("pair_interactions", ctypes.c_double), ("pair_flops", ctypes.c_double),
                ("vector_iterations", ctypes.c_int64), ("vector_ms", ctypes.c_double),
                ("vector_bytes", ctypes.c_double)]


_lib = None
_vp = ctypes.c_void_p


def lib():
    """Load the shared library (built by ``_build.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2510_02135_gb300._build.build()")
        L = ctypes.CDLL(LIB_PATH)
        st = ctypes.c_int
        L.lm_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_char_p, ctypes.c_char_p, ctypes.c_char_p,
                                ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int, _vp]
        L.lm_create.restype = st
        L.lm_destroy.argtypes = [_vp]
        L.lm_destroy.restype = st
        L.lm_set_stream.argtypes = [_vp, _vp]
        L.lm_set_stream.restype = st
        L.lm_set_positions.argtypes = [_vp, _vp, ctypes.c_int64]
        L.lm_set_positions.restype = st
        L.lm_mdot.argtypes = [_vp, _vp, _vp, _vp, _vp]
        L.lm_mdot.restype = st
        L.lm_sqrt_mdot.argtypes = [_vp, _vp, ctypes.c_uint64, ctypes.c_double, ctypes.c_double, ctypes.c_int, _vp,
                                   _vp, ctypes.POINTER(ctypes.c_int)]
        L.lm_sqrt_mdot.restype = st
        L.lm_div_m.argtypes = [_vp, _vp, _vp]
        L.lm_div_m.restype = st
        L.lm_div_m_rfd.argtypes = [_vp, ctypes.c_uint64, ctypes.c_double, _vp, _vp]
        L.lm_div_m_rfd.restype = st
        L.lm_set_wall_height.argtypes = [_vp, ctypes.c_double]
        L.lm_set_wall_height.restype = st
        L.lm_langevin_velocities.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int, _vp, _vp, ctypes.POINTER(ctypes.c_int)]
        L.lm_langevin_velocities.restype = st
        L.lm_set_sqrt_preconditioner.argtypes = [_vp, ctypes.c_int]
        L.lm_set_sqrt_preconditioner.restype = st
        L.lm_set_reorthogonalization.argtypes = [_vp, ctypes.c_int]
        L.lm_set_reorthogonalization.restype = st
        L.lm_batch_set_reorthogonalization.argtypes = [_vp, ctypes.c_int]
        L.lm_batch_set_reorthogonalization.restype = st
        L.lm_soft_repulsion.argtypes = [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, _vp]
        L.lm_soft_repulsion.restype = st
        L.lm_ab_step.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_int)]
        L.lm_ab_step.restype = st
        L.lm_mdot_backward.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.lm_mdot_backward.restype = st
        L.lm_get_pair_config.argtypes = [_vp, ctypes.POINTER(lm_pair_config)]
        L.lm_get_pair_config.restype = st
        L.lm_set_pair_config.argtypes = [_vp, ctypes.POINTER(lm_pair_config)]
        L.lm_set_pair_config.restype = st
        L.lm_get_adjoint_config.argtypes = [_vp, ctypes.POINTER(lm_pair_config)]
        L.lm_get_adjoint_config.restype = st
        L.lm_set_adjoint_config.argtypes = [_vp, ctypes.POINTER(lm_pair_config)]
        L.lm_set_adjoint_config.restype = st
        L.lm_autotune.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(lm_pair_config)]
        L.lm_autotune.restype = st
        L.lm_get_lanczos_stats.argtypes = [_vp, ctypes.POINTER(lm_lanczos_stats)]
        L.lm_get_lanczos_stats.restype = st
        L.lm_profile_enable.argtypes = [_vp, ctypes.c_int]
        L.lm_profile_enable.restype = st
        L.lm_profile_read.argtypes = [_vp, ctypes.POINTER(lm_profile), ctypes.c_int]
        L.lm_profile_read.restype = st
        L.lm_launch_count.argtypes = [_vp]
        L.lm_launch_count.restype = ctypes.c_int64
        L.lm_last_error.argtypes = []
        L.lm_last_error.restype = ctypes.c_char_p
        L.lm_version.argtypes = []
        L.lm_version.restype = ctypes.c_char_p
        L.lm_mdot_noalloc.argtypes = [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                      _vp, _vp, _vp]
        L.lm_mdot_noalloc.restype = st
        L.lm_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int64, _vp, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, _vp]
        L.lm_batch_create.restype = st
        L.lm_batch_destroy.argtypes = [_vp]
        L.lm_batch_destroy.restype = st
        L.lm_batch_set_positions.argtypes = [_vp, _vp]
        L.lm_batch_set_positions.restype = st
        L.lm_batch_get_positions.argtypes = [_vp, _vp]
        L.lm_batch_get_positions.restype = st
        L.lm_batch_mdot.argtypes = [_vp, _vp, _vp]
        L.lm_batch_mdot.restype = st
        L.lm_batch_sqrt_mdot.argtypes = [_vp, _vp, ctypes.c_uint64, ctypes.c_double, ctypes.c_double, _vp, _vp]
        L.lm_batch_sqrt_mdot.restype = st
        L.lm_batch_bd_run.argtypes = [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_int, _vp]
        L.lm_batch_bd_run.restype = st
        L.lm_batch_set_tiling.argtypes = [_vp, ctypes.c_int, ctypes.c_int]
        L.lm_batch_set_tiling.restype = st
        L.lm_batch_autotune.argtypes = [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.lm_batch_autotune.restype = st
        L.lm_batch_profile_enable.argtypes = [_vp, ctypes.c_int]
        L.lm_batch_profile_enable.restype = st
        L.lm_batch_profile_read.argtypes = [_vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.lm_batch_profile_read.restype = st
        L.lm_batch_profile_pairs.argtypes = [_vp, ctypes.POINTER(ctypes.c_uint64)]
        L.lm_batch_profile_pairs.restype = st
        L.lm_tridiag_sqrt_e1_device.argtypes = [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]
        L.lm_tridiag_sqrt_e1_device.restype = st
        L.lm_tridiag_sqrt_e1_device_paths.argtypes = [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp]
        L.lm_tridiag_sqrt_e1_device_paths.restype = st
        L.lm_batch_solve_counts.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        L.lm_batch_solve_counts.restype = st
        L.lm_batch_timeout_selftest.argtypes = [ctypes.c_longlong]
        L.lm_batch_timeout_selftest.restype = st
        L.lm_philox_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _vp, ctypes.c_int64, _vp]
        L.lm_philox_normals.restype = st
        L.lm_philox4x32_10.argtypes = [_vp, _vp, _vp, ctypes.c_int64, _vp]
        L.lm_philox4x32_10.restype = st
        L.lm_fp32_probe.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), _vp]
        L.lm_fp32_probe.restype = st
        L.lm_debug_bounds.argtypes = []
        L.lm_debug_bounds.restype = ctypes.c_int
        L.lm_debug_check.argtypes = []
        L.lm_debug_check.restype = st
        L.lm_tridiag_sqrt_e1.argtypes = [ctypes.c_int, _vp, _vp, _vp]
        L.lm_tridiag_sqrt_e1.restype = ctypes.c_int
        _lib = L
    return _lib


def _check(status: int):
    if status != LM_OK:
        raise LmError(status, lib().lm_last_error().decode(errors="replace"))


def _torch():
    import torch

    return torch


def _is_tensor(x) -> bool:
    try:
        import torch
    except ImportError:  # pragma: no cover
        return False
    return isinstance(x, torch.Tensor)


def _ptr(x, dtype_f64: bool, n_elems: int | None, name: str):
    """Data pointer of a contiguous array of the solver's dtype (or None)."""
    if x is None:
        return None
    if _is_tensor(x):
        torch = _torch()
        want = torch.float64 if dtype_f64 else torch.float32
        if x.dtype != want:
            raise TypeError(f"{name}: expected {want}, got {x.dtype}")
        if not x.is_contiguous():
            raise ValueError(f"{name}: tensor must be contiguous")
        if n_elems is not None and x.numel() != n_elems:
            raise ValueError(f"{name}: expected {n_elems} elements, got {x.numel()}")
        return x.data_ptr()
    a = x
    if not isinstance(a, np.ndarray):
        raise TypeError(f"{name}: expected a torch tensor or numpy array")
    want = np.float64 if dtype_f64 else np.float32
    if a.dtype != want:
        raise TypeError(f"{name}: expected {np.dtype(want)}, got {a.dtype}")
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError(f"{name}: array must be C-contiguous")
    if n_elems is not None and a.size != n_elems:
        raise ValueError(f"{name}: expected {n_elems} elements, got {a.size}")
    return a.ctypes.data


def _like(ref, shape, f64: bool):
    """Allocate an output of the same kind as ``ref``."""
    if _is_tensor(ref):
        torch = _torch()
        return torch.empty(shape, dtype=torch.float64 if f64 else torch.float32, device=ref.device)
    return np.empty(shape, dtype=np.float64 if f64 else np.float32)


def _current_stream(*arrays):
    for a in arrays:
        if _is_tensor(a) and a.is_cuda:
            torch = _torch()
            return torch.cuda.current_stream(a.device).cuda_stream
    return None


class Solver:
    """Handle of an ``lm_solver``; freed with ``lm_destroy`` when collected."""

    def __init__(self, handle: int, eta: float, a: float, angular: bool, precision: int):
        self.handle = ctypes.c_void_p(handle)
        self.eta = eta
        self.a = a
        self.angular = bool(angular)
        self.precision = precision
        self.f64 = precision == LM_FP64
        self.N = 0
        self._stream = None

    def _sync_stream(self, *arrays):
        s = _current_stream(*arrays)
        if s is not None and s != self._stream:
            _check(lib().lm_set_stream(self.handle, s))
            self._stream = s

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.lm_destroy(h)
            self.handle = None


def lm_create(viscosity: float, hydrodynamic_radius: float, include_angular: bool = False,
              precision: int = LM_FP32C, periodicity=("open", "open", "open"), cuda_stream: int | None = None
              ) -> Solver:
    h = ctypes.c_void_p()
    px, py, pz = (p.encode() for p in periodicity)
    _check(lib().lm_create(ctypes.byref(h), px, py, pz, float(viscosity), float(hydrodynamic_radius),
                           int(bool(include_angular)), int(precision), cuda_stream))
    s = Solver(h.value, viscosity, hydrodynamic_radius, include_angular, precision)
    s._stream = cuda_stream
    return s


def lm_set_positions(s: Solver, pos) -> None:
    n = (pos.numel() if _is_tensor(pos) else np.asarray(pos).size) // 3
    s._sync_stream(pos)
    _check(lib().lm_set_positions(s.handle, _ptr(pos, s.f64, 3 * n, "pos"), n))
    s.N = n


def lm_mdot(s: Solver, forces=None, torques=None, lin_out=None, ang_out=None):
    """[lin; ang] = M [F; T].  Returns (lin, ang); ang is None without angular blocks."""
    ref = forces if forces is not None else torques
    if lin_out is None:
        if ref is None:
            raise ValueError("give forces, torques or lin_out")
        lin_out = _like(ref, (s.N, 3), s.f64)
    if s.angular and ang_out is None:
        ang_out = _like(ref if ref is not None else lin_out, (s.N, 3), s.f64)
    s._sync_stream(forces, torques, lin_out, ang_out)
    n3 = 3 * s.N if s.N else None  # size unknown until positions are set
    _check(lib().lm_mdot(s.handle, _ptr(forces, s.f64, n3, "forces"), _ptr(torques, s.f64, n3, "torques"),
                         _ptr(lin_out, s.f64, n3, "lin_out"), _ptr(ang_out, s.f64, n3, "ang_out")))
    return lin_out, ang_out


def lm_sqrt_mdot(s: Solver, W=None, seed: int = 0, prefactor: float = 1.0, tol: float = 1e-5,
                 max_iter: int = 200, lin_out=None, ang_out=None, like=None, raise_not_converged: bool = True):
    """[lin; ang] = prefactor * M^{1/2} W (Lanczos).  Returns (lin, ang, iterations)."""
    ref = W if W is not None else (lin_out if lin_out is not None else like)
    if ref is None:
        raise ValueError("give W, lin_out or like= to choose where outputs live")
    if lin_out is None:
        lin_out = _like(ref, (s.N, 3), s.f64)
    if s.angular and ang_out is None:
        ang_out = _like(ref, (s.N, 3), s.f64)
    s._sync_stream(W, lin_out, ang_out)
    n3 = 3 * s.N if s.N else None  # size unknown until positions are set
    it = ctypes.c_int(0)
    wptr = _ptr(W, True, (6 if s.angular else 3) * s.N if s.N else None, "W")
    st = lib().lm_sqrt_mdot(s.handle, wptr, int(seed), float(prefactor), float(tol), int(max_iter),
                            _ptr(lin_out, s.f64, n3, "lin_out"), _ptr(ang_out, s.f64, n3, "ang_out"),
                            ctypes.byref(it))
    if st != LM_OK and (raise_not_converged or st != LM_ERR_NOT_CONVERGED):
        _check(st)
    return lin_out, ang_out, it.value


def lm_div_m(s: Solver, like):
    lin = _like(like, (s.N, 3), s.f64)
    ang = _like(like, (s.N, 3), s.f64) if s.angular else None
    s._sync_stream(lin, ang)
    n3 = 3 * s.N if s.N else None  # size unknown until positions are set
    _check(lib().lm_div_m(s.handle, _ptr(lin, s.f64, n3, "lin"), _ptr(ang, s.f64, n3, "ang")))
    return lin, ang


def lm_div_m_rfd(s: Solver, seed: int, delta: float, like):
    """One random-finite-difference sample of div M (Sec. 3.4) with noise key ``seed``."""
    lin = _like(like, (s.N, 3), s.f64)
    ang = _like(like, (s.N, 3), s.f64) if s.angular else None
    s._sync_stream(lin, ang)
    n3 = 3 * s.N if s.N else None
    _check(lib().lm_div_m_rfd(s.handle, int(seed), float(delta), _ptr(lin, s.f64, n3, "lin"),
                              _ptr(ang, s.f64, n3, "ang")))
    return lin, ang


def lm_set_wall_height(s: Solver, height: float) -> None:
    """setParameters(wallHeight): the no-slip wall lies at z = height."""
    _check(lib().lm_set_wall_height(s.handle, float(height)))


def lm_langevin_velocities(s: Solver, forces, torques, kT: float, dt: float, W=None, seed: int = 0,
                           tol: float = 1e-5, max_iter: int = 200, like=None):
    """LangevinVelocities (Sec. 3.2): M [F; T] + sqrt(2 kT / dt) M^{1/2} W + kT divM.
    Returns (lin, ang, Lanczos iterations)."""
    ref = forces if forces is not None else like
    lin = _like(ref, (s.N, 3), s.f64)
    ang = _like(ref, (s.N, 3), s.f64) if s.angular else None
    s._sync_stream(lin, ang)
    it = ctypes.c_int(0)
    nW = (6 if s.angular else 3) * s.N
    _check(lib().lm_langevin_velocities(s.handle, _ptr(forces, s.f64, 3 * s.N, "forces"),
                                        _ptr(torques, s.f64, 3 * s.N, "torques"), _ptr(W, True, nW, "W"), int(seed),
                                        float(kT), float(dt), float(tol), int(max_iter),
                                        _ptr(lin, s.f64, 3 * s.N, "lin"), _ptr(ang, s.f64, 3 * s.N, "ang"),
                                        ctypes.byref(it)))
    return lin, ang, it.value


def lm_set_sqrt_preconditioner(s: Solver, kind: int) -> None:
    """0: none (principal root), 1: Jacobi (B = P^-1 (P M P)^1/2, P = diag(M)^-1/2)."""
    _check(lib().lm_set_sqrt_preconditioner(s.handle, int(kind)))


def lm_set_reorthogonalization(s: Solver, mode: int) -> None:
    """Gram-Schmidt passes of the Lanczos root: 0 DGKS-adaptive (default), 1 always two."""
    _check(lib().lm_set_reorthogonalization(s.handle, int(mode)))


def lm_soft_repulsion(s: Solver, U0: float, b: float, d_pair: float, d_wall: float, like, out=None):
    """Soft steric forces, Eq. (soft_potential) of Sec. 5.1, at the solver's positions."""
    out = _like(like, (s.N, 3), s.f64) if out is None else out
    s._sync_stream(out)
    _check(lib().lm_soft_repulsion(s.handle, float(U0), float(b), float(d_pair), float(d_wall),
                                   _ptr(out, s.f64, 3 * s.N, "forces_out")))
    return out


def lm_ab_step(s: Solver, forces, torques, history, first: bool, kT: float, dt: float, W=None, seed: int = 0,
               tol: float = 1e-5, max_iter: int = 200, pos_out=None, like=None):
    """One stochastic Adams-Bashforth step (Sec. 5.1).  ``history``: device
    float64 tensor of 6N values owned by the caller.  Returns (new positions,
    Lanczos iterations)."""
    ref = forces if forces is not None else like
    pos_out = _like(ref, (s.N, 3), s.f64) if pos_out is None else pos_out
    s._sync_stream(pos_out)
    it = ctypes.c_int(0)
    nW = (6 if s.angular else 3) * s.N
    _check(lib().lm_ab_step(s.handle, _ptr(forces, s.f64, 3 * s.N, "forces"), _ptr(torques, s.f64, 3 * s.N, "torques"),
                            _ptr(W, True, nW, "W"), int(seed), float(kT), float(dt), float(tol), int(max_iter),
                            _ptr(history, True, 6 * s.N, "history"), int(bool(first)), _ptr(pos_out, s.f64, 3 * s.N,
                                                                                             "pos_out"),
                            ctypes.byref(it)))
    return pos_out, it.value


def lm_mdot_backward(s: Solver, forces, torques, grad_lin, grad_ang, need_dX: bool = True, need_dF: bool = True):
    """Adjoint of lm_mdot.  Returns (dX, dF, dT)."""
    dX = _like(forces, (s.N, 3), s.f64) if need_dX else None
    dF = _like(forces, (s.N, 3), s.f64) if need_dF else None
    dT = _like(forces, (s.N, 3), s.f64) if (s.angular and need_dF) else None
    s._sync_stream(forces, torques, grad_lin, grad_ang, dX, dF, dT)
    n3 = 3 * s.N if s.N else None  # size unknown until positions are set
    _check(lib().lm_mdot_backward(s.handle, _ptr(forces, s.f64, n3, "forces"), _ptr(torques, s.f64, n3, "torques"),
                                  _ptr(grad_lin, s.f64, n3, "grad_lin"), _ptr(grad_ang, s.f64, n3, "grad_ang"),
                                  _ptr(dX, s.f64, n3, "dX"), _ptr(dF, s.f64, n3, "dF"), _ptr(dT, s.f64, n3, "dT")))
    return dX, dF, dT


LM_NOALLOC_MAX_N = 32768
LM_NOALLOC_SCRATCH_BYTES = 16 << 20


def lm_mdot_noalloc(pos, forces, torques, viscosity: float, hydrodynamic_radius: float,
                    include_angular: bool, lin_out, ang_out=None, cuda_stream=None) -> None:
    """FP32 mobility product that allocates no device memory (all arrays on
    the device, N <= LM_NOALLOC_MAX_N).  For callers that cannot let the
    library allocate: see lm_mdot_noalloc in include/lm.h.  Runs on
    ``cuda_stream`` (default: torch's current stream of lin_out's device)."""
    n = lin_out.numel() // 3
    if cuda_stream is None:
        cuda_stream = _current_stream(lin_out)
    n3 = 3 * n
    _check(lib().lm_mdot_noalloc(_ptr(pos, False, n3, "pos"), _ptr(forces, False, n3, "forces"),
                                 _ptr(torques, False, n3, "torques"), n, float(viscosity),
                                 float(hydrodynamic_radius), int(bool(include_angular)),
                                 _ptr(lin_out, False, n3, "lin_out"), _ptr(ang_out, False, n3, "ang_out"),
                                 cuda_stream))


class Batch:
    """Handle of an ``lm_batch`` (systems concatenated by ``offsets``)."""

    def __init__(self, handle: int, offsets, eta: float, a: float, max_iter: int):
        self.handle = ctypes.c_void_p(handle)
        self.offsets = np.asarray(offsets, dtype=np.int64)
        self.S = self.offsets.size - 1
        self.Ntot = int(self.offsets[-1])
        self.eta = eta
        self.a = a
        self.max_iter = max_iter

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.lm_batch_destroy(h)
            self.handle = None


def lm_batch_create(offsets, viscosity: float, hydrodynamic_radius: float, max_iter: int = 64,
                    cuda_stream: int | None = None) -> Batch:
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    h = ctypes.c_void_p()
    _check(lib().lm_batch_create(ctypes.byref(h), off.size - 1, off.ctypes.data, float(viscosity),
                                 float(hydrodynamic_radius), int(max_iter), cuda_stream))
    return Batch(h.value, off, viscosity, hydrodynamic_radius, max_iter)


def lm_batch_set_positions(b: Batch, pos) -> None:
    _check(lib().lm_batch_set_positions(b.handle, _ptr(pos, False, 3 * b.Ntot, "pos")))


def lm_batch_get_positions(b: Batch, out=None, like=None):
    if out is None:
        out = _like(like if like is not None else np.empty(0, np.float32), (b.Ntot, 3), False)
    _check(lib().lm_batch_get_positions(b.handle, _ptr(out, False, 3 * b.Ntot, "pos_out")))
    return out


def lm_batch_mdot(b: Batch, forces, lin_out=None):
    if lin_out is None:
        lin_out = _like(forces, (b.Ntot, 3), False)
    _check(lib().lm_batch_mdot(b.handle, _ptr(forces, False, 3 * b.Ntot, "forces"),
                               _ptr(lin_out, False, 3 * b.Ntot, "lin_out")))
    return lin_out


def lm_batch_sqrt_mdot(b: Batch, W=None, seed: int = 0, prefactor: float = 1.0, tol: float = 1e-4, lin_out=None,
                       like=None, raise_not_converged: bool = True):
    """Returns (lin, iterations per system)."""
    ref = W if W is not None else (lin_out if lin_out is not None else like)
    if lin_out is None:
        lin_out = _like(ref, (b.Ntot, 3), False)
    its = np.zeros(b.S, dtype=np.int32)
    st = lib().lm_batch_sqrt_mdot(b.handle, _ptr(W, True, 3 * b.Ntot, "W"), int(seed), float(prefactor), float(tol),
                                  _ptr(lin_out, False, 3 * b.Ntot, "lin_out"), its.ctypes.data)
    if st != LM_OK and (raise_not_converged or st != LM_ERR_NOT_CONVERGED):
        _check(st)
    return lin_out, its


def lm_batch_bd_run(b: Batch, kT: float, dt: float, k_trap: float, nsteps: int, step0: int = 0, seed: int = 0,
                    tol: float = 1e-4, use_graph: bool = True, raise_not_converged: bool = True):
    """nsteps Euler-Maruyama steps in one persistent launch.  Returns iterations per system."""
    its = np.zeros(b.S, dtype=np.int32)
    st = lib().lm_batch_bd_run(b.handle, float(kT), float(dt), float(k_trap), int(nsteps), int(step0), int(seed),
                               float(tol), int(bool(use_graph)), its.ctypes.data)
    if st != LM_OK and (raise_not_converged or st != LM_ERR_NOT_CONVERGED):
        _check(st)
    return its


def lm_batch_set_tiling(b: Batch, threads: int, ilp: int) -> None:
    _check(lib().lm_batch_set_tiling(b.handle, int(threads), int(ilp)))


def lm_batch_set_reorthogonalization(b: Batch, mode: int) -> None:
    _check(lib().lm_batch_set_reorthogonalization(b.handle, int(mode)))


def lm_batch_autotune(b: Batch) -> dict:
    t, i = ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().lm_batch_autotune(b.handle, ctypes.byref(t), ctypes.byref(i)))
    return {"threads": t.value, "ilp": i.value}


def lm_batch_profile_enable(b: Batch, enable: bool = True) -> None:
    _check(lib().lm_batch_profile_enable(b.handle, int(bool(enable))))


def lm_batch_profile_pairs(b: Batch) -> int:
    """Pair evaluations of the last profiled run (all steps and systems)."""
    v = ctypes.c_uint64(0)
    _check(lib().lm_batch_profile_pairs(b.handle, ctypes.byref(v)))
    return int(v.value)


def lm_batch_profile_read(b: Batch) -> np.ndarray:
    """Phase end times (ns) of the last step of the last run (see include/lm.h)."""
    out = np.zeros(5 + 5 * b.max_iter, dtype=np.uint64)
    c = ctypes.c_int(0)
    _check(lib().lm_batch_profile_read(b.handle, out.ctypes.data, out.size, ctypes.byref(c)))
    return out[: c.value]


def lm_tridiag_sqrt_e1_device(alpha, beta, out=None, stream=None, paths=False):
    """sqrt(T_c) e1 for each row c of the (count, m) float64 CUDA tensors alpha,
    beta (beta[:, :m-1] used) with the device tridiagonal step.  With
    paths=True also returns an int array: 0 where the quadrature solved T_c,
    1 where the QR form did."""
    import torch

    count, m = alpha.shape
    if beta.shape != alpha.shape or alpha.dtype != torch.float64 or beta.dtype != torch.float64:
        raise ValueError("alpha and beta must be float64 tensors of equal shape (count, m)")
    alpha, beta = alpha.contiguous(), beta.contiguous()
    if out is None:
        out = torch.empty_like(alpha)
    cs = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    pth = np.zeros(max(int(count), 1), dtype=np.int32) if paths else None
    _check(lib().lm_tridiag_sqrt_e1_device_paths(int(count), int(m), alpha.data_ptr(), beta.data_ptr(),
                                                 out.data_ptr(), pth.ctypes.data if paths else None, cs))
    return (out, pth[: int(count)]) if paths else out


def lm_batch_solve_counts(b: Batch):
    """(posted, solved) tridiagonal solve requests of the last batched run."""
    p, q = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(lib().lm_batch_solve_counts(b.handle, ctypes.byref(p), ctypes.byref(q)))
    return int(p.value), int(q.value)


def lm_batch_timeout_selftest(spin_cycles: int = 2_000_000) -> int:
    """Returns the status of the bounded-wait self test (LM_ERR_TIMEOUT when it works)."""
    return int(lib().lm_batch_timeout_selftest(int(spin_cycles)))


def lm_philox_normals(seed: int, stream: int, out, cuda_stream=None) -> None:
    """Fill the device tensor ``out`` (float64) with the library's Philox normals."""
    if cuda_stream is None:
        cuda_stream = _current_stream(out)
    _check(lib().lm_philox_normals(int(seed), int(stream), _ptr(out, True, None, "out"), out.numel(), cuda_stream))


def lm_philox4x32_10(counters, keys, out, cuda_stream=None) -> None:
    """Raw Philox-4x32-10 words on the device: counters (count, 4), keys
    (count, 2) and out (count, 4) are CUDA int32/uint32 tensors."""
    count = counters.numel() // 4
    if keys.numel() != 2 * count or out.numel() != 4 * count:
        raise ValueError("counters (count, 4), keys (count, 2) and out (count, 4) must agree")
    if cuda_stream is None:
        cuda_stream = _current_stream(out)
    _check(lib().lm_philox4x32_10(counters.data_ptr(), keys.data_ptr(), out.data_ptr(), count, cuda_stream))


def lm_get_pair_config(s: Solver) -> dict:
    c = lm_pair_config()
    _check(lib().lm_get_pair_config(s.handle, ctypes.byref(c)))
    return {"threads": c.threads, "ilp": c.ilp, "splits": c.splits, "packed": c.packed}


def lm_set_pair_config(s: Solver, threads: int, ilp: int, splits: int = 0, packed: int = 0) -> None:
    c = lm_pair_config(threads, ilp, splits, packed)
    _check(lib().lm_set_pair_config(s.handle, ctypes.byref(c)))


def lm_get_adjoint_config(s: Solver) -> dict:
    c = lm_pair_config()
    _check(lib().lm_get_adjoint_config(s.handle, ctypes.byref(c)))
    return {"threads": c.threads, "ilp": c.ilp, "splits": c.splits, "packed": c.packed}


def lm_set_adjoint_config(s: Solver, threads: int, ilp: int, splits: int = 0, packed: int = 1) -> None:
    c = lm_pair_config(threads, ilp, splits, packed)
    _check(lib().lm_set_adjoint_config(s.handle, ctypes.byref(c)))


def lm_autotune(s: Solver, reps: int = 3) -> dict:
    c = lm_pair_config()
    _check(lib().lm_autotune(s.handle, int(reps), ctypes.byref(c)))
    return {"threads": c.threads, "ilp": c.ilp, "splits": c.splits, "packed": c.packed}


def lm_get_lanczos_stats(s: Solver) -> dict:
    st = lm_lanczos_stats()
    _check(lib().lm_get_lanczos_stats(s.handle, ctypes.byref(st)))
    return {"iterations": st.iterations, "converged": bool(st.converged), "rel_change": st.rel_change,
            "norm_w": st.norm_w, "clamped_eigs": st.clamped_eigs}


def lm_profile_enable(s: Solver, enable: bool = True) -> None:
    _check(lib().lm_profile_enable(s.handle, int(bool(enable))))


def lm_profile_read(s: Solver, reset: bool = True) -> dict:
    p = lm_profile()
    _check(lib().lm_profile_read(s.handle, ctypes.byref(p), int(bool(reset))))
    return {"pair_launches": p.pair_launches, "pair_ms": p.pair_ms, "pair_interactions": p.pair_interactions,
            "pair_flops": p.pair_flops, "vector_iterations": p.vector_iterations, "vector_ms": p.vector_ms,
            "vector_bytes": p.vector_bytes}


def lm_fp32_probe(mode: int, iters: int = 1 << 14, cuda_stream=None) -> float:
    """Measured FMA rate of the current GPU in TFLOP/s (mode 0 scalar FP32,
    1 packed f32x2, 2 packed with three distinct operand pairs, 3 packed in
    dependent chains of fresh operands, 4 FP64; for mode 4 pass about 2^8
    iterations)."""
    t = ctypes.c_double(0.0)
    _check(lib().lm_fp32_probe(int(mode), int(iters), ctypes.byref(t), cuda_stream))
    return t.value


def lm_debug_bounds() -> bool:
    """True if the loaded library is the bounds-checked build."""
    return bool(lib().lm_debug_bounds())


def lm_debug_check() -> None:
    """Raise LmError if a device bounds check failed since the last call (bounds-checked build)."""
    _check(lib().lm_debug_check())


def lm_launch_count() -> int:
    return int(lib().lm_launch_count(None))


def lm_version() -> str:
    return lib().lm_version().decode()


def lm_tridiag_sqrt_e1(alpha, beta) -> np.ndarray:
    """Host helper: T^{1/2} e1 for the symmetric tridiagonal T (no GPU)."""
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    out = np.zeros(a.size)
    rc = lib().lm_tridiag_sqrt_e1(a.size, a.ctypes.data, b.ctypes.data if b.size else None, out.ctypes.data)
    if rc != 0:
        raise LmError(LM_ERR_NOT_CONVERGED if rc == -1 else LM_ERR_INVALID_ARG, "tridiagonal square root failed")
    return out


# ---------------------------------------------------------------------------
# Autograd: (X, F, T) -> (u, w) with the fused adjoint as backward.
# ---------------------------------------------------------------------------
def _make_function():
    torch = _torch()

    class MobilityFn(torch.autograd.Function):
        """u, w = M(X) [F; T] with gradients through X, F and T (lm_mdot / lm_mdot_backward)."""

        @staticmethod
        def forward(ctx, solver: Solver, X, F, T):
            X = X.contiguous()
            F = F.contiguous()
            T = T.contiguous() if T is not None else None
            lm_set_positions(solver, X)
            u, w = lm_mdot(solver, F, T)
            ctx.solver = solver
            ctx.save_for_backward(X, F, T if T is not None else F)
            ctx.has_T = T is not None
            return (u, w) if solver.angular else (u, torch.zeros(0, device=u.device, dtype=u.dtype))

        @staticmethod
        def backward(ctx, gu, gw):
            X, F, T = ctx.saved_tensors
            s = ctx.solver
            T = T if ctx.has_T else None
            lm_set_positions(s, X)
            gu = gu.contiguous()
            gw = gw.contiguous() if (s.angular and gw is not None and gw.numel()) else None
            dX, dF, dT = lm_mdot_backward(s, F, T, gu, gw, need_dX=ctx.needs_input_grad[1],
                                          need_dF=ctx.needs_input_grad[2] or ctx.needs_input_grad[3])
            return None, dX, dF, (dT if ctx.has_T else None)

    return MobilityFn


_MobilityFn = None


def mobility(solver: Solver, X, F, T=None):
    """Differentiable u, w = M(X) [F; T] on torch tensors (w is None without angular blocks)."""
    global _MobilityFn
    if _MobilityFn is None:
        _MobilityFn = _make_function()
    u, w = _MobilityFn.apply(solver, X, F, T)
    return u, (w if solver.angular else None)


@dataclass
class NBody:
    """The paper's solver interface (Sec. 3.2) over the C ABI: x and y open,
    z "open" or "single_wall" (the Swan-Brady kernel)."""

    viscosity: float
    hydrodynamicRadius: float
    includeAngular: bool = False
    precision: int = LM_FP32C
    periodicityZ: str = "open"

    def __post_init__(self):
        self.solver = lm_create(self.viscosity, self.hydrodynamicRadius, self.includeAngular, self.precision,
                                periodicity=("open", "open", self.periodicityZ))

    def setPositions(self, pos):
        lm_set_positions(self.solver, pos)

    def Mdot(self, forces=None, torques=None):
        return lm_mdot(self.solver, forces, torques)

    def sqrtMdotW(self, W=None, seed=0, prefactor=1.0, tol=1e-5, max_iter=200, like=None):
        lin, ang, _ = lm_sqrt_mdot(self.solver, W, seed, prefactor, tol, max_iter, like=like)
        return lin, ang

    def divM(self, like):
        return lm_div_m(self.solver, like)

    def setParameters(self, wallHeight: float = 0.0):
        if self.periodicityZ == "single_wall":
            lm_set_wall_height(self.solver, wallHeight)

    def LangevinVelocities(self, dt, kbt, forces=None, torques=None, seed=0, tol=1e-5, max_iter=200, like=None):
        lin, ang, _ = lm_langevin_velocities(self.solver, forces, torques, kbt, dt, seed=seed, tol=tol,
                                             max_iter=max_iter, like=like)
        return lin, ang
