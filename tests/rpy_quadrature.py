"""Numerical quadrature of the RPY pair blocks from their defining integral.

The pair mobility is the double envelope integral of the free-space Stokes
Green's function (libMobility paper, Eq. stokestomob, with the coupling of
Eqs. fpcoup / kinetic_constraint).  For the RPY model the force envelope
delta_F is the uniform measure on the sphere surface |x| = a and the torque
envelope delta_T is the uniform density on the ball |x| < a.  With the
divergence theorem the torque coupling becomes a surface integral:

  (1/2) curl(T delta_T)   = (3 / (8 pi a^3)) T x n  on the surface,
  (1/2) int curl v delta_T = (3 / (8 pi a^3)) oint n x v dS,

so, with <.> the surface average over a sphere (area 4 pi a^2) and
G(x) = (I + x x^T / |x|^2) / (8 pi eta |x|):

  M_uF = <G(x - y)>,               M_wF =  (3 / 2a) <[n_x]x G(x - y)>,
  M_uT = -(3 / 2a) <G(x - y) [n_y]x>, M_wT = -(3 / 2a)^2 <[n_x]x G(x - y) [n_y]x>,

x on sphere i (centre d = r e_z), y on sphere j (centre 0).  This module
evaluates those averages with composite Gauss-Legendre rules, graded toward
the point where the integrand is singular when the spheres overlap.  It is a
test helper (an independent route to the same matrices); it shares nothing
with the oracle or the CUDA library.
"""
from __future__ import annotations

import numpy as np


def _graded_panels(lo, hi, s, levels, ratio=0.35):
    """Breakpoints on [lo, hi] graded geometrically toward the point s (lo <= s <= hi)."""
    pts = {lo, hi, s}
    if s > lo:
        for k in range(1, levels + 1):
            pts.add(s - (s - lo) * ratio ** k)
    if s < hi:
        for k in range(1, levels + 1):
            pts.add(s + (hi - s) * ratio ** k)
    return np.array(sorted(pts))


def _composite(bps, order):
    x, w = np.polynomial.legendre.leggauss(order)
    nodes, weights = [], []
    for a, b in zip(bps[:-1], bps[1:]):
        nodes.append(0.5 * (b - a) * x + 0.5 * (b + a))
        weights.append(0.5 * (b - a) * w)
    return np.concatenate(nodes), np.concatenate(weights)


def _cross(v):
    """[v]x for an array of vectors v (..., 3) -> (..., 3, 3)."""
    z = np.zeros(v.shape[:-1])
    return np.stack([
        np.stack([z, -v[..., 2], v[..., 1]], -1),
        np.stack([v[..., 2], z, -v[..., 0]], -1),
        np.stack([-v[..., 1], v[..., 0], z], -1),
    ], -2)


def rpy_blocks_quadrature(r, a=1.0, eta=1.0, order=8, levels=10):
    """Scalar RPY coefficients at separation r (r > 0) by quadrature.

    Returns dict with keys tt_par, tt_perp, g_uT, g_wF, rr_par, rr_perp where,
    for e = e_z, M_uF = tt_perp I + (tt_par - tt_perp) e e^T,
    M_uT = g_uT [e]x, M_wF = g_wF [e]x, M_wT = rr_perp I + (rr_par - rr_perp) e e^T.
    The integrand is averaged over a common rotation about e, so one azimuth
    (phi_x = 0) suffices."""
    # singular point (spheres overlap): cos(theta_x) = -r/2a, cos(theta_y) = r/2a, dphi = 0
    sx = -r / (2 * a)
    sy = r / (2 * a)
    ux, wux = _composite(_graded_panels(-1.0, 1.0, sx if r < 2 * a else -1.0, levels), order)
    uy, wuy = _composite(_graded_panels(-1.0, 1.0, sy if r < 2 * a else 1.0, levels), order)
    # azimuth: graded toward 0 and 2 pi (the same point on the circle)
    ph1, wph1 = _composite(_graded_panels(0.0, np.pi, 0.0, levels), order)
    ph = np.concatenate([ph1, 2 * np.pi - ph1[::-1]])
    wph = np.concatenate([wph1, wph1[::-1]])

    acc = {k: 0.0 for k in ("tt_par", "tt_perp", "g_uT", "g_wF", "rr_par", "rr_perp")}
    sin_x = np.sqrt(np.clip(1 - ux ** 2, 0, None))
    nx = np.stack([sin_x, np.zeros_like(ux), ux], -1)  # (Nx, 3)
    X = nx * a + np.array([0.0, 0.0, r])
    CX = _cross(nx)
    for iy in range(uy.size):
        sy_ = np.sqrt(max(1 - uy[iy] ** 2, 0.0))
        ny = np.stack([sy_ * np.cos(ph), sy_ * np.sin(ph), np.full_like(ph, uy[iy])], -1)  # (Nphi, 3)
        Y = ny * a
        D = X[:, None, :] - Y[None, :, :]  # (Nx, Nphi, 3)
        R = np.linalg.norm(D, axis=-1)
        Rs = np.where(R > 0, R, 1.0)
        E = D / Rs[..., None]
        Gm = (np.eye(3) + E[..., :, None] * E[..., None, :]) / (8 * np.pi * eta * Rs[..., None, None])
        Gm = np.where((R > 0)[..., None, None], Gm, 0.0)
        CY = _cross(ny)  # (Nphi, 3, 3)
        wgt = (wux[:, None] * wuy[iy] * wph[None, :]) / (2.0 * 2.0 * 2.0 * np.pi)
        tt = np.einsum("xp,xpab->ab", wgt, Gm)
        wf = (1.5 / a) * np.einsum("xp,xac,xpcb->ab", wgt, CX, Gm)
        ut = -(1.5 / a) * np.einsum("xp,xpac,pcb->ab", wgt, Gm, CY)
        rr = -(1.5 / a) ** 2 * np.einsum("xp,xac,xpcd,pdb->ab", wgt, CX, Gm, CY)
        acc["tt_par"] += tt[2, 2]
        acc["tt_perp"] += 0.5 * (tt[0, 0] + tt[1, 1])
        # [e_z]x has (1,0) = +1 and (0,1) = -1
        acc["g_wF"] += 0.5 * (wf[1, 0] - wf[0, 1])
        acc["g_uT"] += 0.5 * (ut[1, 0] - ut[0, 1])
        acc["rr_par"] += rr[2, 2]
        acc["rr_perp"] += 0.5 * (rr[0, 0] + rr[1, 1])
    return acc
