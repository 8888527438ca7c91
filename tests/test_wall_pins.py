"""Pins of the single-wall (Swan-Brady) part of the oracle, independent of it.

* The definition: the blocks are the Faxen operators applied to the Blake
  (1971) Green's function of a point force above a no-slip wall (NBody with
  z = "single_wall", Sec. 3.5, which names the Swan-Brady kernel).  The test
  writes the Blake image system out in sympy, applies the Laplacians and curls
  symbolically, and compares with the oracle's closed forms at random pairs.
* The single-sphere mobilities of Swan & Brady (2007) (tests/golden).
* Symmetry, positive definiteness, the far-field limit, the symmetries of the
  half-space, and the damping reading for particles overlapping the wall.
"""
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _blake_blocks():
    """Blocks of the wall part as numpy functions of (x, y, a), eta = 1,
    derived from the definition.  With R = x - y* (y* = (y1, y2, -y3)) and
    h = y3: d/dx_k = d/dR_k, and d/dy = (-d/dR1, -d/dR2, d/dR3 + d/dh)."""
    sp = pytest.importorskip("sympy")
    R = sp.symbols("R1:4", real=True)
    h, a = sp.symbols("h a", positive=True)
    rho = sp.sqrt(R[0] ** 2 + R[1] ** 2 + R[2] ** 2)
    dlt = lambda i, j: 1 if i == j else 0  # noqa: E731
    mirror = [1, 1, -1]

    def q(i):  # h R_i / R^3 - (delta_i3 / R + R_i R_3 / R^3)
        return h * R[i] / rho ** 3 - (dlt(i, 2) / rho + R[i] * R[2] / rho ** 3)

    # image part of the Blake tensor (times 8 pi eta): -S(R) + 2 h M_jk d/dR_k q_i
    G = sp.Matrix(3, 3, lambda i, j: -(dlt(i, j) / rho + R[i] * R[j] / rho ** 3)
                  + 2 * h * mirror[j] * sp.diff(q(i), R[j]))
    dx = lambda e, k: sp.diff(e, R[k])  # noqa: E731

    def dy(e, k):
        return -sp.diff(e, R[k]) if k < 2 else sp.diff(e, R[2]) + sp.diff(e, h)

    lap_x = lambda e: sum(dx(dx(e, k), k) for k in range(3))  # noqa: E731
    lap_y = lambda e: sum(dy(dy(e, k), k) for k in range(3))  # noqa: E731
    eps = sp.LeviCivita
    Gy = G.applyfunc(lambda e: e + a ** 2 / 6 * lap_y(e))
    Gx = G.applyfunc(lambda e: e + a ** 2 / 6 * lap_x(e))
    uF = Gy.applyfunc(lambda e: e + a ** 2 / 6 * lap_x(e))
    wF = sp.Matrix(3, 3, lambda p, s: sp.Rational(1, 2) * sum(eps(p, k, l) * dx(Gy[l, s], k)
                                                               for k in range(3) for l in range(3)))
    uT = sp.Matrix(3, 3, lambda p, s: sp.Rational(1, 2) * sum(eps(s, k, l) * dy(Gx[p, l], k)
                                                               for k in range(3) for l in range(3)))
    wT = sp.Matrix(3, 3, lambda p, s: sp.Rational(1, 4) * sum(eps(p, k, l) * eps(s, m, n) * dy(dx(G[l, n], k), m)
                                                               for k in range(3) for l in range(3)
                                                               for m in range(3) for n in range(3)))
    f = sp.lambdify((R, h, a), [uF, uT, wF, wT], "numpy")

    def blocks(x, y, av):
        Rv = (x[0] - y[0], x[1] - y[1], x[2] + y[2])
        return [np.array(m, dtype=float) / (8 * np.pi) for m in f(Rv, y[2], av)]

    return blocks


def test_wall_blocks_match_blake_definition():
    blocks = _blake_blocks()
    rng = np.random.default_rng(11)
    cases = []
    for _ in range(12):
        av = rng.uniform(0.5, 2.0)
        x = np.array([*rng.uniform(-6, 6, 2), rng.uniform(av, 8 * av)])
        y = np.array([*rng.uniform(-6, 6, 2), rng.uniform(av, 8 * av)])
        cases.append((x, y, av))
    cases.append((np.array([0.3, -0.2, 1.0]), np.array([0.3, -0.2, 1.0]), 1.0))   # self, touching the wall
    cases.append((np.array([1.0, 2.0, 3.5]), np.array([1.0, 2.0, 3.5]), 1.3))     # self
    cases.append((np.array([0.0, 0.0, 2.0]), np.array([0.0, 0.0, 5.0]), 1.0))     # vertically aligned (s = 0)
    for x, y, av in cases:
        ref = blocks(x, y, av)
        got = oracle.wall_blocks(x, y, av, 1.0)
        for name, g, r in zip(("uF", "uT", "wF", "wT"), got, ref):
            scale = np.abs(r).max() + 1e-300
            assert np.abs(g - r).max() <= 1e-12 * scale, (name, x, y, av, g, r)


def _golden():
    rows = {}
    for line in open(os.path.join(HERE, "golden", "wall_self_mobility.txt")):
        if line.startswith("#") or not line.strip():
            continue
        p = line.split()
        rows[(p[0], p[1])] = np.array([float(v) for v in p[2:]])
    return rows


@pytest.mark.parametrize("a,eta", [(1.0, 1.0), (0.7, 2.5)])
def test_wall_self_mobility_matches_swan_brady(a, eta):
    g = _golden()
    for h in (a, 1.3 * a, 2 * a, 5 * a, 40 * a):
        x = np.array([0.4, -1.7, h])
        M = oracle.assemble(x[None, :], a, eta, True, wall=True)
        xi = a / h
        poly = lambda c: sum(ck * xi ** k for k, ck in enumerate(c))  # noqa: E731
        mt = 1 / (6 * np.pi * eta * a)
        mr = 1 / (8 * np.pi * eta * a ** 3)
        np.testing.assert_allclose(M[0, 0], mt * poly(g[("translation", "parallel")]), rtol=1e-13)
        np.testing.assert_allclose(M[1, 1], mt * poly(g[("translation", "parallel")]), rtol=1e-13)
        np.testing.assert_allclose(M[2, 2], mt * poly(g[("translation", "normal")]), rtol=1e-13)
        np.testing.assert_allclose(M[3, 3], mr * poly(g[("rotation", "parallel")]), rtol=1e-13)
        np.testing.assert_allclose(M[5, 5], mr * poly(g[("rotation", "normal")]), rtol=1e-13)
        cpl = poly(g[("coupling", "parallel")]) / (6 * np.pi * eta * a ** 2)
        # the coupling is a difference of O((a/h)^2) terms that cancel to O((a/h)^4):
        # rounding grows like (h/a)^2 eps
        np.testing.assert_allclose(abs(M[0, 4]), cpl, rtol=1e-15 * (h / a) ** 2 + 1e-14)
        np.testing.assert_allclose(abs(M[1, 3]), cpl, rtol=1e-15 * (h / a) ** 2 + 1e-14)
        assert M[0, 4] == pytest.approx(-M[1, 3], rel=1e-13)      # u_x from T_y = -(u_y from T_x)
        assert np.abs(M[:3, 3:][2]).max() == 0.0 and M[2, 3:].any() == False  # noqa: E712


def _above_wall(rng, n, a, spacing=2.0):
    """n non-overlapping spheres above the wall (centres at z >= a, r >= spacing a)."""
    pts = []
    while len(pts) < n:
        p = np.array([*rng.uniform(-6 * a, 6 * a, 2), rng.uniform(a, 7 * a)])
        if all(np.linalg.norm(p - q) >= spacing * a for q in pts):
            pts.append(p)
    return np.array(pts)


@pytest.mark.parametrize("angular", [False, True])
def test_wall_matrix_symmetric_positive_definite(angular):
    rng = np.random.default_rng(5)
    pos = _above_wall(rng, 40, 1.0)
    M = oracle.assemble(pos, 1.0, 1.0, angular, wall=True)
    assert np.abs(M - M.T).max() <= 1e-15 * np.abs(M).max()
    assert np.linalg.eigvalsh(M).min() > 0.0
    # the wall only lowers the mobility: M_open - M_wall is positive semi-definite
    M0 = oracle.assemble(pos, 1.0, 1.0, angular)
    assert np.linalg.eigvalsh(M0 - M).min() > -1e-13 * np.abs(M0).max()


def test_wall_far_field_limit_and_half_space_symmetries():
    rng = np.random.default_rng(8)
    a, eta = 1.0, 1.0
    pos = rng.uniform(-5, 5, size=(12, 3))
    pos[:, 2] += 1e6   # far from the wall
    Mw = oracle.assemble(pos, a, eta, True, wall=True)
    M0 = oracle.assemble(pos, a, eta, True)
    assert np.abs(Mw - M0).max() <= 2e-6 * np.abs(M0).max()
    # translation parallel to the wall and rotation about its normal
    pos = _above_wall(rng, 10, a, 2.2)
    M = oracle.assemble(pos, a, eta, True, wall=True)
    shift = pos + np.array([3.7, -1.2, 0.0])
    assert np.abs(oracle.assemble(shift, a, eta, True, wall=True) - M).max() <= 1e-13 * np.abs(M).max()
    th = 0.73
    Rz = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    Mr = oracle.assemble(pos @ Rz.T, a, eta, True, wall=True)
    Q = np.kron(np.eye(2 * len(pos)), Rz)
    assert np.abs(Mr - Q @ M @ Q.T).max() <= 1e-13 * np.abs(M).max()
    # a reflection through a vertical plane (x -> -x) is a symmetry too; torques are pseudovectors
    P = np.diag([-1.0, 1.0, 1.0])
    Mp = oracle.assemble(pos @ P, a, eta, True, wall=True)
    n = len(pos)
    Q = np.zeros((6 * n, 6 * n))
    Q[:3 * n, :3 * n] = np.kron(np.eye(n), P)
    Q[3 * n:, 3 * n:] = np.kron(np.eye(n), -P)
    assert np.abs(Mp - Q @ M @ Q.T).max() <= 1e-13 * np.abs(M).max()


def test_wall_damping_reading():
    a, eta = 1.0, 1.0
    rng = np.random.default_rng(2)
    pos = _above_wall(rng, 6, a, 2.5)
    n = len(pos)
    for z, f in ((0.5 * a, 0.5), (0.2 * a, 0.2), (0.0, 0.0), (-0.4, 0.0)):
        p2 = pos.copy()
        p2[0, 2] = z
        pc = pos.copy()
        pc[0, 2] = a   # evaluated at the clamped height
        Mc = oracle.assemble(pc, a, eta, True, wall=True)
        D = np.ones(6 * n)
        D[[0, 1, 2, 3 * n, 3 * n + 1, 3 * n + 2]] = f
        M2 = oracle.assemble(p2, a, eta, True, wall=True)
        assert np.abs(M2 - D[:, None] * Mc * D[None, :]).max() <= 1e-15 * np.abs(Mc).max()
        assert np.linalg.eigvalsh(M2).min() >= -1e-14 * np.abs(M2).max()
    # continuous at z = a
    p3 = pos.copy()
    p3[0, 2] = a * (1 + 1e-9)
    p4 = pos.copy()
    p4[0, 2] = a * (1 - 1e-9)
    M3 = oracle.assemble(p3, a, eta, True, wall=True)
    M4 = oracle.assemble(p4, a, eta, True, wall=True)
    assert np.abs(M3 - M4).max() <= 1e-7 * np.abs(M3).max()


def test_wall_mdot_matches_assembled():
    rng = np.random.default_rng(4)
    pos = rng.uniform(-4, 4, size=(30, 3))
    pos[:, 2] = rng.uniform(-0.5, 5.0, 30)    # includes particles overlapping the wall
    F = rng.standard_normal((30, 3))
    T = rng.standard_normal((30, 3))
    M = oracle.assemble(pos, 1.1, 0.9, True, wall=True)
    u, w = oracle.mdot(pos, F, T, 1.1, 0.9, True, wall=True)
    y = M @ np.concatenate([F.ravel(), T.ravel()])
    np.testing.assert_allclose(np.concatenate([u.ravel(), w.ravel()]), y, rtol=1e-12, atol=1e-14)


def test_div_fd_pins():
    """The deterministic divergence: zero in the open geometry (Sec. 2: no
    thermal drift in bulk), and for one sphere above the wall the derivative
    of the normal self-mobility, d/dh [mu_0 (1 - 9/8 xi + 1/2 xi^3 - 1/8 xi^5)]
    (the golden polynomial, differentiated by hand)."""
    rng = np.random.default_rng(6)
    pos = rng.uniform(-3, 3, size=(8, 3))
    lin, ang = oracle.div_fd(pos, 1.0, 1.0, True, False, 1e-4)
    assert np.abs(lin).max() < 1e-8 and np.abs(ang).max() < 1e-8
    a, eta = 0.8, 1.3
    mt = 1 / (6 * np.pi * eta * a)
    for h in (1.05 * a, 1.7 * a, 4.0 * a):   # the damping makes z = a a kink
        lin, ang = oracle.div_fd(np.array([[0.3, 0.1, h]]), a, eta, True, True, 1e-5)
        xi = a / h
        ref = mt * (9 / 8 * xi - 1.5 * xi ** 3 + 5 / 8 * xi ** 5) / h
        assert abs(lin[0, 2] - ref) <= 1e-7 * abs(ref), (h, lin, ref)
        assert np.abs(lin[0, :2]).max() < 1e-10 * abs(ref) and np.abs(ang).max() < 1e-10 * abs(ref)


def test_jacobi_square_root_pins():
    """B = P^{-1} (P M P)^{1/2}, P = diag(M)^{-1/2}: B B^T = M (so the
    fluctuation-dissipation balance of Eq. fdt holds), and B is the principal
    root when diag(M) is constant (open geometry, translation only)."""
    rng = np.random.default_rng(12)
    pos = np.column_stack([rng.uniform(-5, 5, (20, 2)), rng.uniform(-0.3, 4.0, 20)])   # damped and zero rows
    M = oracle.assemble(pos, 1.0, 1.0, True, wall=True)
    n = M.shape[0]
    B = np.column_stack([oracle.sqrt_jacobi_exact(M, e) for e in np.eye(n)])
    assert np.abs(B @ B.T - M).max() <= 1e-12 * np.abs(M).max()
    posf = rng.uniform(-4, 4, (25, 3))
    Mf = oracle.assemble(posf, 1.0, 1.0, False)
    W = rng.standard_normal(75)
    np.testing.assert_allclose(oracle.sqrt_jacobi_exact(Mf, W), oracle.sqrt_exact(Mf, W), rtol=1e-11, atol=1e-14)
