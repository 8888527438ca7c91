"""Pins of the oracle's roller-example pieces (Sec. 5.1): the soft steric
forces of Eq. (soft_potential), the random finite difference of Eq. (rfd),
and the stochastic Adams-Bashforth step."""
import numpy as np

import oracle


def _energy(pos, U0, b, d_pair, d_wall, wall):
    """Total potential energy, Eq. (soft_potential) summed over pairs (and the wall)."""
    def U(r, d):
        return np.where(r < d, U0 * (1.0 + (d - r) / b), U0 * np.exp((d - r) / b))
    n = len(pos)
    E = 0.0
    for i in range(n):
        for j in range(i + 1, n):
            E += float(U(np.linalg.norm(pos[i] - pos[j]), d_pair))
    if wall:
        E += float(np.sum(U(pos[:, 2], d_wall)))
    return E


def test_soft_repulsion_is_minus_energy_gradient():
    rng = np.random.default_rng(3)
    a = 0.656
    U0, b, dp, dw = 4.0 * 4.11e-3, 0.1 * a, 2 * a, a
    pos = np.column_stack([rng.uniform(-2, 2, (9, 2)), rng.uniform(0.3, 2.5, 9)])
    for wall in (False, True):
        F = oracle.soft_repulsion(pos, U0, b, dp, dw, wall)
        h = 1e-6
        Ffd = np.zeros_like(pos)
        for k in range(pos.size):
            p1 = pos.copy(); p1.flat[k] += h
            p2 = pos.copy(); p2.flat[k] -= h
            Ffd.flat[k] = -(_energy(p1, U0, b, dp, dw, wall) - _energy(p2, U0, b, dp, dw, wall)) / (2 * h)
        assert np.abs(F - Ffd).max() <= 1e-6 * np.abs(F).max(), wall
        if not wall:
            assert np.abs(F.sum(axis=0)).max() <= 1e-12 * np.abs(F).max()   # action = reaction


def test_soft_repulsion_two_particles_closed_form():
    U0, b, d = 2.0, 0.2, 1.5
    for r in (0.5, 1.5, 2.3):
        F = oracle.soft_repulsion(np.array([[0.0, 0, 0], [r, 0, 0]]), U0, b, d, 1.0, False)
        mag = U0 / b if r < d else U0 / b * np.exp((d - r) / b)
        np.testing.assert_allclose(F[1], [mag, 0, 0], rtol=1e-14)
        np.testing.assert_allclose(F[0], [-mag, 0, 0], rtol=1e-14)
    # coincident particles exert no force on each other
    F = oracle.soft_repulsion(np.array([[1.0, 2, 3], [1.0, 2, 3]]), U0, b, d, 1.0, False)
    assert not F.any()


def test_rfd_sample_mean_approaches_divergence():
    a, eta = 1.0, 1.0
    pos = np.array([[0.0, 0.0, 1.4], [1.9, 0.4, 2.2], [-0.8, 1.7, 1.2]])
    ref, _ = oracle.div_fd(pos, a, eta, False, True, 1e-6)
    K = 3000
    S = np.array([oracle.rfd_sample(pos, s, 1e-5, a, eta, False, True)[0] for s in range(K)])
    se = S.std(axis=0, ddof=1) / np.sqrt(K)
    assert (np.abs(S.mean(axis=0) - ref) <= 5 * se + 1e-9).all()


def test_ab_step_first_step_is_euler_and_second_order():
    a, eta = 1.0, 1.0
    rng = np.random.default_rng(1)
    pos = rng.uniform(-4, 4, (6, 3))
    F = rng.standard_normal((6, 3))
    W = np.zeros(18)
    new, u, d = oracle.ab_step(pos, F, None, W, None, None, True, 0.0, 0.01, a, eta, False, False, 0, 1e-4)
    uref, _ = oracle.mdot(pos, F, None, a, eta, False)
    np.testing.assert_allclose(new, pos + 0.01 * uref, rtol=1e-14, atol=1e-15)
    assert not d.any()
    # one sphere in a harmonic trap, F = -k x: dx/dt = -mu0 k x, x(t) = x0 exp(-mu0 k t)
    k = 3.0
    mu0 = 1.0 / (6 * np.pi * eta * a)
    lam = mu0 * k
    errs = []
    for nstep in (20, 40, 80):
        dt = 1.0 / nstep
        x = np.array([[1.0, -0.5, 2.0]])
        pu = pdr = None
        for s in range(nstep):
            x, pu, pdr = oracle.ab_step(x, -k * x, None, np.zeros(3), pu, pdr, s == 0, 0.0, dt, a, eta, False,
                                        False, 0, 1e-4)
        errs.append(np.abs(x - np.array([[1.0, -0.5, 2.0]]) * np.exp(-lam)).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, errs     # global error O(dt^2)


def test_ab_step_noise_and_drift_terms():
    a, eta, kT, dt = 1.0, 1.0, 0.7, 0.01
    rng = np.random.default_rng(2)
    pos = np.column_stack([rng.uniform(-3, 3, (5, 2)), rng.uniform(1.2, 4, 5)])
    F = np.zeros((5, 3))
    W = rng.standard_normal(15)
    new, u, d = oracle.ab_step(pos, F, None, W, None, None, True, kT, dt, a, eta, False, True, 11, 1e-5)
    M = oracle.assemble(pos, a, eta, False, wall=True)
    dref, _ = oracle.rfd_sample(pos, 11, 1e-5, a, eta, False, True)
    y = oracle.sqrt_exact(M, W).reshape(5, 3)
    np.testing.assert_allclose(new, pos + dt * kT * dref + np.sqrt(2 * kT * dt) * y, rtol=1e-13, atol=1e-15)
    # a later step weighs the two drift samples 3/2 and -1/2
    new2, u2, d2 = oracle.ab_step(new, F, None, W, u, d, False, kT, dt, a, eta, False, True, 12, 1e-5)
    M2 = oracle.assemble(new, a, eta, False, wall=True)
    y2 = oracle.sqrt_exact(M2, W).reshape(5, 3)
    np.testing.assert_allclose(new2, new + dt * kT * (1.5 * d2 - 0.5 * d) + np.sqrt(2 * kT * dt) * y2,
                               rtol=1e-13, atol=1e-15)


def test_langevin_velocities_are_the_euler_maruyama_step_over_dt():
    """dt times the Langevin velocities equals the displacement of the first
    (Euler-Maruyama) step of the Adams-Bashforth scheme, a separate oracle
    path; at kT = 0 they are M F."""
    a, eta, kT, dt = 1.0, 1.0, 0.8, 0.01
    rng = np.random.default_rng(9)
    pos = np.column_stack([rng.uniform(-3, 3, (7, 2)), rng.uniform(1.1, 4, 7)])
    F = rng.standard_normal((7, 3))
    T = rng.standard_normal((7, 3))
    W = rng.standard_normal(42)
    lin, ang = oracle.langevin_velocities(pos, F, T, W, kT, dt, a, eta, True, True, 5, 1e-5)
    new, _, _ = oracle.ab_step(pos, F, T, W, None, None, True, kT, dt, a, eta, True, True, 5, 1e-5)
    np.testing.assert_allclose(dt * lin, new - pos, rtol=1e-10, atol=1e-15)
    lin0, ang0 = oracle.langevin_velocities(pos, F, T, W, 0.0, dt, a, eta, True, True, 5, 1e-5)
    u, w = oracle.mdot(pos, F, T, a, eta, True, wall=True)
    np.testing.assert_array_equal(lin0, u)
    np.testing.assert_array_equal(ang0, w)
