"""The roller example's time stepping on the GPU (Sec. 5.1): the soft steric
forces of Eq. (soft_potential) and the stochastic Adams-Bashforth step,
against the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2510_02135_gb300 import lm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2510_02135_gb300 import _build

    _build.build()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def rel(y, ref):
    y = np.asarray(y, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    return np.linalg.norm(y - ref) / np.linalg.norm(ref)


def slab(seed, n, a, zlo, zhi, side):
    rng = np.random.default_rng(seed)
    return np.column_stack([rng.uniform(-side / 2, side / 2, (n, 2)), rng.uniform(zlo, zhi, n)]), rng


@pytest.mark.parametrize("fp64,wall", [(False, False), (False, True), (True, True)])
def test_soft_repulsion_matches_oracle(orc, fp64, wall):
    a = 0.656
    U0, b, dp, dw = 4 * 4.11e-3, 0.1 * a, 2 * a, a
    pos, _ = slab(31, 1500, a, -0.2 * a, 6 * a, 40 * a)     # 5 tiles of 256 and a ragged tail
    pos[7] = pos[3]                                           # a coincident pair
    dt_ = np.float64 if fp64 else np.float32
    pos = pos.astype(dt_)
    geo = ("open", "open", "single_wall" if wall else "open")
    s = lm.lm_create(1.0, a, False, lm.LM_FP64 if fp64 else lm.LM_FP32C, periodicity=geo)
    lm.lm_set_positions(s, dev(pos))
    F = lm.lm_soft_repulsion(s, U0, b, dp, dw, like=dev(pos))
    torch.cuda.synchronize()
    ref = orc.soft_repulsion(pos, U0, b, dp, dw, wall)
    assert rel(F.cpu().numpy(), ref) <= (1e-12 if fp64 else 1e-5), rel(F.cpu().numpy(), ref)


def test_ab_step_matches_oracle_fp64_wall(orc):
    a, eta, kT, dt = 1.0, 1.0, 0.5, 1e-3
    n = 150
    pos, rng = slab(32, n, a, 0.6 * a, 6 * a, 24 * a)
    s = lm.lm_create(eta, a, True, lm.LM_FP64, periodicity=("open", "open", "single_wall"))
    lm.lm_set_positions(s, dev(pos))
    hist = torch.zeros(6 * n, dtype=torch.float64, device="cuda")
    X = pos.copy()
    pu = pd = None
    for step in range(2):
        F = orc.soft_repulsion(X, 4 * kT, 0.1 * a, 2 * a, a, True) + np.array([0, 0, -0.5 * kT])   # + gravity
        T = rng.standard_normal((n, 3))
        W = rng.standard_normal(6 * n)
        Xg, it = lm.lm_ab_step(s, dev(F), dev(T), hist, step == 0, kT, dt, W=dev(W), seed=100 + step, tol=1e-11,
                               max_iter=400)
        torch.cuda.synchronize()
        Xr, pu, pd = orc.ab_step(X, F, T, W, pu, pd, step == 0, kT, dt, a, eta, True, True, 100 + step, 1e-4)
        disp = np.abs(Xr - X).max()
        assert np.abs(Xg.cpu().numpy() - Xr).max() <= 1e-7 * disp, (step, np.abs(Xg.cpu().numpy() - Xr).max(), disp)
        h = hist.cpu().numpy()
        np.testing.assert_allclose(h[:3 * n], pu.ravel(), rtol=1e-10, atol=1e-14)
        # (P - Q) / delta amplifies the 1e-13 rounding differences of the two FP64 products by 1 / delta
        np.testing.assert_allclose(h[3 * n:], pd.ravel(), rtol=1e-6, atol=1e-9 * np.abs(pd).max())
        X = Xr


def test_ab_step_deterministic_fp32_open(orc):
    a, eta, dt = 1.0, 1.0, 0.05
    n = 700
    pos, rng = slab(33, n, a, -10, 10, 20)
    pos = pos.astype(np.float32)
    s = lm.lm_create(eta, a, False, lm.LM_FP32C)
    lm.lm_set_positions(s, dev(pos))
    hist = torch.zeros(6 * n, dtype=torch.float64, device="cuda")
    F = rng.standard_normal((n, 3)).astype(np.float32)
    X1, _ = lm.lm_ab_step(s, dev(F), None, hist, True, 0.0, dt)
    X2, _ = lm.lm_ab_step(s, dev(F), None, hist, False, 0.0, dt)
    torch.cuda.synchronize()
    Xr1, pu, pd = orc.ab_step(pos, F, None, np.zeros(3 * n), None, None, True, 0.0, dt, a, eta, False, False, 0, 1e-2)
    Xr2, _, _ = orc.ab_step(X1.cpu().numpy(), F, None, np.zeros(3 * n), pu, pd, False, 0.0, dt, a, eta, False, False,
                            0, 1e-2)
    # FP32 positions: the new coordinates are rounded to FP32 (half an ulp of |x|) on top of the
    # 1e-5 relative parity of the FP32 product
    x1 = X1.cpu().numpy().astype(np.float64)
    x2 = X2.cpu().numpy().astype(np.float64)
    ulp = np.spacing(np.abs(Xr1).astype(np.float32)).astype(np.float64)
    assert (np.abs(x1 - Xr1) <= 1e-5 * np.abs(Xr1 - pos).max() + ulp).all()
    ulp = np.spacing(np.abs(Xr2).astype(np.float32)).astype(np.float64)
    assert (np.abs(x2 - Xr2) <= 1e-5 * np.abs(Xr2 - x1).max() + ulp).all()


def test_roller_like_trajectory_stays_finite():
    """20 stochastic steps of the roller setting: single wall, soft repulsion
    with the wall and between particles, gravity, a torque about y."""
    a, eta, kT, dt = 0.656, 1e-3, 4.11e-3, 0.01
    n = 2000
    pos, rng = slab(34, n, a, 1.0 * a, 3.0 * a, 120 * a)
    pos = pos.astype(np.float32)
    s = lm.lm_create(eta, a, True, lm.LM_FP32C, periodicity=("open", "open", "single_wall"))
    lm.lm_set_positions(s, dev(pos))
    hist = torch.zeros(6 * n, dtype=torch.float64, device="cuda")
    mg = kT / (1.5 * a - a)
    T = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    T[:, 1] = 8 * np.pi * eta * a ** 3 * 10.0
    X = dev(pos)
    for step in range(20):
        F = lm.lm_soft_repulsion(s, 4 * kT, 0.1 * a, 2 * a, a, like=X)
        F[:, 2] -= mg
        X, it = lm.lm_ab_step(s, F, T, hist, step == 0, kT, dt, seed=step, tol=1e-3, max_iter=100)
        assert 0 < it <= 100
    torch.cuda.synchronize()
    Xh = X.cpu().numpy()
    assert np.isfinite(Xh).all()
    assert Xh[:, 2].min() > -a and Xh[:, 2].mean() > 0.5 * a
    assert np.abs(Xh[:, 0] - pos[:, 0]).mean() > 0.0


@pytest.mark.parametrize("fp64,wall,angular", [(True, True, True), (False, True, False), (True, False, True)])
def test_langevin_velocities_match_oracle(orc, fp64, wall, angular):
    """LangevinVelocities (Sec. 3.2): M [F; T] + sqrt(2 kT/dt) M^{1/2} W +
    kT divM against the oracle with the same W and RFD seed."""
    a, eta, kT, dt = 1.0, 1.0, 0.6, 1e-3
    n = 140
    pos, rng = slab(35, n, a, 0.6 * a, 5 * a, 18 * a)
    dt_ = np.float64 if fp64 else np.float32
    pos = pos.astype(dt_)
    F = rng.standard_normal((n, 3)).astype(dt_)
    T = rng.standard_normal((n, 3)).astype(dt_) if angular else None
    W = rng.standard_normal((6 if angular else 3) * n)
    geo = ("open", "open", "single_wall" if wall else "open")
    s = lm.lm_create(eta, a, angular, lm.LM_FP64 if fp64 else lm.LM_FP32C, periodicity=geo)
    lm.lm_set_positions(s, dev(pos))
    tol = 1e-11 if fp64 else 1e-6
    lin, ang, it = lm.lm_langevin_velocities(s, dev(F), dev(T) if angular else None, kT, dt, W=dev(W), seed=17,
                                             tol=tol, max_iter=400)
    torch.cuda.synchronize()
    rl, ra = orc.langevin_velocities(pos, F, T, W, kT, dt, a, eta, angular, wall, 17, 1e-4 if fp64 else 1e-2)
    got = lin.double().cpu().numpy() if not angular else np.concatenate([lin.double().cpu().numpy(),
                                                                          ang.double().cpu().numpy()])
    ref = rl if not angular else np.concatenate([rl, ra])
    # FP32: the RFD difference amplifies the 1e-7 rounding of the FP32 products by 1/delta, and the
    # displaced positions are rounded to FP32 (ulp(|x|) against displacements of delta/2 = 5e-3 a)
    assert rel(got, ref) <= (1e-8 if fp64 else 1e-3), (rel(got, ref), it)


def test_wall_height_shifts_the_geometry(orc):
    """setParameters(wallHeight): positions lifted by h above a wall at z = h
    give the mobility of the unlifted positions above a wall at z = 0."""
    a, eta, h = 1.0, 1.0, 3.25
    pos, rng = slab(36, 300, a, -0.2 * a, 6 * a, 20 * a)
    F = rng.standard_normal((300, 3))
    T = rng.standard_normal((300, 3))
    s = lm.lm_create(eta, a, True, lm.LM_FP64, periodicity=("open", "open", "single_wall"))
    lm.lm_set_positions(s, dev(pos + np.array([0.0, 0.0, h])))
    lm.lm_set_wall_height(s, h)
    u, w = lm.lm_mdot(s, dev(F), dev(T))
    ur, wr = orc.mdot(pos, F, T, a, eta, True, wall=True)
    assert rel(u.cpu().numpy(), ur) <= 1e-12 and rel(w.cpu().numpy(), wr) <= 1e-12
    Fs = lm.lm_soft_repulsion(s, 1.0, 0.1, 2.0, 1.0, like=dev(F))
    Fr = orc.soft_repulsion(pos, 1.0, 0.1, 2.0, 1.0, True)
    assert rel(Fs.cpu().numpy(), Fr) <= 1e-12
    so = lm.lm_create(eta, a, True, lm.LM_FP64)
    with pytest.raises(lm.LmError):
        lm.lm_set_wall_height(so, 1.0)
