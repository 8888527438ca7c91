"""Single-wall geometry (NBody with z = "single_wall", Sec. 3.5) on the GPU
against the FP64 oracle: per block, every launch configuration, the wall
damping edge cases, and the Lanczos square root."""
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


def wall_suspension(seed, n, a, fp32, zlo=-0.3, zhi=10.0, side=None):
    """Spheres uniform in a slab above the wall; z in [zlo a, zhi a], so some
    overlap the wall and a few sit below it (the damping cases)."""
    rng = np.random.default_rng(seed)
    side = side or (n * 4.0 / 3.0 * np.pi * a ** 3 / (0.1 * (zhi - zlo) * a)) ** 0.5
    pos = np.column_stack([rng.uniform(-side / 2, side / 2, (n, 2)), rng.uniform(zlo * a, zhi * a, n)])
    F = rng.standard_normal((n, 3))
    T = rng.standard_normal((n, 3))
    W = rng.standard_normal(6 * n)
    if fp32:
        pos, F, T = pos.astype(np.float32), F.astype(np.float32), T.astype(np.float32)
    return pos, F, T, W


def make_solver(eta, a, angular, fp64, pos):
    s = lm.lm_create(eta, a, angular, lm.LM_FP64 if fp64 else lm.LM_FP32C, periodicity=("open", "open", "single_wall"))
    lm.lm_set_positions(s, dev(pos))
    return s


make = make_solver


def gpu_mdot(s, F, T):
    u, w = lm.lm_mdot(s, dev(F), dev(T) if s.angular else None)
    torch.cuda.synchronize()
    return u.double().cpu().numpy(), (w.double().cpu().numpy() if w is not None else None)


@pytest.mark.parametrize("fp64,packed", [(False, 0), (False, 1), (True, 0)])
def test_wall_mdot_blocks_match_oracle(orc, fp64, packed):
    n, a, eta = 1500, 1.0, 0.8        # 11 tiles of 128 and a ragged tail of 92
    pos, F, T, _ = wall_suspension(21, n, a, not fp64)
    s = make(eta, a, True, fp64, pos)
    lm.lm_set_pair_config(s, 128, 2 if packed else 1, 0, packed)
    tol = 1e-12 if fp64 else 1e-5
    zero = np.zeros_like(F)
    for name, Fv, Tv in (("F", F, zero), ("T", zero, T), ("FT", F, T)):
        u, w = gpu_mdot(s, Fv, Tv)
        ur, wr = orc.mdot(pos, Fv, Tv, a, eta, True, wall=True)
        assert rel(u, ur) <= tol, (name, "u", rel(u, ur))
        assert rel(w, wr) <= tol, (name, "w", rel(w, wr))
    # translation only
    s3 = make(eta, a, False, fp64, pos)
    lm.lm_set_pair_config(s3, 128, 2 if packed else 1, 0, packed)
    u, _ = gpu_mdot(s3, F, None)
    ur, _ = orc.mdot(pos, F, None, a, eta, False, wall=True)
    assert rel(u, ur) <= tol, rel(u, ur)


@pytest.mark.parametrize("fp64,angular", [(False, False), (False, True), (True, True)])
def test_wall_launch_configs_agree(orc, fp64, angular):
    n, a, eta = 1100, 1.3, 1.0
    pos, F, T, _ = wall_suspension(22, n, a, not fp64)
    s = make(eta, a, angular, fp64, pos)
    ur, wr = orc.mdot(pos, F, T, a, eta, angular, wall=True)
    tol = 1e-12 if fp64 else 1e-5
    for packed in ((0,) if fp64 else (0, 1)):
        for threads in (128, 256):
            for ilp in ((1,) if fp64 else ((2, 4) if packed else (1, 2, 4))):
                for splits in (1, 4, 11):
                    lm.lm_set_pair_config(s, threads, ilp, splits, packed)
                    u, w = gpu_mdot(s, F, T)
                    cfg = (threads, ilp, splits, packed)
                    assert rel(u, ur) <= tol, (cfg, rel(u, ur))
                    if angular:
                        assert rel(w, wr) <= tol, (cfg, rel(w, wr))
    with pytest.raises(lm.LmError) as e:
        lm.lm_set_pair_config(s, 128, 1, 1, packed=1)   # the packed form needs an even ilp
    assert e.value.status == lm.LM_ERR_INVALID_ARG


@pytest.mark.parametrize("fp64,packed", [(False, 0), (False, 1), (True, 0)])
def test_wall_edge_cases(orc, fp64, packed):
    dt = np.float64 if fp64 else np.float32

    def make(eta, a, angular, fp64, pos):
        s = make_solver(eta, a, angular, fp64, pos)
        if packed:
            lm.lm_set_pair_config(s, 128, 2, 0, packed=1)
        return s

    a, eta = 1.3, 0.7
    tol = 1e-12 if fp64 else 2e-6
    rng = np.random.default_rng(9)
    # one sphere at several heights: the Swan-Brady single-sphere mobilities, damped below z = a
    for z in (10.0, 3.0 * a, 1.5 * a, a, 0.6 * a, 0.0, -1.0):
        pos = np.array([[0.2, -0.4, z]], dt)
        F = rng.standard_normal((1, 3)).astype(dt)
        T = rng.standard_normal((1, 3)).astype(dt)
        s = make(eta, a, True, fp64, pos)
        u, w = gpu_mdot(s, F, T)
        ur, wr = orc.mdot(pos, F, T, a, eta, True, wall=True)
        if z <= 0.0:
            assert not u.any() and not w.any()
        else:
            assert np.abs(u - ur).max() <= tol * np.abs(ur).max(), (z, u, ur)
            assert np.abs(w - wr).max() <= tol * np.abs(wr).max(), (z, w, wr)
    # overlapping pair, coincident pair, one particle below the wall, pairs stacked vertically
    for pos in (np.array([[0, 0, 2.0], [0.7, 0.2, 2.3]], dt),
                np.array([[1, 2, 3], [1, 2, 3], [4, 2, 3]], dt),
                np.array([[0, 0, 2.0], [0.5, 0.1, -0.5], [3.0, 0.0, 1.0]], dt),
                np.array([[0, 0, 1.5], [0, 0, 4.5], [0, 0, 9.0]], dt),
                np.column_stack([rng.uniform(-4, 4, (129, 2)), rng.uniform(0.5, 6, 129)]).astype(dt)):
        n = pos.shape[0]
        F = rng.standard_normal((n, 3)).astype(dt)
        T = rng.standard_normal((n, 3)).astype(dt)
        s = make(eta, a, True, fp64, pos)
        u, w = gpu_mdot(s, F, T)
        ur, wr = orc.mdot(pos, F, T, a, eta, True, wall=True)
        assert rel(u, ur) <= tol and rel(w, wr) <= tol, (n, rel(u, ur), rel(w, wr))


def test_wall_sqrt_mdot_matches_exact_root(orc):
    n, a, eta = 300, 1.0, 1.0
    pos, _, _, W = wall_suspension(23, n, a, False, zlo=0.2, zhi=8.0)
    s = make(eta, a, True, True, pos)
    tol = 1e-8
    lin, ang, it = lm.lm_sqrt_mdot(s, dev(W), tol=tol, max_iter=300)
    y = np.concatenate([lin.cpu().numpy().ravel(), ang.cpu().numpy().ravel()])
    M = orc.assemble(pos, a, eta, True, wall=True)
    assert np.linalg.eigvalsh(M).min() > 0.0
    assert rel(y, orc.sqrt_exact(M, W)) <= 20 * tol, (rel(y, orc.sqrt_exact(M, W)), it)
    # FP32 pairs
    s32 = make(eta, a, True, False, pos.astype(np.float32))
    lin, ang, it = lm.lm_sqrt_mdot(s32, dev(W), tol=1e-5, max_iter=300)
    y = np.concatenate([lin.cpu().numpy().ravel(), ang.cpu().numpy().ravel()])
    M32 = orc.assemble(pos.astype(np.float32), a, eta, True, wall=True)
    assert rel(y, orc.sqrt_exact(M32, W)) <= 2e-4, rel(y, orc.sqrt_exact(M32, W))


def test_wall_rejects_the_adjoint():
    pos, F, _, _ = wall_suspension(24, 50, 1.0, True)
    s = make(1.0, 1.0, False, False, pos)
    with pytest.raises(lm.LmError) as e:
        lm.lm_mdot_backward(s, dev(F), None, dev(F), None)
    assert e.value.status == lm.LM_ERR_UNSUPPORTED_GEOMETRY


def _rfd_samples(s, K, delta):
    like = torch.empty((s.N, 3), dtype=torch.float64 if s.f64 else torch.float32, device="cuda")
    L, A = [], []
    for seed in range(K):
        lin, ang = lm.lm_div_m_rfd(s, seed, delta, like)
        L.append(lin.double())
        A.append(ang.double() if ang is not None else lin.double() * 0)
    torch.cuda.synchronize()
    return torch.stack(L).cpu().numpy(), torch.stack(A).cpu().numpy()


@pytest.mark.parametrize("fp64", [True, False])
def test_wall_rfd_mean_matches_fd_divergence(orc, fp64):
    """The thermal-drift test of Sec. 4: the average of random finite
    differences (Eq. rfd) converges to the deterministic central-difference
    divergence of M; compared component-wise within 5 standard errors (plus
    the O(delta^2) bias and, in FP32, the rounding of displaced positions)."""
    a, eta = 1.0, 1.0
    pos = np.array([[0.0, 0.0, 1.3], [2.5, 0.3, 1.8], [-1.0, 2.2, 2.6], [0.4, -2.4, 1.1], [3.0, 3.0, 4.0],
                    [-2.5, -1.5, 1.5]])
    if not fp64:
        pos = pos.astype(np.float32)
    s = make(eta, a, True, fp64, pos)
    ref_l, ref_w = orc.div_fd(pos, a, eta, True, True, 1e-6)
    K = 4000
    delta = 1e-4 if fp64 else 1e-2
    L, A = _rfd_samples(s, K, delta)
    assert np.isfinite(L).all() and np.isfinite(A).all()
    for got, ref in ((L, ref_l), (A, ref_w)):
        mean = got.mean(axis=0)
        se = got.std(axis=0, ddof=1) / np.sqrt(K)
        slack = 5 * se + (1e-8 if fp64 else 3e-3 * np.abs(ref).max())
        assert (np.abs(mean - ref) <= slack).all(), (mean, ref, se)
    # the normal drift of the lowest particles is the largest term and points away from the wall
    assert ref_l[3, 2] > 0 and ref_l[0, 2] > 0


def test_wall_div_m_draws_fresh_samples_and_open_is_zero(orc):
    pos = np.array([[0.0, 0.0, 1.2], [1.5, 0.5, 2.0], [-0.7, 1.1, 3.1]])
    s = make(1.0, 1.0, False, True, pos)
    like = torch.empty((3, 3), dtype=torch.float64, device="cuda")
    d1, _ = lm.lm_div_m(s, like)
    d2, _ = lm.lm_div_m(s, like)
    r0, _ = lm.lm_div_m_rfd(s, 0, 1e-4, like)
    torch.cuda.synchronize()
    assert torch.isfinite(d1).all() and not torch.equal(d1, d2)
    assert torch.equal(d1, r0)          # the first call uses seed 0 and delta = 1e-4 a
    so = lm.lm_create(1.0, 1.0, False, lm.LM_FP64)
    lm.lm_set_positions(so, dev(pos))
    z, _ = lm.lm_div_m_rfd(so, 3, 1e-4, like)
    assert not z.any()


@pytest.mark.parametrize("fp64,wall", [(True, True), (False, True), (True, False)])
def test_jacobi_preconditioned_sqrt_matches_oracle(orc, fp64, wall):
    """lm_sqrt_mdot with the Jacobi preconditioner against the oracle's
    P^{-1} (P M P)^{1/2} W; with a wall the preconditioned iteration needs
    fewer iterations (damped particles spread the spectrum of M)."""
    n, a, eta = 300, 1.0, 1.0
    pos, _, _, W = wall_suspension(25, n, a, False, zlo=-0.2, zhi=8.0)
    if not fp64:
        pos = pos.astype(np.float32)
    geo = ("open", "open", "single_wall" if wall else "open")
    tol = 1e-8 if fp64 else 1e-5
    pre = lm.lm_create(eta, a, True, lm.LM_FP64 if fp64 else lm.LM_FP32C, periodicity=geo)
    lm.lm_set_positions(pre, dev(pos))
    lm.lm_set_sqrt_preconditioner(pre, 1)
    lin, ang, it_pre = lm.lm_sqrt_mdot(pre, dev(W), tol=tol, max_iter=600)
    y = np.concatenate([lin.double().cpu().numpy().ravel(), ang.double().cpu().numpy().ravel()])
    M = orc.assemble(pos, a, eta, True, wall=wall)
    ref = orc.sqrt_jacobi_exact(M, W)
    assert rel(y, ref) <= (20 * tol if fp64 else 2e-4), (rel(y, ref), it_pre)
    plain = lm.lm_create(eta, a, True, lm.LM_FP64 if fp64 else lm.LM_FP32C, periodicity=geo)
    lm.lm_set_positions(plain, dev(pos))
    _, _, it_plain = lm.lm_sqrt_mdot(plain, dev(W), tol=tol, max_iter=600)
    if wall:
        assert it_pre < it_plain, (it_pre, it_plain)
    with pytest.raises(lm.LmError):
        lm.lm_set_sqrt_preconditioner(pre, 2)


def test_wall_n32768_sampled_rows_bench_configuration(orc):
    """The single-wall benchmark workload at full size (N = 32768 on the wall
    at number density 0.1/a^3, forces only) in the autotuned launch
    configuration the benchmark times; 256 sampled rows against the oracle,
    and all blocks on the same positions."""
    from paper_2510_02135_gb300 import inputs as I

    c = I.WALL_N32768
    s_ = I.wall_suspension(c["seed"], c["n"], c["rho"], c["a"], angular=True, fp32=True)
    rows = np.random.default_rng(3).choice(c["n"], 256, replace=False)
    for angular in (False, True):
        s = make(c["eta"], c["a"], angular, False, s_.pos)
        lm.lm_autotune(s, reps=1)
        u, w = gpu_mdot(s, s_.F, s_.T if angular else None)
        ur, wr = orc.mdot(s_.pos, s_.F, s_.T if angular else None, c["a"], c["eta"], angular, rows=rows, wall=True)
        assert rel(u[rows], ur) <= 1e-5, (angular, rel(u[rows], ur))
        if angular:
            assert rel(w[rows], wr) <= 1e-5, rel(w[rows], wr)
        assert np.isfinite(u).all()
