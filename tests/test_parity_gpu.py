"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances (relative L2 error per output block, |y - y_ref| / |y_ref|):
  * FP64 path: 1e-12 for M [F; T] (the stated target); the adjoint 1e-11.
  * FP32 compensated path: 1e-5 for M [F; T] per block (the stated target),
    with the max-abs error below 1e-4 x RMS(y_ref); the adjoint 1e-5.
  * Lanczos: against the oracle's Lanczos at the same W and tol, and
    against the exact eigen-root within 20 x tol (the stopping rule bounds the
    change of successive iterates, not the error).
Inputs come from the seeded generators; FP32 workloads use the same
FP32-rounded values on both sides."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2510_02135_gb300 import inputs as I  # noqa: E402
from paper_2510_02135_gb300 import lm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2510_02135_gb300 import _build

    _build.build()


def dev(x):
    return None if x is None else torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    return None if t is None else t.detach().cpu().numpy().astype(np.float64)


def rel(y, ref):
    y = np.asarray(y, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    n = np.linalg.norm(ref)
    return np.linalg.norm(y - ref) / (n if n > 0 else 1.0)


def maxabs_over_rms(y, ref):
    y = np.asarray(y, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    rms = np.sqrt(np.mean(ref ** 2))
    return np.abs(y - ref).max() / (rms if rms > 0 else 1.0)


def make_solver(eta, a, angular, fp64, pos):
    s = lm.lm_create(eta, a, angular, lm.LM_FP64 if fp64 else lm.LM_FP32C)
    lm.lm_set_positions(s, dev(pos))
    return s


make = make_solver


def gpu_mdot(s, F, T):
    u, w = lm.lm_mdot(s, dev(F), dev(T) if s.angular else None,
                      lin_out=torch.empty((s.N, 3), dtype=torch.float64 if s.f64 else torch.float32, device="cuda"),
                      ang_out=(torch.empty((s.N, 3), dtype=torch.float64 if s.f64 else torch.float32,
                                           device="cuda") if s.angular else None))
    torch.cuda.synchronize()
    return host(u), host(w)


# ---------------------------------------------------------------------------
# M [F; T]
# ---------------------------------------------------------------------------
def test_mdot_fp64_translational_n1024(orc):
    c = I.RPY_FP64_N1024
    s_ = I.cube_suspension(c["seed"], c["n"], c["phi"], c["a"], angular=False, fp32=False)
    s = make(c["eta"], c["a"], False, True, s_.pos)
    u, _ = gpu_mdot(s, s_.F, None)
    ur, _ = orc.mdot(s_.pos, s_.F, None, c["a"], c["eta"], False)
    assert rel(u, ur) <= 1e-12


@pytest.mark.parametrize("fp64,packed", [(False, 0), (False, 1), (False, 2), (True, 0)])
def test_mdot_blocks_match_oracle(orc, fp64, packed):
    n = 2500  # 19 tiles of 128 and a ragged tail of 68
    a, eta = 1.0, 1.0
    s_ = I.cube_suspension(77, n, 0.2, a, angular=True, fp32=not fp64)
    s = make(eta, a, True, fp64, s_.pos)
    if packed:
        lm.lm_set_pair_config(s, 128, 8, 0, packed=packed)
    tol = 1e-12 if fp64 else 1e-5
    zero = np.zeros_like(s_.F)
    for name, F, T in (("F", s_.F, zero), ("T", zero, s_.T), ("FT", s_.F, s_.T)):
        u, w = gpu_mdot(s, F, T)
        ur, wr = orc.mdot(s_.pos, F, T, a, eta, True)
        assert rel(u, ur) <= tol, (name, "u", rel(u, ur))
        assert rel(w, wr) <= tol, (name, "w", rel(w, wr))
        if not fp64:
            assert maxabs_over_rms(u, ur) <= 1e-4, (name, maxabs_over_rms(u, ur))
            assert maxabs_over_rms(w, wr) <= 1e-4, (name, maxabs_over_rms(w, wr))


@pytest.mark.parametrize("fp64,angular", [(False, False), (False, True), (True, False), (True, True)])
def test_mdot_launch_configs_agree(orc, fp64, angular):
    n = 1100
    s_ = I.cube_suspension(5, n, 0.15, 1.0, angular=angular, fp32=not fp64)
    s = make(1.0, 1.0, angular, fp64, s_.pos)
    ur, wr = orc.mdot(s_.pos, s_.F, s_.T, 1.0, 1.0, angular)
    tol = 1e-12 if fp64 else 1e-5
    for packed in ((0,) if fp64 else (0, 1, 2, 4)):
        for threads in (128, 256):
            for ilp in ((1, 2) if fp64 else ((4, 8) if packed == 4 else ((2, 4, 8) if packed else (1, 2, 4, 8)))):
                for splits in (1, 3, 9):
                    lm.lm_set_pair_config(s, threads, ilp, splits, packed)
                    u, w = gpu_mdot(s, s_.F, s_.T)
                    cfg = (threads, ilp, splits, packed)
                    assert rel(u, ur) <= tol, (cfg, rel(u, ur))
                    if angular:
                        assert rel(w, wr) <= tol, (cfg, rel(w, wr))
                    if not fp64:
                        assert maxabs_over_rms(u, ur) <= 1e-4, (cfg, maxabs_over_rms(u, ur))


@pytest.mark.parametrize("fp64,packed", [(False, 0), (False, 1), (False, 2), (False, 4), (True, 0)])
def test_mdot_edge_cases(orc, fp64, packed):
    dt = np.float64 if fp64 else np.float32

    def make(eta, a, angular, fp64, pos):
        s = make_solver(eta, a, angular, fp64, pos)
        if packed:
            lm.lm_set_pair_config(s, 128, 4 if packed == 4 else 2, 0, packed=packed)
        return s

    a, eta = 1.3, 0.7
    rng = np.random.default_rng(3)
    tol = 1e-12 if fp64 else 1e-6
    # N = 1: the self mobilities (6 pi eta a)^-1 and (8 pi eta a^3)^-1
    pos = np.zeros((1, 3), dt) + dt(5.0)
    F = rng.standard_normal((1, 3)).astype(dt)
    T = rng.standard_normal((1, 3)).astype(dt)
    s = make(eta, a, True, fp64, pos)
    u, w = gpu_mdot(s, F, T)
    np.testing.assert_allclose(u, F / (6 * np.pi * eta * a), rtol=tol)
    np.testing.assert_allclose(w, T / (8 * np.pi * eta * a ** 3), rtol=tol)
    # overlapping pair, coincident pair, pair at exactly 2a, and a ragged N
    for pos in (np.array([[0, 0, 0], [0.7, 0.2, -0.1]], dt),
                np.array([[1, 2, 3], [1, 2, 3], [4, 2, 3]], dt),
                np.array([[0, 0, 0], [2 * a, 0, 0]], dt),
                rng.uniform(-4, 4, size=(129, 3)).astype(dt),
                rng.uniform(-4, 4, size=(257, 3)).astype(dt)):
        n = pos.shape[0]
        F = rng.standard_normal((n, 3)).astype(dt)
        T = rng.standard_normal((n, 3)).astype(dt)
        s = make(eta, a, True, fp64, pos)
        u, w = gpu_mdot(s, F, T)
        ur, wr = orc.mdot(pos, F, T, a, eta, True)
        assert rel(u, ur) <= tol and rel(w, wr) <= tol, (n, rel(u, ur), rel(w, wr))
        # forces only, torques only, neither
        u1, w1 = lm.lm_mdot(s, dev(F), None)
        ur1, wr1 = orc.mdot(pos, F, None, a, eta, True)
        assert rel(host(u1), ur1) <= tol and rel(host(w1), wr1) <= tol
        u2, w2 = lm.lm_mdot(s, None, dev(T))
        ur2, wr2 = orc.mdot(pos, np.zeros_like(F), T, a, eta, True)
        assert rel(host(u2), ur2) <= tol and rel(host(w2), wr2) <= tol
        lin = torch.full((n, 3), 7.0, dtype=torch.float64 if fp64 else torch.float32, device="cuda")
        ang = torch.full((n, 3), 7.0, dtype=lin.dtype, device="cuda")
        lm.lm_mdot(s, None, None, lin, ang)
        assert not lin.any() and not ang.any()


def test_mdot_rpy6_n32768_sampled_rows(orc):
    """Full-size 6N FP32 workload (N = 32768, phi = 0.2) in the benchmark's
    launch configuration (autotuned, as bench.py does); 256 sampled rows
    against the oracle, per block."""
    c = I.RPY6_FP32_N32768
    s_ = I.cube_suspension(c["seed"], c["n"], c["phi"], c["a"], angular=True, fp32=True)
    s = make(c["eta"], c["a"], True, False, s_.pos)
    lm.lm_autotune(s, reps=2)
    rows = np.random.default_rng(0).choice(c["n"], 256, replace=False)
    zero = np.zeros_like(s_.F)
    for name, F, T in (("F", s_.F, zero), ("T", zero, s_.T), ("FT", s_.F, s_.T)):
        u, w = gpu_mdot(s, F, T)
        ur, wr = orc.mdot(s_.pos, F, T, c["a"], c["eta"], True, rows=rows)
        assert rel(u[rows], ur) <= 1e-5, (name, rel(u[rows], ur))
        assert rel(w[rows], wr) <= 1e-5, (name, rel(w[rows], wr))
        assert np.isfinite(u).all() and np.isfinite(w).all()


def test_mdot_melt_n524288_sampled_rows(orc):
    """Largest workload: 1024 chains x 512 beads, 6N, FP32; 48 sampled rows,
    in the default launch configuration and in the one the autotuner picks
    there (256 threads x 8 i-particles, two j per vote)."""
    c = I.MELT_N524288
    m = I.polymer_melt(c["seed"], c["n_chains"], c["beads"], c["bond"], c["sigma"], c["phi"], c["a"])
    s = make(c["eta"], c["a"], True, False, m.pos)
    rows = np.random.default_rng(1).choice(m.pos.shape[0], 48, replace=False)
    ur, wr = orc.mdot(m.pos, m.F, m.T, c["a"], c["eta"], True, rows=rows)
    for cfg in (None, (256, 8, 20, 2)):
        if cfg is not None:
            lm.lm_set_pair_config(s, *cfg)
        u, w = gpu_mdot(s, m.F, m.T)
        assert rel(u[rows], ur) <= 1e-5, (cfg, rel(u[rows], ur))
        assert rel(w[rows], wr) <= 1e-5, (cfg, rel(w[rows], wr))
        assert np.isfinite(u).all() and np.isfinite(w).all()


@pytest.mark.parametrize("n,angular", [(1 << 20, True), (1 << 21, False)])
def test_mdot_beyond_the_benchmark_sizes_sampled_rows(orc, n, angular):
    """Sizes above the largest benchmark workload (2^20 particles with all four
    blocks, 2^21 translation only; random cube at phi = 0.1): 48 sampled rows
    against the oracle, in the default launch configuration (and, with the
    angular blocks, in the headline tiling of 256 threads x 8 i-particles with
    four j per vote).  Indices, split counts and grids are all far from the
    sizes the smaller tests reach."""
    s_ = I.cube_suspension(77 + angular, n, 0.1, 1.0, angular=angular, fp32=True)
    s = make(1.0, 1.0, angular, False, s_.pos)
    rows = np.random.default_rng(3).choice(n, 48, replace=False)
    ur, wr = orc.mdot(s_.pos, s_.F, s_.T if angular else None, 1.0, 1.0, angular, rows=rows)
    for cfg in (None, (256, 8, 19, 4)) if angular else (None,):
        if cfg is not None:
            lm.lm_set_pair_config(s, *cfg)
        u, w = gpu_mdot(s, s_.F, s_.T if angular else None)
        assert rel(u[rows], ur) <= 1e-5, (cfg, rel(u[rows], ur))
        assert np.isfinite(u).all()
        if angular:
            assert rel(w[rows], wr) <= 1e-5, (cfg, rel(w[rows], wr))
            assert np.isfinite(w).all()


def test_mdot_tt_n65536_sampled_rows(orc):
    """Full-size translation workload of the adjoint benchmark (N = 65536,
    phi = 0.1) in the autotuned forward configuration; 256 sampled rows."""
    c = I.ADJOINT_N65536
    s_ = I.cube_suspension(c["seed"], c["n"], c["phi"], c["a"], angular=False, fp32=True)
    s = make(c["eta"], c["a"], False, False, s_.pos)
    lm.lm_autotune(s, reps=2)
    rows = np.random.default_rng(2).choice(c["n"], 256, replace=False)
    u, _ = gpu_mdot(s, s_.F, None)
    ur, _ = orc.mdot(s_.pos, s_.F, None, c["a"], c["eta"], False, rows=rows)
    assert rel(u[rows], ur) <= 1e-5, rel(u[rows], ur)
    assert np.isfinite(u).all()


def test_host_arrays_are_copied_by_the_library(orc):
    n = 700
    s_ = I.cube_suspension(9, n, 0.1, 1.0, angular=True, fp32=True)
    s = lm.lm_create(1.0, 1.0, True, lm.LM_FP32C)
    lm.lm_set_positions(s, s_.pos)  # numpy (pageable host memory)
    u_h, w_h = lm.lm_mdot(s, s_.F, s_.T)
    assert isinstance(u_h, np.ndarray)
    pin = torch.from_numpy(s_.F).pin_memory()
    pinT = torch.from_numpy(s_.T).pin_memory()
    u_p, w_p = lm.lm_mdot(s, pin, pinT)
    assert not u_p.is_cuda
    u_d, w_d = lm.lm_mdot(s, dev(s_.F), dev(s_.T))
    np.testing.assert_array_equal(u_h, host(u_d))
    np.testing.assert_array_equal(u_p.numpy(), host(u_d))
    np.testing.assert_array_equal(w_h, host(w_d))


# ---------------------------------------------------------------------------
# Lanczos M^{1/2} W
# ---------------------------------------------------------------------------
def test_sqrt_fp64_n1024_matches_eigen_root(orc):
    c = I.RPY_FP64_N1024
    s_ = I.cube_suspension(c["seed"], c["n"], c["phi"], c["a"], angular=False, fp32=False)
    s = make(c["eta"], c["a"], False, True, s_.pos)
    y, _, it = lm.lm_sqrt_mdot(s, dev(s_.W), tol=c["tol"], max_iter=200)
    y = host(y).ravel()
    M = orc.assemble(s_.pos, c["a"], c["eta"], False)
    exact = orc.sqrt_exact(M, s_.W)
    assert rel(y, exact) <= 20 * c["tol"], (rel(y, exact), it)
    yo, ito, conv = orc.lanczos_sqrt(lambda v: M @ v, s_.W, tol=c["tol"], max_iter=200)
    assert conv and abs(ito - it) <= 1
    if ito == it:
        assert rel(y, yo) <= 1e-10, rel(y, yo)
    st = lm.lm_get_lanczos_stats(s)
    assert st["converged"] and st["iterations"] == it
    # prefactor scales linearly
    y2, _, _ = lm.lm_sqrt_mdot(s, dev(s_.W), prefactor=-0.25, tol=c["tol"], max_iter=200)
    np.testing.assert_allclose(host(y2).ravel(), -0.25 * y, rtol=1e-14, atol=1e-300)


def test_sqrt_long_basis_matches_eigen_root(orc):
    """tol = 0 runs up to max_iter = 200 iterations (NOT_CONVERGED by design):
    a basis of more than 128 rows takes more than 16 row groups of the
    Gram-Schmidt multi-dot and its counters; the result stays the exact root
    (converged long before), and a second call reuses the counters."""
    n = 300
    s_ = I.cube_suspension(31, n, 0.3, 1.0, angular=True, fp32=False)
    s = make(1.0, 1.0, True, True, s_.pos)
    M = orc.assemble(s_.pos, 1.0, 1.0, True)
    exact = orc.sqrt_exact(M, s_.W)
    for _ in range(2):
        lin, ang, it = lm.lm_sqrt_mdot(s, dev(s_.W), tol=0.0, max_iter=200, raise_not_converged=False)
        y = np.concatenate([host(lin).ravel(), host(ang).ravel()])
        assert it >= 130, it   # (a breakdown, |beta| ~ 0, may end it before 200)
        assert rel(y, exact) <= 1e-10, rel(y, exact)


@pytest.mark.parametrize("fp64", [False, True])
def test_sqrt_forced_second_gram_schmidt_pass(orc, fp64):
    """Mode 1 runs the second Gram-Schmidt pass at every iteration (the DGKS
    pass that mode 0 skips unless the first pass cancelled): the same
    iterates to rounding, the exact root within the stopping rule, and the
    profile counts two passes at every iteration."""
    n = 300
    s_ = I.cube_suspension(41, n, 0.2, 1.0, angular=True, fp32=not fp64)
    s = make(1.0, 1.0, True, fp64, s_.pos)
    tol = 1e-8 if fp64 else 1e-5
    lin0, ang0, it0 = lm.lm_sqrt_mdot(s, dev(s_.W), tol=tol, max_iter=300)
    lm.lm_set_reorthogonalization(s, 1)
    lm.lm_profile_read(s, reset=True)
    lm.lm_profile_enable(s, True)
    lin1, ang1, it1 = lm.lm_sqrt_mdot(s, dev(s_.W), tol=tol, max_iter=300)
    lm.lm_profile_enable(s, False)
    p = lm.lm_profile_read(s, reset=True)
    y0 = np.concatenate([host(lin0).ravel(), host(ang0).ravel()])
    y1 = np.concatenate([host(lin1).ravel(), host(ang1).ravel()])
    assert abs(it1 - it0) <= 1
    assert rel(y1, y0) <= (1e-12 if fp64 else 1e-5), rel(y1, y0)
    M = orc.assemble(s_.pos, 1.0, 1.0, True)
    assert rel(y1, orc.sqrt_exact(M, s_.W)) <= 20 * tol
    nv = p["vector_iterations"]
    two = sum(2 + (4 if k else 3) + 2 * (2 * k + 5) for k in range(nv)) * 8.0 * 6 * n
    assert it1 <= nv <= it1 + 1 and p["vector_bytes"] == two
    with pytest.raises(lm.LmError):
        lm.lm_set_reorthogonalization(s, 3)


@pytest.mark.parametrize("fp64", [False, True])
def test_sqrt_rpy6_small_matches_oracle(orc, fp64):
    n = 600
    a, eta = 1.0, 1.0
    s_ = I.cube_suspension(12, n, 0.2, a, angular=True, fp32=not fp64)
    s = make(eta, a, True, fp64, s_.pos)
    tol = 1e-5
    lin, ang, it = lm.lm_sqrt_mdot(s, dev(s_.W), tol=tol, max_iter=300)
    y = np.concatenate([host(lin).ravel(), host(ang).ravel()])
    M = orc.assemble(s_.pos, a, eta, True)
    exact = orc.sqrt_exact(M, s_.W)
    assert rel(y, exact) <= 20 * tol, rel(y, exact)
    yo, ito, conv = orc.lanczos_sqrt(lambda v: M @ v, s_.W, tol=tol, max_iter=300)
    if ito == it:
        assert rel(y, yo) <= (1e-10 if fp64 else 1e-5), rel(y, yo)


def test_sqrt_philox_noise_matches_oracle_generator(orc):
    n = 300
    s_ = I.cube_suspension(21, n, 0.1, 1.0, angular=True, fp32=False)
    s = make(1.0, 1.0, True, True, s_.pos)
    seed = 0x1234_5678_9ABC
    lin, ang, it = lm.lm_sqrt_mdot(s, None, seed=seed, tol=1e-10, max_iter=300, like=dev(s_.F))
    y = np.concatenate([host(lin).ravel(), host(ang).ravel()])
    ntot = 6 * n
    q = np.arange((ntot + 3) // 4, dtype=np.uint64)
    ctr = np.zeros((q.size, 4), dtype=np.uint32)
    ctr[:, 0] = (q & 0xFFFFFFFF).astype(np.uint32)
    ctr[:, 1] = (q >> 32).astype(np.uint32)
    words = orc.philox4x32(ctr, np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32))
    z0, z1 = orc.box_muller(words[:, 0:2])
    z2, z3 = orc.box_muller(words[:, 2:4])
    W = np.stack([z0, z1, z2, z3], axis=1).ravel()[:ntot]
    # the library's generator reproduces the oracle's W (to Box-Muller rounding)
    lin_b, ang_b, _ = lm.lm_sqrt_mdot(s, dev(W), tol=1e-10, max_iter=300)
    yb = np.concatenate([host(lin_b).ravel(), host(ang_b).ravel()])
    assert rel(y, yb) <= 1e-13, rel(y, yb)
    M = orc.assemble(s_.pos, 1.0, 1.0, True)
    assert rel(y, orc.sqrt_exact(M, W)) <= 1e-8


def test_fdt_whitening_of_library_noise(orc):
    """The FDT test of Sec. 4 on the library's own output: samples
    y = M^{1/2} W with W from the library's Philox generator (one seed per
    sample), whitened by the oracle's SVD inverse root, are N(0, I):
    component-wise Kolmogorov-Smirnov p-values and the sample covariance."""
    from scipy.stats import kstest

    n = 6
    s_ = I.cube_suspension(53, n, 0.3, 1.0, angular=True, fp32=False)
    s = make(1.0, 1.0, True, True, s_.pos)
    M = orc.assemble(s_.pos, 1.0, 1.0, True)
    U, sv, Vt = np.linalg.svd(M)
    Minvsqrt = U @ np.diag(1.0 / np.sqrt(sv)) @ Vt
    ns = 3000
    like = dev(s_.F)
    Z = np.empty((6 * n, ns))
    for q in range(ns):
        lin, ang, _ = lm.lm_sqrt_mdot(s, None, seed=1000 + q, tol=1e-10, max_iter=6 * n, like=like)
        Z[:, q] = Minvsqrt @ np.concatenate([host(lin).ravel(), host(ang).ravel()])
    pvals = [kstest(Z[c], "norm").pvalue for c in range(6 * n)]
    assert min(pvals) > 1e-4, min(pvals)
    np.testing.assert_allclose(np.cov(Z), np.eye(6 * n), atol=0.12)


def _lanczos_golden():
    """Expected M^{1/2} W of the 6N N = 32768 workload: the oracle's FP64
    Lanczos at tol 1e-10 (written by tests/golden/make_lanczos_rpy6_n32768.py,
    which calls only the oracle): |y|, 8 random projections, 4096 entries."""
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "lanczos_rpy6_n32768.txt")
    g = {"proj": {}, "idx": [], "val": []}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] == "iterations":
            g["iterations"] = int(f[1])
        elif f[0] == "norm_y":
            g["norm_y"] = float(f[1])
        elif f[0] == "proj":
            g["proj"][int(f[1])] = float(f[2])
        elif f[0] == "y":
            g["idx"].append(int(f[1]))
            g["val"].append(float(f[2]))
    g["idx"] = np.array(g["idx"], dtype=np.int64)
    g["val"] = np.array(g["val"])
    return g


def _compare_with_golden(y, g, bound):
    """Relative L2 error of y against the stored oracle vector on the sampled
    entries, and the full-vector error estimated from the random projections
    (g_k . (y - y_ref) ~ N(0, |y - y_ref|^2) for Gaussian g_k)."""
    e_rows = rel(y[g["idx"]], g["val"])
    d = [float(np.random.default_rng(k).standard_normal(y.size) @ y) - p for k, p in g["proj"].items()]
    e_proj = float(np.sqrt(np.mean(np.square(d)))) / g["norm_y"]
    e_norm = abs(float(np.linalg.norm(y)) - g["norm_y"]) / g["norm_y"]
    print(f"vs oracle Lanczos: sampled entries {e_rows:.2e}, projections {e_proj:.2e}, norm {e_norm:.2e}")
    assert e_rows <= bound and e_proj <= bound and e_norm <= bound, (e_rows, e_proj, e_norm)
    return e_rows, e_proj, e_norm


def test_sqrt_rpy6_n32768_matches_oracle_lanczos():
    """Full-size Lanczos (N = 32768, 6N, FP32 pairs, tol 1e-5) in the
    benchmark's autotuned configuration, element by element against the
    oracle's FP64 Lanczos of the same W at tol 1e-10: within 20 x tol on 4096
    sampled entries, on the whole vector (random projections) and in norm."""
    c = I.RPY6_FP32_N32768
    s_ = I.cube_suspension(c["seed"], c["n"], c["phi"], c["a"], angular=True, fp32=True)
    s = make(c["eta"], c["a"], True, False, s_.pos)
    lm.lm_autotune(s, reps=2)
    lin, ang, it = lm.lm_sqrt_mdot(s, dev(s_.W), tol=c["tol"], max_iter=200)
    y = np.concatenate([host(lin).ravel(), host(ang).ravel()])
    g = _lanczos_golden()
    _compare_with_golden(y, g, 20 * c["tol"])
    st = lm.lm_get_lanczos_stats(s)
    assert st["converged"] and 2 <= it < g["iterations"]


def test_sqrt_rpy6_n32768_fp64_matches_oracle_lanczos():
    """The same W through the FP64 path at the oracle's own tolerance (1e-10):
    both run the FP64 iteration with FP64 products, so they agree far inside
    the stopping tolerance (1e-8 relative on the sampled entries)."""
    c = I.RPY6_FP32_N32768
    s_ = I.cube_suspension(c["seed"], c["n"], c["phi"], c["a"], angular=True, fp32=True)
    s = make(c["eta"], c["a"], True, True, s_.pos.astype(np.float64))
    g = _lanczos_golden()
    lin, ang, it = lm.lm_sqrt_mdot(s, dev(s_.W), tol=1e-10, max_iter=g["iterations"] + 20)
    y = np.concatenate([host(lin).ravel(), host(ang).ravel()])
    _compare_with_golden(y, g, 1e-8)
    assert abs(it - g["iterations"]) <= 2, (it, g["iterations"])


def test_sqrt_melt_n524288_self_convergence():
    """Largest workload (N = 524288, 6N, FP32 pairs): no oracle can give the
    root here, so the tol 1e-3 result of the benchmark must lie within
    20 x tol of the tol 1e-4 result for the same W (self-convergence), and
    both must have converged."""
    c = I.MELT_N524288
    m = I.polymer_melt(c["seed"], c["n_chains"], c["beads"], c["bond"], c["sigma"], c["phi"], c["a"])
    s = make(c["eta"], c["a"], True, False, m.pos)
    lm.lm_set_pair_config(s, 256, 8, 20, 2)
    W = dev(m.W)
    ys, its = [], []
    for tol in (c["tol"], 0.1 * c["tol"]):
        lin, ang, it = lm.lm_sqrt_mdot(s, W, tol=tol, max_iter=200)
        assert lm.lm_get_lanczos_stats(s)["converged"]
        ys.append(np.concatenate([host(lin).ravel(), host(ang).ravel()]))
        its.append(it)
        del lin, ang
    assert its[1] > its[0]
    assert np.isfinite(ys[0]).all()
    print(f"self-convergence: tol {c['tol']:g} vs {0.1 * c['tol']:g}: {rel(ys[0], ys[1]):.2e} ({its} iterations)")
    assert rel(ys[0], ys[1]) <= 20 * c["tol"], (rel(ys[0], ys[1]), its)


def test_fp32_probe_rates_are_plausible():
    """The roofline probe: every mode gives a finite rate below twice the
    nominal FP32 peak, and packed FMA with reused operands reaches at least
    half of it."""
    props = torch.cuda.get_device_properties(0)
    nominal = props.multi_processor_count * 128 * 2 * 2.07e9 / 1e12
    rates = [lm.lm_fp32_probe(m, 1 << 10) for m in range(4)]
    assert all(0 < r < 2 * nominal for r in rates), rates
    assert rates[1] > 0.5 * nominal, rates
    # FP64 (mode 4): well below the FP32 rate on this GPU, and above a 1/256 floor
    fp64 = lm.lm_fp32_probe(4, 1 << 6)
    assert nominal / 256 < fp64 < 0.25 * nominal, (fp64, nominal)


def test_profile_counts_pairs_and_lanczos_vector_bytes():
    """The device-time profile: one pair launch and N^2 pairs per product
    (86 flops each with all blocks); one vector-kernel record per Lanczos
    iteration enqueued (the speculative one included), with the algorithmic
    bytes of the rule stated in the header, between the one-pass and the
    two-pass counts."""
    n = 2000
    s_ = I.cube_suspension(5, n, 0.2, 1.0, angular=True, fp32=True)
    s = make(1.0, 1.0, True, False, s_.pos)
    lm.lm_sqrt_mdot(s, dev(s_.W), tol=1e-5, max_iter=200)   # warm-up, not profiled
    lm.lm_profile_read(s, reset=True)
    lm.lm_profile_enable(s, True)
    lm.lm_mdot(s, dev(s_.F), dev(s_.T))
    _, _, it = lm.lm_sqrt_mdot(s, dev(s_.W), tol=1e-5, max_iter=200)
    lm.lm_profile_enable(s, False)
    p = lm.lm_profile_read(s, reset=True)
    nv = p["vector_iterations"]
    assert it <= nv <= it + 1, (it, nv)
    assert p["pair_launches"] == 1 + nv
    assert p["pair_interactions"] == float(n) * n * (1 + nv)
    assert p["pair_flops"] == 86.0 * p["pair_interactions"]
    assert p["pair_ms"] > 0 and p["vector_ms"] > 0
    vec = 8.0 * 6 * n
    one = sum(2 + (4 if k else 3) + (2 * k + 5) for k in range(nv)) * vec
    two = sum(2 + (4 if k else 3) + 2 * (2 * k + 5) for k in range(nv)) * vec
    assert one <= p["vector_bytes"] <= two, (one, p["vector_bytes"], two)
    # reset cleared everything
    p2 = lm.lm_profile_read(s, reset=False)
    assert p2["pair_launches"] == 0 and p2["vector_iterations"] == 0 and p2["vector_bytes"] == 0.0


def test_sqrt_error_paths(orc):
    n = 200
    s_ = I.cube_suspension(4, n, 0.2, 1.0, angular=False, fp32=False)
    s = make(1.0, 1.0, False, True, s_.pos)
    with pytest.raises(lm.LmError) as e:
        lm.lm_sqrt_mdot(s, dev(s_.W), tol=1e-14, max_iter=2)
    assert e.value.status == lm.LM_ERR_NOT_CONVERGED
    y, _, it = lm.lm_sqrt_mdot(s, dev(s_.W), tol=1e-14, max_iter=2, raise_not_converged=False)
    assert it == 2 and torch.isfinite(y).all()
    y0, _, it0 = lm.lm_sqrt_mdot(s, dev(np.zeros(3 * n)), tol=1e-6)
    assert it0 == 0 and not y0.any()
    # an eigenvector of M converges in one iteration
    M = orc.assemble(s_.pos, 1.0, 1.0, False)
    lam, Q = np.linalg.eigh(M)
    W = Q[:, 10] * 2.0
    y1, _, it1 = lm.lm_sqrt_mdot(s, dev(W), tol=1e-10, max_iter=50)
    assert it1 == 1
    np.testing.assert_allclose(host(y1).ravel(), np.sqrt(lam[10]) * W, atol=1e-12)


# ---------------------------------------------------------------------------
# Errors and call order
# ---------------------------------------------------------------------------
def test_call_order_and_argument_errors():
    s = lm.lm_create(1.0, 1.0, False, lm.LM_FP32C)
    F = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(lm.LmError) as e:
        lm.lm_mdot(s, F, None, lin_out=torch.empty_like(F))
    assert e.value.status == lm.LM_ERR_STATE
    bad = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    bad[2, 1] = float("nan")
    with pytest.raises(lm.LmError) as e:
        lm.lm_set_positions(s, bad)
    assert e.value.status == lm.LM_ERR_NONFINITE
    bad[2, 1] = float("inf")
    with pytest.raises(lm.LmError):
        lm.lm_set_positions(s, bad)
    lm.lm_set_positions(s, torch.rand((4, 3), device="cuda"))
    with pytest.raises(lm.LmError) as e:
        lm.lm_mdot(s, F, F)  # torques without angular blocks
    assert e.value.status == lm.LM_ERR_INVALID_ARG
    with pytest.raises(lm.LmError) as e:
        lm.lm_sqrt_mdot(s, torch.zeros(12, dtype=torch.float64, device="cuda"), tol=-1.0)
    assert e.value.status == lm.LM_ERR_INVALID_ARG
    with pytest.raises(lm.LmError) as e:
        lm.lm_set_pair_config(s, 96, 3, 1)
    assert e.value.status == lm.LM_ERR_INVALID_ARG
    with pytest.raises(lm.LmError) as e:
        lm.lm_set_pair_config(s, 128, 1, 1, packed=1)  # the packed form needs an even ilp
    assert e.value.status == lm.LM_ERR_INVALID_ARG
    z, _ = lm.lm_div_m(s, F)
    assert not z.any()


def test_autotune_keeps_results(orc):
    n = 3000
    s_ = I.cube_suspension(31, n, 0.1, 1.0, angular=False, fp32=True)
    s = make(1.0, 1.0, False, False, s_.pos)
    cfg = lm.lm_autotune(s, reps=2)
    assert cfg["threads"] in (128, 256) and cfg["ilp"] in (1, 2, 4, 8) and cfg["splits"] >= 1
    assert lm.lm_get_pair_config(s) == cfg
    u, _ = gpu_mdot(s, s_.F, None)
    ur, _ = orc.mdot(s_.pos, s_.F, None, 1.0, 1.0, False)
    assert rel(u, ur) <= 1e-5


def test_autotune_choice_shared_within_n_bucket(orc):
    """lm_autotune records its choice per (precision, angular, geometry,
    floor(log2 N)): a new solver of the same kind whose N falls in the same
    bucket starts from it (pair and adjoint kernels); other precisions keep
    their own defaults; results stay exact."""
    s_a = I.cube_suspension(61, 2600, 0.1, 1.0, angular=False, fp32=True)
    a = make(1.0, 1.0, False, False, s_a.pos)
    tuned = lm.lm_autotune(a, reps=2)
    tuned_adj = lm.lm_get_adjoint_config(a)
    n_b = 3900                                    # same bucket [2048, 4096)
    s_b = I.cube_suspension(62, n_b, 0.1, 1.0, angular=False, fp32=True)
    b = make(1.0, 1.0, False, False, s_b.pos)
    cb = lm.lm_get_pair_config(b)
    assert (cb["threads"], cb["ilp"], cb["packed"]) == (tuned["threads"], tuned["ilp"], tuned["packed"])
    ab = lm.lm_get_adjoint_config(b)
    assert (ab["threads"], ab["ilp"], ab["packed"]) == (tuned_adj["threads"], tuned_adj["ilp"], tuned_adj["packed"])
    u, _ = gpu_mdot(b, s_b.F, None)
    ur, _ = orc.mdot(s_b.pos, s_b.F, None, 1.0, 1.0, False)
    assert rel(u, ur) <= 1e-5
    c64 = lm.lm_get_pair_config(make(1.0, 1.0, False, True, s_b.pos.astype(np.float64)))
    assert c64["packed"] == 0
