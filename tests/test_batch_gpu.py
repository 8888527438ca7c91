"""GPU parity of the batched persistent kernel (lm_batch_*) and its noise
generator, against the FP64 oracle and against the single-system API.

Batched Euler-Maruyama step (Eq. bdhi, open geometry, drift 0):
  x' = x + dt M F + sqrt(2 kT dt) M^{1/2} W,   F = -k x,
with W of system s at step t drawn from Philox-4x32-10 (key seed, stream
(t << 32) | s); the oracle draws the same numbers from its own
implementation of the generator."""
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
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def rel(y, r):
    y = np.asarray(y, np.float64).ravel()
    r = np.asarray(r, np.float64).ravel()
    return np.linalg.norm(y - r) / max(np.linalg.norm(r), 1e-300)


def small_batch(seed=7, S=6, nmin=20, nmax=700):
    return I.batch_suspensions(seed, S=S, nmin=nmin, nmax=nmax)


def test_philox_normals_match_oracle(orc):
    for seed, stream, n in ((0, 0, 1000), (123456789012345, (7 << 32) | 3, 4099)):
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        lm.lm_philox_normals(seed, stream, out)
        torch.cuda.synchronize()
        ref = orc.philox_normals(seed, stream, n)
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=0, atol=1e-13)


def test_device_philox_known_answer_vectors():
    """The device generator (the one source of the library's noise) against
    the published Philox-4x32-10 known-answer vectors, read from
    tests/golden/philox4x32_10_kat.txt, bitwise."""
    import os

    rows = []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append([int(w, 16) for w in line.split()])
    a = np.array(rows, dtype=np.uint64).astype(np.uint32).view(np.int32)
    ctr = torch.from_numpy(np.ascontiguousarray(a[:, 0:4])).cuda()
    key = torch.from_numpy(np.ascontiguousarray(a[:, 4:6])).cuda()
    out = torch.zeros_like(ctr)
    lm.lm_philox4x32_10(ctr, key, out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), a[:, 6:10].view(np.uint32))


def test_batch_mdot_matches_oracle(orc):
    b_ = small_batch()
    rng = np.random.default_rng(1)
    F = rng.standard_normal((b_.pos.shape[0], 3)).astype(np.float32)
    b = lm.lm_batch_create(b_.offsets, 1.0, 1.0)
    lm.lm_batch_set_positions(b, dev(b_.pos))
    for threads, ilp in ((128, 1), (64, 2), (128, 2), (64, 1)):
        lm.lm_batch_set_tiling(b, threads, ilp)
        u = lm.lm_batch_mdot(b, dev(F)).cpu().numpy()
        for s in range(b.S):
            o0, o1 = b_.offsets[s], b_.offsets[s + 1]
            ur, _ = orc.mdot(b_.pos[o0:o1], F[o0:o1], None, 1.0, 1.0, False)
            assert rel(u[o0:o1], ur) <= 1e-5, (threads, ilp, s, rel(u[o0:o1], ur))


def test_batch_sqrt_matches_oracle(orc):
    b_ = small_batch(seed=9)
    n = b_.pos.shape[0]
    W = np.random.default_rng(2).standard_normal(3 * n)
    b = lm.lm_batch_create(b_.offsets, 1.0, 1.0, max_iter=100)
    lm.lm_batch_set_positions(b, dev(b_.pos))
    tol = 1e-6
    y, its = lm.lm_batch_sqrt_mdot(b, dev(W), tol=tol, prefactor=0.5)
    y = y.cpu().numpy()
    for s in range(b.S):
        o0, o1 = b_.offsets[s], b_.offsets[s + 1]
        M = orc.assemble(b_.pos[o0:o1], 1.0, 1.0, False)
        ws = W[3 * o0:3 * o1]
        exact = 0.5 * orc.sqrt_exact(M, ws)
        assert rel(y[o0:o1], exact) <= 20 * tol, (s, rel(y[o0:o1], exact), its[s])
        yo, ito, conv = orc.lanczos_sqrt(lambda v: M @ v, ws, tol=tol, max_iter=100)
        assert abs(int(its[s]) - ito) <= 1, (s, its[s], ito)


def test_batch_profile_counts_pair_evaluations():
    """The profiling pair counter: one batched product evaluates exactly
    sum_s N_s^2 pairs; a batched square root at least sum_s N_s^2 per
    Lanczos iteration of system s (speculative iterations on top)."""
    b_ = small_batch(seed=23, S=5)
    sizes = np.diff(b_.offsets)
    F = np.random.default_rng(2).standard_normal((b_.pos.shape[0], 3)).astype(np.float32)
    b = lm.lm_batch_create(b_.offsets, 1.0, 1.0)
    lm.lm_batch_set_positions(b, dev(b_.pos))
    lm.lm_batch_profile_enable(b, True)
    for threads, ilp in ((64, 1), (128, 2)):
        lm.lm_batch_set_tiling(b, threads, ilp)
        lm.lm_batch_mdot(b, dev(F))
        assert lm.lm_batch_profile_pairs(b) == int(np.sum(sizes.astype(np.int64) ** 2))
    W = np.random.default_rng(3).standard_normal(3 * b_.pos.shape[0])
    _, its = lm.lm_batch_sqrt_mdot(b, dev(W), tol=1e-6)
    assert lm.lm_batch_profile_pairs(b) >= int(np.sum(sizes.astype(np.int64) ** 2 * np.asarray(its)))


def test_batch_sqrt_philox_equals_explicit_noise(orc):
    b_ = small_batch(seed=11)
    n = b_.pos.shape[0]
    b = lm.lm_batch_create(b_.offsets, 1.0, 1.0)
    lm.lm_batch_set_positions(b, dev(b_.pos))
    seed = 99
    y1, it1 = lm.lm_batch_sqrt_mdot(b, None, seed=seed, tol=1e-5, like=dev(b_.pos))
    W = np.concatenate([orc.philox_normals(seed, s, 3 * int(b_.sizes[s])) for s in range(b.S)])
    y2, it2 = lm.lm_batch_sqrt_mdot(b, dev(W), tol=1e-5)
    np.testing.assert_array_equal(it1, it2)
    assert rel(y1.cpu().numpy(), y2.cpu().numpy()) <= 1e-12


def test_batch_forced_second_gram_schmidt_pass(orc):
    """Two Gram-Schmidt passes at every iteration (the DGKS pass that the
    adaptive test rarely asks for) give the same iterates to rounding, and the
    results stay within the stopping tolerance of the exact root."""
    b_ = small_batch(seed=17, S=5)
    n = b_.pos.shape[0]
    W = np.random.default_rng(5).standard_normal(3 * n)
    b = lm.lm_batch_create(b_.offsets, 1.0, 1.0)
    lm.lm_batch_set_positions(b, dev(b_.pos))
    y0, it0 = lm.lm_batch_sqrt_mdot(b, dev(W), tol=1e-6)
    lm.lm_batch_set_reorthogonalization(b, 1)
    y1, it1 = lm.lm_batch_sqrt_mdot(b, dev(W), tol=1e-6)
    y0, y1 = y0.cpu().numpy(), y1.cpu().numpy()
    for s in range(b.S):
        o0, o1 = b_.offsets[s], b_.offsets[s + 1]
        assert abs(int(it0[s]) - int(it1[s])) <= 1
        assert rel(y1[o0:o1], y0[o0:o1]) <= 1e-5, s
        M = orc.assemble(b_.pos[o0:o1], 1.0, 1.0, False)
        exact = orc.sqrt_exact(M, W[3 * o0:3 * o1])
        assert rel(y1[o0:o1], exact) <= 20 * 1e-6, (s, rel(y1[o0:o1], exact))
    with pytest.raises(lm.LmError):
        lm.lm_batch_set_reorthogonalization(b, 2)


def test_batch_sqrt_mixed_breakdown_and_large_systems(orc):
    """Systems that end almost at once (one particle: W is an eigenvector of M),
    after a few iterations with round-off residuals (two far-apart particles,
    three touching ones), next to two suspensions: in one iteration some
    systems end in the first Gram-Schmidt pass and others may take the DGKS
    pass, all in the same launch.  Every system matches the exact root and the
    oracle's iteration count; the forced second pass agrees to rounding."""
    rng = np.random.default_rng(31)
    parts = [np.array([[0.3, -0.2, 0.1]]),
             np.array([[0.0, 0.0, 0.0], [40.0, 5.0, -3.0]]),
             np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0], [1.0, 1.7, 0.0]]),
             I.batch_suspensions(3, S=1, nmin=150, nmax=150).pos,
             I.batch_suspensions(4, S=1, nmin=400, nmax=400).pos]
    offsets = np.cumsum([0] + [p_.shape[0] for p_ in parts]).astype(np.int64)
    pos = np.concatenate(parts).astype(np.float32)
    n = pos.shape[0]
    W = rng.standard_normal(3 * n)
    b = lm.lm_batch_create(offsets, 1.0, 1.0, max_iter=100)
    lm.lm_batch_set_positions(b, dev(pos))
    tol = 1e-6
    y0, it0 = lm.lm_batch_sqrt_mdot(b, dev(W), tol=tol)
    lm.lm_batch_set_reorthogonalization(b, 1)
    y1, it1 = lm.lm_batch_sqrt_mdot(b, dev(W), tol=tol)
    y0, y1 = y0.cpu().numpy(), y1.cpu().numpy()
    for s in range(b.S):
        o0, o1 = offsets[s], offsets[s + 1]
        M = orc.assemble(pos[o0:o1].astype(np.float64), 1.0, 1.0, False)
        ws = W[3 * o0:3 * o1]
        exact = orc.sqrt_exact(M, ws)
        # FP32 pairs: the product itself carries about 1e-7 relative error
        assert rel(y0[o0:o1], exact) <= 20 * tol + 1e-6, (s, rel(y0[o0:o1], exact), it0[s])
        assert rel(y1[o0:o1], y0[o0:o1]) <= 1e-6, (s, rel(y1[o0:o1], y0[o0:o1]))
        assert abs(int(it1[s]) - int(it0[s])) <= 1, (s, it0[s], it1[s])
        _, ito, _ = orc.lanczos_sqrt(lambda v: M @ v, ws, tol=tol, max_iter=100)
        assert abs(int(it0[s]) - ito) <= 2, (s, it0[s], ito)


def test_batch_sqrt_runs_to_the_largest_basis(orc):
    """max_iter = 128 (the largest basis a batch holds) with a tolerance that
    FP32 products cannot reach: the systems iterate until the FP32 breakdown
    test (beta below 1e-7 of the largest alpha) or m = 128, so the solver
    warps solve tridiagonal matrices up to their scratch limit; the call
    reports non-convergence for the systems that hit the cap, and all results
    match the exact root to the accuracy of the FP32 products."""
    b_ = small_batch(seed=43, S=4, nmin=300, nmax=600)
    n = b_.pos.shape[0]
    W = np.random.default_rng(8).standard_normal(3 * n)
    b = lm.lm_batch_create(b_.offsets, 1.0, 1.0, max_iter=128)
    lm.lm_batch_set_positions(b, dev(b_.pos))
    with pytest.raises(lm.LmError) as e:
        lm.lm_batch_sqrt_mdot(b, dev(W), tol=1e-15)
    assert e.value.status == lm.LM_ERR_NOT_CONVERGED
    y, its = lm.lm_batch_sqrt_mdot(b, dev(W), tol=1e-15, raise_not_converged=False)
    y = y.cpu().numpy()
    its = np.asarray(its)
    assert (its >= 100).all() and (its <= 128).all() and (its == 128).any(), its
    for s in range(b.S):
        o0, o1 = b_.offsets[s], b_.offsets[s + 1]
        M = orc.assemble(b_.pos[o0:o1], 1.0, 1.0, False)
        assert rel(y[o0:o1], orc.sqrt_exact(M, W[3 * o0:3 * o1])) <= 1e-5, s


def test_batch_sqrt_matches_single_system_api(orc):
    b_ = small_batch(seed=13, S=4)
    n = b_.pos.shape[0]
    W = np.random.default_rng(3).standard_normal(3 * n)
    b = lm.lm_batch_create(b_.offsets, 1.0, 1.0)
    lm.lm_batch_set_positions(b, dev(b_.pos))
    y, its = lm.lm_batch_sqrt_mdot(b, dev(W), tol=1e-6)
    y = y.cpu().numpy()
    for s in range(b.S):
        o0, o1 = b_.offsets[s], b_.offsets[s + 1]
        sv = lm.lm_create(1.0, 1.0, False, lm.LM_FP32C)
        lm.lm_set_positions(sv, dev(b_.pos[o0:o1]))
        ys, _, it = lm.lm_sqrt_mdot(sv, dev(W[3 * o0:3 * o1]), tol=1e-6, max_iter=64)
        assert abs(it - int(its[s])) <= 1
        assert rel(y[o0:o1], ys.cpu().numpy()) <= 1e-5


def test_batch_bd_one_step_matches_oracle(orc):
    b_ = small_batch(seed=17, S=5, nmin=30, nmax=400)
    b = lm.lm_batch_create(b_.offsets, 1.0, 1.0, max_iter=100)
    lm.lm_batch_set_positions(b, dev(b_.pos))
    kT, dt, k, seed, tol = 1.0, 1e-3, 1.0, 4242, 1e-8
    its = lm.lm_batch_bd_run(b, kT, dt, k, 1, step0=0, seed=seed, tol=tol, use_graph=True)
    x1 = lm.lm_batch_get_positions(b, like=dev(b_.pos)).cpu().numpy()
    for s in range(b.S):
        o0, o1 = b_.offsets[s], b_.offsets[s + 1]
        x0 = b_.pos[o0:o1].astype(np.float64)
        W = orc.philox_normals(seed, orc.bd_noise_stream(s, 0), 3 * (o1 - o0))
        xr, itr = orc.em_step(x0, 1.0, 1.0, kT, dt, k, W, tol)
        # compare displacements; x1 is rounded to FP32 on read-back
        d_gpu = x1[o0:o1] - x0
        d_ref = xr - x0
        atol = 2 * np.abs(x0).max() * 2 ** -24
        assert np.abs(d_gpu - d_ref).max() <= 1e-5 * np.abs(d_ref).max() + atol, s
        assert abs(int(its[s]) - itr) <= 1


def test_batch_bd_full_size_step_on_sampled_systems(orc):
    """The benchmark's batch (256 systems, N log-uniform in [64, 4096]) in
    its launch configuration (autotuned tiling, max_iter 64, tol 1e-4): one
    Euler-Maruyama step against the oracle's step with the same Philox noise,
    on the smallest systems and a few of a few hundred particles."""
    c = I.BATCH_BD_256
    b_ = I.batch_suspensions(c["seed"], c["S"], c["nmin"], c["nmax"], c["phi_lo"], c["phi_hi"], c["a"])
    b = lm.lm_batch_create(b_.offsets, c["eta"], c["a"], max_iter=64)
    lm.lm_batch_set_positions(b, dev(b_.pos))
    lm.lm_batch_autotune(b)
    its = lm.lm_batch_bd_run(b, c["kT"], c["dt"], c["k_trap"], 1, step0=0, seed=c["seed"], tol=c["tol"],
                             use_graph=True)
    x1 = lm.lm_batch_get_positions(b, like=dev(b_.pos)).cpu().numpy()
    order = np.argsort(b_.sizes)
    mid = [s for s in order if 300 <= b_.sizes[s] <= 700][:3]
    for s in list(order[:3]) + mid:
        o0, o1 = b_.offsets[s], b_.offsets[s + 1]
        x0 = b_.pos[o0:o1].astype(np.float64)
        W = orc.philox_normals(c["seed"], orc.bd_noise_stream(s, 0), 3 * (o1 - o0))
        xr, itr = orc.em_step(x0, c["a"], c["eta"], c["kT"], c["dt"], c["k_trap"], W, c["tol"])
        d_gpu, d_ref = x1[o0:o1] - x0, xr - x0
        atol = 2 * np.abs(x0).max() * 2 ** -24
        # iteration counts may differ by one near the stopping rule: then the
        # iterates differ by about tol
        assert abs(int(its[s]) - itr) <= 1, (s, its[s], itr)
        lim = (1e-5 if int(its[s]) == itr else 20 * c["tol"]) * np.abs(d_ref).max() + atol
        assert np.abs(d_gpu - d_ref).max() <= lim, (s, int(b_.sizes[s]))


def test_batch_bd_graph_direct_and_resume_agree():
    b_ = small_batch(seed=19, S=7, nmin=16, nmax=300)
    args = dict(kT=1.0, dt=1e-3, k_trap=1.0, seed=5, tol=1e-4)
    res = []
    for mode in ("graph4", "direct4", "resume2+2"):
        b = lm.lm_batch_create(b_.offsets, 1.0, 1.0)
        lm.lm_batch_set_positions(b, dev(b_.pos))
        if mode == "graph4":
            lm.lm_batch_bd_run(b, nsteps=4, use_graph=True, **args)
        elif mode == "direct4":
            lm.lm_batch_bd_run(b, nsteps=4, use_graph=False, **args)
        else:
            lm.lm_batch_bd_run(b, nsteps=2, step0=0, use_graph=True, **args)
            lm.lm_batch_bd_run(b, nsteps=2, step0=2, use_graph=False, **args)
        res.append(lm.lm_batch_get_positions(b, like=dev(b_.pos)).cpu().numpy())
    np.testing.assert_array_equal(res[0], res[1])
    np.testing.assert_array_equal(res[0], res[2])
    assert np.abs(res[0] - b_.pos).max() > 0


def test_batch_trap_statistics_single_particles():
    """Isolated spheres in the trap: x' = (1 - k mu dt) x + sqrt(2 kT mu dt) xi with
    mu = 1/(6 pi eta a); the displacement variance after one step is 2 kT mu dt."""
    S = 4000
    offsets = np.arange(S + 1, dtype=np.int64)
    pos = np.zeros((S, 3), np.float32)
    b = lm.lm_batch_create(offsets, 1.0, 1.0, max_iter=8)
    lm.lm_batch_set_positions(b, dev(pos))
    lm.lm_batch_bd_run(b, 1.0, 1e-2, 1.0, 1, seed=3, tol=1e-10)
    x = lm.lm_batch_get_positions(b, like=dev(pos)).cpu().numpy().astype(np.float64)
    var = 2 * 1.0 * (1 / (6 * np.pi)) * 1e-2
    assert abs(x.var() / var - 1) < 0.05
    assert abs(x.mean()) < 5 * np.sqrt(var / x.size)


def test_batch_errors_and_timeout_selftest():
    with pytest.raises(lm.LmError) as e:
        lm.lm_batch_create(np.array([0, 0], np.int64), 1.0, 1.0)
    assert e.value.status == lm.LM_ERR_INVALID_ARG
    b = lm.lm_batch_create(np.array([0, 5, 9], np.int64), 1.0, 1.0)
    with pytest.raises(lm.LmError) as e:
        lm.lm_batch_bd_run(b, 1.0, 1e-3, 1.0, 1)
    assert e.value.status == lm.LM_ERR_STATE
    with pytest.raises(lm.LmError):
        lm.lm_batch_set_tiling(b, 96, 3)
    assert lm.lm_batch_timeout_selftest(2_000_000) == lm.LM_ERR_TIMEOUT
    # the context stays usable after the expired waits
    lm.lm_batch_set_positions(b, dev(np.random.default_rng(0).uniform(-3, 3, (9, 3)).astype(np.float32)))
    lm.lm_batch_bd_run(b, 1.0, 1e-3, 1.0, 2)


def test_batch_autotune_keeps_results(orc):
    b_ = small_batch(seed=23)
    F = np.random.default_rng(4).standard_normal((b_.pos.shape[0], 3)).astype(np.float32)
    b = lm.lm_batch_create(b_.offsets, 1.0, 1.0)
    lm.lm_batch_set_positions(b, dev(b_.pos))
    t = lm.lm_batch_autotune(b)
    assert (t["threads"], t["ilp"]) in ((64, 1), (64, 2), (128, 1), (128, 2))
    u = lm.lm_batch_mdot(b, dev(F)).cpu().numpy()
    o0, o1 = b_.offsets[0], b_.offsets[1]
    ur, _ = orc.mdot(b_.pos[o0:o1], F[o0:o1], None, 1.0, 1.0, False)
    assert rel(u[o0:o1], ur) <= 1e-5
