"""GPU parity of the fused adjoint (lm_mdot_backward) and the autograd wrapper.

L = sum_i G_i.u_i + H_i.w_i with [u; w] = M(X)[F; T].  References:
  * the oracle's analytic gradient (chain rule over its pair-block
    derivatives) at N = 512 (volume fraction 0.1);
  * central finite differences in FP64 at the full N = 65536 workload, on
    the part of L that moves with x_k:
        L_k = [G_k; H_k].(M [F; T])_k + [F_k; T_k].(M [G; H])_k
    (all other terms of L are constant in x_k; M is symmetric), computed with
    the oracle's row products, h = 1e-4 a, on 64 random (particle, axis) pairs;
  * dL/dF = (M [G; H])_u, dL/dT = (M [G; H])_w from the oracle's product."""
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
    return np.linalg.norm(y - ref) / max(np.linalg.norm(ref), 1e-300)


@pytest.mark.parametrize("fp64,angular", [(False, False), (False, True), (True, False), (True, True)])
def test_adjoint_matches_oracle_gradient(orc, fp64, angular):
    c = I.ADJOINT_N65536
    s_ = I.cube_suspension(c["seed"], 512, c["phi"], c["a"], angular=angular, fp32=not fp64)
    s = lm.lm_create(c["eta"], c["a"], angular, lm.LM_FP64 if fp64 else lm.LM_FP32C)
    lm.lm_set_positions(s, dev(s_.pos))
    dX, dF, dT = lm.lm_mdot_backward(s, dev(s_.F), dev(s_.T), dev(s_.G), dev(s_.H))
    gX = orc.grad(s_.pos, s_.F, s_.T, s_.G, s_.H, c["a"], c["eta"], angular)
    gF, gT = orc.mdot(s_.pos, s_.G, s_.H, c["a"], c["eta"], angular)
    tol = 1e-11 if fp64 else 1e-5
    assert rel(host(dX), gX) <= tol, rel(host(dX), gX)
    assert rel(host(dF), gF) <= tol, rel(host(dF), gF)
    if angular:
        assert rel(host(dT), gT) <= tol, rel(host(dT), gT)


def test_adjoint_launch_configs_agree(orc):
    """Every configuration of the packed translation adjoint (threads x ilp x
    j per vote x splits) against the oracle gradient; N = 1100 is ragged for
    every tile size."""
    n = 1100
    s_ = I.cube_suspension(61, n, 0.15, 1.0, angular=False, fp32=True)
    s = lm.lm_create(1.0, 1.0, False, lm.LM_FP32C)
    lm.lm_set_positions(s, dev(s_.pos))
    gX = orc.grad(s_.pos, s_.F, None, s_.G, None, 1.0, 1.0, False)
    gF, _ = orc.mdot(s_.pos, s_.G, None, 1.0, 1.0, False)
    for threads in (128, 256):
        for ilp in (2, 4):
            for uj in (1, 2, 3):
                for splits in (1, 3, 9):
                    lm.lm_set_adjoint_config(s, threads, ilp, splits, uj)
                    dX, dF, _ = lm.lm_mdot_backward(s, dev(s_.F), None, dev(s_.G), None)
                    cfg = (threads, ilp, uj, splits)
                    assert rel(host(dX), gX) <= 1e-5, (cfg, rel(host(dX), gX))
                    assert rel(host(dF), gF) <= 1e-5, (cfg, rel(host(dF), gF))
    with pytest.raises(lm.LmError):
        lm.lm_set_adjoint_config(s, 128, 3, 1, 1)
    with pytest.raises(lm.LmError):
        lm.lm_set_adjoint_config(s, 128, 4, 1, 0)


def test_adjoint_symmetric_form_overlaps_across_blocks(orc):
    """The symmetric form (each unordered pair once, added to both particles)
    where the exact branch falls in symmetric tiles: a coincident pair and an
    overlapping pair whose particles lie in different i-blocks, N ragged for
    every tile; dF alone and dX alone."""
    n = 700
    s_ = I.cube_suspension(62, n, 0.15, 1.0, angular=False, fp32=True)
    pos = s_.pos.copy()
    pos[500] = pos[10]                                           # coincident, blocks 0 and 1
    pos[600] = pos[20] + np.array([0.5, 0.1, 0.0], np.float32)  # overlapping, blocks 0 and 2
    s = lm.lm_create(1.0, 1.0, False, lm.LM_FP32C)
    lm.lm_set_positions(s, dev(pos))
    gX = orc.grad(pos, s_.F, None, s_.G, None, 1.0, 1.0, False)
    gF, _ = orc.mdot(pos, s_.G, None, 1.0, 1.0, False)
    for threads, ilp, chunk in ((128, 2, 1), (128, 2, 0), (256, 4, 2), (128, 4, 5)):
        lm.lm_set_adjoint_config(s, threads, ilp, chunk, 3)
        dX, dF, _ = lm.lm_mdot_backward(s, dev(s_.F), None, dev(s_.G), None)
        assert rel(host(dX), gX) <= 1e-5, (threads, ilp, chunk, rel(host(dX), gX))
        assert rel(host(dF), gF) <= 1e-5, (threads, ilp, chunk, rel(host(dF), gF))
        dX2, dF2, _ = lm.lm_mdot_backward(s, dev(s_.F), None, dev(s_.G), None, need_dF=False)
        assert dF2 is None and rel(host(dX2), gX) <= 1e-5
        _, dF3, _ = lm.lm_mdot_backward(s, dev(s_.F), None, dev(s_.G), None, need_dX=False)
        assert rel(host(dF3), gF) <= 1e-5


@pytest.mark.parametrize("fp64,angular,ilp,packed", [(False, True, 2, 3), (False, True, 4, 3), (True, True, 1, 3),
                                                     (True, False, 1, 3), (False, True, 2, 4), (False, True, 4, 4)])
def test_adjoint_symmetric_6n_and_fp64_forms(orc, fp64, angular, ilp, packed):
    """The symmetric forms of the adjoint with angular blocks (FP32 scalar,
    packed = 3, and packed f32x2, packed = 4) and in FP64 (scalar): each
    unordered pair evaluated once and added to both particles.
    A coincident and an overlapping pair whose particles lie in different
    i-blocks, N ragged for every tile; items of one tile, of the automatic
    size and of five tiles; dX alone and dF, dT alone."""
    n = 700
    s_ = I.cube_suspension(63, n, 0.15, 1.0, angular=angular, fp32=not fp64)
    pos = s_.pos.copy()
    pos[500] = pos[10]                                          # coincident
    pos[600] = pos[20] + np.array([0.5, 0.1, 0.0], pos.dtype)  # overlapping
    s = lm.lm_create(1.0, 1.0, angular, lm.LM_FP64 if fp64 else lm.LM_FP32C)
    lm.lm_set_positions(s, dev(pos))
    gX = orc.grad(pos, s_.F, s_.T, s_.G, s_.H, 1.0, 1.0, angular)
    gF, gT = orc.mdot(pos, s_.G, s_.H, 1.0, 1.0, angular)
    tol = 1e-11 if fp64 else 1e-5
    args = (dev(s_.F), dev(s_.T), dev(s_.G), dev(s_.H))
    for chunk in (1, 0, 5):
        lm.lm_set_adjoint_config(s, 128, ilp, chunk, packed)
        assert lm.lm_get_adjoint_config(s)["packed"] == packed
        dX, dF, dT = lm.lm_mdot_backward(s, *args)
        assert rel(host(dX), gX) <= tol, (chunk, rel(host(dX), gX))
        assert rel(host(dF), gF) <= tol, (chunk, rel(host(dF), gF))
        if angular:
            assert rel(host(dT), gT) <= tol, (chunk, rel(host(dT), gT))
    dX2, dF2, dT2 = lm.lm_mdot_backward(s, *args, need_dF=False)
    assert dF2 is None and dT2 is None and rel(host(dX2), gX) <= tol
    dX3, dF3, dT3 = lm.lm_mdot_backward(s, *args, need_dX=False)
    assert dX3 is None and rel(host(dF3), gF) <= tol
    if angular:
        assert rel(host(dT3), gT) <= tol


@pytest.mark.parametrize("packed", [0, 3, 4])
def test_adjoint_6n_full_size_sampled_rows(orc, packed):
    """The FP32 adjoint with angular blocks at N = 65536 (the adjoint
    benchmark's suspension, with torques and their cotangents), one-sided
    (packed 0), symmetric scalar (3) and symmetric packed (4), against the
    oracle's gradient and products on 64 sampled particles."""
    c = I.ADJOINT_N65536
    s_ = I.cube_suspension(c["seed"], c["n"], c["phi"], c["a"], angular=True, fp32=True)
    s = lm.lm_create(c["eta"], c["a"], True, lm.LM_FP32C)
    lm.lm_set_positions(s, dev(s_.pos))
    lm.lm_set_adjoint_config(s, 128, 2, 0, packed)
    dX, dF, dT = lm.lm_mdot_backward(s, dev(s_.F), dev(s_.T), dev(s_.G), dev(s_.H))
    rows = np.sort(np.random.default_rng(8).choice(c["n"], 64, replace=False))
    gX = orc.grad(s_.pos, s_.F, s_.T, s_.G, s_.H, c["a"], c["eta"], True, rows=rows)
    gF, gT = orc.mdot(s_.pos, s_.G, s_.H, c["a"], c["eta"], True, rows=rows)
    assert rel(host(dX)[rows], gX) <= 1e-5, rel(host(dX)[rows], gX)
    assert rel(host(dF)[rows], gF) <= 1e-5, rel(host(dF)[rows], gF)
    assert rel(host(dT)[rows], gT) <= 1e-5, rel(host(dT)[rows], gT)


def test_adjoint_6n_beyond_the_benchmark_size_sampled_rows(orc):
    """The default adjoint with angular blocks (the packed symmetric form) at
    N = 2^20, sixteen times the adjoint benchmark's N (random cube at
    phi = 0.1): dX, dF and dT on 32 sampled particles against the oracle.
    Work-item counts, accumulator indices and grids are far from the sizes
    the smaller tests reach."""
    n = 1 << 20
    s_ = I.cube_suspension(79, n, 0.1, 1.0, angular=True, fp32=True)
    s = lm.lm_create(1.0, 1.0, True, lm.LM_FP32C)
    lm.lm_set_positions(s, dev(s_.pos))
    assert lm.lm_get_adjoint_config(s)["packed"] == 4
    dX, dF, dT = (host(t) for t in lm.lm_mdot_backward(s, dev(s_.F), dev(s_.T), dev(s_.G), dev(s_.H)))
    rows = np.sort(np.random.default_rng(9).choice(n, 32, replace=False))
    gX = orc.grad(s_.pos, s_.F, s_.T, s_.G, s_.H, 1.0, 1.0, True, rows=rows)
    gF, gT = orc.mdot(s_.pos, s_.G, s_.H, 1.0, 1.0, True, rows=rows)
    assert rel(dX[rows], gX) <= 1e-5, rel(dX[rows], gX)
    assert rel(dF[rows], gF) <= 1e-5, rel(dF[rows], gF)
    assert rel(dT[rows], gT) <= 1e-5, rel(dT[rows], gT)
    assert np.isfinite(dX).all() and np.isfinite(dF).all() and np.isfinite(dT).all()


def test_adjoint_skips_outputs_and_handles_coincident(orc):
    pos = np.array([[0, 0, 0], [0, 0, 0], [0.5, 0.1, 0.0], [3.0, 0.0, 1.0]], np.float64)
    rng = np.random.default_rng(2)
    F, T, G, H = (rng.standard_normal((4, 3)) for _ in range(4))
    s = lm.lm_create(1.0, 1.0, True, lm.LM_FP64)
    lm.lm_set_positions(s, dev(pos))
    dX, dF, dT = lm.lm_mdot_backward(s, dev(F), dev(T), dev(G), dev(H))
    gX = orc.grad(pos, F, T, G, H, 1.0, 1.0, True)
    assert rel(host(dX), gX) <= 1e-12
    dX2, dF2, dT2 = lm.lm_mdot_backward(s, dev(F), dev(T), dev(G), dev(H), need_dF=False)
    assert dF2 is None and dT2 is None
    np.testing.assert_array_equal(host(dX2), host(dX))


def test_adjoint_n65536_finite_differences(orc):
    c = I.ADJOINT_N65536
    s_ = I.cube_suspension(c["seed"], c["n"], c["phi"], c["a"], angular=False, fp32=True)
    s = lm.lm_create(c["eta"], c["a"], False, lm.LM_FP32C)
    lm.lm_set_positions(s, dev(s_.pos))
    lm.lm_autotune(s, reps=1)        # the launch configuration the benchmark times
    dX, dF, _ = lm.lm_mdot_backward(s, dev(s_.F), None, dev(s_.G), None)
    dX, dF = host(dX), host(dF)
    rng = np.random.default_rng(7)
    ks = rng.choice(c["n"], 64, replace=False)
    axes = rng.integers(0, 3, 64)
    h = 1e-4 * c["a"]
    pos = s_.pos.astype(np.float64)
    F = s_.F.astype(np.float64)
    G = s_.G.astype(np.float64)
    errs = []
    for k, ax in zip(ks, axes):
        vals = []
        for sgn in (1.0, -1.0):
            p = pos.copy()
            p[k, ax] += sgn * h
            uF, _ = orc.mdot(p, F, None, c["a"], c["eta"], False, rows=[k])
            uG, _ = orc.mdot(p, G, None, c["a"], c["eta"], False, rows=[k])
            vals.append(G[k] @ uF[0] + F[k] @ uG[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        scale = max(abs(fd), np.abs(dX[k]).max(), 1e-30)
        errs.append(abs(dX[k, ax] - fd) / scale)
    assert max(errs) <= 1e-4, max(errs)
    rows = ks[:16]
    gF, _ = orc.mdot(pos, G, None, c["a"], c["eta"], False, rows=rows)
    assert rel(dF[rows], gF) <= 1e-5


def test_autograd_mobility_function(orc):
    n = 300
    s_ = I.cube_suspension(55, n, 0.15, 1.0, angular=True, fp32=True)
    s = lm.lm_create(1.0, 1.0, True, lm.LM_FP32C)
    X = dev(s_.pos).requires_grad_(True)
    F = dev(s_.F).requires_grad_(True)
    T = dev(s_.T).requires_grad_(True)
    u, w = lm.mobility(s, X, F, T)
    G, H = dev(s_.G), dev(s_.H)
    L = (u * G).sum() + (w * H).sum()
    L.backward()
    gX = orc.grad(s_.pos, s_.F, s_.T, s_.G, s_.H, 1.0, 1.0, True)
    gF, gT = orc.mdot(s_.pos, s_.G, s_.H, 1.0, 1.0, True)
    assert rel(host(X.grad), gX) <= 1e-5
    assert rel(host(F.grad), gF) <= 1e-5
    assert rel(host(T.grad), gT) <= 1e-5
    ur, wr = orc.mdot(s_.pos, s_.F, s_.T, 1.0, 1.0, True)
    assert rel(host(u), ur) <= 1e-5 and rel(host(w), wr) <= 1e-5
