"""C-ABI checks that need no GPU: the library loads, exports every entry
point that ``include/lm.h`` declares, rejects bad arguments before touching
the device, and its host-side tridiagonal step agrees with LAPACK."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2510_02135_gb300 import _build, lm

    _build.build()
    return lm.lib()


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(lm_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(L):
    names = _declared_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_version_and_empty_error(L):
    from paper_2510_02135_gb300 import lm

    assert "sm_103a" in lm.lm_version()
    assert isinstance(L.lm_last_error(), bytes)


def test_create_rejects_bad_arguments_without_gpu(L):
    from paper_2510_02135_gb300 import lm

    h = ctypes.c_void_p()
    cases = [
        ((b"open", b"open", b"two_walls", 1.0, 1.0, 0, 0), lm.LM_ERR_UNSUPPORTED_GEOMETRY),
        ((b"single_wall", b"open", b"open", 1.0, 1.0, 0, 0), lm.LM_ERR_UNSUPPORTED_GEOMETRY),
        ((b"periodic", b"periodic", b"periodic", 1.0, 1.0, 0, 0), lm.LM_ERR_UNSUPPORTED_GEOMETRY),
        ((b"open", b"open", b"single_wall", -1.0, 1.0, 0, 0), lm.LM_ERR_INVALID_ARG),
        ((b"open", b"open", b"bogus", 1.0, 1.0, 0, 0), lm.LM_ERR_INVALID_ARG),
        ((b"open", b"open", b"open", -1.0, 1.0, 0, 0), lm.LM_ERR_INVALID_ARG),
        ((b"open", b"open", b"open", 1.0, 0.0, 0, 0), lm.LM_ERR_INVALID_ARG),
        ((b"open", b"open", b"open", float("nan"), 1.0, 0, 0), lm.LM_ERR_INVALID_ARG),
        ((b"open", b"open", b"open", 1.0, 1.0, 0, 7), lm.LM_ERR_INVALID_ARG),
    ]
    for args, want in cases:
        st = L.lm_create(ctypes.byref(h), *args, None)
        assert st == want, (args, st)
        assert not h.value
        assert L.lm_last_error()


def test_null_solver_and_null_pointers(L):
    from paper_2510_02135_gb300 import lm

    assert L.lm_destroy(None) == lm.LM_OK
    assert L.lm_set_positions(None, None, 1) == lm.LM_ERR_INVALID_ARG
    assert L.lm_mdot(None, None, None, None, None) == lm.LM_ERR_INVALID_ARG
    assert L.lm_sqrt_mdot(None, None, 0, 1.0, 1e-5, 10, None, None, None) == lm.LM_ERR_INVALID_ARG
    assert L.lm_mdot_backward(None, None, None, None, None, None, None, None) == lm.LM_ERR_INVALID_ARG
    assert L.lm_create(None, b"open", b"open", b"open", 1.0, 1.0, 0, 0, None) == lm.LM_ERR_INVALID_ARG
    # entry points added for the single wall, the drift, the time stepping and the tuning
    assert L.lm_div_m_rfd(None, 0, 1e-3, None, None) == lm.LM_ERR_INVALID_ARG
    assert L.lm_set_wall_height(None, 0.0) == lm.LM_ERR_INVALID_ARG
    assert L.lm_set_sqrt_preconditioner(None, 1) == lm.LM_ERR_INVALID_ARG
    assert L.lm_set_reorthogonalization(None, 1) == lm.LM_ERR_INVALID_ARG
    assert L.lm_batch_set_reorthogonalization(None, 1) == lm.LM_ERR_INVALID_ARG
    assert L.lm_batch_profile_pairs(None, None) == lm.LM_ERR_INVALID_ARG
    assert L.lm_soft_repulsion(None, 1.0, 0.1, 2.0, 1.0, None) == lm.LM_ERR_INVALID_ARG
    assert L.lm_ab_step(None, None, None, None, 0, 1.0, 1e-3, 1e-5, 10, None, 1, None, None) == lm.LM_ERR_INVALID_ARG
    assert L.lm_langevin_velocities(None, None, None, None, 0, 1.0, 1e-3, 1e-5, 10, None, None,
                                    None) == lm.LM_ERR_INVALID_ARG
    cfg = lm.lm_pair_config(128, 4, 0, 1)
    assert L.lm_get_adjoint_config(None, ctypes.byref(cfg)) == lm.LM_ERR_INVALID_ARG
    assert L.lm_set_adjoint_config(None, ctypes.byref(cfg)) == lm.LM_ERR_INVALID_ARG


def test_create_without_gpu_reports_cuda_error(L):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2510_02135_gb300 import lm

    h = ctypes.c_void_p()
    st = L.lm_create(ctypes.byref(h), b"open", b"open", b"open", 1.0, 1.0, 0, 0, None)
    assert st in (lm.LM_ERR_CUDA, lm.LM_ERR_OOM)
    assert not h.value


@pytest.mark.parametrize("m", [1, 2, 3, 7, 40, 150])
def test_tridiagonal_root_matches_lapack(orc, L, m):
    from paper_2510_02135_gb300 import lm

    rng = np.random.default_rng(m)
    alpha = rng.uniform(0.5, 3.0, m)
    beta = rng.uniform(0.05, 0.8, max(m - 1, 0))
    got = lm.lm_tridiag_sqrt_e1(alpha, beta)
    want = orc.tridiag_sqrt_e1(alpha, beta)
    np.testing.assert_allclose(got, want, atol=1e-13 * max(1.0, np.abs(want).max()))


def test_tridiagonal_root_graded_and_clustered(orc, L):
    """Eigenvalues spanning many decades and near-multiple ones (Lanczos late iterations)."""
    from paper_2510_02135_gb300 import lm

    m = 30
    alpha = np.full(m, 2.0)
    beta = np.array([10.0 ** (-k / 3.0) for k in range(m - 1)])
    np.testing.assert_allclose(lm.lm_tridiag_sqrt_e1(alpha, beta), orc.tridiag_sqrt_e1(alpha, beta), atol=1e-13)
    alpha = np.linspace(1e-6, 1.0, m)
    beta = np.full(m - 1, 1e-9)
    np.testing.assert_allclose(lm.lm_tridiag_sqrt_e1(alpha, beta), orc.tridiag_sqrt_e1(alpha, beta), atol=1e-13)


def test_tridiagonal_root_clamps_negative(orc, L):
    from paper_2510_02135_gb300 import lm

    alpha = np.array([-1e-18, 1.0])
    beta = np.array([0.0])
    np.testing.assert_allclose(lm.lm_tridiag_sqrt_e1(alpha, beta), [0.0, 0.0], atol=1e-15)


def test_fp32_probe_rejects_bad_arguments_without_gpu(L):
    """The FP32 throughput probe checks its arguments before touching the GPU."""
    import ctypes as C

    from paper_2510_02135_gb300 import lm

    t = C.c_double(0.0)
    for mode, iters in ((5, 100), (-1, 100), (1, 0), (1, (1 << 24) + 1)):
        assert L.lm_fp32_probe(mode, iters, C.byref(t), None) == lm.LM_ERR_INVALID_ARG
    assert L.lm_fp32_probe(1, 100, None, None) == lm.LM_ERR_INVALID_ARG


def test_release_build_has_no_bounds_checks_and_debug_check_is_free(L):
    """The release library reports no device bounds checks, and lm_debug_check
    returns LM_OK there without touching a GPU."""
    from paper_2510_02135_gb300 import lm

    assert L.lm_debug_bounds() == 0
    assert L.lm_debug_check() == lm.LM_OK
