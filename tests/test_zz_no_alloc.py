"""The no-allocation product (lm_mdot_noalloc) against the regular lm_mdot
and the FP64 oracle.

lm_mdot_noalloc serves callers that cannot let a library allocate device
memory (their own memory pool owns the GPU, or a latency-critical loop cannot
take the synchronisation of cudaMalloc/cudaFree).  It keeps its scratch in a
fixed array inside the library, shared by all calls.  These tests call it
through the C ABI several times in a row, with different sizes, inputs and
block sets, and check each result against lm_mdot on the same inputs and
against the oracle on sampled rows, at the FP32 parity tolerance (1e-5
relative L2), so a stale or mis-addressed scratch array shows up.  The file
is named to be collected last."""
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


def _rel(y, ref):
    y = y.double().cpu().numpy().ravel()
    ref = ref.double().cpu().numpy().ravel()
    return np.linalg.norm(y - ref) / np.linalg.norm(ref)


def _rel_np(y, ref):
    y = np.asarray(y, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    return np.linalg.norm(y - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("angular", [True, False])
def test_noalloc_matches_lm_mdot_on_two_calls_in_a_row(orc, angular):
    eta, a = 1.0, 1.0
    cases = [(32768, 0.2, 101), (5000, 0.1, 102)]   # full size first, then a smaller, ragged N
    for n, phi, seed in cases:
        s_ = I.cube_suspension(seed, n, phi, a, angular=angular, fp32=True)
        pos = torch.from_numpy(s_.pos).cuda()
        F = torch.from_numpy(s_.F).cuda()
        T = torch.from_numpy(s_.T).cuda() if angular else None
        solver = lm.lm_create(eta, a, angular, lm.LM_FP32C)
        lm.lm_set_positions(solver, pos)
        u_ref, w_ref = lm.lm_mdot(solver, F, T)
        u = torch.full((n, 3), float("nan"), dtype=torch.float32, device="cuda")
        w = torch.full((n, 3), float("nan"), dtype=torch.float32, device="cuda") if angular else None
        lm.lm_mdot_noalloc(pos, F, T, eta, a, angular, u, w)
        torch.cuda.synchronize()
        assert torch.isfinite(u).all()
        assert _rel(u, u_ref) <= 1e-5, (n, _rel(u, u_ref))
        rows = np.random.default_rng(seed).choice(n, 64, replace=False)
        ur, wr = orc.mdot(s_.pos, s_.F, s_.T, a, eta, angular, rows=rows)
        assert _rel_np(u.cpu().numpy()[rows], ur) <= 1e-5, (n, _rel_np(u.cpu().numpy()[rows], ur))
        if angular:
            assert torch.isfinite(w).all()
            assert _rel(w, w_ref) <= 1e-5, (n, _rel(w, w_ref))
            assert _rel_np(w.cpu().numpy()[rows], wr) <= 1e-5, (n, _rel_np(w.cpu().numpy()[rows], wr))


def test_noalloc_zero_forces_and_argument_checks():
    """forces = torques = NULL gives exact zeros (over stale NaNs); torques or
    ang_out without angular blocks, and host arrays, are rejected."""
    n = 3000
    s_ = I.cube_suspension(103, n, 0.1, 1.0, angular=True, fp32=True)
    pos = torch.from_numpy(s_.pos).cuda()
    u = torch.full((n, 3), float("nan"), dtype=torch.float32, device="cuda")
    w = torch.full((n, 3), float("nan"), dtype=torch.float32, device="cuda")
    lm.lm_mdot_noalloc(pos, None, None, 1.0, 1.0, True, u, w)
    torch.cuda.synchronize()
    assert not u.any() and not w.any()
    T = torch.from_numpy(s_.T).cuda()
    F = torch.from_numpy(s_.F).cuda()
    for kwargs in ({"torques": T, "ang_out": None}, {"torques": None, "ang_out": w}):
        with pytest.raises(lm.LmError) as e:
            lm.lm_mdot_noalloc(pos, F, kwargs["torques"], 1.0, 1.0, False, u, kwargs["ang_out"])
        assert e.value.status == lm.LM_ERR_INVALID_ARG
    with pytest.raises(lm.LmError) as e:
        lm.lm_mdot_noalloc(torch.from_numpy(s_.pos), F, None, 1.0, 1.0, False, u)
    assert e.value.status == lm.LM_ERR_INVALID_ARG


def test_noalloc_rejects_sizes_beyond_its_limit():
    n = lm.LM_NOALLOC_MAX_N + 1
    x = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    out = torch.empty_like(x)
    with pytest.raises(lm.LmError) as e:
        lm.lm_mdot_noalloc(x, x, None, 1.0, 1.0, False, out)
    assert e.value.status == lm.LM_ERR_INVALID_ARG
    assert "no-allocation limit" in str(e.value)
