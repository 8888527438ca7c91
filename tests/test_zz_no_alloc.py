"""The no-allocation product (lm_mdot_noalloc) against the regular lm_mdot.

lm_mdot_noalloc serves callers that cannot let a library allocate device
memory (their own memory pool owns the GPU, or a latency-critical loop cannot
take the synchronisation of cudaMalloc/cudaFree).  It keeps its scratch in a
fixed array inside the library, shared by all calls.  This test calls it
through the C ABI twice in a row, with different sizes and inputs, and checks
each result against lm_mdot on the same inputs at the FP32 parity tolerance
(1e-5 relative L2), so a stale or mis-addressed scratch array shows up.  The
file is named to be collected last."""
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


def test_noalloc_matches_lm_mdot_on_two_calls_in_a_row():
    eta, a = 1.0, 1.0
    cases = [(32768, 0.2, 101), (5000, 0.1, 102)]   # full size first, then a smaller, ragged N
    for n, phi, seed in cases:
        s_ = I.cube_suspension(seed, n, phi, a, angular=True, fp32=True)
        pos = torch.from_numpy(s_.pos).cuda()
        F = torch.from_numpy(s_.F).cuda()
        T = torch.from_numpy(s_.T).cuda()
        solver = lm.lm_create(eta, a, True, lm.LM_FP32C)
        lm.lm_set_positions(solver, pos)
        u_ref, w_ref = lm.lm_mdot(solver, F, T)
        u = torch.full((n, 3), float("nan"), dtype=torch.float32, device="cuda")
        w = torch.full((n, 3), float("nan"), dtype=torch.float32, device="cuda")
        lm.lm_mdot_noalloc(pos, F, T, eta, a, True, u, w)
        torch.cuda.synchronize()
        assert torch.isfinite(u).all() and torch.isfinite(w).all()
        assert _rel(u, u_ref) <= 1e-5, (n, _rel(u, u_ref))
        assert _rel(w, w_ref) <= 1e-5, (n, _rel(w, w_ref))


def test_noalloc_rejects_sizes_beyond_its_limit():
    n = lm.LM_NOALLOC_MAX_N + 1
    x = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    out = torch.empty_like(x)
    with pytest.raises(lm.LmError) as e:
        lm.lm_mdot_noalloc(x, x, None, 1.0, 1.0, False, out)
    assert e.value.status == lm.LM_ERR_INVALID_ARG
    assert "no-allocation limit" in str(e.value)
