"""The device tridiagonal step sqrt(T) e1 (Sec. 3.3; the form the batched
kernel runs, one warp per system: the quadrature for a T certified positive
definite, the QR iteration otherwise) against the oracle's LAPACK
eigendecomposition."""
import numpy as np
import pytest

from paper_2510_02135_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lm():
    import torch

    from paper_2510_02135_gb300 import lm as lm_

    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    lm_.lib()
    return lm_


def _run(lm, alpha, beta, paths=False):
    """alpha, beta: (count, m) arrays (beta[:, m-1] ignored).  paths=True also
    returns which form solved each system (0 quadrature, 1 QR)."""
    import torch

    a = torch.from_numpy(np.ascontiguousarray(alpha, dtype=np.float64)).cuda()
    b = torch.from_numpy(np.ascontiguousarray(beta, dtype=np.float64)).cuda()
    out, pth = lm.lm_tridiag_sqrt_e1_device(a, b, paths=True)
    torch.cuda.synchronize()
    return (out.cpu().numpy(), pth) if paths else out.cpu().numpy()


def _check(orc, got, alpha, beta, rtol):
    for c in range(alpha.shape[0]):
        m = alpha.shape[1]
        want = orc.tridiag_sqrt_e1(alpha[c], beta[c, : m - 1])
        np.testing.assert_allclose(got[c], want, atol=rtol * max(1.0, np.abs(want).max()), err_msg=f"system {c}")


@pytest.mark.parametrize("m", [1, 2, 3, 7, 40, 64, 128])
def test_random_spd(orc, lm, m):
    rng = np.random.default_rng(100 + m)
    count = 70   # more than two warps, ragged
    alpha = rng.uniform(0.5, 3.0, (count, m))
    beta = rng.uniform(0.05, 0.8, (count, m))
    got, paths = _run(lm, alpha, beta, paths=True)
    _check(orc, got, alpha, beta, 1e-12)
    # positive definite where the Sturm bound certifies it: the quadrature ran
    for c in range(count):
        T = np.diag(alpha[c]) + np.diag(beta[c, : m - 1], 1) + np.diag(beta[c, : m - 1], -1)
        if np.linalg.eigvalsh(T).min() > 1e-3 * np.abs(T).max():
            assert paths[c] == 0, f"system {c}"


def test_graded_clustered_and_split(orc, lm):
    m = 30
    rows_a, rows_b = [], []
    rows_a.append(np.full(m, 2.0))                                   # decaying couplings
    rows_b.append(np.array([10.0 ** (-k / 3.0) for k in range(m)]))
    rows_a.append(np.linspace(1e-6, 1.0, m))                         # nearly diagonal, graded
    rows_b.append(np.full(m, 1e-9))
    a = np.full(m, 1.0)                                              # exactly split in two blocks
    b = np.full(m, 0.3)
    b[m // 2] = 0.0
    rows_a.append(a)
    rows_b.append(b)
    rows_a.append(np.full(m, 0.7))                                   # diagonal: sqrt(alpha_0) e1
    rows_b.append(np.zeros(m))
    alpha, beta = np.array(rows_a), np.array(rows_b)
    got, paths = _run(lm, alpha, beta, paths=True)
    _check(orc, got, alpha, beta, 1e-12)
    np.testing.assert_allclose(got[3], np.r_[np.sqrt(0.7), np.zeros(m - 1)], rtol=1e-12, atol=0)
    # the graded matrix (smallest eigenvalue 1e-6 of the largest entry) is not
    # certified and takes the QR form; the split and diagonal ones are
    assert paths[1] == 1 and paths[2] == 0 and paths[3] == 0


def test_quadrature_near_the_certification_limit(orc, lm):
    """Smallest eigenvalues from 1e-1 down to 1e-4 of the largest entry: the
    quadrature's node range grows with log(kappa) and its error stays at the
    1e-13 level."""
    m = 48
    rng = np.random.default_rng(11)
    rows_a, rows_b = [], []
    for lmin in (1e-1, 1e-2, 1e-3, 1e-4):
        lam = np.r_[lmin, np.exp(rng.uniform(np.log(lmin), 0.0, m - 1))]
        Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
        A = (Q * lam) @ Q.T
        # Householder tridiagonalisation of A keeps its spectrum
        from scipy.linalg import hessenberg

        H = hessenberg(A)
        rows_a.append(np.diag(H).copy())
        rows_b.append(np.r_[np.diag(H, 1), 0.0])
    alpha, beta = np.array(rows_a), np.array(rows_b)
    got, paths = _run(lm, alpha, beta, paths=True)
    _check(orc, got, alpha, beta, 1e-12)
    assert list(paths) == [0, 0, 0, 0]


def test_clamps_negative_eigenvalue(lm):
    alpha = np.array([[-1e-18, 1.0]])
    beta = np.array([[0.0, 0.0]])
    got, paths = _run(lm, alpha, beta, paths=True)
    np.testing.assert_allclose(got, [[0.0, 0.0]], atol=1e-15)
    assert paths[0] == 1


def test_lanczos_tridiagonals_of_a_mobility_matrix(orc, lm):
    """T_k of the Lanczos process on an RPY mobility matrix for k = 1..40:
    the spectra the batched kernel meets."""
    s = inputs.cube_suspension(seed=7, n=100, phi=0.2, a=1.0, angular=False, fp32=False)
    M = orc.assemble(s.pos, 1.0, 1.0, False)
    rng = np.random.default_rng(3)
    v = rng.standard_normal(M.shape[0])
    V = [v / np.linalg.norm(v)]
    al, be = [], []
    for k in range(40):
        w = M @ V[-1]
        al.append(V[-1] @ w)
        w -= al[-1] * V[-1] + (be[-1] * V[-2] if k else 0.0)
        for u in V:                       # full reorthogonalisation, twice
            w -= (u @ w) * u
        for u in V:
            w -= (u @ w) * u
        be.append(np.linalg.norm(w))
        V.append(w / be[-1])
    alpha = np.zeros((40, 40))
    beta = np.zeros((40, 40))
    for k in range(1, 41):
        alpha[k - 1, :k] = al[:k]
        beta[k - 1, : k - 1] = be[: k - 1]
    for k in range(1, 41):   # one launch per size (rows of a launch share m)
        got, paths = _run(lm, alpha[k - 1: k, :k], beta[k - 1: k, :k], paths=True)
        want = orc.tridiag_sqrt_e1(alpha[k - 1, :k], beta[k - 1, : k - 1])
        np.testing.assert_allclose(got[0], want, atol=1e-12 * np.abs(want).max())
        assert paths[0] == 0, f"k = {k}: the quadrature solves the Lanczos matrices of a mobility"


def test_rejects_bad_arguments(lm):
    import torch

    a = torch.zeros((2, 200), dtype=torch.float64, device="cuda")
    with pytest.raises(lm.LmError):
        lm.lm_tridiag_sqrt_e1_device(a, a)
