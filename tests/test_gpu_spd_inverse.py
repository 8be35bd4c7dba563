"""xm_spd_inverse (the adjoint preconditioner's dense inverse, formed on the tensor cores)
against the FP64 inverse of the same FP32 matrix, element by element.

Error model: each product of the Schur-complement recursion has the accuracy of an FP32 GEMM
(three BF16 digits per operand, FP32 accumulation), so the computed inverse X of an SPD A with
condition number kappa satisfies |X - A^{-1}| <~ c sqrt(n) u kappa max|A^{-1}| (u = 2^-24);
the test takes c = 8.  A wrong sign, a dropped product or a misplaced tile gives O(1) errors."""
import numpy as np
import pytest

from tests.gpu_util import EPS32, ctx, torch

pytestmark = pytest.mark.gpu

U32 = EPS32


@pytest.fixture(scope="module")
def C():
    c = ctx()
    yield c
    c.close()


def _spd(n, kappa, seed):
    rng = np.random.default_rng(seed)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.exp(rng.uniform(0.0, np.log(kappa), n))
    lam[0], lam[-1] = 1.0, kappa
    A = (Qm * lam) @ Qm.T
    return 0.5 * (A + A.T)


@pytest.mark.parametrize("n", [1, 50, 128, 129, 300, 700, 2100, 4000])
def test_spd_inverse_matches_fp64_inverse(C, n):
    from paper_2502_04640_b300 import xm
    kappa = 100.0
    A32 = _spd(n, kappa, seed=n).astype(np.float32)
    ref = np.linalg.inv(A32.astype(np.float64))
    X = torch.from_numpy(A32.copy()).cuda()
    xm.xm_spd_inverse(C, X)
    X = X.cpu().numpy().astype(np.float64)
    tol = 8.0 * np.sqrt(n) * U32 * kappa * np.abs(ref).max()
    err = np.abs(X - ref).max()
    assert err <= tol, (n, err, tol)
    assert np.abs(X - X.T).max() == 0.0          # both triangles written, exactly symmetric


def test_spd_inverse_ill_conditioned_residual(C):
    from paper_2502_04640_b300 import xm
    # kappa = 1e4 at n = 1500 (several recursion levels, ragged tiles): the residual A X - I
    # stays at the FP32 level times kappa
    n, kappa = 1500, 1.0e4
    A32 = _spd(n, kappa, seed=7).astype(np.float32)
    X = torch.from_numpy(A32.copy()).cuda()
    xm.xm_spd_inverse(C, X)
    X = X.cpu().numpy().astype(np.float64)
    R = A32.astype(np.float64) @ X - np.eye(n)
    assert np.abs(R).max() <= 8.0 * np.sqrt(n) * U32 * kappa, np.abs(R).max()


def test_spd_inverse_rejects_an_indefinite_matrix(C):
    from paper_2502_04640_b300 import xm
    n = 300
    rng = np.random.default_rng(3)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.linspace(1.0, 10.0, n)
    lam[n // 2] = -1.0
    A32 = ((Qm * lam) @ Qm.T).astype(np.float32)
    A32 = 0.5 * (A32 + A32.T)
    X = torch.from_numpy(A32.copy()).cuda()
    with pytest.raises(xm.XmError) as ei:
        xm.xm_spd_inverse(C, X)
    assert ei.value.status == xm.XM_ENUMERIC
    # the context stays usable
    A2 = _spd(200, 10.0, 1).astype(np.float32)
    B = torch.from_numpy(A2.copy()).cuda()
    xm.xm_spd_inverse(C, B)
    ref = np.linalg.inv(A2.astype(np.float64))
    assert np.abs(B.cpu().numpy() - ref).max() <= 8.0 * np.sqrt(200) * U32 * 10.0 * np.abs(ref).max()
