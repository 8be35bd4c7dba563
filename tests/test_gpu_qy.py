"""Q.Y sweep kernel (packed symmetric tiles, bulk-async pipeline) against the exact product,
element by element, within the a-priori rounding bound of each storage precision."""
import numpy as np
import pytest

from tests.gpu_util import EPS32, EPS64, EPS_BF16, ctx, gamma, rand_sym, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    c = ctx()
    yield c
    c.close()


@pytest.mark.parametrize("N", [1, 20, 43, 86, 300])   # n = 3 .. 900: one tile, ragged tails, many tiles
@pytest.mark.parametrize("r", [1, 3, 4, 5, 8])
def test_sweep_matches_dense_product(C, N, r):
    from paper_2502_04640_b300 import xm
    n = 3 * N
    Q = rand_sym(n, 1000 + N)
    Y = np.random.default_rng(r).standard_normal((n, r))
    W_ref = Q @ Y
    bound = np.abs(Q) @ np.abs(Y)
    q = xm.xm_qmat_from_dense(C, torch.tensor(Q, device="cuda"))
    W64 = xm.xm_qy(q, torch.tensor(Y, device="cuda"), xm.XM_FP64).cpu().numpy()
    assert np.all(np.abs(W64 - W_ref) <= gamma(n + 2, EPS64) * bound + 1e-300)
    Y32 = Y.astype(np.float32)
    W_ref32 = Q @ Y32.astype(np.float64)
    b32 = np.abs(Q) @ np.abs(Y32.astype(np.float64))
    W32 = xm.xm_qy(q, torch.tensor(Y32, device="cuda"), xm.XM_FP32_BULK).cpu().numpy()
    assert np.all(np.abs(W32 - W_ref32) <= (EPS32 + gamma(n + 2, EPS32)) * b32 + 1e-30)
    W16 = xm.xm_qy(q, torch.tensor(Y32, device="cuda"), xm.XM_BF16Q_BULK).cpu().numpy()
    assert np.all(np.abs(W16 - W_ref32) <= (EPS_BF16 + gamma(n + 2, EPS32)) * b32 + 1e-30)
    q.free()


@pytest.mark.parametrize("r", [1, 4, 8])
def test_sweep_several_tiles_per_cta(C, r):
    """n = 6000 (2000 cameras): 1128 packed tiles over the persistent grid, so every CTA walks a
    range of about eight tiles across tile-row changes and around its copy ring; the full W is
    checked element by element in all three storage precisions."""
    from paper_2502_04640_b300 import xm
    n = 6000
    Q = rand_sym(n, 6000 + r)
    Y = np.random.default_rng(60 + r).standard_normal((n, r))
    q = xm.xm_qmat_from_dense(C, torch.tensor(Q, device="cuda"))
    W64 = xm.xm_qy(q, torch.tensor(Y, device="cuda"), xm.XM_FP64).cpu().numpy()
    assert np.all(np.abs(W64 - Q @ Y) <= gamma(n + 2, EPS64) * (np.abs(Q) @ np.abs(Y)))
    Y32 = Y.astype(np.float32)
    ref32 = Q @ Y32.astype(np.float64)
    b32 = np.abs(Q) @ np.abs(Y32.astype(np.float64))
    W32 = xm.xm_qy(q, torch.tensor(Y32, device="cuda"), xm.XM_FP32_BULK).cpu().numpy()
    assert np.all(np.abs(W32 - ref32) <= (EPS32 + gamma(n + 2, EPS32)) * b32)
    W16 = xm.xm_qy(q, torch.tensor(Y32, device="cuda"), xm.XM_BF16Q_BULK).cpu().numpy()
    assert np.all(np.abs(W16 - ref32) <= (EPS_BF16 + gamma(n + 2, EPS32)) * b32)
    q.free()


def test_dense_roundtrip_and_symmetry(C):
    from paper_2502_04640_b300 import xm
    for N in (1, 43, 100):
        Q = rand_sym(3 * N, N)
        q = xm.xm_qmat_from_dense(C, torch.tensor(Q, device="cuda"))
        back = xm.xm_qmat_to_dense(q).cpu().numpy()
        assert np.array_equal(back, Q)
        q.free()


def test_sweep_rejects_bad_arguments(C):
    from paper_2502_04640_b300 import xm
    q = xm.xm_qmat_from_dense(C, torch.tensor(rand_sym(6, 1), device="cuda"), xm.XM_STORE_FP64)
    with pytest.raises(xm.XmError):   # no FP32 copy stored
        xm.xm_qy(q, torch.zeros((6, 2), dtype=torch.float32, device="cuda"), xm.XM_FP32_BULK)
    Y = torch.zeros((6, 9), dtype=torch.float64, device="cuda")
    W = torch.zeros_like(Y)
    assert xm.lib().xm_qy(C.h, q.h, xm.XM_FP64, 9, Y.data_ptr(), W.data_ptr()) == xm.XM_EINVAL
    q.free()


def test_sweep_full_size_sampled_rows(C):
    """Largest workload's size (n = 30465, 10155 cameras), FP32 and FP64 storage, in the launch
    configuration the benchmark times; sampled rows checked against exact row products."""
    from paper_2502_04640_b300 import xm
    n = 3 * 10155
    g = torch.Generator(device="cuda").manual_seed(7)
    Qt = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
    Qt = (Qt + Qt.T) * 0.5
    q = xm.xm_qmat_from_dense(C, Qt, xm.XM_STORE_FP64 | xm.XM_STORE_FP32)
    rows = np.r_[0:3, 127:131, 15000:15003, n - 5:n]
    Qs = Qt[rows].cpu().numpy()
    del Qt
    torch.cuda.empty_cache()
    Y = np.random.default_rng(3).standard_normal((n, 4))
    W64 = xm.xm_qy(q, torch.tensor(Y, device="cuda"), xm.XM_FP64)[rows].cpu().numpy()
    ref = Qs @ Y
    bound = np.abs(Qs) @ np.abs(Y)
    assert np.all(np.abs(W64 - ref) <= gamma(n + 2, EPS64) * bound)
    Y32 = Y.astype(np.float32)
    W32 = xm.xm_qy(q, torch.tensor(Y32, device="cuda"), xm.XM_FP32_BULK)[rows].cpu().numpy()
    ref32 = Qs @ Y32.astype(np.float64)
    b32 = np.abs(Qs) @ np.abs(Y32.astype(np.float64))
    assert np.all(np.abs(W32 - ref32) <= (EPS32 + gamma(n + 2, EPS32)) * b32)
    q.free()
