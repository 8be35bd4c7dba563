"""Q built on the tensor cores (XM_BUILD_SPLIT_BF16: the blocked triangular solve C = L^-1 Bbar^T
and the rank-(N-1) product C^T C of App. A's translation elimination, by error-free digit
splitting on tcgen05) against
the oracle's FP64 Schur-form Q and against the FP64 DSYRK build; its packed FP32 / BF16 copies;
the automatic choice; and a certified solve on it."""
import numpy as np
import pytest

import scenes
from oracle import xm_oracle as O
from tests.gpu_util import EPS32, EPS_BF16, ctx, gamma, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    c = ctx()
    yield c
    c.close()


def _build(C, sc, mode, mask=7):
    from paper_2502_04640_b300 import xm
    xm.xm_set_build_mode(C, mode)
    try:
        q = xm.xm_build_Q(C, sc.N, sc.M, *xm.scene_tensors(sc), store_mask=mask)
    finally:
        xm.xm_set_build_mode(C, xm.XM_BUILD_AUTO)
    return q


CASES = [
    # one tile, K = 19 (one ragged k-block)
    ("c1", lambda: scenes.config1()),
    # 10 tiles with a ragged edge, K = 129
    ("tiles", lambda: scenes.random_scene(130, 3000, noise=0.02, outlier_frac=0.02, seed=6)),
    # chain-like view graph: an ill-conditioned translation block
    ("traj", lambda: scenes.sub_scene(scenes.trajectory_scene(300, 20000, seed=7), 120)),
    # 55 tiles; K = 399: levels of up to 56 k-blocks, several exact-accumulation chunks each
    ("chunks", lambda: scenes.random_scene(400, 8000, noise=0.02, outlier_frac=0.05, seed=8)),
    # K = 699: one ragged diagonal block of the triangular solve, a blocked Cholesky factor
    # (blocks 512 + 187); 17 tile rows, so the last 256-column tile is half outside
    ("trsm-blocks", lambda: scenes.random_scene(700, 12000, noise=0.02, outlier_frac=0.02, seed=15)),
]


@pytest.mark.parametrize("name,make", CASES)
def test_split_build_matches_oracle(C, name, make):
    from paper_2502_04640_b300 import xm
    sc = make()
    q = _build(C, sc, xm.XM_BUILD_SPLIT_BF16)
    assert xm.xm_qmat_build_info(q)[0] == xm.XM_BUILD_SPLIT_BF16
    Qs = xm.xm_qmat_to_dense(q).cpu().numpy()
    Qo = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    scale = np.abs(Qo).max()
    assert np.abs(Qs - Qo).max() <= 1e-9 * scale
    Y = np.random.default_rng(0).standard_normal((3 * sc.N, 4))
    assert abs(np.sum(Y * (Qs @ Y)) - np.sum(Y * (Qo @ Y))) <= \
        1e-9 * np.sum(np.abs(Y) * (np.abs(Qo) @ np.abs(Y)))
    # the FP64-unit build of the same scene: both are FP64-accurate rank-k updates
    qf = _build(C, sc, xm.XM_BUILD_FP64)
    assert xm.xm_qmat_build_info(qf)[0] == xm.XM_BUILD_FP64
    Qf = xm.xm_qmat_to_dense(qf).cpu().numpy()
    assert np.abs(Qs - Qf).max() <= 1e-11 * scale
    q.free()
    qf.free()


@pytest.mark.parametrize("N", [1500, 2200])
def test_split_build_large_against_fp64_build(C, N):
    """K = 1499: a single digit pair spans two exact-accumulation chunks; diagonal blocks of
    1024 + 475 rows in the triangular solve (one block update), 512 x 3 in the Cholesky factor.
    K = 2199: diagonal blocks 1024 + 1024 + 151 (two block updates, the second with a ragged
    row tile)."""
    from paper_2502_04640_b300 import xm
    sc = scenes.random_scene(N, 27 * N, noise=0.02, outlier_frac=0.05, seed=9)
    qs = _build(C, sc, xm.XM_BUILD_SPLIT_BF16)
    qf = _build(C, sc, xm.XM_BUILD_FP64)
    Qs = xm.xm_qmat_to_dense(qs)
    Qf = xm.xm_qmat_to_dense(qf)
    scale = Qf.abs().max().item()
    assert (Qs - Qf).abs().max().item() <= 1e-11 * scale
    Y = torch.randn((3 * sc.N, 4), dtype=torch.float64, device="cuda",
                    generator=torch.Generator(device="cuda").manual_seed(1))
    fs, ff = (Y * (Qs @ Y)).sum().item(), (Y * (Qf @ Y)).sum().item()
    assert abs(fs - ff) <= 1e-11 * (Y.abs() * (Qf.abs() @ Y.abs())).sum().item()
    qs.free()
    qf.free()


def test_split_build_packed_copies(C):
    """The FP32 and BF16 tiles the update writes are the FP64 tiles rounded: a sweep on each
    stays within the sweep's a-priori bound of the exact product with the FP64 Q."""
    from paper_2502_04640_b300 import xm
    sc = scenes.random_scene(200, 4000, noise=0.02, outlier_frac=0.02, seed=10)
    q = _build(C, sc, xm.XM_BUILD_SPLIT_BF16)
    Q = xm.xm_qmat_to_dense(q).cpu().numpy()
    n = 3 * sc.N
    Y = np.random.default_rng(2).standard_normal((n, 4))
    Y32 = Y.astype(np.float32)
    exact = Q @ Y32.astype(np.float64)
    absb = np.abs(Q) @ np.abs(Y32.astype(np.float64))
    for prec, eps_store in ((xm.XM_FP32_BULK, EPS32), (xm.XM_BF16Q_BULK, EPS_BF16)):
        W = xm.xm_qy(q, torch.as_tensor(Y32, device="cuda"), prec).cpu().numpy().astype(np.float64)
        bound = (gamma(n + 2, EPS32) + eps_store * (1 + gamma(n + 2, EPS32))) * absb
        assert np.all(np.abs(W - exact) <= bound + 1e-300), prec
    q.free()


def test_split_build_without_fp64_copy(C):
    """Store masks without the FP64 copy accumulate in a scratch FP64 buffer."""
    from paper_2502_04640_b300 import xm
    sc = scenes.random_scene(130, 3000, noise=0.02, seed=11)
    qs = _build(C, sc, xm.XM_BUILD_SPLIT_BF16, mask=xm.XM_STORE_FP32)
    qf = _build(C, sc, xm.XM_BUILD_FP64, mask=xm.XM_STORE_FP32)
    Y = torch.randn((3 * sc.N, 4), dtype=torch.float32, device="cuda",
                    generator=torch.Generator(device="cuda").manual_seed(3))
    Ws = xm.xm_qy(qs, Y, xm.XM_FP32_BULK)
    Wf = xm.xm_qy(qf, Y, xm.XM_FP32_BULK)
    assert torch.allclose(Ws, Wf, rtol=1e-5, atol=1e-5 * Wf.abs().max().item())
    qs.free()
    qf.free()


def test_auto_mode_and_bad_mode(C):
    from paper_2502_04640_b300 import xm
    small = scenes.circle_scene(30, 300, 4, 0.01, seed=12)
    q = xm.xm_build_Q(C, small.N, small.M, *xm.scene_tensors(small))
    assert xm.xm_qmat_build_info(q)[0] == xm.XM_BUILD_FP64
    q.free()
    big = scenes.random_scene(520, 10000, noise=0.02, seed=13)
    q = xm.xm_build_Q(C, big.N, big.M, *xm.scene_tensors(big))
    path, t = xm.xm_qmat_build_info(q)
    assert path == xm.XM_BUILD_SPLIT_BF16 and t > 0.0
    q.free()
    one = scenes.circle_scene(1, 20, 1, 0.0, seed=1)
    q = _build(C, one, xm.XM_BUILD_SPLIT_BF16)        # N = 1: no translation update at all
    assert xm.xm_qmat_build_info(q)[0] == xm.XM_BUILD_AUTO
    q.free()
    with pytest.raises(xm.XmError) as e:
        xm.xm_set_build_mode(C, 7)
    assert e.value.status == xm.XM_EINVAL


def test_certified_solve_on_split_build(C):
    from paper_2502_04640_b300 import xm
    sc = scenes.random_scene(60, 1200, noise=0.02, outlier_frac=0.02, seed=14, center_sigma=3.0)
    q = _build(C, sc, xm.XM_BUILD_SPLIT_BF16)
    out = xm.xm_solve(q, xm.xm_default_opts(prec=xm.XM_FP64))
    info = out["info"]
    ref = O.solve(O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w), r0=4)
    assert info["certified"] == 1 and ref.certified
    assert abs(info["f"] - ref.f) / (1.0 + abs(ref.f)) <= 1e-9
    q.free()
