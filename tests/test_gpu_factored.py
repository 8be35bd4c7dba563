"""Factored Q operator (App. A's elimination in product form) against the oracle's dense Q Y,
element by element.

Bound: both sides evaluate the same exact product in FP64 by different routes.  With the
magnitudes T_P = |Q1||Y| + |V2 D^-1 V2^T||Y| (the landmark-eliminated part) and
T_S = |Bbar||Sbar^-1||Bbar^T||Y| (the translation part), each route's error is at most
gamma_K (T_P + kappa(Sbar) T_S) with K the longest chain of sums (observations of a camera and of
a landmark plus N); the test allows the sum of the two.  On the CPU the same difference measured
below one ulp of T_P + T_S."""
import numpy as np
import pytest

import scenes
from oracle import xm_oracle as O
from tests.gpu_util import EPS64, ctx, gamma, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    c = ctx()
    yield c
    c.close()


def _bound(sc, Y):
    N, M = sc.N, sc.M
    dm = O.data_matrices(N, M, sc.cam, sc.lmk, sc.ukp, sc.w)
    d = np.asarray(dm["Q3"].diagonal()).ravel()
    di = np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0)
    aY = np.abs(Y)
    V2 = abs(dm["V2"])
    TP = abs(dm["Q1"]) @ aY + V2 @ (di[:, None] * (V2.T @ aY))
    K = 2 * (np.bincount(sc.cam, minlength=N).max() + np.bincount(sc.lmk, minlength=M).max() + N + 8)
    if N == 1:
        return 2 * gamma(K, EPS64) * TP
    V3 = dm["V3"].toarray()
    S = dm["Q2"].toarray() - (V3 * di[None, :]) @ V3.T
    Sb_inv = np.linalg.inv(S[1:, 1:])
    B = dm["V1"].toarray() - (dm["V2"] @ (di[:, None] * V3.T))
    Bb = np.abs(B[:, 1:])
    TS = Bb @ (np.abs(Sb_inv) @ (Bb.T @ aY))
    return 2 * gamma(K, EPS64) * (TP + np.linalg.cond(S[1:, 1:]) * TS)


def _check(C, sc, rs, seed=0):
    from paper_2502_04640_b300 import xm
    Q = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    f = xm.xm_qfact_create(C, sc.N, sc.M, *xm.scene_tensors(sc))
    for r in rs:
        Y = np.random.default_rng(seed + r).standard_normal((3 * sc.N, r))
        W = xm.xm_qy_factored(f, torch.tensor(Y, device="cuda")).cpu().numpy()
        err = np.abs(W - Q @ Y)
        bnd = _bound(sc, Y)
        assert np.all(err <= bnd), (r, float((err / bnd).max()))
    f.free()


@pytest.mark.parametrize("N,M,seed", [(2, 60, 3), (20, 400, 1), (90, 4000, 21), (300, 6000, 31)])
def test_factored_product_matches_dense_Q(C, N, M, seed):
    """Two cameras to 300 (the -Sbar^-1 sweep from a single tile to three tile rows with a ragged
    tail), outliers, every padded width of the kernels (r = 1, 3, 4, 5, 8)."""
    sc = scenes.random_scene(N, M, noise=0.03, outlier_frac=0.05, seed=seed, center_sigma=3.0)
    _check(C, sc, (1, 3, 4, 5, 8))


def test_single_camera_and_unobserved_landmarks(C):
    """N = 1 (no translation block: Q = P), and a scene whose landmark list has entries without
    observations and with a single one (both contribute nothing)."""
    _check(C, scenes.circle_scene(1, 30, 1, 0.0, seed=2), (1, 4))
    sc = scenes.circle_scene(12, 200, 3, 0.02, seed=5)
    keep = sc.lmk % 7 != 3                       # landmarks 3, 10, ... lose every observation
    one = (sc.lmk % 11 == 5) & (np.arange(sc.E) % 3 != 0)    # some keep a single observation
    sel = keep & ~one
    sub = scenes.Scene(sc.name + "-holes", sc.N, sc.M, sc.cam[sel], sc.lmk[sel], sc.ukp[sel], sc.w[sel],
                       sc.R_gt, sc.s_gt, sc.t_gt, sc.p_gt, sc.outlier[sel])
    assert O.graph_is_connected(sub.N, sub.M, sub.cam, sub.lmk)
    _check(C, sub, (3, 8))


def test_factored_product_at_1934_cameras(C):
    """The 1934-camera workload itself (about 1.5 M observations; -Sbar^-1 of 15 x 15 tiles)."""
    sc = scenes.config2()
    from paper_2502_04640_b300 import xm
    Q = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    f = xm.xm_qfact_create(C, sc.N, sc.M, *xm.scene_tensors(sc))
    Y = np.random.default_rng(7).standard_normal((3 * sc.N, 4))
    W = xm.xm_qy_factored(f, torch.tensor(Y, device="cuda")).cpu().numpy()
    err = np.abs(W - Q @ Y)
    bnd = _bound(sc, Y)
    assert np.all(err <= bnd), float((err / bnd).max())
    f.free()


def test_factored_product_properties_at_10155_cameras(C):
    """The 10155-camera size, where the oracle cannot form Q: (a) on the noise-free scene the
    ground truth is in Q's null space (every residual vanishes), (b) <Z1, Q Z2> = <Z2, Q Z1>,
    (c) agreement with the dense FP64 sweep of the tensor-core-built Q within that build's tested
    entrywise bar (1e-9 of max|Q|, max|Q| <= max diag(Q1) for the PSD Q <= Q1) times each column's
    1-norm."""
    from paper_2502_04640_b300 import xm
    clean = scenes.random_scene(10155, 1_500_000, noise=0.0, outlier_frac=0.0, seed=1)
    f = xm.xm_qfact_create(C, clean.N, clean.M, *xm.scene_tensors(clean))
    R, s, _, _ = clean.anchored_gt()
    Ygt = np.concatenate([s[i] * R[i] for i in range(clean.N)], axis=1).T
    W = xm.xm_qy_factored(f, torch.tensor(Ygt, device="cuda")).cpu().numpy()
    q1 = np.zeros((clean.N, 3))
    np.add.at(q1, clean.cam, clean.w[:, None] * np.abs(clean.ukp) * np.abs(clean.ukp).sum(1, keepdims=True))
    scale = (q1.reshape(-1)[:, None] * np.abs(Ygt).max())
    assert np.all(np.abs(W) <= 1e-9 * scale.max())
    f.free()
    sc = scenes.config3()
    t = xm.scene_tensors(sc)
    f = xm.xm_qfact_create(C, sc.N, sc.M, *t)
    rng = np.random.default_rng(11)
    Z1, Z2 = rng.standard_normal((3 * sc.N, 4)), rng.standard_normal((3 * sc.N, 4))
    W1 = xm.xm_qy_factored(f, torch.tensor(Z1, device="cuda")).cpu().numpy()
    W2 = xm.xm_qy_factored(f, torch.tensor(Z2, device="cuda")).cpu().numpy()
    a, b = np.sum(Z2 * W1), np.sum(Z1 * W2)
    assert abs(a - b) <= 1e-10 * (np.abs(Z2) * np.abs(W1)).sum()
    q = xm.xm_build_Q(C, sc.N, sc.M, *t, xm.XM_STORE_FP64)
    Wd = xm.xm_qy(q, torch.tensor(Z1, device="cuda"), xm.XM_FP64).cpu().numpy()
    q1 = np.zeros((sc.N, 3))
    np.add.at(q1, sc.cam, sc.w[:, None] * sc.ukp ** 2)
    tol = 1e-9 * q1.max() * np.abs(Z1).sum(axis=0)[None, :]
    assert np.all(np.abs(W1 - Wd) <= tol)
    q.free()
    f.free()


def test_factored_operator_errors(C):
    from paper_2502_04640_b300 import xm
    a = scenes.circle_scene(3, 10, 3, 0.01, seed=6)
    cam = np.concatenate([a.cam, a.cam + 3]); lmk = np.concatenate([a.lmk, a.lmk + 10])
    ukp = np.concatenate([a.ukp, a.ukp]); w = np.concatenate([a.w, a.w])
    two = scenes.Scene("two", 6, 20, cam.astype(np.int32), lmk.astype(np.int32), ukp, w, a.R_gt, a.s_gt,
                       a.t_gt, a.p_gt, np.zeros(cam.size, bool))
    with pytest.raises(xm.XmError) as e:
        xm.xm_qfact_create(C, two.N, two.M, *xm.scene_tensors(two))
    assert e.value.status == xm.XM_EDISCONNECTED
    sc = scenes.circle_scene(6, 40, 3, 0.01, seed=7)
    f = xm.xm_qfact_create(C, sc.N, sc.M, *xm.scene_tensors(sc))
    Y = torch.zeros((18, 9), dtype=torch.float64, device="cuda")
    assert xm.lib().xm_qy_factored(C.h, f.h, 9, Y.data_ptr(), Y.data_ptr()) == xm.XM_EINVAL
    f.free()


@pytest.mark.parametrize("mask,prec", [("factored", 0), ("fp32+factored", 1)])
@pytest.mark.parametrize("scene", ["config1", "outliers"])
def test_solve_on_the_factored_operator(C, mask, prec, scene):
    """XM_STORE_FACTORED: every FP64 product (the FP64 RTR, the mixed modes' polish, the
    certificate's Z products, rounding) goes through the factored operator.  Alone, Q is never
    formed and the solve runs in FP64; with the FP32 tiles, the bulk phase reads them.  Either
    way the certified optimum is the oracle's."""
    from paper_2502_04640_b300 import xm
    from tests.oracle_checks import check_at_returned_point
    sc = scenes.config1() if scene == "config1" else scenes.random_scene(
        90, 4000, noise=0.03, outlier_frac=0.05, seed=21)
    Qo = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    ref = O.solve(Qo, r0=4)
    store = xm.XM_STORE_FACTORED | (xm.XM_STORE_FP32 if mask == "fp32+factored" else 0)
    q = xm.xm_build_Q(C, sc.N, sc.M, *xm.scene_tensors(sc), store)
    assert q.mask == store
    out = xm.xm_solve(q, xm.xm_default_opts(prec=prec))
    info = out["info"]
    assert info["certified"] == int(ref.certified) == 1
    assert abs(info["f"] - ref.f) <= 1e-6 * (1 + abs(ref.f))
    assert abs(info["lambda_min_deflated"] - ref.cert.lam_min_deflated) <= 1e-5 * ref.cert.lam_max_Q
    if ref.eta <= 1e-9:
        assert np.abs(out["R"].cpu().numpy() - ref.R).max() <= 1e-5
    check_at_returned_point(Qo, out)
    if prec == 0:
        assert info["n_sweeps_fp64"] == info["n_sweeps"]
    if mask == "factored":                 # no FP32 tiles for a mixed-mode solve
        with pytest.raises(xm.XmError) as e:
            xm.xm_solve(q, xm.xm_default_opts(prec=xm.XM_FP32_BULK))
        assert e.value.status == xm.XM_EINVAL
    q.free()
