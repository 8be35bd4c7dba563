"""Translations and landmarks (Eq. 7), per-measurement residual terms and the XM^2 re-run on
the GPU against the FP64 oracle.  Recovery at the same (R, s) is FP64 least squares on both
sides: t and p agree to 1e-9 of their scale and the residual terms to 1e-9 relative.  XM^2's
keep rule compares FP64 residual terms computed from two different (agreeing to ~1e-6)
first solves, so the kept sets may differ only at the threshold: every disagreement must sit
within 1e-4 (relative) of it, and the final rotations agree to 1e-5."""
import numpy as np
import pytest

import scenes
from oracle import xm_oracle as O
from tests.gpu_util import ctx, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    c = ctx()
    yield c
    c.close()


def test_recover_tp_matches_oracle(C):
    from paper_2502_04640_b300 import xm
    sc = scenes.random_scene(25, 400, noise=0.03, outlier_frac=0.02, seed=91, center_sigma=3.0)
    Q = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    ref = O.solve(Q, r0=4)
    U3 = np.concatenate([ref.s[i] * ref.R[i] for i in range(sc.N)], axis=1)
    t_ref, p_ref = O.recover_tp(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w, U3)
    r2_ref = O.observation_residuals(sc.cam, sc.lmk, sc.ukp, sc.w, ref.R, ref.s, t_ref, p_ref)
    cam, lmk, ukp, w = xm.scene_tensors(sc)
    t, p, r2 = xm.xm_recover_tp(C, sc.N, sc.M, cam, lmk, ukp, w, torch.tensor(ref.R, device="cuda"),
                                torch.tensor(ref.s, device="cuda"))
    scale = max(np.abs(t_ref).max(), np.abs(p_ref).max())
    assert np.abs(t.cpu().numpy() - t_ref).max() <= 1e-9 * scale
    assert np.abs(p.cpu().numpy() - p_ref).max() <= 1e-9 * scale
    assert np.abs(r2.cpu().numpy() - r2_ref).max() <= 1e-9 * (1 + np.abs(r2_ref).max())


def test_noise_free_recovery_of_translations_and_landmarks(C):
    from paper_2502_04640_b300 import xm
    sc = scenes.circle_scene(12, 120, 4, 0.0, seed=18)
    q = xm.xm_build_Q(C, sc.N, sc.M, *xm.scene_tensors(sc))
    out = xm.xm_solve(q, xm.xm_default_opts(prec=0), allow_notcert=False)
    t, p, r2 = xm.xm_recover_tp(C, sc.N, sc.M, *xm.scene_tensors(sc), out["R"], out["s"])
    R, s, t_gt, p_gt = sc.anchored_gt()
    assert np.abs(t.cpu().numpy() - t_gt).max() <= 1e-7 and np.abs(p.cpu().numpy() - p_gt).max() <= 1e-7
    assert float(r2.abs().max()) <= 1e-12
    q.free()


def test_xm2_matches_oracle(C):
    from paper_2502_04640_b300 import xm
    sc = scenes.random_scene(15, 300, noise=0.01, outlier_frac=0.05, seed=82, center_sigma=3.0)
    x = O.solve_xm2(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    first, second, keep_ref, t_ref, p_ref = x.first, x.second, x.keep, x.t, x.p
    out = xm.xm_solve_xm2(C, sc.N, sc.M, *xm.scene_tensors(sc), xm.xm_default_opts(), 0.1,
                          allow_notcert=False)
    keep = out["keep"].cpu().numpy()
    assert keep.sum() == keep_ref.sum() == sc.E - int(0.1 * sc.E)
    diff = np.nonzero(keep != keep_ref)[0]
    if diff.size:
        U3 = np.concatenate([first.s[i] * first.R[i] for i in range(sc.N)], axis=1)
        t1, p1 = O.recover_tp(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w, U3)
        r2 = O.observation_residuals(sc.cam, sc.lmk, sc.ukp, sc.w, first.R, first.s, t1, p1)
        thr = r2[~keep_ref].min()
        assert np.all(np.abs(r2[diff] - thr) <= 1e-4 * thr)
    assert out["info_first"]["certified"] == 1 and out["info_second"]["certified"] == 1
    assert np.abs(out["R"].cpu().numpy() - second.R).max() <= 1e-5
    scale = max(np.abs(t_ref).max(), np.abs(p_ref).max())
    assert np.abs(out["t"].cpu().numpy() - t_ref).max() <= 1e-4 * scale
    assert np.abs(out["p"].cpu().numpy() - p_ref).max() <= 1e-4 * scale


def test_xm2_on_a_split_view_graph_matches_oracle(C):
    """The cut drops every measurement of a camera with planted outliers and of the anchor (the
    unregularised optimum shrinks the other scales): both sides solve the largest remaining
    component, anchored at camera 1, and report cameras 0 and 7 with zero scale and rotation."""
    from paper_2502_04640_b300 import xm
    sc = scenes.random_scene(40, 500, noise=0.01, outlier_frac=0.0, seed=83, center_sigma=3.0)
    rng = np.random.default_rng(83)
    ukp = sc.ukp.copy()
    ukp[sc.cam == 7] = rng.uniform(-100.0, 100.0, size=(int((sc.cam == 7).sum()), 3))
    x = O.solve_xm2(sc.N, sc.M, sc.cam, sc.lmk, ukp, sc.w)
    assert list(np.nonzero(~x.cams)[0]) == [0, 7]
    cam, lmk, _, w = xm.scene_tensors(sc)
    out = xm.xm_solve_xm2(C, sc.N, sc.M, cam, lmk, torch.tensor(ukp, device="cuda"), w,
                          xm.xm_default_opts(), 0.1, allow_notcert=False)
    s, R = out["s"].cpu().numpy(), out["R"].cpu().numpy()
    assert out["status"] == xm.XM_OK and out["info_second"]["certified"] == 1
    assert np.array_equal(s > 0, x.cams) and not R[[0, 7]].any()
    keep = out["keep"].cpu().numpy()
    if not np.array_equal(keep, x.keep):
        # the two first solves agree to ~1e-6, so the cut may differ at its threshold only
        U3 = np.concatenate([x.first.s[i] * x.first.R[i] for i in range(sc.N)], axis=1)
        t1, p1 = O.recover_tp(sc.N, sc.M, sc.cam, sc.lmk, ukp, sc.w, U3)
        r2 = O.observation_residuals(sc.cam, sc.lmk, ukp, sc.w, x.first.R, x.first.s, t1, p1)
        thr = np.sort(r2)[::-1][int(0.1 * sc.E) - 1]
        diff = np.nonzero(keep != x.keep)[0]
        assert np.all(np.abs(r2[diff] - thr) <= 1e-4 * thr), r2[diff] / thr
        return
    assert abs(out["info_second"]["f"] - x.second.f) <= 1e-6 * (1 + abs(x.second.f))
    assert np.abs(R - x.R).max() <= 1e-5 and np.abs(s - x.s).max() <= 1e-5 * x.s.max()
    scale = max(np.abs(x.t).max(), np.abs(x.p).max())
    assert np.abs(out["t"].cpu().numpy() - x.t).max() <= 1e-4 * scale
    assert np.abs(out["p"].cpu().numpy() - x.p).max() <= 1e-4 * scale
