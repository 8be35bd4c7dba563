"""Pins for the oracle's translation/landmark recovery (Eq. 7) and the XM^2 re-run
(Sec. 5: drop the 10 % of measurements with the largest residuals and solve again)."""
import numpy as np

import scenes
from oracle import xm_oracle as O


def test_recovered_tp_minimise_the_sba_cost_and_match_the_objective():
    """For fixed rotations and scales, (t, p) of Eq. 7 is the least-squares minimiser of Eq. 3:
    the cost equals f = tr(Y^T Q Y) at the rounded Y and no perturbation of (t, p) lowers it."""
    sc = scenes.random_scene(12, 150, noise=0.05, seed=81, center_sigma=3.0)
    Q = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    res = O.solve(Q, r0=4)
    U3 = np.concatenate([res.s[i] * res.R[i] for i in range(sc.N)], axis=1)
    t, p = O.recover_tp(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w, U3)
    assert np.abs(t[0]).max() == 0.0                          # the anchor (gauge)
    c = O.sba_cost(sc.cam, sc.lmk, sc.ukp, sc.w, res.R, res.s, t, p)
    assert abs(c - res.rho_hat) <= 1e-9 * (1 + c)
    assert abs(np.sum(O.observation_residuals(sc.cam, sc.lmk, sc.ukp, sc.w, res.R, res.s, t, p)) - c) \
        <= 1e-12 * (1 + c)
    rng = np.random.default_rng(81)
    for _ in range(5):
        dt = 1e-4 * rng.standard_normal(t.shape); dt[0] = 0.0
        dp = 1e-4 * rng.standard_normal(p.shape)
        assert O.sba_cost(sc.cam, sc.lmk, sc.ukp, sc.w, res.R, res.s, t + dt, p + dp) >= c


def test_keep_rule_drops_exactly_the_largest_terms():
    res2 = np.array([5.0, 1.0, 9.0, 9.0, 0.5, 7.0, 2.0, 3.0, 4.0, 6.0, 8.0])
    keep = O.xm2_keep(res2, 0.2)                              # floor(0.2 * 11) = 2 dropped
    assert list(np.nonzero(~keep)[0]) == [2, 3]
    assert O.xm2_keep(res2, 0.0).all()


def test_xm2_drops_the_largest_terms_and_resolves_the_rest():
    """The second solve is the certified solve of the kept measurements, and the dropped tenth
    is the tenth with the largest residual terms at the first solve's (R, s, t, p).  The rule is
    a greedy heuristic: on a scene with 5 % planted outliers the dropped set is strongly
    enriched in them (not a guarantee of a better estimate)."""
    sc = scenes.random_scene(15, 300, noise=0.01, outlier_frac=0.05, seed=82, center_sigma=3.0)
    x = O.solve_xm2(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    first, second, keep = x.first, x.second, x.keep
    assert first.certified and second.certified and x.cams.all()
    assert keep.sum() == sc.E - int(0.1 * sc.E)
    U3 = np.concatenate([first.s[i] * first.R[i] for i in range(sc.N)], axis=1)
    t1, p1 = O.recover_tp(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w, U3)
    r2 = O.observation_residuals(sc.cam, sc.lmk, sc.ukp, sc.w, first.R, first.s, t1, p1)
    assert r2[~keep].min() >= r2[keep].max()
    Q2 = O.build_Q_schur(sc.N, sc.M, sc.cam[keep], sc.lmk[keep], sc.ukp[keep], sc.w[keep])
    ref = O.solve(Q2, r0=4)
    assert abs(ref.f - second.f) <= 1e-8 * (1 + abs(ref.f))
    assert np.abs(ref.R - second.R).max() <= 1e-6
    frac_outliers_in_dropped = np.mean(sc.outlier[~keep])
    assert frac_outliers_in_dropped >= 3 * np.mean(sc.outlier)


def _isolating_scene():
    """40 cameras in which every measurement of camera 7 is a planted outlier (uniform in a box
    of side 200 in its frame): its residual terms are the largest, XM^2's cut drops all of them
    and leaves camera 7 without a measurement."""
    sc = scenes.random_scene(40, 500, noise=0.01, outlier_frac=0.0, seed=83, center_sigma=3.0)
    rng = np.random.default_rng(83)
    ukp = sc.ukp.copy()
    bad = sc.cam == 7
    ukp[bad] = rng.uniform(-100.0, 100.0, size=(int(bad.sum()), 3))
    return sc, ukp, bad


def test_xm2_solves_the_largest_component_when_the_cut_isolates_cameras():
    """Cameras whose every measurement is dropped leave the view graph: here camera 7 (planted
    outliers) and the anchor itself (the unregularised optimum shrinks the other scales, so the
    anchor's unit-scale terms are among the largest).  The second solve is the certified solve of
    the largest component (the other 38 cameras and the landmarks they still see, re-indexed,
    anchored at camera 1), and the isolated cameras are reported with zero scale and rotation."""
    sc, ukp, bad = _isolating_scene()
    assert bad.sum() < int(0.1 * sc.E)            # all of them fit inside the dropped tenth
    x = O.solve_xm2(sc.N, sc.M, sc.cam, sc.lmk, ukp, sc.w)
    assert not x.keep[bad].any() and x.keep.sum() <= sc.E - int(0.1 * sc.E)
    kept_any = np.bincount(sc.cam[x.keep],
                           minlength=sc.N) > 0
    assert list(np.nonzero(~x.cams)[0]) == [0, 7]
    assert np.array_equal(x.cams, kept_any)
    for i in (0, 7):
        assert x.s[i] == 0.0 and not x.R[i].any() and not x.t[i].any()
    assert x.second.certified and np.all(x.s[x.cams] > 0)
    assert np.allclose(x.R[1], np.eye(3)) and x.s[1] == 1.0 and not x.t[1].any()   # new anchor
    # the same solve written out by hand on the component (cameras 0 and 7 removed, re-indexed)
    use = x.keep
    cidx = np.setdiff1d(np.arange(sc.N), [0, 7])
    cmap = -np.ones(sc.N, np.int64); cmap[cidx] = np.arange(cidx.size)
    lm = np.unique(sc.lmk[use])
    lmap = -np.ones(sc.M, np.int64); lmap[lm] = np.arange(lm.size)
    Q2 = O.build_Q_schur(cidx.size, lm.size, cmap[sc.cam[use]], lmap[sc.lmk[use]], ukp[use], sc.w[use])
    ref = O.solve(Q2, r0=4)
    assert abs(ref.f - x.second.f) <= 1e-9 * (1 + abs(ref.f))
    assert np.abs(x.R[cidx] - ref.R).max() <= 1e-6
    # landmarks seen only through dropped measurements get no position
    unseen = np.setdiff1d(np.arange(sc.M), lm)
    assert unseen.size and not x.p[unseen].any()
