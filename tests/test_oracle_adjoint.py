"""Pins for the oracle's adjoint: finite differences of complete re-solves (FP64) of a
gauge-invariant loss of the anchored scaled rotations G_i = s_i R_i."""
import numpy as np
import pytest

import scenes
from oracle import xm_oracle as O


def _solve_G(sc, ukp, w, Y0):
    Q = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, ukp, w)
    res = O.solve(Q, r0=Y0.shape[1], Y0=Y0, grad_tol_rel=1e-13)
    G = res.s[:, None, None] * res.R
    return G, res


def test_adjoint_matches_finite_differences():
    sc = scenes.circle_scene(6, 60, 3, 0.02, seed=31, w_range=(0.5, 1.5))
    rng = np.random.default_rng(31)
    C = rng.standard_normal((sc.N, 3, 3))
    C[0] = 0.0
    Q = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    base = O.solve(Q, r0=4, grad_tol_rel=1e-13)
    assert base.certified
    np.testing.assert_allclose(np.linalg.matrix_rank(base.Y, tol=1e-6 * np.abs(base.Y).max()), 3)
    d_u, d_w, _ = O.adjoint(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w, base.Y, C, Q=Q)
    loss = lambda G: float(np.sum(C * G))
    h = 1e-6
    for e, comp in [(0, 0), (5, 2), (37, 1), (101, 0)]:
        up, um = sc.ukp.copy(), sc.ukp.copy()
        up[e, comp] += h; um[e, comp] -= h
        fd = (loss(_solve_G(sc, up, sc.w, base.Y)[0]) - loss(_solve_G(sc, um, sc.w, base.Y)[0])) / (2 * h)
        assert abs(fd - d_u[e, comp]) <= 2e-5 * (1 + abs(fd)), (e, comp, fd, d_u[e, comp])
    for e in (3, 64, 150):
        wp, wm = sc.w.copy(), sc.w.copy()
        wp[e] += h; wm[e] -= h
        fd = (loss(_solve_G(sc, sc.ukp, wp, base.Y)[0]) - loss(_solve_G(sc, sc.ukp, wm, base.Y)[0])) / (2 * h)
        assert abs(fd - d_w[e]) <= 2e-5 * (1 + abs(fd)), (e, fd, d_w[e])


def test_optimal_residuals_reproduce_the_objective():
    """sum_e w_e e_e^2 = tr(U^T Q U) (Prop. 1) for the residual routine used by the adjoint."""
    sc = scenes.random_scene(7, 80, noise=0.05, seed=32, center_sigma=2.0)
    Q = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    U = np.random.default_rng(32).standard_normal((3 * sc.N, 5))
    e = O.optimal_residuals(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w, U)
    assert abs(np.sum(sc.w[:, None] * e * e) - O.cost(Q, U)) <= 1e-10 * O.cost(Q, U)


def test_adjoint_ignores_gauge_directions():
    """The loss of G_i = Y_0 Y_i^T is constant along Y -> Y O; the adjoint's lambda has no part
    along the gauge directions Y Omega, and the outputs do not change when the point moves along
    the orbit (Y -> Y O, a different representative of the same X)."""
    sc = scenes.circle_scene(8, 80, 3, 0.03, seed=33, w_range=(0.5, 1.5))
    Q = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    res = O.solve(Q, r0=4, grad_tol_rel=1e-13)
    assert res.certified
    C = np.random.default_rng(34).standard_normal((sc.N, 3, 3)); C[0] = 0.0
    d_u, d_w, lam = O.adjoint(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w, res.Y, C, Q=Q)
    Ng = O.gauge_basis(res.Y)
    assert np.abs(Ng.T @ lam.ravel()).max() <= 1e-10 * np.abs(lam).max()
    r = res.Y.shape[1]
    Oq, _ = np.linalg.qr(np.random.default_rng(35).standard_normal((r, r)))
    d_u2, d_w2, _ = O.adjoint(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w, res.Y @ Oq, C, Q=Q)
    assert np.abs(d_u2 - d_u).max() <= 1e-8 * np.abs(d_u).max()
    assert np.abs(d_w2 - d_w).max() <= 1e-8 * np.abs(d_w).max()
