"""Pins for the oracle's scale-regularised problem (App. D): F(X) = mu sum_{i>=2} (X_{3i,3i}-1)^2
added to tr(QX), its gradient, Hessian, modified certificate matrix Z and dual value.  Each
test checks against something other than the oracle's own formulas: the two-view closed form
(Umeyama rotation plus the scalar cubic of the regularised scale), finite differences of the
cost along retraction curves, the dense X = Y Y^T entry by entry, weak duality over random
feasible points (convexity of F, App. E), and the large-mu limit.  CPU only."""
import numpy as np
import pytest

import scenes
from oracle import xm_oracle as O


def _Q(sc):
    return O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)


def _scaled_point(N, r, rng):
    Y = O.random_point(N, r, rng) * np.repeat(rng.uniform(0.5, 2.0, N), 3)[:, None]
    Y[:3] /= np.sqrt(O.alphas(Y)[0])
    return Y


def test_regulariser_reads_the_third_diagonal_entry_of_each_non_anchor_block():
    rng = np.random.default_rng(50)
    Y = _scaled_point(5, 4, rng)
    X = Y @ Y.T
    mu = 0.7
    want = mu * sum((X[3 * i + 2, 3 * i + 2] - 1.0) ** 2 for i in range(1, 5))
    assert abs(O.scale_reg_F(Y, mu) - want) <= 1e-14 * (1 + want)
    # on the feasible set X_ii = alpha_i I_3, so the entry equals the squared scale
    assert np.allclose(np.diag(X)[2::3], O.alphas(Y), rtol=1e-13)


@pytest.mark.parametrize("mu", [0.3, 4.0])
def test_regularised_gradient_and_hessian_match_finite_differences(mu):
    sc = scenes.circle_scene(6, 40, 3, 0.05, seed=51)
    Q = _Q(sc)
    rng = np.random.default_rng(51)
    Y = _scaled_point(6, 4, rng)
    Xi = O.proj_tangent(Y, rng.standard_normal(Y.shape))
    g = O.rgrad(Q, Y, mu=mu)
    H = O.hess(Q, Y, Xi, mu=mu)
    h = 1e-4
    fp, f0, fm = (O.cost(Q, O.retract(Y, t * Xi), mu) for t in (h, 0.0, -h))
    d1 = (fp - fm) / (2 * h)
    d2 = (fp - 2 * f0 + fm) / (h * h)
    assert abs(d1 - O.inner(g, Xi)) <= 1e-6 * (1 + abs(d1))
    assert abs(d2 - O.inner(H, Xi)) <= 1e-4 * (1 + abs(d2))
    # the regulariser's share is not negligible in this check
    g0 = O.rgrad(Q, Y)
    assert np.linalg.norm(g - g0) > 1e-2 * np.linalg.norm(g)
    Eta = O.proj_tangent(Y, rng.standard_normal(Y.shape))
    assert abs(O.inner(O.hess(Q, Y, Eta, mu=mu), Xi) - O.inner(H, Eta)) <= 1e-10 * np.abs(H).sum()


@pytest.mark.parametrize("mu", [0.5, 20.0])
def test_two_views_regularised_scale_is_the_root_of_the_cubic(mu):
    """N = 2, every landmark seen by both cameras: the problem is scaled registration
    (Umeyama 1991) with cost A s^2 - 2 B s + C after eliminating t, plus mu (s^2 - 1)^2.
    The rotation is Umeyama's (independent of s); s minimises the quartic, a root of
    4 mu s^3 + (2A - 4 mu) s - 2B = 0."""
    sc = scenes.circle_scene(2, 60, 2, 0.05, seed=17, w_range=(0.5, 1.5))
    Q = _Q(sc)
    res = O.solve(Q, r0=4, mu=mu, grad_tol_rel=1e-13)
    x = np.zeros((sc.M, 3)); y = np.zeros((sc.M, 3)); w1 = np.zeros(sc.M); w2 = np.zeros(sc.M)
    for e in range(sc.E):
        if sc.cam[e] == 0:
            y[sc.lmk[e]] = sc.ukp[e]; w1[sc.lmk[e]] = sc.w[e]
        else:
            x[sc.lmk[e]] = sc.ukp[e]; w2[sc.lmk[e]] = sc.w[e]
    om = w1 * w2 / (w1 + w2)
    _, R, _, _ = O.umeyama_weighted(x, y, om)
    xc = x - (om[:, None] * x).sum(0) / om.sum()
    yc = y - (om[:, None] * y).sum(0) / om.sum()
    A = float((om * (xc * xc).sum(1)).sum())
    B = float((om * (yc * (xc @ R.T)).sum(1)).sum())
    C = float((om * (yc * yc).sum(1)).sum())
    roots = np.roots([4 * mu, 0.0, 2 * A - 4 * mu, -2 * B])
    cand = [z.real for z in roots if abs(z.imag) < 1e-9 and z.real > 0]
    obj = lambda s: A * s * s - 2 * B * s + C + mu * (s * s - 1) ** 2
    s_star = min(cand, key=obj)
    assert res.certified
    assert abs(res.s[1] - s_star) <= 1e-8 * s_star
    assert np.abs(res.R[1] - R).max() <= 1e-7
    assert abs(res.rho_hat - obj(s_star)) <= 1e-9 * (1 + obj(s_star))
    assert abs(res.f - obj(s_star)) <= 1e-9 * (1 + obj(s_star))


def test_weak_duality_over_random_feasible_points():
    """App. E: for every feasible X, tr(QX) + F(X) >= <Z, X> + dual >= dual when Z >= 0 (F
    convex).  At the certified regularised optimum the gap is zero and no sampled feasible
    point of any rank goes below the dual value."""
    sc = scenes.circle_scene(8, 80, 3, 0.1, seed=52, w_range=(0.5, 1.5))
    Q = _Q(sc)
    mu = 2.0
    res = O.solve(Q, r0=4, mu=mu, grad_tol_rel=1e-12)
    assert res.certified
    c = res.cert
    assert abs(res.f - c.dual) <= 1e-9 * (1 + abs(res.f))
    assert c.lam_min >= -1e-8 * c.lam_max_Q
    rng = np.random.default_rng(52)
    worst = np.inf
    for k in range(300):
        r = int(rng.integers(3, 9))
        Y = O.random_point(sc.N, r, rng) * np.repeat(rng.uniform(0.2, 3.0, sc.N), 3)[:, None]
        Y[:3] /= np.sqrt(O.alphas(Y)[0])
        # half the samples near the optimum, where the bound is tight
        if k % 2:
            Yo = np.hstack([res.Y, np.zeros((res.Y.shape[0], max(0, r - res.Y.shape[1])))])[:, :r]
            Y = O.retract(Yo, 0.05 * O.proj_tangent(Yo, rng.standard_normal(Yo.shape)))
        worst = min(worst, O.cost(Q, Y, mu) - c.dual)
    assert worst >= -1e-9 * (1 + abs(res.f))


def test_large_mu_pins_every_scale_to_one():
    sc = scenes.circle_scene(6, 60, 3, 0.02, seed=53, s_range=(0.5, 2.0))
    Q = _Q(sc)
    res = O.solve(Q, r0=4, mu=1e6, grad_tol_rel=1e-12)
    assert res.certified
    assert np.abs(res.s - 1.0).max() <= 1e-3
    free = O.solve(Q, r0=4)
    assert np.abs(free.s - 1.0).max() > 0.1        # without the regulariser they are not
