"""Pins for the FP64 oracle: each test checks it against something other than itself
(closed forms, brute force, an independent SDP solver, the paper's printed matrices,
invariances and finite differences).  CPU only."""
import math
import os

import numpy as np
import pytest

import scenes
from oracle import xm_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _Q(sc, literal=False):
    f = O.build_Q_literal if literal else O.build_Q_schur
    return f(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)


def _Ygt(sc):
    R, s, _, _ = sc.anchored_gt()
    return np.concatenate([s[i] * R[i] for i in range(sc.N)], axis=1).T


# ------------------------------------------------------------------ Q construction (App. A)

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_literal_formula_equals_schur_form(seed):
    sc = scenes.random_scene(7, 60, noise=0.05, outlier_frac=0.1, seed=seed, center_sigma=2.0)
    Ql, Qs = _Q(sc, True), _Q(sc)
    assert np.abs(Ql - Qs).max() <= 1e-10 * np.abs(Qs).max()


@pytest.mark.parametrize("r", [3, 4, 5])
def test_trace_form_equals_brute_force_least_squares(r):
    """tr(Q U^T U) = min over t, p of the SBA cost (Prop. 1), for arbitrary U."""
    sc = scenes.circle_scene(6, 50, 3, 0.05, seed=3 + r)
    Q = _Q(sc)
    Y = np.random.default_rng(r).standard_normal((3 * sc.N, r))
    c, _, _ = O.min_over_tp(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w, Y)
    assert abs(O.cost(Q, Y) - c) <= 1e-9 * abs(c)


def test_observation_order_does_not_matter():
    sc = scenes.circle_scene(8, 60, 3, 0.02, seed=4)
    Q1, Q2 = _Q(sc), _Q(scenes.shuffled(sc))
    assert np.abs(Q1 - Q2).max() <= 1e-12 * np.abs(Q1).max()


def test_laplacian_rank_and_connectivity():
    """Lemma (App. A): Q_tp is the weighted Laplacian, rank N + M - 1 iff connected."""
    sc = scenes.circle_scene(6, 30, 3, 0.01, seed=5)
    Qtp, _ = O.laplacian_blocks(O.data_matrices(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w))
    L = Qtp.toarray()
    assert np.allclose(L.sum(1), 0) and np.allclose(L, L.T)
    assert np.linalg.matrix_rank(L) == sc.N + sc.M - 1
    assert O.graph_is_connected(sc.N, sc.M, sc.cam, sc.lmk)
    # two disjoint halves: rank drops by one, connectivity check fails
    a = scenes.circle_scene(3, 10, 3, 0.01, seed=6)
    cam = np.concatenate([a.cam, a.cam + 3]); lmk = np.concatenate([a.lmk, a.lmk + 10])
    ukp = np.concatenate([a.ukp, a.ukp]); w = np.concatenate([a.w, a.w])
    Qtp2, _ = O.laplacian_blocks(O.data_matrices(6, 20, cam, lmk, ukp, w))
    assert np.linalg.matrix_rank(Qtp2.toarray()) == 6 + 20 - 2
    assert not O.graph_is_connected(6, 20, cam, lmk)


def test_Q_is_psd_and_symmetric():
    sc = scenes.random_scene(9, 80, noise=0.1, outlier_frac=0.05, seed=7, center_sigma=2.0)
    Q = _Q(sc)
    ev = np.linalg.eigvalsh(Q)
    assert np.allclose(Q, Q.T, atol=0)
    assert ev.min() >= -1e-11 * ev.max()


def test_noise_free_scene_has_zero_cost_at_ground_truth():
    sc = scenes.circle_scene(10, 80, 4, 0.0, seed=8)
    Q = _Q(sc)
    Y = _Ygt(sc)
    assert np.abs(Q @ Y).max() <= 1e-11 * np.abs(Q).max() * np.abs(Y).max()
    assert abs(O.cost(Q, Y)) <= 1e-10 * np.abs(Q).sum()


def test_scaling_and_permutation_invariances():
    sc = scenes.circle_scene(6, 40, 3, 0.03, seed=9)
    Q = _Q(sc)
    Qu = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, 3.0 * sc.ukp, sc.w)
    Qw = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, 2.5 * sc.w)
    assert np.allclose(Qu, 9.0 * Q, rtol=1e-11, atol=1e-11 * np.abs(Q).max())
    assert np.allclose(Qw, 2.5 * Q, rtol=1e-11, atol=1e-11 * np.abs(Q).max())
    # relabel cameras 1..N-1 (anchor fixed): Q's blocks permute the same way
    perm = np.array([0, 3, 1, 5, 2, 4])
    inv = np.argsort(perm)
    Qp = O.build_Q_schur(sc.N, sc.M, inv[sc.cam], sc.lmk, sc.ukp, sc.w)
    idx = (3 * perm[:, None] + np.arange(3)).ravel()
    assert np.allclose(Qp, Q[np.ix_(idx, idx)], atol=1e-11 * np.abs(Q).max())


# ------------------------------------------------------------------ manifold calculus

def test_tangent_projection_is_orthogonal_projector():
    rng = np.random.default_rng(10)
    Y = O.random_point(5, 4, rng) * np.repeat([1.0, 2.0, 0.5, 1.5, 3.0], 3)[:, None]
    A = rng.standard_normal(Y.shape)
    P = O.proj_tangent(Y, A)
    assert np.allclose(O.proj_tangent(Y, P), P, atol=1e-13)
    # normal component S Y with S symmetric (anchor) / traceless symmetric (others)
    Nrm = A - P
    B = rng.standard_normal(Y.shape)
    assert abs(O.inner(Nrm, O.proj_tangent(Y, B))) <= 1e-12 * np.abs(A).sum() * np.abs(B).sum()
    # tangency: sym(Xi_i Y_i^T) is 0 (anchor) or a multiple of I (others)
    S = O._sym(np.einsum("iar,ibr->iab", O.blocks(P), O.blocks(Y)))
    assert np.abs(S[0]).max() < 1e-12
    dev = S[1:] - np.trace(S[1:], axis1=1, axis2=2)[:, None, None] / 3 * np.eye(3)
    assert np.abs(dev).max() < 1e-12


def test_retraction_is_feasible_and_first_order():
    rng = np.random.default_rng(11)
    Y = O.random_point(6, 5, rng) * np.repeat(rng.uniform(0.5, 2, 6), 3)[:, None]
    Y[:3] /= np.sqrt(O.alphas(Y)[0])
    Xi = O.proj_tangent(Y, rng.standard_normal(Y.shape))
    Yp = O.retract(Y, 0.3 * Xi)
    G = np.einsum("iar,ibr->iab", O.blocks(Yp), O.blocks(Yp))
    a = np.trace(G, axis1=1, axis2=2) / 3
    assert np.abs(G - a[:, None, None] * np.eye(3)).max() < 1e-12 and abs(a[0] - 1) < 1e-12
    h = 1e-6
    assert np.abs((O.retract(Y, h * Xi) - Y) / h - Xi).max() < 1e-5


def test_riemannian_gradient_and_hessian_match_finite_differences():
    sc = scenes.circle_scene(6, 40, 3, 0.05, seed=12)
    Q = _Q(sc)
    rng = np.random.default_rng(12)
    Y = O.random_point(6, 4, rng) * np.repeat(rng.uniform(0.5, 2, 6), 3)[:, None]
    Y[:3] /= np.sqrt(O.alphas(Y)[0])
    Xi = O.proj_tangent(Y, rng.standard_normal(Y.shape))
    g = O.rgrad(Q, Y)
    H = O.hess(Q, Y, Xi)
    h = 1e-4
    fp, f0, fm = (O.cost(Q, O.retract(Y, t * Xi)) for t in (h, 0.0, -h))
    d1 = (fp - fm) / (2 * h)
    d2 = (fp - 2 * f0 + fm) / (h * h)
    assert abs(d1 - O.inner(g, Xi)) <= 1e-6 * (1 + abs(d1))
    # metric projection is a second-order retraction: the identity holds away from critical points
    assert abs(d2 - O.inner(H, Xi)) <= 1e-4 * (1 + abs(d2))
    Eta = O.proj_tangent(Y, rng.standard_normal(Y.shape))
    assert abs(O.inner(O.hess(Q, Y, Eta), Xi) - O.inner(H, Eta)) <= 1e-10 * np.abs(H).sum()


# ------------------------------------------------------------------ SDP, certificate, staircase

def _paper_constraint_matrices(N):
    """A_i of Eq. 19 from the paper's printed B^1..B^5 (tests/golden/licq_basis.txt) for the
    non-anchor blocks; the anchor block's six constraints fix X_00 = I_3."""
    Bs = []
    with open(os.path.join(GOLDEN, "licq_basis.txt")) as fh:
        for line in fh:
            if line.startswith("B"):
                Bs.append(np.array(line.split(":")[1].split(), float).reshape(3, 3))
    n = 3 * N
    A = []
    for (p, q) in [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]:
        M = np.zeros((n, n)); M[p, q] = M[q, p] = 1.0; A.append(M)
    for k in range(1, N):
        for B in Bs:
            M = np.zeros((n, n)); M[3 * k:3 * k + 3, 3 * k:3 * k + 3] = B; A.append(M)
    return np.array(A), Bs


def test_closed_form_dual_matches_paper_constraint_basis():
    """Eq. 24 solved by least squares over the paper's printed A_i equals the closed form,
    there are 5N+1 constraints, and LICQ (App. C) makes the solution unique."""
    sc = scenes.circle_scene(5, 40, 3, 0.02, seed=13)
    Q = _Q(sc)
    res = O.rtr(Q, O.random_point(5, 4, np.random.default_rng(13)))
    A, Bs = _paper_constraint_matrices(5)
    assert A.shape[0] == 5 * 5 + 1
    Bm = np.array([B.ravel() for B in Bs])
    assert np.linalg.matrix_rank(Bm) == 5 and np.allclose(Bm[:, [0, 4, 8]].sum(1), 0)
    QY = Q @ res.Y
    cols = np.array([(Ai @ res.Y).ravel() for Ai in A]).T
    assert np.linalg.matrix_rank(cols) == A.shape[0]                  # LICQ
    y, *_ = np.linalg.lstsq(cols, QY.ravel(), rcond=None)
    Lam_ls = np.einsum("j,jab->ab", y, A)
    L = O.lambdas(res.Y, QY)
    Lam_cf = np.zeros_like(Q)
    for i in range(5):
        Lam_cf[3 * i:3 * i + 3, 3 * i:3 * i + 3] = L[i]
    assert np.abs(Lam_ls - Lam_cf).max() <= 1e-8 * np.abs(Lam_cf).max()
    # dual objective sum b_i y_i = tr(Lambda_0) = f at stationarity (zero duality gap)
    assert abs(y[:3].sum() - res.f) <= 1e-9 * (1 + abs(res.f))


@pytest.mark.parametrize("seed,outl", [(14, 0.0), (15, 0.1), (16, 0.0)])
def test_staircase_matches_independent_barrier_sdp(seed, outl):
    sc = scenes.random_scene(4, 40, noise=0.05, outlier_frac=outl, seed=seed, center_sigma=2.0)
    Q = _Q(sc)
    rho_sdp, X = O.sdp_barrier(Q)
    res = O.solve(Q, r0=4)
    assert res.certified
    assert abs(res.f - rho_sdp) <= 1e-7 * (1 + abs(rho_sdp))
    if np.linalg.matrix_rank(X, tol=1e-5 * np.abs(X).max()) == 3:
        Xbm = res.Y @ res.Y.T
        assert np.abs(Xbm - X).max() <= 1e-4 * np.abs(X).max()


def test_two_views_reduce_to_umeyama():
    """N = 2 with both cameras seeing every landmark: scaled point-cloud registration
    (Sec. 1, remark), solved in closed form (Umeyama 1991)."""
    rng = np.random.default_rng(17)
    sc = scenes.circle_scene(2, 60, 2, 0.05, seed=17, w_range=(0.5, 1.5))
    Q = _Q(sc)
    res = O.solve(Q, r0=4)
    x = np.zeros((sc.M, 3)); y = np.zeros((sc.M, 3)); w1 = np.zeros(sc.M); w2 = np.zeros(sc.M)
    for e in range(sc.E):
        if sc.cam[e] == 0:
            y[sc.lmk[e]] = sc.ukp[e]; w1[sc.lmk[e]] = sc.w[e]
        else:
            x[sc.lmk[e]] = sc.ukp[e]; w2[sc.lmk[e]] = sc.w[e]
    s, R, t, c = O.umeyama_weighted(x, y, w1 * w2 / (w1 + w2))
    assert res.certified
    assert abs(res.rho_hat - c) <= 1e-9 * (1 + c)
    assert np.abs(res.R[1] - R).max() < 1e-7 and abs(res.s[1] - s) < 1e-8


def test_noise_free_solve_recovers_ground_truth():
    sc = scenes.circle_scene(12, 120, 4, 0.0, seed=18)
    res = O.solve(_Q(sc), r0=4)
    R, s, t, p = sc.anchored_gt()
    assert res.certified and abs(res.f) < 1e-10
    assert np.abs(res.R - R).max() < 1e-8 and np.abs(res.s - s).max() < 1e-8
    U3 = np.concatenate([res.s[i] * res.R[i] for i in range(sc.N)], axis=1)
    tt, pp = O.recover_tp(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w, U3)
    assert np.abs(tt - t).max() < 1e-7 and np.abs(pp - p).max() < 1e-7


def test_certificate_structure_at_tight_optimum():
    sc = scenes.config1()
    Q = _Q(sc)
    res = O.solve(Q, r0=4)
    c = res.cert
    assert res.certified and c.ZY_norm <= 1e-9 * np.abs(Q).max()
    assert abs(res.f - c.dual) <= 1e-10 * (1 + abs(res.f))             # zero duality gap
    Z = Q.copy()
    for i in range(sc.N):
        Z[3 * i:3 * i + 3, 3 * i:3 * i + 3] -= c.Lambda[i]
    ev = np.linalg.eigvalsh(Z)
    assert np.sum(np.abs(ev) < 1e-8 * ev.max()) == 3                 # exactly rank(Y) zeros
    assert c.lam_min_deflated > 1e-3 * ev.max() * 1e-2               # positive gap
    assert res.eta >= -1e-12 and res.eta < 1e-6


def test_bad_local_minimum_is_rejected_and_escaped():
    """Alg. 1 from [I, ..., I]: the rank-3 local optimum of config 1 is not certified
    (Thm. 1 fails), the escape direction of Thm. 2 decreases f, and the staircase ends at
    the same certified value as random initial points (Thm. 3)."""
    sc = scenes.config1()
    Q = _Q(sc)
    r3 = O.rtr(Q, O.initial_point(sc.N, 3))
    c3 = O.certify(Q, r3.Y)
    assert c3.lam_min < -1e-3
    Yn, fn, alpha = O.escape(Q, r3.Y, c3.v, r3.f)
    assert Yn is not None and fn < r3.f
    fs = [O.solve(Q, r0=4).f]
    for k in range(3):
        fs.append(O.solve(Q, r0=5, Y0=O.random_point(sc.N, 5, np.random.default_rng(k))).f)
    assert max(fs) - min(fs) <= 1e-9 * (1 + abs(fs[0]))
    assert fs[0] < r3.f


def test_rounding_projects_reflections_onto_SO3():
    """A camera whose keypoints are mirrored has an O(3)-but-not-SO(3) optimum (Prop. 2,
    det < 0): rounding must return proper rotations and a feasible value rho_hat >= f."""
    sc = scenes.circle_scene(6, 60, 4, 0.0, seed=19)
    ukp = sc.ukp.copy()
    ukp[sc.cam == 3] *= np.array([1.0, 1.0, -1.0])
    Q = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, ukp, sc.w)
    res = O.solve(Q, r0=4)
    dets = np.linalg.det(res.R)
    assert np.all(dets > 0.999)
    assert res.rho_hat >= res.f - 1e-9 * (1 + abs(res.f))
    # the mirrored camera's rounded rotation is the SO(3) projection of its O(3) block
    Yb = np.swapaxes(O.blocks(res.Y @ np.linalg.eigh(res.Y.T @ res.Y)[1][:, ::-1][:, :3]), 1, 2)
    assert np.linalg.det(Yb[3]) * np.linalg.det(Yb[0]) < 0


# ------------------------------------------------------------------ Eq. 18 and App. E's bound

def _rounded_cost_brute_force(sc, R, s):
    """rho_hat evaluated independently of the oracle's Q: the SBA cost (Eq. 3) at the rounded
    rotations and scales, minimised over translations and landmarks by dense least squares."""
    U = np.concatenate([s[i] * R[i] for i in range(sc.N)], axis=1)
    c, _, _ = O.min_over_tp(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w, U.T)
    return c


def test_eta_against_barrier_sdp_value_and_brute_force_rounding():
    """A 6-camera scene whose rank-3 SDP optimum holds a reflected block (Prop. 2: O(3) but not
    SO(3)), so rounding to SO(3) costs something and the chain rho_SDP <= rho_hat of Eq. 17 is
    strict.  eta must equal Eq. 18 evaluated on independent values: rho_SDP from the primal
    log-barrier solver and rho_hat from brute-force least squares over t, p at the rounded
    (R, s).  A swapped numerator sign gives eta < 0; a dropped "1 +" in the denominator moves eta
    by 0.2 %."""
    sc = scenes.random_scene(6, 40, noise=0.3, outlier_frac=0.2, seed=7, center_sigma=2.0)
    Q = _Q(sc)
    res = O.solve(Q, r0=4)
    rho_sdp, X = O.sdp_barrier(Q)
    rho_hat = _rounded_cost_brute_force(sc, res.R, res.s)
    assert res.certified
    assert np.all(np.linalg.det(res.R) > 0.999)
    assert abs(res.rho_hat - rho_hat) <= 1e-9 * (1 + rho_hat)
    assert abs(res.f - rho_sdp) <= 1e-7 * (1 + rho_sdp)
    eta = (rho_hat - rho_sdp) / (1.0 + abs(rho_hat) + abs(rho_sdp))
    assert eta > 1e-2                                                    # rounding is not free here
    assert abs(res.eta - eta) <= 1e-6 * eta
    # at a certified optimum lambda_min ~ 0, so App. E's bound gives the same value
    assert abs(res.eta_robust - eta) <= 1e-6 * eta


@pytest.mark.parametrize("N,seed", [(4, 2), (5, 1), (5, 7)])
def test_app_e_lower_bound_brackets_the_sdp_value(N, seed):
    """At an uncertified stationary point (the rank-3 saddle reached from [I, ..., I]) the dual
    value alone exceeds rho_SDP; App. E's bound with the sign kept, tr(Lambda_0) +
    min(0, lambda_min(Z)) tr(X), is a valid lower bound (weak duality) for the optimal X* of the
    independent barrier solver, and in these instances also with tr(X) at the computed point.
    The staircase stopped at rank 3 reports eta_robust >= the true relative gap (Eq. 18 with the
    barrier's rho_SDP): the bound can only overstate the suboptimality."""
    sc = scenes.random_scene(N, 40, noise=0.3, outlier_frac=0.2, seed=seed, center_sigma=2.0)
    Q = _Q(sc)
    rho_sdp, Xs = O.sdp_barrier(Q)
    r3 = O.rtr(Q, O.initial_point(N, 3))
    c3 = O.certify(Q, r3.Y)
    assert c3.lam_min < -1.0                                             # not certified
    assert c3.dual > rho_sdp + 1.0 and r3.f >= rho_sdp                   # the dual value alone is no bound
    lower_star = c3.dual + min(0.0, c3.lam_min) * np.trace(Xs)
    lower_here = c3.dual + min(0.0, c3.lam_min) * float(np.sum(r3.Y * r3.Y))
    assert lower_star <= rho_sdp + 1e-8 * (1 + abs(rho_sdp))
    assert lower_here <= rho_sdp
    res = O.solve(Q, r0=3, r_max=3)
    assert not res.certified and res.rank == 3
    rho_hat = _rounded_cost_brute_force(sc, res.R, res.s)
    eta_true = (rho_hat - rho_sdp) / (1.0 + abs(rho_hat) + abs(rho_sdp))
    assert eta_true > 0
    assert res.eta_robust >= eta_true
    assert res.eta_robust < 1.0


def test_iterative_certificate_branch_matches_dense_branch():
    """certify's branch for large n (ARPACK on the Z operator, deflated) against its dense eigh
    branch on the same small instance, at the certified optimum and at the rank-3 saddle."""
    sc = scenes.config1()
    Q = _Q(sc)
    opt = O.solve(Q, r0=4)
    r3 = O.rtr(Q, O.initial_point(sc.N, 3))
    for Y in (opt.Y, r3.Y):
        d = O.certify(Q, Y)
        it = O.certify(Q, Y, dense_limit=0)
        scale = d.lam_max_Q
        assert abs(it.lam_max_Q - d.lam_max_Q) <= 1e-8 * scale
        assert abs(it.lam_min - d.lam_min) <= 1e-8 * scale
        assert abs(it.lam_min_deflated - d.lam_min_deflated) <= 1e-8 * scale
        assert it.dual == d.dual and np.array_equal(it.Lambda, d.Lambda)
        Z = Q.copy()
        for i in range(sc.N):
            Z[3 * i:3 * i + 3, 3 * i:3 * i + 3] -= d.Lambda[i]
        # the returned vector is an eigenvector of lambda_min in both branches
        for c in (d, it):
            assert np.linalg.norm(Z @ c.v - c.lam_min * c.v) <= 1e-6 * scale
