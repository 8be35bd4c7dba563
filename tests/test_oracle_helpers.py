"""Pins for the oracle's helper steps that the solve pins cover only indirectly: each is checked
against a route that does not reuse its own formula (a library routine, the diagonal of the full
product, central finite differences, a dense solve, the closed form of Steihaug's first step, exact
recovery from noise-free data).  CPU only."""
import math

import numpy as np
import pytest
import scipy.linalg

import scenes
from oracle import xm_oracle as O


def _small_problem(seed=0, N=6, r=4):
    sc = scenes.circle_scene(N, 60, 3, 0.02, seed=seed)
    Q = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    Y = O.random_point(sc.N, r, np.random.default_rng(seed + 100))
    return Q, Y


def _rotations(N, rng):
    R = []
    for _ in range(N):
        A = rng.standard_normal((3, 3))
        U, _, Vt = np.linalg.svd(A)
        Ri = U @ Vt
        if np.linalg.det(Ri) < 0:
            Ri = U @ np.diag([1.0, 1.0, -1.0]) @ Vt
        R.append(Ri)
    return np.array(R)


def test_apply_blockdiag_is_block_diagonal_product():
    rng = np.random.default_rng(1)
    N, r = 5, 4
    L = rng.standard_normal((N, 3, 3))
    X = rng.standard_normal((3 * N, r))
    ref = scipy.linalg.block_diag(*L) @ X
    assert np.allclose(O.apply_blockdiag(L, X), ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_scale_reg_x_is_the_diagonal_of_YYt():
    rng = np.random.default_rng(2)
    Y = rng.standard_normal((3 * 7, 5))
    X = Y @ Y.T
    assert np.allclose(O.scale_reg_x(Y), np.diag(X)[2::3], rtol=1e-14, atol=0)


@pytest.mark.parametrize("mu", [0.0, 3.0])
def test_egrad_matches_central_differences(mu):
    Q, Y = _small_problem(seed=3)
    D = np.random.default_rng(4).standard_normal(Y.shape)
    t = 1e-6
    fd = (O.cost(Q, Y + t * D, mu) - O.cost(Q, Y - t * D, mu)) / (2 * t)
    an = O.inner(O.egrad(Q, Y, mu), D)
    assert abs(fd - an) <= 1e-6 * (abs(an) + 1.0)


def test_scale_reg_diag_is_the_gradient_of_F():
    """d/dY F(Y Y^T) = 2 diag(d) Y with d the diagonal of grad_X F (the anchor row excluded)."""
    rng = np.random.default_rng(5)
    Y = rng.standard_normal((3 * 6, 4))
    D = rng.standard_normal(Y.shape)
    mu, t = 2.5, 1e-6
    fd = (O.scale_reg_F(Y + t * D, mu) - O.scale_reg_F(Y - t * D, mu)) / (2 * t)
    an = O.inner(2.0 * O.scale_reg_diag(Y, mu)[:, None] * Y, D)
    assert abs(fd - an) <= 1e-6 * (abs(an) + 1.0)
    assert O.scale_reg_diag(Y, mu)[2] == 0.0 and O.scale_reg_F(Y, 0.0) == 0.0


def test_anchored_blocks_grad_matches_central_differences():
    rng = np.random.default_rng(6)
    N, r = 5, 4
    Y = rng.standard_normal((3 * N, r))
    Dl = rng.standard_normal((N, 3, 3))

    def loss(Yv):
        Yb = O.blocks(Yv)
        return sum(float(np.sum(Dl[i] * (Yb[0] @ Yb[i].T))) for i in range(1, N))

    E = rng.standard_normal(Y.shape)
    t = 1e-6
    fd = (loss(Y + t * E) - loss(Y - t * E)) / (2 * t)
    an = O.inner(O.anchored_blocks_grad(Y, Dl), E)
    assert abs(fd - an) <= 1e-7 * (abs(an) + 1.0)


def test_conjugate_gradient_against_dense_solve():
    rng = np.random.default_rng(7)
    B = rng.standard_normal((30, 30))
    A = B @ B.T + 0.5 * np.eye(30)
    b = rng.standard_normal(30)
    x = O.conjugate_gradient(lambda v: A @ v, b, tol=1e-14)
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    # a consistent singular system: the residual vanishes
    C = B[:, :12] @ B[:, :12].T
    c = C @ rng.standard_normal(30)
    y = O.conjugate_gradient(lambda v: C @ v, c, tol=1e-13)
    assert np.linalg.norm(C @ y - c) <= 1e-9 * np.linalg.norm(c)


def test_tcg_first_step_at_a_tiny_radius_is_the_scaled_negative_gradient():
    """Steihaug-Toint's first direction is -grad; a radius below the first CG step makes the
    step the boundary point -Delta grad / ||grad|| after one iteration."""
    Q, Y = _small_problem(seed=8)
    G = O.qeff(Q, Y)
    L = O.lambdas(Y, G)
    grad = O.rgrad(Q, Y, G)
    Delta = 1e-9 * math.sqrt(O.inner(Y, Y))
    eta, _, its, boundary = O.tcg(Q, Y, grad, L, Delta)
    ref = -Delta * grad / math.sqrt(O.inner(grad, grad))
    assert boundary and its == 1
    assert np.abs(eta - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("seed", [9, 10])
def test_tcg_step_is_tangent_bounded_and_beats_the_cauchy_step(seed):
    Q, Y = _small_problem(seed=seed)
    G = O.qeff(Q, Y)
    L = O.lambdas(Y, G)
    grad = O.rgrad(Q, Y, G)
    Delta = 0.3 * math.sqrt(O.inner(Y, Y))

    def model(e):   # with a fresh Hessian product, not the tCG's accumulated one
        return O.inner(grad, e) + 0.5 * O.inner(e, O.hess(Q, Y, e, L))

    eta, _, its, _ = O.tcg(Q, Y, grad, L, Delta)
    eta1, _, _, _ = O.tcg(Q, Y, grad, L, Delta, max_inner=1)
    assert np.abs(O.proj_tangent(Y, eta) - eta).max() <= 1e-10 * np.abs(eta).max()
    assert math.sqrt(O.inner(eta, eta)) <= Delta * (1 + 1e-12)
    assert model(eta) <= model(eta1) + 1e-12 * abs(model(eta1))
    assert model(eta1) < 0.0


def test_round_solution_recovers_rotations_and_scales_exactly():
    """Noise-free data: Y = [s_i R_i]^T (anchor R_0 = I, s_0 = 1) padded to rank 5 and mixed by a
    random orthogonal gauge; rounding returns every R_i and s_i."""
    rng = np.random.default_rng(11)
    N = 7
    R = _rotations(N, rng)
    R[0] = np.eye(3)
    s = rng.uniform(0.5, 2.0, N)
    s[0] = 1.0
    Yt = np.concatenate([s[i] * R[i] for i in range(N)], axis=1).T          # 3N x 3
    Og, _ = np.linalg.qr(rng.standard_normal((5, 5)))
    Y = np.concatenate([Yt, np.zeros((3 * N, 2))], axis=1) @ Og
    Rh, sh, Yhat, rho = O.round_solution(np.zeros((3 * N, 3 * N)), Y)
    assert np.abs(Rh - R).max() <= 1e-10
    assert np.abs(sh - s).max() <= 1e-10
    assert np.abs(Yhat - Yt).max() <= 1e-10 and rho == 0.0


def test_deflation_basis_is_an_orthonormal_basis_of_range_Y():
    rng = np.random.default_rng(12)
    Y = np.concatenate([rng.standard_normal((24, 3)), np.zeros((24, 2))], axis=1) @ \
        np.linalg.qr(rng.standard_normal((5, 5)))[0]
    U = O._deflation_basis(Y)
    assert U.shape == (24, 3)
    assert np.abs(U.T @ U - np.eye(3)).max() <= 1e-12
    assert np.abs(U @ (U.T @ Y) - Y).max() <= 1e-12 * np.abs(Y).max()


def test_retraction_returns_the_closest_feasible_block():
    """retract(Y, Xi) is, per non-anchor block, the nearest c U (c > 0, U U^T = I) to
    Y_i + Xi_i: no feasible point obtained by perturbing its scale and rotating its rows or its
    row space is closer."""
    rng = np.random.default_rng(13)
    N, r = 4, 5
    Y = O.random_point(N, r, rng)
    Xi = 0.4 * rng.standard_normal(Y.shape)
    A = O.blocks(Y + Xi)
    P = O.blocks(O.retract(Y, Xi))
    for i in range(1, N):
        c = math.sqrt(np.trace(P[i] @ P[i].T) / 3.0)
        U = P[i] / c
        assert np.abs(U @ U.T - np.eye(3)).max() <= 1e-12
        best = np.linalg.norm(A[i] - P[i])
        for _ in range(200):
            W = 1e-3 * rng.standard_normal((3, 3)); W = W - W.T            # row rotation
            V = 1e-3 * rng.standard_normal((r, r)); V = V - V.T            # row-space rotation
            Up = scipy.linalg.expm(W) @ U @ scipy.linalg.expm(V)
            cp = c * math.exp(1e-3 * rng.standard_normal())
            assert np.linalg.norm(A[i] - cp * Up) >= best - 1e-12
