"""FP64 CPU oracle for XM (scaled bundle adjustment via SDP + Burer-Monteiro).

TEST INFRASTRUCTURE ONLY.  Nothing in the CUDA library, its Python binding or the
timed path of the benchmark imports or executes this module; only ``tests/``, the
smoke check and the benchmark's CPU-baseline leg do.  It shares no code with the
CUDA path: it is a plain, slow, obviously correct restatement of the paper in
numpy/scipy, in float64 throughout.

Notation (paper, Sec. 2-3 and App. A):
    N cameras, M landmarks, observations (i, k, u_ik, w_ik), n = 3N.
    U = [Rbar_1 ... Rbar_N] in R^{r x 3N} (BM factor, Prop. 4); this module works with
    Y := U^T in R^{n x r}, so Y_i := U_i^T is the 3 x r block of camera i and the
    constraint Rbar_i^T Rbar_i = alpha_i I_3 reads Y_i Y_i^T = alpha_i I_3.
    f(Y) = tr(Q U^T U) = tr(Y^T Q Y)   (Eq. 5 / Eq. 17).
    Camera 0 is the anchor (the paper's camera 1): alpha_0 = 1.

Readings of the paper taken here:
  * App. A writes Q1 with a stray "p_{i,k}^T"; the sum of w (e_i (x) u)(e_i (x) u)^T is used.
  * App. A's anchored least-squares solve carries a sign slip in two places that cancel;
    ``build_Q_literal`` follows the printed A and Q formulas, ``build_Q_schur`` the
    sign-free Schur complement, and tests assert both agree.
  * Alg. 1's line search compares tr(Q U U^T); read as tr(Q U^T U) = f.
  * Alg. 1's U_{r+1} = [U_r; alpha v^T] leaves the feasible set; the escape point is the
    retraction of [Y, 0] along the tangent vector [0, alpha v] (Thm. 2's direction).
  * App. E's bound uses max(0, lambda_min) tr(X); the valid lower bound keeps the sign,
    min(0, lambda_min) tr(X), with tr(X) taken at the computed X (not rigorous).
  * Sec. 3.2 cites Absil et al. (2008) / Boumal (2023) for RTR-tCG without constants;
    the textbook defaults are used (rho' = 0.1, shrink 1/4, expand 2, theta = 1, kappa = 0.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# ======================================================================================
# Appendix A: data matrices, the view-graph Laplacian and the reduced data matrix Q
# ======================================================================================


def _validated(N, M, cam, lmk, ukp, w):
    cam = np.asarray(cam, dtype=np.int64)
    lmk = np.asarray(lmk, dtype=np.int64)
    ukp = np.asarray(ukp, dtype=np.float64).reshape(-1, 3)
    w = np.asarray(w, dtype=np.float64).reshape(-1)
    E = cam.size
    if not (lmk.size == E and ukp.shape[0] == E and w.size == E):
        raise ValueError("observation arrays disagree in length")
    if E and (cam.min() < 0 or cam.max() >= N or lmk.min() < 0 or lmk.max() >= M):
        raise ValueError("camera or landmark index out of range")
    if not np.all(w > 0) or not np.all(np.isfinite(w)) or not np.all(np.isfinite(ukp)):
        raise ValueError("weights must be positive and keypoints finite")
    return cam, lmk, ukp, w


def data_matrices(N, M, cam, lmk, ukp, w):
    """Q1, Q2, Q3, V1, V2, V3 of App. A (Proof of Prop. 1), as scipy.sparse matrices.

    Q1 = sum w (e_i (x) u)(e_i (x) u)^T   (3N x 3N, block diagonal)
    Q2 = sum w e_i e_i^T                  (N x N)
    Q3 = sum w ebar_k ebar_k^T            (M x M)
    V1 = sum w (e_i (x) u) e_i^T          (3N x N)
    V2 = sum w (e_i (x) u) ebar_k^T       (3N x M)
    V3 = sum w e_i ebar_k^T               (N x M)
    """
    cam, lmk, ukp, w = _validated(N, M, cam, lmk, ukp, w)
    n = 3 * N
    rows3 = (3 * cam[:, None] + np.arange(3)[None, :])            # E x 3 row indices of e_i (x) u
    wu = w[:, None] * ukp                                          # E x 3
    # Q1: for each obs, the 3x3 block w u u^T at (i, i)
    r_q1 = np.repeat(rows3, 3, axis=1).ravel()
    c_q1 = np.tile(rows3, (1, 3)).ravel()
    v_q1 = (wu[:, :, None] * ukp[:, None, :]).ravel()
    Q1 = sp.csr_matrix((v_q1, (r_q1, c_q1)), shape=(n, n))
    Q2 = sp.csr_matrix((w, (cam, cam)), shape=(N, N))
    Q3 = sp.csr_matrix((w, (lmk, lmk)), shape=(M, M))
    V1 = sp.csr_matrix((wu.ravel(), (rows3.ravel(), np.repeat(cam, 3))), shape=(n, N))
    V2 = sp.csr_matrix((wu.ravel(), (rows3.ravel(), np.repeat(lmk, 3))), shape=(n, M))
    V3 = sp.csr_matrix((w, (cam, lmk)), shape=(N, M))
    return dict(Q1=Q1, Q2=Q2, Q3=Q3, V1=V1, V2=V2, V3=V3)


def laplacian_blocks(dm):
    """Q_tp = [[Q2, -V3], [-V3^T, Q3]] and V_tp = [-V1, V2] (Eq. 33-34, App. A)."""
    Qtp = sp.bmat([[dm["Q2"], -dm["V3"]], [-dm["V3"].T, dm["Q3"]]]).tocsr()
    Vtp = sp.hstack([-dm["V1"], dm["V2"]]).tocsr()
    return Qtp, Vtp


def graph_is_connected(N, M, cam, lmk) -> bool:
    """Connectivity of the camera-landmark view graph over the vertices that carry an edge."""
    cam = np.asarray(cam, np.int64); lmk = np.asarray(lmk, np.int64)
    A = sp.csr_matrix((np.ones(cam.size), (cam, N + lmk)), shape=(N + M, N + M))
    ncomp, lab = sp.csgraph.connected_components(A, directed=False)
    used = np.zeros(N + M, bool); used[:N] = True; used[N + lmk] = True
    return np.unique(lab[used]).size == 1


def build_Q_literal(N, M, cam, lmk, ukp, w):
    """Q exactly as printed in App. A: Q = A^T Q_tp A + V_tp A + A^T V_tp^T + Q1 with
    A = [0_{1 x 3N}; -(Qbar^T Qbar)^{-1} Qbar^T V_tp^T], Qbar = Q_tp without its first column.
    Dense; tiny instances only."""
    dm = data_matrices(N, M, cam, lmk, ukp, w)
    Qtp, Vtp = laplacian_blocks(dm)
    Qtp = Qtp.toarray(); Vtp = Vtp.toarray(); Q1 = dm["Q1"].toarray()
    Qbar = Qtp[:, 1:]
    Abar = -np.linalg.solve(Qbar.T @ Qbar, Qbar.T @ Vtp.T)
    A = np.vstack([np.zeros((1, 3 * N)), Abar])
    Q = A.T @ Qtp @ A + Vtp @ A + A.T @ Vtp.T + Q1
    return 0.5 * (Q + Q.T)


def build_Q_schur(N, M, cam, lmk, ukp, w):
    """Q by eliminating landmarks, then translations (anchored t_0 = 0):
        D = Q3,  P = Q1 - V2 D^-1 V2^T,  B = V1 - V2 D^-1 V3^T,  S = Q2 - V3 D^-1 V3^T,
        Q = P - Bbar Sbar^-1 Bbar^T   (bars drop camera 0's column / row).
    Same matrix as App. A's formula (the minimiser over t, p of Eq. 3 in closed form)."""
    dm = data_matrices(N, M, cam, lmk, ukp, w)
    d = np.asarray(dm["Q3"].diagonal()).copy()
    used = d > 0
    dinv = np.zeros_like(d); dinv[used] = 1.0 / d[used]
    Dinv = sp.diags(dinv)
    V2, V3 = dm["V2"], dm["V3"]
    P = (dm["Q1"] - V2 @ Dinv @ V2.T).toarray()
    B = (dm["V1"] - V2 @ Dinv @ V3.T).toarray()
    S = (dm["Q2"] - V3 @ Dinv @ V3.T).toarray()
    if N == 1:
        return 0.5 * (P + P.T)
    Sbar = S[1:, 1:]
    Bbar = B[:, 1:]
    c, low = sla.cho_factor(Sbar, lower=True)
    X = sla.cho_solve((c, low), Bbar.T)
    Q = P - Bbar @ X
    return 0.5 * (Q + Q.T)


def sba_cost(cam, lmk, ukp, w, R, s, t, p):
    """Eq. 3: sum_{(i,k)} w_ik || R_i (s_i u_ik) + t_i - p_k ||^2."""
    res = np.einsum("eab,eb->ea", R[cam], s[cam][:, None] * ukp) + t[cam] - p[lmk]
    return float(np.sum(w * np.sum(res * res, axis=1)))


def min_over_tp(N, M, cam, lmk, ukp, w, Y):
    """Brute force: min over t (t_0 = 0) and p of sum w || Y_i^T u + t_i - p_k ||^2 for a
    given Y (n x r, any r), by dense least squares.  Returns (cost, t (N x r), p (M x r)).
    Tiny instances only."""
    cam, lmk, ukp, w = _validated(N, M, cam, lmk, ukp, w)
    E = cam.size
    r = Y.shape[1]
    Yb = Y.reshape(N, 3, r)
    a = np.einsum("eab,ea->eb", Yb[cam], ukp)                      # E x r : U_i u_ik
    # unknowns: t_1..t_{N-1}, p_0..p_{M-1}
    G = np.zeros((E, N - 1 + M))
    m = cam > 0
    G[np.nonzero(m)[0], cam[m] - 1] = 1.0
    G[np.arange(E), N - 1 + lmk] = -1.0
    sw = np.sqrt(w)
    sol, *_ = np.linalg.lstsq(sw[:, None] * G, -(sw[:, None] * a), rcond=None)
    res = a + G @ sol
    cost = float(np.sum(w[:, None] * res * res))
    t = np.vstack([np.zeros((1, r)), sol[: N - 1]])
    return cost, t, sol[N - 1:]


def recover_tp(N, M, cam, lmk, ukp, w, U3):
    """Eq. 7 (t*, p* from U*): the least-squares translations and landmarks for the rounded
    3 x 3N solution, computed by the sparse normal equations of Eq. 31 with t_0 = 0."""
    cam, lmk, ukp, w = _validated(N, M, cam, lmk, ukp, w)
    Yb = np.asarray(U3).T.reshape(N, 3, 3)
    a = np.einsum("eab,ea->eb", Yb[cam], ukp)
    E = cam.size
    # a landmark without observations leaves p_k free: it is left out and reported as 0
    seen = np.bincount(lmk, minlength=M) > 0
    idx = -np.ones(M, dtype=np.int64)
    idx[seen] = np.arange(int(seen.sum()))
    Ms = int(seen.sum())
    rows = np.concatenate([np.arange(E)[cam > 0], np.arange(E)])
    cols = np.concatenate([cam[cam > 0] - 1, N - 1 + idx[lmk]])
    vals = np.concatenate([np.ones(int((cam > 0).sum())), -np.ones(E)])
    G = sp.csr_matrix((vals, (rows, cols)), shape=(E, N - 1 + Ms))
    Wd = sp.diags(w)
    Hm = (G.T @ Wd @ G).tocsc()
    rhs = -(G.T @ (w[:, None] * a))
    sol = spla.splu(Hm).solve(rhs)
    t = np.vstack([np.zeros((1, 3)), sol[: N - 1]])
    p = np.zeros((M, 3))
    p[seen] = sol[N - 1:]
    return t, p


# ======================================================================================
# Sec. 3.2 / Prop. 5: the Riemannian structure of the BM problem (Eq. 21)
# ======================================================================================

def blocks(Y):
    n, r = Y.shape
    return Y.reshape(n // 3, 3, r)


def alphas(Y):
    """alpha_i = tr(Y_i Y_i^T) / 3 (equal to the scale^2 on the feasible set)."""
    Yb = blocks(Y)
    return np.einsum("iab,iab->i", Yb, Yb) / 3.0


def _sym(A):
    return 0.5 * (A + np.swapaxes(A, -1, -2))


def _dev_except_anchor(S):
    """P_i: identity on symmetric 3x3 for the anchor, trace removal for the others
    (the span of the constraint matrices A_i of one block, App. 'Proof of LICQ')."""
    out = S.copy()
    tr = np.trace(S[1:], axis1=1, axis2=2)
    out[1:] -= (tr / 3.0)[:, None, None] * np.eye(3)
    return out


def lambdas(Y, G):
    """Closed-form dual blocks: Lambda_i = P_i(sym(G_i Y_i^T)) / alpha_i with G = Q Y.

    At a first-order critical point this is the unique y* of Eq. 24 (LICQ holds, App. C),
    giving Z(y*) = Q - blockdiag(Lambda)."""
    Yb, Gb = blocks(Y), blocks(G)
    S = _sym(np.einsum("iar,ibr->iab", Gb, Yb))
    return _dev_except_anchor(S) / alphas(Y)[:, None, None]


def apply_blockdiag(L, X):
    Xb = blocks(X)
    return np.einsum("iab,ibr->iar", L, Xb).reshape(X.shape)


def proj_tangent(Y, Xi):
    """Orthogonal projection onto T_Y M: Xi_i - P_i(sym(Xi_i Y_i^T)) Y_i / alpha_i."""
    S = lambdas(Y, Xi)
    return Xi - apply_blockdiag(S, Y)


# App. D scale regularisation: F(X) = mu * sum_{i >= 2} (X_{3i,3i} - 1)^2 in the paper's 1-based
# indexing, i.e. the third diagonal entry of every non-anchor block; here row 3i + 2 of camera
# i >= 1 (0-based), with X_{3i+2,3i+2} = ||Y_{3i+2,:}||^2.  mu = 0 is the plain problem of Eq. 17.

def scale_reg_x(Y):
    """x_i = X_{3i+2,3i+2} for every camera (the regularised diagonal entries)."""
    return np.sum(Y[2::3] * Y[2::3], axis=1)


def scale_reg_F(Y, mu):
    """F(X) = mu sum_{i >= 1} (x_i - 1)^2."""
    if mu == 0.0:
        return 0.0
    x = scale_reg_x(Y)[1:]
    return float(mu * np.sum((x - 1.0) ** 2))


def scale_reg_diag(Y, mu):
    """grad_X F as the n-vector of its diagonal: 2 mu (x_i - 1) on row 3i + 2, i >= 1."""
    d = np.zeros(Y.shape[0])
    if mu != 0.0:
        d[2::3] = 2.0 * mu * (scale_reg_x(Y) - 1.0)
        d[2] = 0.0
    return d


def qeff(Q, Y, mu=0.0):
    """(Q + grad_X F) Y: half the Euclidean gradient of f(Y) = tr(Y^T Q Y) + F(Y Y^T)."""
    G = Q @ Y
    if mu != 0.0:
        G = G + scale_reg_diag(Y, mu)[:, None] * Y
    return G


def cost(Q, Y, mu=0.0):
    return float(np.sum(Y * (Q @ Y))) + scale_reg_F(Y, mu)


def egrad(Q, Y, mu=0.0):
    return 2.0 * qeff(Q, Y, mu)


def rgrad(Q, Y, G=None, mu=0.0):
    """Riemannian gradient 2 (Q + grad F - blockdiag(Lambda)) Y = 2 Z Y (App. D's Z)."""
    G = qeff(Q, Y, mu) if G is None else G
    L = lambdas(Y, G)
    return 2.0 * (G - apply_blockdiag(L, Y))


def hess(Q, Y, Xi, L=None, mu=0.0):
    """Riemannian Hessian of f on the embedded manifold: P_Y(Euclidean Hessian - 2 Lambda Xi)
    with the Euclidean Hessian 2 Q Xi + 2 D Xi + 2 Ddot Y of f(Y) = tr(Y^T Q Y) + F(Y Y^T):
    D = grad_X F (diagonal), Ddot = 2 mu dX_{jj} = 4 mu <y_j, xi_j> on the regularised rows j."""
    if L is None:
        L = lambdas(Y, qeff(Q, Y, mu))
    E = Q @ Xi - apply_blockdiag(L, Xi)
    if mu != 0.0:
        d = scale_reg_diag(Y, mu)
        dd = np.zeros(Y.shape[0])
        dd[2::3] = 4.0 * mu * np.sum(Y[2::3] * Xi[2::3], axis=1)
        dd[2] = 0.0
        E = E + d[:, None] * Xi + dd[:, None] * Y
    return proj_tangent(Y, 2.0 * E)


def retract(Y, Xi):
    """Metric-projection retraction: per block, the closest point of {sqrt(a) * (3 x r with
    orthonormal rows)} to Y_i + Xi_i, i.e. polar factor times the mean singular value;
    the anchor keeps unit scale (Stiefel polar retraction)."""
    A = blocks(Y + Xi)
    Uu, sv, Vt = np.linalg.svd(A, full_matrices=False)           # A = Uu diag(sv) Vt
    P = np.einsum("iab,ibr->iar", Uu, Vt)
    scale = sv.mean(axis=1)
    scale[0] = 1.0
    return (scale[:, None, None] * P).reshape(Y.shape)


def inner(A, B):
    return float(np.sum(A * B))


def initial_point(N, r):
    """Alg. 1's initialisation [I_3, ..., I_3] padded with zero rows to rank r."""
    Y = np.zeros((3 * N, r))
    for i in range(N):
        Y[3 * i:3 * i + 3, :3] = np.eye(3)
    return Y


def random_point(N, r, rng):
    """A random feasible point (random orthonormal-row blocks, unit scales)."""
    A = rng.standard_normal((N, 3, r))
    Uu, sv, Vt = np.linalg.svd(A, full_matrices=False)
    return np.einsum("iab,ibr->iar", Uu, Vt).reshape(3 * N, r)


# ======================================================================================
# Riemannian trust region with truncated CG (Sec. 3.2; Absil et al. 2008, Boumal 2023)
# ======================================================================================

@dataclass
class RTRResult:
    Y: np.ndarray
    f: float
    grad_norm: float
    outer: int
    inner: int
    sweeps: int
    history: list = field(default_factory=list)


def tcg(Q, Y, grad, L, Delta, theta=1.0, kappa=0.1, max_inner=1000, mu=0.0):
    """Steihaug-Toint truncated CG on the model m(eta) = <grad, eta> + 1/2 <Hess eta, eta>,
    ||eta|| <= Delta.  Returns (eta, Heta, inner iterations, hit-boundary flag)."""
    eta = np.zeros_like(Y)
    Heta = np.zeros_like(Y)
    r = grad.copy()
    r0 = math.sqrt(inner(r, r))
    rr = r0 * r0
    delta = -r
    for j in range(max_inner):
        Hd = hess(Q, Y, delta, L, mu)
        kap = inner(delta, Hd)
        ee, ed, dd = inner(eta, eta), inner(eta, delta), inner(delta, delta)
        alpha = rr / kap if kap > 0 else 0.0
        if kap <= 0 or ee + 2 * alpha * ed + alpha * alpha * dd >= Delta * Delta:
            tau = (-ed + math.sqrt(max(ed * ed + dd * (Delta * Delta - ee), 0.0))) / dd
            return eta + tau * delta, Heta + tau * Hd, j + 1, True
        eta = eta + alpha * delta
        Heta = Heta + alpha * Hd
        r = r + alpha * Hd
        r = proj_tangent(Y, r)
        rr_new = inner(r, r)
        if math.sqrt(rr_new) <= r0 * min(r0 ** theta, kappa):
            return eta, Heta, j + 1, False
        beta = rr_new / rr
        rr = rr_new
        delta = -r + beta * delta
    return eta, Heta, max_inner, False


def rtr(Q, Y0, grad_tol_rel=1e-10, grad_tol_abs=0.0, max_outer=500, max_inner=1000,
        Delta_bar=None, rho_prime=0.1, verbose=False, mu=0.0) -> RTRResult:
    """Riemannian trust-region method (Absil et al. 2008, Alg. 10): tCG model step,
    retraction, ratio test rho, radius update, until ||rgrad|| <= tol."""
    Y = Y0.copy()
    G = qeff(Q, Y, mu)
    f = cost(Q, Y, mu)
    L = lambdas(Y, G)
    grad = 2.0 * (G - apply_blockdiag(L, Y))
    gn = math.sqrt(inner(grad, grad))
    g0 = gn
    Delta_bar = math.sqrt(inner(Y, Y)) if Delta_bar is None else Delta_bar
    Delta = Delta_bar / 8.0
    sweeps, inner_total = 1, 0
    hist = [(f, gn)]
    k = 0
    eps_reg = 1e3 * np.finfo(np.float64).eps
    # Rounding floor of the Riemannian gradient: FP64 products Q Y carry errors of order
    # eps * ||Q Y||; below ~1e4 eps * ||2 Q Y0|| a first-order point is reached for all purposes.
    floor = 1e4 * np.finfo(np.float64).eps * float(np.linalg.norm(2.0 * G))
    best = (gn, Y, f)
    for k in range(1, max_outer + 1):
        if gn <= max(grad_tol_abs, grad_tol_rel * g0, floor):
            break
        eta, Heta, nin, _ = tcg(Q, Y, grad, L, Delta, max_inner=max_inner, mu=mu)
        inner_total += nin
        sweeps += nin
        Yp = retract(Y, eta)
        Gp = qeff(Q, Yp, mu)
        sweeps += 1
        fp = cost(Q, Yp, mu)
        model_dec = -(inner(grad, eta) + 0.5 * inner(eta, Heta))
        reg = max(1.0, abs(f)) * eps_reg
        rho = (f - fp + reg) / (model_dec + reg)
        en = math.sqrt(inner(eta, eta))
        if rho < 0.25:
            Delta *= 0.25
        elif rho > 0.75 and en >= Delta * (1 - 1e-10):
            Delta = min(2.0 * Delta, Delta_bar)
        if rho > rho_prime and fp <= f + reg:
            Y, G, f = Yp, Gp, fp
            L = lambdas(Y, G)
            grad = 2.0 * (G - apply_blockdiag(L, Y))
            gn = math.sqrt(inner(grad, grad))
        hist.append((f, gn))
        if gn < best[0]:
            best = (gn, Y, f)
        if verbose:
            print(f"rtr {k:3d} f={f:.12e} |g|={gn:.3e} rho={rho:.3f} D={Delta:.3e} inner={nin}")
        if Delta < 1e-15 * Delta_bar:
            break
    # near the rounding floor accepted steps along flat directions can raise ||grad||; return the
    # most stationary iterate seen
    gn, Y, f = best
    return RTRResult(Y, f, gn, k, inner_total, sweeps, hist)


# ======================================================================================
# Thm. 1 (dual certificate), Thm. 2 (descent direction), Alg. 1 (staircase)
# ======================================================================================

@dataclass
class Certificate:
    Lambda: np.ndarray
    f: float
    dual: float           # tr(Lambda_0) = sum_i b_i y_i (+ F - <grad F, X> with App. D's term)
    lam_min: float        # lambda_min(Z)
    lam_min_deflated: float
    v: np.ndarray         # eigenvector of lambda_min(Z)
    lam_max_Q: float
    ZY_norm: float


def _deflation_basis(Y):
    Uu, sv, _ = np.linalg.svd(Y, full_matrices=False)
    keep = sv > sv.max() * 1e-8 if sv.size else sv > 0
    return Uu[:, keep]


def certify(Q, Y, dense_limit=4000, tol=1e-12, mu=0.0):
    """Z = Q - blockdiag(Lambda) with the closed-form Lambda (App. D: Z = Q + grad F(X) -
    blockdiag(Lambda)); lambda_min(Z) (raw, for the escape direction) and lambda_min of Z
    restricted to range(Y)^perp (the gap).  The dual value is tr(Lambda_0), plus
    F(X) - <grad F(X), X> with the regulariser (App. E)."""
    n = Q.shape[0]
    d = scale_reg_diag(Y, mu)
    G = qeff(Q, Y, mu)
    L = lambdas(Y, G)
    f = cost(Q, Y, mu)
    dual = float(np.trace(L[0])) + scale_reg_F(Y, mu) - float(np.sum(d * np.sum(Y * Y, axis=1)))
    ZY = G - apply_blockdiag(L, Y)
    Vd = _deflation_basis(Y)
    if n <= dense_limit:
        Z = Q.copy() + np.diag(d)
        for i in range(n // 3):
            Z[3 * i:3 * i + 3, 3 * i:3 * i + 3] -= L[i]
        Z = 0.5 * (Z + Z.T)
        ev, evec = np.linalg.eigh(Z)
        lam_min, v = float(ev[0]), evec[:, 0]
        Pp = np.eye(n) - Vd @ Vd.T
        Zd = Pp @ Z @ Pp
        # add a large multiple of the projector onto range(Y) so it never wins the minimum
        Zd = Zd + (abs(ev).max() + 1.0) * 10 * (Vd @ Vd.T)
        lam_def = float(np.linalg.eigvalsh(0.5 * (Zd + Zd.T))[0])
        lmQ = float(np.linalg.eigvalsh(Q)[-1])
    else:
        def zmul(x):
            x = x.reshape(n, -1)
            return Q @ x + d[:, None] * x - apply_blockdiag(L, x)
        Zop = spla.LinearOperator((n, n), matvec=lambda x: zmul(x[:, None]).ravel(), dtype=np.float64)
        lmQ = float(spla.eigsh(spla.aslinearoperator(Q), k=1, which="LA", tol=1e-8,
                               return_eigenvectors=False)[0])
        evs, vecs = spla.eigsh(Zop, k=1, which="SA", tol=tol, maxiter=20 * n)
        lam_min, v = float(evs[0]), vecs[:, 0]
        big = 10 * lmQ + 1.0

        def zdmul(x):
            x = x - Vd @ (Vd.T @ x)
            y = zmul(x[:, None]).ravel()
            y = y - Vd @ (Vd.T @ y)
            return y
        Zd = spla.LinearOperator((n, n), matvec=lambda x: zdmul(x) + big * (Vd @ (Vd.T @ x)),
                                 dtype=np.float64)
        ed, vd = spla.eigsh(Zd, k=1, which="SA", tol=tol, maxiter=20 * n)
        lam_def = float(ed[0])
        # lambda_min(Z) is the least Rayleigh quotient of Z; the Ritz values on range(Y) (the
        # r x r block Vd^T Z Vd) and on its complement (lam_def) are Rayleigh quotients too, so
        # the least of the three is still an upper bound of lambda_min(Z), and does not depend
        # on one Lanczos run finding the near-null cluster that range(Y) gives Z
        ZVd = zmul(Vd)
        zr = 0.5 * (Vd.T @ ZVd + (Vd.T @ ZVd).T)
        if zr.size:
            ew, ev = np.linalg.eigh(zr)
            if ew[0] < lam_min:
                lam_min, v = float(ew[0]), Vd @ ev[:, 0]
        if lam_def < lam_min:
            lam_min, v = lam_def, vd[:, 0]
    return Certificate(L, f, dual, lam_min, lam_def, v, lmQ, float(np.linalg.norm(ZY)))


def escape(Q, Y, v, f, max_halvings=30, mu=0.0):
    """Thm. 2 / Alg. 1 escape: step along the tangent direction [0, v] at [Y, 0] with
    step alpha = 1, 1/2, 1/4, ... until the retracted point strictly decreases f."""
    n, r = Y.shape
    Y0 = np.hstack([Y, np.zeros((n, 1))])
    D = np.zeros((n, r + 1)); D[:, r] = v / np.linalg.norm(v)
    alpha = 1.0
    for _ in range(max_halvings + 1):
        Yp = retract(Y0, alpha * D)
        fp = cost(Q, Yp, mu)
        if fp < f:
            return Yp, fp, alpha
        alpha *= 0.5
    return None, f, 0.0


def round_solution(Q, Y, mu=0.0):
    """Rounding (Sec. 2.2): top-3 eigenvectors of X = Y Y^T (via the r x r Gram Y^T Y),
    gauge by the anchor's orthogonal factor (Prop. 3), per-camera scale ||.||_F / sqrt(3)
    and projection onto SO(3) (det fix, Prop. 2).  Returns (R, s, Yhat (n x 3), rho_hat)."""
    n, r = Y.shape
    N = n // 3
    ev, V = np.linalg.eigh(Y.T @ Y)
    V3 = V[:, ::-1][:, :3]
    Yh = Y @ V3                                                  # n x 3, X ~ Yh Yh^T
    Ub = np.swapaxes(blocks(Yh), 1, 2)                           # Ubar_i = Yh_i^T (3 x 3)
    Uu, _, Vt = np.linalg.svd(Ub[0])
    O0 = Uu @ Vt                                                 # polar factor of Ubar_0 (in O(3))
    G = np.einsum("ba,ibc->iac", O0, Ub)                         # O0^T Ubar_i
    s = np.linalg.norm(G, axis=(1, 2)) / math.sqrt(3.0)
    Uu, _, Vt = np.linalg.svd(G)
    d = np.sign(np.linalg.det(np.einsum("iab,ibc->iac", Uu, Vt)))
    Dm = np.tile(np.eye(3), (N, 1, 1)); Dm[:, 2, 2] = d
    R = np.einsum("iab,ibc,icd->iad", Uu, Dm, Vt)
    R[0] = np.eye(3); s[0] = 1.0
    Uhat = np.concatenate([s[i] * R[i] for i in range(N)], axis=1)   # 3 x 3N
    Yhat = Uhat.T
    return R, s, Yhat, cost(Q, Yhat, mu)


@dataclass
class SolveResult:
    Y: np.ndarray
    rank: int
    f: float
    grad_norm: float
    cert: Certificate
    certified: bool
    R: np.ndarray
    s: np.ndarray
    rho_hat: float
    eta: float
    eta_robust: float
    sweeps: int
    ranks_visited: list


def suboptimality(rho_hat, rho_sdp):
    """Eq. 18: eta = (rho_hat - rho_sdp) / (1 + |rho_hat| + |rho_sdp|)."""
    return (rho_hat - rho_sdp) / (1.0 + abs(rho_hat) + abs(rho_sdp))


def solve(Q, r0=4, r_max=None, cert_tau_rel=1e-6, Y0=None, grad_tol_rel=1e-10,
          max_outer=500, verbose=False, mu=0.0) -> SolveResult:
    """Alg. 1 (Riemannian staircase): RTR at rank r, certificate, escape to rank r+1.
    mu > 0 solves App. D's scale-regularised problem."""
    n = Q.shape[0]
    N = n // 3
    r_max = n if r_max is None else r_max
    Y = initial_point(N, r0) if Y0 is None else Y0.copy()
    sweeps = 0
    visited = []
    while True:
        r = Y.shape[1]
        visited.append(r)
        res = rtr(Q, Y, grad_tol_rel=grad_tol_rel, max_outer=max_outer, verbose=verbose, mu=mu)
        sweeps += res.sweeps
        Y = res.Y
        cert = certify(Q, Y, mu=mu)
        tau = cert_tau_rel * max(cert.lam_max_Q, 1e-300)
        ok = cert.lam_min >= -tau
        if ok or r >= r_max:
            break
        Yn, fn, alpha = escape(Q, Y, cert.v, res.f, mu=mu)
        if Yn is None:
            break
        Y = Yn
    R, s, Yhat, rho_hat = round_solution(Q, Y, mu)
    trX = float(np.sum(Y * Y))
    lower = cert.dual + min(0.0, cert.lam_min) * trX
    return SolveResult(Y, Y.shape[1], res.f, res.grad_norm, cert, bool(ok), R, s, rho_hat,
                       suboptimality(rho_hat, res.f), suboptimality(rho_hat, lower), sweeps,
                       visited)


def observation_residuals(cam, lmk, ukp, w, R, s, t, p):
    """Per-measurement terms of Eq. 3: w_e || R_i (s_i u_e) + t_i - p_k ||^2."""
    res = np.einsum("eab,eb->ea", R[cam], s[cam][:, None] * ukp) + t[cam] - p[lmk]
    return w * np.sum(res * res, axis=1)


def xm2_keep(res2, drop_frac=0.1):
    """XM^2's greedy outlier rule: drop the fraction drop_frac of measurements with the largest
    residual terms (ties broken by index), keep the rest; returns a boolean mask."""
    E = res2.size
    k = int(math.floor(drop_frac * E))
    keep = np.ones(E, dtype=bool)
    if k > 0:
        order = np.lexsort((np.arange(E), -res2))     # largest first, then lower index
        keep[order[:k]] = False
    return keep


@dataclass
class XM2Result:
    first: "SolveResult"
    second: "SolveResult"       # the solve on the kept measurements of the anchor's component
    keep: np.ndarray            # bool[E]: measurement used by the second solve
    cams: np.ndarray            # bool[N]: camera in the anchor's component of the kept view graph
    R: np.ndarray               # N x 3 x 3 (zero for excluded cameras)
    s: np.ndarray               # N (zero for excluded cameras)
    t: np.ndarray               # N x 3 (zero for excluded cameras)
    p: np.ndarray               # M x 3 (zero for landmarks outside the component)


def solve_xm2(N, M, cam, lmk, ukp, w, drop_frac=0.1, mu=0.0, **kw) -> XM2Result:
    """XM^2 (running twice, Sec. 5): solve, recover t and p (Eq. 7), drop the drop_frac
    measurements with the largest residual terms, solve again on the rest.  Dropping can split
    the view graph (a camera whose every measurement was dropped: without App. D's regulariser
    even the anchor, whose unit-scale terms can be the largest); the second solve then runs on
    the connected component with the most cameras (ties: the one holding the lowest camera
    index), anchored at its lowest-index camera (R = I, s = 1, t = 0 there), and reports the
    cameras and landmarks outside it with zero rotation, scale, translation and position."""
    cam, lmk, ukp, w = _validated(N, M, cam, lmk, ukp, w)
    Q = build_Q_schur(N, M, cam, lmk, ukp, w)
    first = solve(Q, mu=mu, **kw)
    U3 = np.concatenate([first.s[i] * first.R[i] for i in range(N)], axis=1)
    t, p = recover_tp(N, M, cam, lmk, ukp, w, U3)
    keep = xm2_keep(observation_residuals(cam, lmk, ukp, w, first.R, first.s, t, p), drop_frac)
    # components of the camera-landmark graph of the kept measurements (vertices: N cameras, then
    # M landmarks)
    A = sp.csr_matrix((np.ones(int(keep.sum())), (cam[keep], N + lmk[keep])), shape=(N + M, N + M))
    _, lab = sp.csgraph.connected_components(A, directed=False)
    size = np.bincount(lab[:N])
    best = lab[:N][np.argmax(size[lab[:N]] == size.max())]   # first camera of a largest component
    cams = lab[:N] == best
    use = keep & cams[cam]
    cidx = np.nonzero(cams)[0]
    cmap = -np.ones(N, np.int64); cmap[cidx] = np.arange(cidx.size)
    lidx = np.unique(lmk[use])
    lmap = -np.ones(M, np.int64); lmap[lidx] = np.arange(lidx.size)
    N2, M2 = int(cidx.size), int(lidx.size)
    c2, l2, u2, w2 = cmap[cam[use]], lmap[lmk[use]], ukp[use], w[use]
    second = solve(build_Q_schur(N2, M2, c2, l2, u2, w2), mu=mu, **kw)
    U3 = np.concatenate([second.s[i] * second.R[i] for i in range(N2)], axis=1)
    t2, p2 = recover_tp(N2, M2, c2, l2, u2, w2, U3)
    R = np.zeros((N, 3, 3)); s = np.zeros(N); tt = np.zeros((N, 3)); pp = np.zeros((M, 3))
    R[cidx], s[cidx], tt[cidx], pp[lidx] = second.R, second.s, t2, p2
    return XM2Result(first, second, use, cams, R, s, tt, pp)


# ======================================================================================
# Independent checks: a primal log-barrier SDP solver (Prop. 3, Eq. 13) and Umeyama (N=2)
# ======================================================================================

def sdp_barrier(Q, mu_final_rel=1e-13, verbose=False):
    """Solve Eq. 13 (min tr(QX), X >= 0, X_00 = I_3, X_ii = alpha_i I_3) by a primal
    log-barrier path-following Newton method in the affine coordinates of the feasible set.
    Independent of the BM machinery; tiny N only.  Returns (rho_sdp, X)."""
    n = Q.shape[0]
    N = n // 3
    Fs = []
    for i in range(1, N):                                        # free scales alpha_i
        F = np.zeros((n, n)); F[3 * i:3 * i + 3, 3 * i:3 * i + 3] = np.eye(3); Fs.append(F)
    for a in range(N):                                           # free off-diagonal blocks
        for b in range(a + 1, N):
            for p_ in range(3):
                for q_ in range(3):
                    F = np.zeros((n, n))
                    F[3 * a + p_, 3 * b + q_] = 1.0
                    F[3 * b + q_, 3 * a + p_] = 1.0
                    Fs.append(F)
    F = np.array(Fs)
    c = np.einsum("ab,jab->j", Q, F)
    x = np.zeros(F.shape[0])
    X0 = np.eye(n)
    scale = max(np.abs(Q).max(), 1e-300)
    mu = scale
    while True:
        for _ in range(200):
            X = X0 + np.einsum("j,jab->ab", x, F)
            W = np.linalg.inv(X)
            g = c - mu * np.einsum("ab,jba->j", W, F)
            A = np.einsum("ab,jbc->jac", W, F)
            H = mu * np.einsum("jab,kba->jk", A, A)
            dx = -np.linalg.solve(H, g)
            lam2 = -g @ dx
            phi = c @ x - mu * np.linalg.slogdet(X)[1]
            t = 1.0
            while True:
                Xt = X0 + np.einsum("j,jab->ab", x + t * dx, F)
                try:
                    np.linalg.cholesky(Xt)
                    phit = c @ (x + t * dx) - mu * np.linalg.slogdet(Xt)[1]
                    if phit <= phi - 0.25 * t * lam2 or t < 1e-12:
                        break
                except np.linalg.LinAlgError:
                    pass
                t *= 0.5
            x = x + t * dx
            if lam2 < 1e-20 * max(1.0, abs(phi)):
                break
        if verbose:
            print("mu", mu, "obj", c @ x + np.trace(Q))
        if mu < mu_final_rel * scale:
            break
        mu *= 0.1
    X = X0 + np.einsum("j,jab->ab", x, F)
    return float(np.sum(Q * X)), X


def umeyama_weighted(x, y, omega):
    """Closed-form weighted scaled registration (Umeyama 1991): argmin over s > 0,
    R in SO(3), t of sum omega_k || s R x_k + t - y_k ||^2.  Returns (s, R, t, cost)."""
    wsum = omega.sum()
    mx = (omega[:, None] * x).sum(0) / wsum
    my = (omega[:, None] * y).sum(0) / wsum
    xc, yc = x - mx, y - my
    Sxy = (omega[:, None, None] * yc[:, :, None] * xc[:, None, :]).sum(0) / wsum
    sx2 = (omega * (xc * xc).sum(1)).sum() / wsum
    Uu, D, Vt = np.linalg.svd(Sxy)
    Sm = np.diag([1.0, 1.0, np.sign(np.linalg.det(Uu) * np.linalg.det(Vt))])
    R = Uu @ Sm @ Vt
    s = float(np.trace(np.diag(D) @ Sm) / sx2)
    t = my - s * R @ mx
    res = s * x @ R.T + t - y
    return s, R, t, float((omega * (res * res).sum(1)).sum())


# ======================================================================================
# Adjoint of the certified optimum (implicit differentiation of the stationarity condition)
# ======================================================================================

def anchored_blocks_grad(Y, dL_dG):
    """Euclidean gradient in Y of L(G) with G_i = Y_0 Y_i^T (i >= 1): the anchored scaled
    rotations s_i R_i of a tight (rank-3) optimum are exactly the blocks X_0i of X = Y Y^T."""
    Yb = blocks(Y)
    dY = np.zeros_like(Yb)
    for i in range(1, Yb.shape[0]):
        dY[i] = dL_dG[i].T @ Yb[0]
        dY[0] += dL_dG[i] @ Yb[i]
    return dY.reshape(Y.shape)


def gauge_basis(Y):
    """Orthonormal basis (columns, vectorised n*r) of the gauge directions {Y Omega : Omega skew}:
    f(Y O) = f(Y) for every orthogonal O, so the Riemannian Hessian vanishes on them at a
    critical point and the loss of G_i = Y_0 Y_i^T is constant along them."""
    n, r = Y.shape
    cols = []
    for a in range(r):
        for b in range(a + 1, r):
            Om = np.zeros((r, r)); Om[a, b] = 1.0; Om[b, a] = -1.0
            cols.append((Y @ Om).ravel())
    if not cols:
        return np.zeros((n * r, 0))
    A = np.array(cols).T
    U, sv, _ = np.linalg.svd(A, full_matrices=False)
    return U[:, sv > 1e-10 * max(sv.max(), 1e-300)]


def conjugate_gradient(apply, b, tol=1e-14, maxit=10000):
    """Plain CG for a symmetric positive semi-definite operator and a consistent right side."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = inner(r, r)
    r0 = math.sqrt(rr)
    for _ in range(maxit):
        if math.sqrt(rr) <= tol * r0:
            break
        Ap = apply(p)
        pAp = inner(p, Ap)
        if pAp <= 0:
            break
        a = rr / pAp
        x = x + a * p
        r = r - a * Ap
        rr_new = inner(r, r)
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x


def optimal_residuals(N, M, cam, lmk, ukp, w, U):
    """Residuals e_e = U_i^T u_e + t_i - p_k at the least-squares t (t_0 = 0) and p for every
    column of U (n x c), by the sparse normal equations (the elimination of App. A)."""
    cam, lmk, ukp, w = _validated(N, M, cam, lmk, ukp, w)
    E = cam.size
    a = np.einsum("eab,ea->eb", blocks(U)[cam], ukp)              # E x c
    rows = np.concatenate([np.arange(E)[cam > 0], np.arange(E)])
    cols = np.concatenate([cam[cam > 0] - 1, N - 1 + lmk])
    vals = np.concatenate([np.ones(int((cam > 0).sum())), -np.ones(E)])
    Gm = sp.csr_matrix((vals, (rows, cols)), shape=(E, N - 1 + M))
    Hm = (Gm.T @ sp.diags(w) @ Gm).tocsc()
    sol = spla.splu(Hm).solve(-(Gm.T @ (w[:, None] * a)))
    return a + Gm @ sol


def adjoint(N, M, cam, lmk, ukp, w, Y, dL_dG, Q=None, tol=1e-14, mu=0.0):
    """Gradient of L(G(theta)) w.r.t. the lifted keypoints u (E x 3) and weights w (E) at a
    certified optimum Y of rank 3 (G_i = s_i R_i).  Implicit differentiation: the Riemannian
    gradient 2 P_Y(Q Y) vanishes, so Hess[Ydot] = -P_Y(2 Qdot Y); with Hess[lam] = P_Y(dL/dY),
    dL/dQ = -(lam Y^T + Y lam^T).  The bilinear form a^T Q b equals sum_e w_e e_a e_b at the
    optimal residuals (Prop. 1), whose derivatives follow from the envelope theorem (App. D's
    regulariser F(X) does not depend on the observations and enters only the Hessian):
        d(a^T Q b)/du_e = w_e (e_a b_i + e_b a_i),   d(a^T Q b)/dw_e = e_a e_b."""
    cam, lmk, ukp, w = _validated(N, M, cam, lmk, ukp, w)
    Q = build_Q_schur(N, M, cam, lmk, ukp, w) if Q is None else Q
    L = lambdas(Y, qeff(Q, Y, mu))
    # CG on the Hessian restricted to the complement of the gauge directions (its null space at a
    # critical point; dL/dY is orthogonal to them, and a gauge part of lambda cancels in dL/dQ)
    Ng = gauge_basis(Y)
    shp = Y.shape

    def deflate(v):
        x = v.ravel()
        return (x - Ng @ (Ng.T @ x)).reshape(shp)

    gL = deflate(proj_tangent(Y, anchored_blocks_grad(Y, dL_dG)))
    lam = conjugate_gradient(lambda v: deflate(hess(Q, Y, deflate(v), L, mu)), gL, tol=tol)
    r = Y.shape[1]
    e = optimal_residuals(N, M, cam, lmk, ukp, w, np.hstack([Y, lam]))
    eY, eL = e[:, :r], e[:, r:]
    Yb, Lb = blocks(Y)[cam], blocks(lam)[cam]                     # E x 3 x r
    d_u = -2.0 * w[:, None] * (np.einsum("ear,er->ea", Yb, eL) + np.einsum("ear,er->ea", Lb, eY))
    d_w = -2.0 * np.sum(eL * eY, axis=1)
    return d_u, d_w, lam
