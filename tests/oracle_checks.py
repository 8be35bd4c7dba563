"""Parity of a GPU solve at the point it returned (test infrastructure): the oracle's objective,
certificate, rounding and suboptimality values evaluated at the GPU's own Y, so the comparison
holds also where the optimum is not unique (an SDP optimum of rank > 3, whose optimal face holds
many X with the same value, or a saddle along flat directions)."""
import numpy as np

from oracle import xm_oracle as O


def _np(x):
    return x.detach().cpu().numpy() if hasattr(x, "detach") else np.asarray(x)


def _rel(a, b):
    return abs(a - b) / (1.0 + abs(b))


def check_at_returned_point(Qo, out, lam_tol_rel=1e-5, mu=0.0):
    """Every reported quantity against the oracle at the returned Y: f and the dual value (FP64
    on both sides: 1e-9), lambda_min raw and deflated (lam_tol_rel of lambda_max(Q)), the
    rounding (_check_rounding), Eq. 18's eta (1e-9) and App. E's eta_robust (1e-9 plus what the
    lambda_min tolerance moves its bound by), both from the reported rho_hat."""
    info = out["info"]
    r = info["rank"]
    Y = _np(out["Y"])[:, :r]
    f = O.cost(Qo, Y, mu)
    c = O.certify(Qo, Y, mu=mu)
    lam_tol = lam_tol_rel * c.lam_max_Q
    assert _rel(info["f"], f) <= 1e-9, (info["f"], f)
    assert abs(info["dual"] - c.dual) <= 1e-9 * (1 + abs(f)), (info["dual"], c.dual)
    assert abs(info["lambda_min_deflated"] - c.lam_min_deflated) <= lam_tol, \
        (info["lambda_min_deflated"], c.lam_min_deflated, lam_tol)
    assert abs(info["lambda_min"] - c.lam_min) <= lam_tol, \
        (info["lambda_min"], c.lam_min, c.lam_min_deflated, lam_tol, info["grad_norm"], c.ZY_norm)
    _check_rounding(Qo, Y, out, mu)
    rho = info["rho_hat"]
    assert abs(info["eta"] - O.suboptimality(rho, f)) <= 1e-9
    trX = float(np.sum(Y * Y))
    lower = c.dual + min(0.0, c.lam_min) * trX
    slack = lam_tol * trX / (1.0 + abs(rho) + abs(lower))
    assert abs(info["eta_robust"] - O.suboptimality(rho, lower)) <= 1e-9 + slack


def _check_rounding(Qo, Y, out, mu):
    """Rounding (Sec. 2.2) at the returned Y.  The anchored blocks G_i of the top-3 eigenvectors
    and the scales s_i = ||G_i||_F / sqrt(3) are unique when the top-3 eigenspace of Y^T Y is
    (always for rank 3); the nearest rotation to G_i / s_i is unique unless G_i is a reflection
    whose two smallest singular values tie (then every choice of the flipped axis is as near).
    So: s against the oracle's, each R_i a proper rotation exactly as near to G_i as the
    oracle's (equal distance), R_i itself where it is unique, and rho_hat as the oracle's cost
    at the GPU's own rounded point (1e-9)."""
    info = out["info"]
    R_g, s_g = _np(out["R"]), _np(out["s"])
    N = R_g.shape[0]
    assert np.allclose(np.einsum("iab,icb->iac", R_g, R_g), np.eye(3), atol=1e-10)
    assert np.all(np.linalg.det(R_g) > 0.0)
    Yhat = np.concatenate([s_g[i] * R_g[i] for i in range(N)], axis=1).T
    assert _rel(info["rho_hat"], O.cost(Qo, Yhat, mu)) <= 1e-9
    ew = np.sort(np.linalg.eigvalsh(Y.T @ Y))[::-1]
    if Y.shape[1] > 3 and ew[2] - ew[3] <= 1e-6 * ew[0]:
        return                                    # top-3 eigenspace not unique: nothing more is fixed
    R_o, s_o, _, _ = O.round_solution(Qo, Y, mu)
    assert np.abs(s_g - s_o).max() <= 1e-9 * s_o.max()
    # the anchored blocks G_i (the oracle's construction, before the SO(3) projection)
    Vt = np.linalg.eigh(Y.T @ Y)[1][:, ::-1][:, :3]
    Ub = np.swapaxes(O.blocks(Y @ Vt), 1, 2)
    u, _, vt = np.linalg.svd(Ub[0])
    G = np.einsum("ba,ibc->iac", u @ vt, Ub)
    d_g = np.linalg.norm(s_g[:, None, None] * R_g - G, axis=(1, 2))
    d_o = np.linalg.norm(s_o[:, None, None] * R_o - G, axis=(1, 2))
    assert np.abs(d_g - d_o).max() <= 1e-7 * s_o.max()
    sv = np.linalg.svd(G, compute_uv=False)
    unique = (np.linalg.det(G) > 0) | (sv[:, 1] - sv[:, 2] > 1e-6 * sv[:, 0])
    unique[0] = True
    sR_g, sR_o = s_g[:, None, None] * R_g, s_o[:, None, None] * R_o
    assert np.abs(sR_g - sR_o)[unique].max() <= 1e-7 * s_o.max()
