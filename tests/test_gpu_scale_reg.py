"""Parity of the CUDA path with the oracle on App. D's scale-regularised problem: the solve
(objective, dual value of App. E, certificate, rounded rotations and scales) in FP64 and in the
FP32-bulk mode, and the adjoint.  Tolerances as in the unregularised solve tests: relative
objective 1e-6, rotations 1e-5, scales 1e-5 relative, and the adjoint at the same Y 1e-6."""
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


def _rel(a, b):
    return abs(a - b) / (1.0 + abs(b))


CASES = {
    "circle-mu2": (lambda: scenes.circle_scene(16, 200, 4, 0.05, seed=61, w_range=(0.5, 1.5)), 2.0),
    "traj50-mu10": (lambda: scenes.sub_scene(scenes.config4(), 50), 10.0),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", [0, 1])
def test_regularised_solve_matches_oracle(C, case, prec):
    from paper_2502_04640_b300 import xm
    mk, mu = CASES[case]
    sc = mk()
    Qo = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    ref = O.solve(Qo, r0=4, mu=mu, grad_tol_rel=1e-12)
    assert ref.certified
    t = xm.scene_tensors(sc)
    q = xm.xm_build_Q(C, sc.N, sc.M, *t)
    out = xm.xm_solve(q, xm.xm_default_opts(prec=prec, scale_reg=mu), allow_notcert=False)
    info = out["info"]
    assert info["certified"] == 1
    assert _rel(info["f"], ref.f) <= 1e-6
    assert _rel(info["rho_hat"], ref.rho_hat) <= 1e-6
    assert abs(info["dual"] - ref.cert.dual) <= 1e-6 * (1 + abs(ref.f))
    assert np.abs(out["R"].cpu().numpy() - ref.R).max() <= 1e-5
    assert np.abs(out["s"].cpu().numpy() - ref.s).max() <= 1e-5 * ref.s.max()
    # the regulariser matters here: the unregularised optimum is elsewhere
    free = O.solve(Qo, r0=4)
    assert np.abs(free.s - ref.s).max() > 1e-3
    q.free()


@pytest.mark.parametrize("prec", [0, 1])
def test_regularised_adjoint_matches_oracle(C, prec):
    from paper_2502_04640_b300 import xm
    mk, mu = CASES["circle-mu2"]
    sc = mk()
    t = xm.scene_tensors(sc)
    q = xm.xm_build_Q(C, sc.N, sc.M, *t)
    out = xm.xm_solve(q, xm.xm_default_opts(prec=0, scale_reg=mu, grad_tol_rel=1e-12),
                      allow_notcert=False)
    r = out["info"]["rank"]
    D = np.random.default_rng(62).standard_normal((sc.N, 3, 3))
    d_u, d_w, _, info, st = xm.xm_backward(q, out["Y"], r, sc.M, *t, torch.as_tensor(D, device="cuda:0"),
                                           xm.xm_default_opts(prec=prec, scale_reg=mu, grad_tol_rel=1e-12))
    assert st == 0
    Y = out["Y"].cpu().numpy()[:, :r]
    ref_u, ref_w, _ = O.adjoint(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w, Y, D, mu=mu)
    scale = np.abs(ref_u).max()
    assert np.abs(d_u.cpu().numpy() - ref_u).max() <= 1e-6 * scale
    assert np.abs(d_w.cpu().numpy() - ref_w).max() <= 1e-6 * np.abs(ref_w).max()
    # the unregularised Hessian gives a different adjoint at this point
    u0, _, _ = O.adjoint(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w, Y, D)
    assert np.abs(u0 - ref_u).max() > 1e-4 * scale
    q.free()


def test_negative_scale_reg_is_rejected(C):
    from paper_2502_04640_b300 import xm
    sc = scenes.circle_scene(6, 40, 3, 0.02, seed=63)
    q = xm.xm_build_Q(C, sc.N, sc.M, *xm.scene_tensors(sc))
    with pytest.raises(xm.XmError, match="XM_EINVAL"):
        xm.xm_solve(q, xm.xm_default_opts(scale_reg=-1.0))
    q.free()
