"""End-to-end parity of the CUDA solver (Alg. 1 + RTR-tCG + certificate + rounding) with the
FP64 oracle, in every precision mode.  Compared quantities are gauge invariant: the objective,
the certificate decision and gap, and the rounded rotations / scales in the anchored gauge.
Tolerances: relative objective 1e-6 (1 + |f| denominator) for the FP64 path and the mixed
modes (both end with an FP64 polish and an FP64 certificate)."""
import numpy as np
import pytest

import scenes
from oracle import xm_oracle as O
from tests.gpu_util import ctx, torch
from tests.oracle_checks import check_at_returned_point

pytestmark = pytest.mark.gpu

PRECS = {"fp64": 0, "fp32": 1, "bf16": 2}


@pytest.fixture(scope="module")
def C():
    c = ctx()
    yield c
    c.close()


def _solve(C, sc, prec, **kw):
    from paper_2502_04640_b300 import xm
    q = xm.xm_build_Q(C, sc.N, sc.M, *xm.scene_tensors(sc))
    opts = xm.xm_default_opts(prec=prec, **kw)
    out = xm.xm_solve(q, opts)
    out["R"] = out["R"].cpu().numpy(); out["s"] = out["s"].cpu().numpy(); out["Y"] = out["Y"].cpu().numpy()
    out["G"] = out["G"].cpu().numpy()
    # the library's G_i is s_i R_i of the same rounding
    assert np.abs(out["G"] - out["s"][:, None, None] * out["R"]).max() <= 1e-14 * max(1.0, out["s"].max())
    return q, out


def _rel(a, b):
    return abs(a - b) / (1.0 + abs(b))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("jitter", [0.0, 0.1])
def test_config1_matches_oracle(C, prec, jitter):
    sc = scenes.config1()
    Qo = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    ref = O.solve(Qo, r0=4)
    q, out = _solve(C, sc, PRECS[prec], init_jitter=jitter)
    info = out["info"]
    assert out["status"] == 0 and info["certified"] == 1 and ref.certified
    assert _rel(info["f"], ref.f) <= 1e-6
    assert _rel(info["rho_hat"], ref.rho_hat) <= 1e-6
    assert abs(info["dual"] - ref.cert.dual) <= 1e-6 * (1 + abs(ref.f))
    assert abs(info["lambda_min_deflated"] - ref.cert.lam_min_deflated) <= 1e-4 * ref.cert.lam_max_Q
    # raw lambda_min(Z) (range(Y) is Z-invariant at a stationary point, so it is the smaller of
    # the deflated minimum and Z's zero block on range(Y)), Eq. 18 and App. E's bound
    assert abs(info["lambda_min"] - ref.cert.lam_min) <= 1e-5 * ref.cert.lam_max_Q
    assert abs(info["eta"] - ref.eta) <= 2e-6
    assert abs(info["eta_robust"] - ref.eta_robust) <= 2e-6
    assert np.abs(out["R"] - ref.R).max() <= 1e-5
    assert np.abs(out["s"] - ref.s).max() <= 1e-5 * ref.s.max()
    if jitter == 0.0:
        assert info["n_escapes"] >= 1     # Alg. 1's exact start needs the escape of Thm. 2
    check_at_returned_point(Qo, out)
    q.free()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_start_above_rank_4_reaches_the_same_optimum(C, prec):
    """r0 = 5 runs every RTR phase in the 8-column layout (the R = 8 kernels); X = Y Y^T of a
    certified optimum is unique, so the certified result is the oracle's rank-4 one."""
    sc = scenes.config1()
    ref = O.solve(O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w), r0=4)
    q, out = _solve(C, sc, PRECS[prec], r0=5)
    info = out["info"]
    assert out["status"] == 0 and info["certified"] == 1 and info["rank"] >= 5
    assert _rel(info["f"], ref.f) <= 1e-6
    assert np.abs(out["R"] - ref.R).max() <= 1e-5
    assert np.abs(out["s"] - ref.s).max() <= 1e-5 * ref.s.max()
    q.free()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noise_free_recovery(C, prec):
    sc = scenes.circle_scene(40, 600, 4, 0.0, seed=11)
    q, out = _solve(C, sc, PRECS[prec])
    R, s, _, _ = sc.anchored_gt()
    info = out["info"]
    assert info["certified"] == 1
    assert abs(info["f"]) <= 1e-8 * np.sum(sc.w * np.sum(sc.ukp ** 2, 1))
    assert np.abs(out["R"] - R).max() <= 1e-6 and np.abs(out["s"] - s).max() <= 1e-6
    q.free()


def test_two_views_umeyama(C):
    sc = scenes.circle_scene(2, 60, 2, 0.05, seed=17, w_range=(0.5, 1.5))
    q, out = _solve(C, sc, 0)
    x = np.zeros((sc.M, 3)); y = np.zeros((sc.M, 3)); w1 = np.zeros(sc.M); w2 = np.zeros(sc.M)
    for e in range(sc.E):
        if sc.cam[e] == 0:
            y[sc.lmk[e]] = sc.ukp[e]; w1[sc.lmk[e]] = sc.w[e]
        else:
            x[sc.lmk[e]] = sc.ukp[e]; w2[sc.lmk[e]] = sc.w[e]
    s, R, t, c = O.umeyama_weighted(x, y, w1 * w2 / (w1 + w2))
    assert out["info"]["certified"] == 1
    assert _rel(out["info"]["rho_hat"], c) <= 1e-8
    assert np.abs(out["R"][1] - R).max() <= 1e-6 and abs(out["s"][1] - s) <= 1e-6
    q.free()


@pytest.mark.parametrize("thr", [1e-2, 1e-6])
def test_bf16_hessian_products_early_in_the_bulk_phase(C, thr):
    """bf16_hvp_until: the FP32 bulk phase takes its Hessian products from the BF16 tiles (the
    tensor-core sweep) until ||rgrad|| falls below thr of the start, then from the FP32 tiles;
    the certified optimum is the oracle's.  Without a BF16 copy the option is refused."""
    from paper_2502_04640_b300 import xm
    sc = scenes.random_scene(90, 4000, noise=0.03, outlier_frac=0.05, seed=21)
    Qo = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    ref = O.solve(Qo, r0=4)
    q, out = _solve(C, sc, PRECS["fp32"], bf16_hvp_until=thr)
    info = out["info"]
    assert ref.certified and info["certified"] == 1
    assert _rel(info["f"], ref.f) <= 1e-6 and _rel(info["rho_hat"], ref.rho_hat) <= 1e-6
    assert abs(info["lambda_min_deflated"] - ref.cert.lam_min_deflated) <= 1e-5 * ref.cert.lam_max_Q
    q.free()
    q = xm.xm_build_Q(C, sc.N, sc.M, *xm.scene_tensors(sc), xm.XM_STORE_FP32 | xm.XM_STORE_FP64)
    with pytest.raises(xm.XmError) as e:
        xm.xm_solve(q, xm.xm_default_opts(bf16_hvp_until=thr))
    assert e.value.status == xm.XM_EINVAL
    q.free()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_outliers_and_tiles_match_oracle(C, prec):
    sc = scenes.random_scene(90, 4000, noise=0.03, outlier_frac=0.05, seed=21)
    Qo = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    ref = O.solve(Qo, r0=4)
    q, out = _solve(C, sc, PRECS[prec])
    info = out["info"]
    assert info["certified"] == int(ref.certified)
    assert _rel(info["f"], ref.f) <= 1e-6
    if ref.certified:
        assert _rel(info["rho_hat"], ref.rho_hat) <= 1e-6
    q.free()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_certify_entry_point_matches_oracle(C, prec):
    """The FP32 mode keeps its Krylov basis in FP32 (FP64 recurrence coefficients): the deflated
    minimum agrees with the oracle's to 1e-5 of lambda_max in both modes."""
    from paper_2502_04640_b300 import xm
    sc = scenes.config1()
    Qo = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    ref = O.solve(Qo, r0=4)
    q = xm.xm_build_Q(C, sc.N, sc.M, *xm.scene_tensors(sc))
    out = xm.xm_certify(q, torch.tensor(ref.Y, device="cuda"), xm.xm_default_opts(prec=PRECS[prec]))
    Lam = out["Lambda"].cpu().numpy()
    cert = O.certify(Qo, ref.Y)
    assert np.abs(Lam - cert.Lambda).max() <= 1e-8 * np.abs(cert.Lambda).max()
    assert abs(out["info"]["lambda_min_deflated"] - cert.lam_min_deflated) <= 1e-5 * cert.lam_max_Q
    assert out["info"]["certified"] == 1 and out["info"]["lanczos_converged"] == 1
    if prec == "fp32":
        q.free()
        return
    # at the rank-3 local optimum of the [I..I] start the certificate fails (Thm. 2)
    r3 = O.rtr(Qo, O.initial_point(sc.N, 3))
    bad = xm.xm_certify(q, torch.tensor(r3.Y, device="cuda"), xm.xm_default_opts(prec=0))
    c3 = O.certify(Qo, r3.Y)
    assert bad["info"]["certified"] == 0
    assert abs(bad["info"]["lambda_min_deflated"] - c3.lam_min_deflated) <= 1e-5 * c3.lam_max_Q
    assert abs(bad["info"]["lambda_min"] - c3.lam_min) <= 1e-5 * c3.lam_max_Q
    assert abs(bad["info"]["dual"] - c3.dual) <= 1e-8 * (1 + abs(c3.f))
    q.free()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_uncertified_stop_reports_app_e_bound(C, prec):
    """The staircase capped at rank 3 from Alg. 1's start stops at config 1's rank-3 saddle
    (Thm. 1 fails: lambda_min < 0): XM_ENOTCERT with the oracle's objective, dual value and raw
    lambda_min, and at the returned point the oracle's rounding, Eq. 18's eta and App. E's
    eta_robust (whose bound now carries min(0, lambda_min) tr(X) < 0)."""
    from paper_2502_04640_b300 import xm
    sc = scenes.config1()
    ref = O.solve(O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w), r0=3, r_max=3)
    assert not ref.certified and ref.cert.lam_min < 0
    q, out = _solve(C, sc, PRECS[prec], r0=3, r_max=3, init_jitter=0.0)
    info = out["info"]
    assert out["status"] == xm.XM_ENOTCERT and info["certified"] == 0 and info["rank"] == 3
    assert _rel(info["f"], ref.f) <= 1e-6
    assert abs(info["dual"] - ref.cert.dual) <= 1e-6 * (1 + abs(ref.f))
    assert abs(info["lambda_min"] - ref.cert.lam_min) <= 1e-5 * ref.cert.lam_max_Q
    # a saddle is not an isolated point (scale-collapsed cameras move along flat directions), so
    # the rounding and both bounds are compared at the GPU's own point
    check_at_returned_point(O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w), out)
    assert info["eta_robust"] > info["eta"] > 0
    q.free()


def test_pipeline_from_host_arrays(C):
    from paper_2502_04640_b300 import xm
    sc = scenes.config1()
    ref = O.solve(O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w), r0=4)
    R, s, info, st = xm.xm_pipeline_host(C, sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w,
                                         xm.xm_default_opts(prec=1))
    assert st == 0 and info["certified"] == 1
    assert np.abs(R - ref.R).max() <= 1e-5 and np.abs(s - ref.s).max() <= 1e-5 * ref.s.max()


@pytest.mark.parametrize("name", ["config1", "bal"])
def test_block_jacobi_tcg_reaches_the_oracle_optimum(C, name):
    """opts.precond = 1 (block-Jacobi preconditioned tCG with the trust region in its norm)
    changes the path, not the certified optimum."""
    sc = scenes.config1() if name == "config1" else scenes.random_scene(
        60, 1500, noise=0.02, outlier_frac=0.02, seed=71, s_range=(0.3, 3.0))
    Qo = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    ref = O.solve(Qo, r0=4)
    assert ref.certified
    for prec in (0, 1):
        q, out = _solve(C, sc, prec, precond=1)
        info = out["info"]
        assert out["status"] == 0 and info["certified"] == 1
        assert _rel(info["f"], ref.f) <= 1e-6
        assert np.abs(out["R"] - ref.R).max() <= 1e-5
        q.free()


@pytest.mark.parametrize("stall,precond", [(5, 0), (-1, 2), (0, 0), (0, 1)])
def test_bulk_stall_option(stall, precond):
    """The FP32 bulk phase's hand-over rules (opts.bulk_stall: k = 5 after five outer steps
    without an FP32 objective improvement beyond its noise, -1 automatic at the gradient's
    noise floor, 0 none) and the tCG preconditioner settings (0 plain, 1 block Jacobi, 2
    adaptive) all reach the oracle's certified optimum; out-of-range values are rejected."""
    from paper_2502_04640_b300 import xm
    from oracle import xm_oracle as O
    sc = scenes.random_scene(80, 1600, noise=0.02, outlier_frac=0.02, seed=21, center_sigma=3.0)
    ctx = xm.Context(0)
    q = xm.xm_build_Q(ctx, sc.N, sc.M, *xm.scene_tensors(sc))
    out = xm.xm_solve(q, xm.xm_default_opts(prec=xm.XM_FP32_BULK, bulk_stall=stall, precond=precond))
    ref = O.solve(O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w), r0=4)
    assert out["info"]["certified"] == 1 and ref.certified
    assert abs(out["info"]["f"] - ref.f) / (1.0 + abs(ref.f)) <= 1e-6
    for bad in (dict(bulk_stall=-2), dict(precond=3), dict(precond=-1)):
        with pytest.raises(xm.XmError) as e:
            xm.xm_solve(q, xm.xm_default_opts(prec=xm.XM_FP32_BULK, **bad))
        assert e.value.status == xm.XM_EINVAL
    q.free()
    ctx.close()


@pytest.mark.parametrize("lob", [0, 1])
def test_fp32_certificate_lobpcg_and_lanczos(C, lob):
    """The FP32-Z certificate by block-Jacobi LOBPCG (opts.cert_lobpcg = 1, the default) and by
    Lanczos (0) both match the oracle's deflated minimum to 1e-5 of lambda_max, at the certified
    optimum and at the rank-3 saddle of the [I..I] start (Thm. 2: not certified)."""
    from paper_2502_04640_b300 import xm
    sc = scenes.config1()
    Qo = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    q = xm.xm_build_Q(C, sc.N, sc.M, *xm.scene_tensors(sc))
    opts = xm.xm_default_opts(prec=xm.XM_FP32_BULK, cert_lobpcg=lob)
    ref = O.solve(Qo, r0=4)
    good = xm.xm_certify(q, torch.tensor(ref.Y, device="cuda"), opts)
    cg = O.certify(Qo, ref.Y)
    assert good["info"]["certified"] == 1 and good["info"]["lanczos_converged"] == 1
    assert abs(good["info"]["lambda_min_deflated"] - cg.lam_min_deflated) <= 1e-5 * cg.lam_max_Q
    r3 = O.rtr(Qo, O.initial_point(sc.N, 3))
    bad = xm.xm_certify(q, torch.tensor(r3.Y, device="cuda"), opts)
    c3 = O.certify(Qo, r3.Y)
    assert bad["info"]["certified"] == 0
    assert abs(bad["info"]["lambda_min_deflated"] - c3.lam_min_deflated) <= 1e-5 * c3.lam_max_Q
    q.free()


def test_lobpcg_certificate_agrees_with_lanczos_mid_size(C):
    """300 cameras with outliers: the two FP32-Z certificates agree on the decision and on
    lambda_min to 1e-5 of lambda_max."""
    from paper_2502_04640_b300 import xm
    sc = scenes.random_scene(300, 6000, noise=0.02, outlier_frac=0.05, seed=31)
    q = xm.xm_build_Q(C, sc.N, sc.M, *xm.scene_tensors(sc))
    out = xm.xm_solve(q, xm.xm_default_opts(prec=xm.XM_FP64))
    assert out["info"]["certified"] == 1
    r = out["info"]["rank"]
    Y = out["Y"][:, :r].contiguous()
    res = {}
    for lob in (0, 1):
        res[lob] = xm.xm_certify(q, Y, xm.xm_default_opts(prec=xm.XM_FP32_BULK, cert_lobpcg=lob))["info"]
    assert res[0]["certified"] == res[1]["certified"] == 1
    assert abs(res[0]["lambda_min_deflated"] - res[1]["lambda_min_deflated"]) <= 1e-5 * res[0]["lambda_max"]
    q.free()
