"""Q construction on the GPU (App. A, FP64) against the oracle's Schur-form Q, plus the
input validation and connectivity errors of the boundary."""
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


def _gpu_Q(C, sc, mask=7):
    from paper_2502_04640_b300 import xm
    q = xm.xm_build_Q(C, sc.N, sc.M, *xm.scene_tensors(sc), store_mask=mask)
    Q = xm.xm_qmat_to_dense(q).cpu().numpy()
    return q, Q


CASES = [
    ("c1", lambda: scenes.config1()),
    ("outliers", lambda: scenes.random_scene(30, 400, noise=0.05, outlier_frac=0.1, seed=3, center_sigma=3.0)),
    ("shuffled", lambda: scenes.shuffled(scenes.random_scene(50, 600, noise=0.02, seed=4))),
    ("two-cams", lambda: scenes.circle_scene(2, 30, 2, 0.02, seed=5)),
    ("tiles", lambda: scenes.random_scene(130, 3000, noise=0.02, outlier_frac=0.02, seed=6)),
    ("traj", lambda: scenes.sub_scene(scenes.trajectory_scene(300, 20000, seed=7), 120)),
]


@pytest.mark.parametrize("name,make", CASES)
def test_build_matches_oracle(C, name, make):
    sc = make()
    q, Qg = _gpu_Q(C, sc)
    Qo = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    scale = np.abs(Qo).max()
    assert np.abs(Qg - Qo).max() <= 1e-9 * scale
    # the quadratic form, which is what the solver uses, agrees to near machine precision
    Y = np.random.default_rng(0).standard_normal((3 * sc.N, 4))
    assert abs(np.sum(Y * (Qg @ Y)) - np.sum(Y * (Qo @ Y))) <= \
        1e-9 * np.sum(np.abs(Y) * (np.abs(Qo) @ np.abs(Y)))
    q.free()


def test_single_camera_and_single_observation_landmarks(C):
    sc = scenes.circle_scene(1, 20, 1, 0.0, seed=1)
    q, Qg = _gpu_Q(C, sc)
    assert np.abs(Qg).max() <= 1e-12 * max(1.0, np.abs(sc.ukp).max() ** 2)
    q.free()


def test_invalid_inputs_are_rejected(C):
    from paper_2502_04640_b300 import xm
    sc = scenes.circle_scene(5, 30, 3, 0.01, seed=2)
    cam, lmk, ukp, w = xm.scene_tensors(sc)
    bad = cam.clone(); bad[3] = sc.N
    with pytest.raises(xm.XmError) as e:
        xm.xm_build_Q(C, sc.N, sc.M, bad, lmk, ukp, w)
    assert e.value.status == xm.XM_EINVAL
    bw = w.clone(); bw[0] = 0.0
    with pytest.raises(xm.XmError) as e:
        xm.xm_build_Q(C, sc.N, sc.M, cam, lmk, ukp, bw)
    assert e.value.status == xm.XM_EINVAL
    bu = ukp.clone(); bu[1, 2] = float("nan")
    with pytest.raises(xm.XmError) as e:
        xm.xm_build_Q(C, sc.N, sc.M, cam, lmk, bu, w)
    assert e.value.status == xm.XM_EINVAL
    # two disjoint scenes: the view graph is disconnected (App. A lemma)
    a = scenes.circle_scene(3, 10, 3, 0.01, seed=6)
    cam2 = np.concatenate([a.cam, a.cam + 3]); lmk2 = np.concatenate([a.lmk, a.lmk + 10])
    t = lambda x, dt: torch.as_tensor(x, dtype=dt, device="cuda").contiguous()
    with pytest.raises(xm.XmError) as e:
        xm.xm_build_Q(C, 6, 20, t(cam2, torch.int32), t(lmk2, torch.int32),
                      t(np.concatenate([a.ukp, a.ukp]), torch.float64), t(np.concatenate([a.w, a.w]), torch.float64))
    assert e.value.status == xm.XM_EDISCONNECTED
    # a camera with no observation is unconstrained: also disconnected
    with pytest.raises(xm.XmError) as e:
        xm.xm_build_Q(C, sc.N + 1, sc.M, cam, lmk, ukp, w)
    assert e.value.status == xm.XM_EDISCONNECTED
