"""The depth-noise model of the paper's noise analysis, s = (1 + eps)^x with x ~ U(-1, 1) per
observation (generator checks), and the oracle's behaviour on it: the paper reports the SDP
relaxation to stay tight up to eps = 5.  CPU only."""
import math

import numpy as np
import pytest

import scenes
from oracle import xm_oracle as O


def test_zero_noise_level_is_the_noise_free_scene():
    a = scenes.depth_noise_scenes(0.0, count=2, N=12, M=150)
    b = [scenes.random_scene(12, 150, noise=0.0, seed=4000 + j, w_range=(1.0, 1.0)) for j in range(2)]
    for x, y in zip(a, b):
        assert np.array_equal(x.ukp, y.ukp) and np.array_equal(x.cam, y.cam)


@pytest.mark.parametrize("eps", [0.1, 1.5, 5.0])
def test_depth_factor_is_log_uniform_on_the_stated_range(eps):
    """Every lifted keypoint is the noise-free one times (1 + eps)^x: its direction is unchanged
    and log(factor) / log(1 + eps) is uniform on (-1, 1) (Kolmogorov-Smirnov at 1e-3); the
    geometry (poses, scales, landmarks, observers) is the same at every noise level."""
    from scipy import stats
    clean = scenes.depth_noise_scenes(0.0, count=1, N=40, M=3000)[0]
    noisy = scenes.depth_noise_scenes(eps, count=1, N=40, M=3000)[0]
    assert np.array_equal(clean.cam, noisy.cam) and np.array_equal(clean.R_gt, noisy.R_gt)
    ratio = np.linalg.norm(noisy.ukp, axis=1) / np.linalg.norm(clean.ukp, axis=1)
    cosang = np.sum(noisy.ukp * clean.ukp, axis=1) / (
        np.linalg.norm(noisy.ukp, axis=1) * np.linalg.norm(clean.ukp, axis=1))
    assert np.all(cosang > 1 - 1e-12)
    x = np.log(ratio) / math.log1p(eps)
    assert x.min() >= -1 - 1e-12 and x.max() <= 1 + 1e-12
    assert stats.kstest(x, "uniform", args=(-1.0, 2.0)).pvalue > 1e-3


@pytest.mark.parametrize("eps", [0.5, 5.0])
def test_relaxation_stays_tight_under_depth_noise(eps):
    """The paper's noise analysis finds the SDP relaxation tight up to eps = 5: on the synthetic
    stand-in the staircase ends certified with a small relative suboptimality (Eq. 18)."""
    sc = scenes.depth_noise_scenes(eps, count=1, N=12, M=200)[0]
    res = O.solve(O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w), r0=4)
    assert res.certified
    assert 0 <= res.eta < 1e-2
