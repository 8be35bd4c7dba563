"""Seeded synthetic scenes for scaled bundle adjustment (SBA, Eq. 3).

This module only draws random inputs: camera poses, scales, landmarks and
lifted keypoints.  It holds none of the method's arithmetic (no data matrix,
no elimination, no solver) and is shared by the FP64 oracle tests and the
CUDA path alike.

Model (Eq. 3): a lifted keypoint of landmark k seen by camera i satisfies
    R_i (s_i u_ik) + t_i = p_k     (noise free),
so u_ik = R_i^T (p_k - t_i) / s_i in the (scaled) camera frame.

Every generator is deterministic in its seed.  Observations are emitted in
landmark-major order unless ``shuffle`` is set.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

__all__ = [
    "Scene", "haar_rotations", "circle_scene", "random_scene", "trajectory_scene",
    "config1", "config2", "config3", "config4", "config5", "sub_scene",
    "batch_scenes", "shuffled", "depth_noise_scenes", "DEPTH_NOISE_EPS",
]


@dataclass
class Scene:
    """One SBA instance: N cameras, M landmarks, E observations (i, k, u_ik, w_ik)."""
    name: str
    N: int
    M: int
    cam: np.ndarray          # int32[E]   camera index i (0 = anchor)
    lmk: np.ndarray          # int32[E]   landmark index k
    ukp: np.ndarray          # float64[E,3] lifted keypoint u_ik (camera frame)
    w: np.ndarray            # float64[E] weight w_ik > 0
    R_gt: np.ndarray         # float64[N,3,3]
    s_gt: np.ndarray         # float64[N]
    t_gt: np.ndarray         # float64[N,3]
    p_gt: np.ndarray         # float64[M,3]
    outlier: np.ndarray      # bool[E]
    meta: dict = field(default_factory=dict)

    @property
    def E(self) -> int:
        return int(self.cam.shape[0])

    def anchored_gt(self):
        """Ground truth expressed in the gauge R_0 = I, t_0 = 0, s_0 = 1 (anchoring, Sec. 2)."""
        R0, s0, t0 = self.R_gt[0], self.s_gt[0], self.t_gt[0]
        R = np.einsum("ba,nbc->nac", R0, self.R_gt)          # R0^T R_i
        s = self.s_gt / s0
        t = (self.t_gt - t0) @ R0 / s0                          # R0^T (t_i - t0) / s0
        p = (self.p_gt - t0) @ R0 / s0
        return R, s, t, p


def haar_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """n rotations uniform on SO(3) (unit quaternions uniform on S^3)."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def _euler_zyx(yaw, pitch, roll) -> np.ndarray:
    cy, sy = np.cos(yaw), np.sin(yaw)
    cp, sp = np.cos(pitch), np.sin(pitch)
    cr, sr = np.cos(roll), np.sin(roll)
    n = np.size(yaw)
    Rz = np.zeros((n, 3, 3)); Rz[:, 0, 0] = cy; Rz[:, 0, 1] = -sy; Rz[:, 1, 0] = sy; Rz[:, 1, 1] = cy; Rz[:, 2, 2] = 1
    Ry = np.zeros((n, 3, 3)); Ry[:, 0, 0] = cp; Ry[:, 0, 2] = sp; Ry[:, 2, 0] = -sp; Ry[:, 2, 2] = cp; Ry[:, 1, 1] = 1
    Rx = np.zeros((n, 3, 3)); Rx[:, 1, 1] = cr; Rx[:, 1, 2] = -sr; Rx[:, 2, 1] = sr; Rx[:, 2, 2] = cr; Rx[:, 0, 0] = 1
    return Rz @ Ry @ Rx


def _distinct_observers(rng, N: int, L: np.ndarray):
    """For landmark k draw L[k] distinct cameras uniformly at random.

    Returns (cam, lmk) in landmark-major order."""
    cams, lmks = [], []
    for Lv in np.unique(L):
        idx = np.nonzero(L == Lv)[0]
        if Lv * Lv > N:
            # long tracks relative to N: the first Lv entries of a random permutation per row
            rows = np.argsort(rng.random((idx.size, N)), axis=1)[:, :Lv]
        else:
            rows = rng.integers(0, N, size=(idx.size, Lv))
            while Lv > 1:
                srt = np.sort(rows, axis=1)
                bad = np.nonzero((srt[:, 1:] == srt[:, :-1]).any(axis=1))[0]
                if bad.size == 0:
                    break
                rows[bad] = rng.integers(0, N, size=(bad.size, Lv))
        cams.append(rows.ravel())
        lmks.append(np.repeat(idx, Lv))
    if not cams:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    cam, lmk = np.concatenate(cams), np.concatenate(lmks)
    order = np.argsort(lmk, kind="stable")
    return cam[order].astype(np.int32), lmk[order].astype(np.int32)


def _observe(name, rng, R, s, t, p, obs, noise_sigma, outlier_frac, outlier_half,
             w_lo, w_hi, mult_noise=0.0, meta=None, depth_eps=0.0) -> Scene:
    N, M = R.shape[0], p.shape[0]
    cam, lmk = obs
    E = cam.size
    # u_ik = R_i^T (p_k - t_i) / s_i
    d = p[lmk] - t[cam]
    ukp = np.einsum("eba,eb->ea", R[cam], d) / s[cam][:, None]
    if mult_noise > 0:
        ukp *= (1.0 + mult_noise * rng.standard_normal(E))[:, None]
    if depth_eps > 0:
        # depth-noise model of the paper's noise analysis: every observation's depth (hence its
        # lifted keypoint) is scaled by (1 + eps)^x with x ~ U(-1, 1) drawn per observation
        x = rng.uniform(-1.0, 1.0, size=E)
        ukp *= np.power(1.0 + depth_eps, x)[:, None]
    if noise_sigma > 0:
        ukp += noise_sigma * rng.standard_normal((E, 3))
    outlier = np.zeros(E, dtype=bool)
    if outlier_frac > 0:
        outlier = rng.random(E) < outlier_frac
        ukp[outlier] = rng.uniform(-outlier_half, outlier_half, size=(int(outlier.sum()), 3))
    w = np.ones(E) if w_lo == w_hi else rng.uniform(w_lo, w_hi, size=E)
    return Scene(name, N, M, cam, lmk, ukp, w.astype(np.float64), R, s, t, p, outlier, meta or {})


def circle_scene(N: int = 20, M: int = 200, obs_per_lmk: int = 4, noise: float = 0.01,
                 seed: int = 0, radius: float = 5.0, s_range=(0.5, 2.0), w_range=(1.0, 1.0),
                 name: str | None = None, depth_eps: float = 0.0) -> Scene:
    """Cameras on a circle of the given radius, Haar rotations, landmarks in [-1,1]^3,
    each landmark seen by ``obs_per_lmk`` distinct random cameras (the tiny FP64 workload).
    depth_eps > 0 adds the depth-noise factor (1 + depth_eps)^x, x ~ U(-1, 1), per observation."""
    rng = np.random.default_rng(seed)
    R = haar_rotations(rng, N)
    th = 2 * math.pi * np.arange(N) / N
    t = np.stack([radius * np.cos(th), radius * np.sin(th), np.zeros(N)], axis=1)
    s = rng.uniform(s_range[0], s_range[1], size=N)
    p = rng.uniform(-1.0, 1.0, size=(M, 3))
    L = np.full(M, min(obs_per_lmk, N), dtype=np.int64)
    obs = _distinct_observers(rng, N, L)
    return _observe(name or f"circle-N{N}-M{M}", rng, R, s, t, p, obs, noise, 0.0, 0.0,
                    w_range[0], w_range[1], meta=dict(kind="circle", seed=seed, depth_eps=depth_eps),
                    depth_eps=depth_eps)


def random_scene(N: int, M: int, noise: float = 0.02, outlier_frac: float = 0.0, seed: int = 1,
                 geom_p: float = 0.25, min_track: int = 2, center_sigma: float = 10.0,
                 s_range=(0.3, 3.0), w_range=(0.5, 1.0), lmk_half: float = 10.0,
                 outlier_half: float = 5.0, name: str | None = None,
                 depth_eps: float = 0.0) -> Scene:
    """Community-photo-shaped scene: Haar rotations, Gaussian-clustered centres, track length
    min_track + Geometric(geom_p) (mean 5 for the defaults) clipped to N, a fraction of
    observations replaced by outliers uniform in a box of side 2*outlier_half.  depth_eps > 0
    adds the depth-noise factor (1 + depth_eps)^x, x ~ U(-1, 1), per observation."""
    rng = np.random.default_rng(seed)
    R = haar_rotations(rng, N)
    t = center_sigma * rng.standard_normal((N, 3))
    s = rng.uniform(s_range[0], s_range[1], size=N)
    p = rng.uniform(-lmk_half, lmk_half, size=(M, 3))
    L = np.minimum(min_track + rng.geometric(geom_p, size=M) - 1, N)
    obs = _distinct_observers(rng, N, L)
    return _observe(name or f"random-N{N}-M{M}", rng, R, s, t, p, obs, noise, outlier_frac,
                    outlier_half, w_range[0], w_range[1],
                    meta=dict(kind="random", seed=seed, outlier_frac=outlier_frac, depth_eps=depth_eps),
                    depth_eps=depth_eps)


def trajectory_scene(N: int = 2000, M: int = 400000, seed: int = 2, step: float = 0.05,
                     room=(10.0, 10.0, 3.0), window: int = 10, track=(3, 10),
                     depth_noise: float = 0.03, s_range=(0.5, 2.0), w_range=(0.5, 1.0),
                     name: str | None = None) -> Scene:
    """Indoor trajectory: random-walk centres (fixed step) inside a room, yaw-dominant
    rotations (yaw random walk, small pitch/roll), each landmark seen by 3..10 frames of a
    10-frame covisibility window, multiplicative depth noise (1 + eps), eps ~ N(0, sigma^2)."""
    rng = np.random.default_rng(seed)
    room = np.asarray(room, dtype=np.float64)
    c = np.empty((N, 3))
    c[0] = room / 2
    for i in range(1, N):
        d = rng.standard_normal(3)
        d[2] *= 0.2
        d /= np.linalg.norm(d)
        c[i] = np.clip(c[i - 1] + step * d, 0.05 * room, 0.95 * room)
    yaw = rng.uniform(-math.pi, math.pi) + np.cumsum(rng.normal(0.0, 0.1, size=N))
    pitch = rng.normal(0.0, math.radians(5.0), size=N)
    roll = rng.normal(0.0, math.radians(5.0), size=N)
    R = _euler_zyx(yaw, pitch, roll)
    s = rng.uniform(s_range[0], s_range[1], size=N)
    p = rng.uniform(0.0, 1.0, size=(M, 3)) * room
    W = min(window, N)
    start = rng.integers(0, N - W + 1, size=M)
    L = rng.integers(min(track[0], W), min(track[1], W) + 1, size=M)
    cams, lmks = [], []
    for Lv in np.unique(L):
        idx = np.nonzero(L == Lv)[0]
        perm = np.argsort(rng.random((idx.size, W)), axis=1)[:, :Lv]
        cams.append((start[idx][:, None] + perm).ravel())
        lmks.append(np.repeat(idx, Lv))
    cam, lmk = np.concatenate(cams), np.concatenate(lmks)
    order = np.argsort(lmk, kind="stable")
    obs = (cam[order].astype(np.int32), lmk[order].astype(np.int32))
    return _observe(name or f"trajectory-N{N}-M{M}", rng, R, s, c, p, obs, 0.0, 0.0, 0.0,
                    w_range[0], w_range[1], mult_noise=depth_noise,
                    meta=dict(kind="trajectory", seed=seed))


def sub_scene(sc: Scene, n_cams: int, name: str | None = None) -> Scene:
    """The first n_cams cameras and the observations of landmarks they see (re-indexed);
    landmarks left with fewer than 2 observations are dropped."""
    keep = sc.cam < n_cams
    lmk = sc.lmk[keep]
    cnt = np.bincount(lmk, minlength=sc.M)
    keep2 = cnt[lmk] >= 2
    cam, lmk = sc.cam[keep][keep2], lmk[keep2]
    used = np.unique(lmk)
    remap = -np.ones(sc.M, dtype=np.int64)
    remap[used] = np.arange(used.size)
    sel = np.nonzero(keep)[0][keep2]
    return Scene(name or f"{sc.name}-sub{n_cams}", n_cams, int(used.size), cam.astype(np.int32),
                 remap[lmk].astype(np.int32), sc.ukp[sel].copy(), sc.w[sel].copy(),
                 sc.R_gt[:n_cams].copy(), sc.s_gt[:n_cams].copy(), sc.t_gt[:n_cams].copy(),
                 sc.p_gt[used].copy(), sc.outlier[sel].copy(), dict(sc.meta, parent=sc.name))


def shuffled(sc: Scene, seed: int = 123) -> Scene:
    """The same scene with its observations in a random order."""
    perm = np.random.default_rng(seed).permutation(sc.E)
    return Scene(sc.name + "-shuf", sc.N, sc.M, sc.cam[perm].copy(), sc.lmk[perm].copy(),
                 sc.ukp[perm].copy(), sc.w[perm].copy(), sc.R_gt, sc.s_gt, sc.t_gt, sc.p_gt,
                 sc.outlier[perm].copy(), dict(sc.meta))


# ---------------------------------------------------------------------------------------
# The five workloads.  Sizes follow the paper's datasets (BAL-1934 / BAL-10155, a 2000-frame
# indoor sequence); every input is synthetic and stands in for those datasets.
# ---------------------------------------------------------------------------------------

def config1(seed: int = 0) -> Scene:
    """Tiny FP64 scene: 20 cameras on a radius-5 circle, 200 landmarks x 4 observers."""
    return circle_scene(20, 200, 4, 0.01, seed=seed, name="c1-circle-N20")


def config2(seed: int = 1) -> Scene:
    """Mid-size community-photo shape: 1934 cameras, 300k landmarks, 2% outliers."""
    return random_scene(1934, 300_000, noise=0.02, outlier_frac=0.02, seed=seed, name="c2-N1934")


def config3(seed: int = 1) -> Scene:
    """Large scene: 10155 cameras, 1.5M landmarks (~7.5M observations), 5% outliers."""
    return random_scene(10155, 1_500_000, noise=0.02, outlier_frac=0.05, seed=seed, name="c3-N10155")


def config4(seed: int = 2) -> Scene:
    """Indoor 2000-frame trajectory with 400k landmarks and multiplicative depth noise."""
    return trajectory_scene(2000, 400_000, seed=seed, name="c4-traj-N2000")


def batch_sizes(count: int = 256, seed: int = 3, lo: int = 10, hi: int = 400) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)


def batch_scenes(count: int = 256, seed: int = 3, lo: int = 10, hi: int = 400,
                 lmk_per_cam: int = 50, obs_per_lmk: int = 4, noise: float = 0.01) -> list:
    """Serving-style batch: camera counts log-uniform in [lo, hi], 50 landmarks per camera,
    4 observers per landmark, the tiny scene's noise."""
    sizes = batch_sizes(count, seed, lo, hi)
    return [circle_scene(int(n), int(lmk_per_cam * n), obs_per_lmk, noise, seed=seed * 100003 + j,
                         name=f"c5-{j}-N{int(n)}") for j, n in enumerate(sizes)]


def config5(seed: int = 3, count: int = 256) -> list:
    return batch_scenes(count, seed)


# Depth-noise robustness sweep (the paper's noise analysis): noise levels eps of the factor
# (1 + eps)^x, x ~ U(-1, 1), applied to every observation's depth, from mild to the level where
# the paper reports the SDP relaxation itself to break (eps = 5).
DEPTH_NOISE_EPS = (0.0, 0.1, 0.25, 0.5, 1.0, 1.5, 2.0, 3.0, 5.0)


def depth_noise_scenes(eps: float, count: int = 8, N: int = 100, M: int = 2000,
                       seed: int = 4) -> list:
    """``count`` community-photo-shaped scenes (N cameras, M landmarks, track 2 + Geom(1/4), unit
    weights) whose only perturbation is the depth-noise factor (1 + eps)^x per observation; scene
    j uses seed seed * 1000 + j, so every noise level sees the same geometry."""
    return [random_scene(N, M, noise=0.0, outlier_frac=0.0, seed=seed * 1000 + j, w_range=(1.0, 1.0),
                         depth_eps=eps, name=f"depthnoise-eps{eps:g}-{j}-N{N}") for j in range(count)]
