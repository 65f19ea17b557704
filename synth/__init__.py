"""Seeded synthetic scenes and cameras for the 6D Gaussian render path.

This module only draws inputs.  It holds no part of the render arithmetic:
no slicing, projection, colour or blending.  Both the FP64 oracle and the
CUDA library consume what it produces.

Scene layout (structure of arrays, float32, one plane per scalar, length n):

* ``mu_p``          (3, n)   position means
* ``mu_d``          (3, n)   direction means
* ``l_raw``         (21, n)  raw Cholesky parameters; planes 0-5 hold the six
  diagonal entries in log space, planes 6-20 the fifteen strictly-lower
  entries in row-major order (1,0) (2,0) (2,1) (3,0) ... (5,4), stored as the
  pre-activation value of the off-diagonal map v = 2*sigmoid(raw) - 1
* ``opacity_logit`` (n,)     pre-sigmoid opacity
* ``sh``            ((deg+1)^2 * 3, n)  SH coefficients, plane k*3 + c for
  basis function k = l*l + l + m and colour channel c

The five workloads follow the shapes of the paper's scenes (10^4-10^6
Gaussians, 800^2-1920x1080 images, section 5.1, Tables 1-2) since the paper's
datasets and trained scenes are not available:

0. 4,096 Gaussians in [-1,1]^3, one 128x128 camera (small parity case)
1. 200k Gaussians on a noisy unit shell, one 800x800 camera
2. 300k shell Gaussians with strong position-direction coupling, 8 x 800^2
   cameras on a ring (the differentiable fwd+bwd workload)
3. 500k Gaussians as 2, 64 cameras on a hemisphere with mixed resolutions
4. 2M Gaussians with strongly view-dependent covariances, 4 x 1920x1080
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

N_RAW_L = 21
OFFDIAG_ORDER = [(i, j) for i in range(6) for j in range(i)]  # row-major lower

CONFIG_SEED_BASE = 6000


@dataclasses.dataclass
class Scene:
    mu_p: np.ndarray
    mu_d: np.ndarray
    l_raw: np.ndarray
    opacity_logit: np.ndarray
    sh: np.ndarray
    sh_degree: int
    lambda_raw: np.ndarray | None = None   # optional per-Gaussian pre-sigmoid lambda_opa

    @property
    def n(self) -> int:
        return int(self.mu_p.shape[1])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.mu_p[:, idx].copy(), self.mu_d[:, idx].copy(),
                     self.l_raw[:, idx].copy(), self.opacity_logit[idx].copy(),
                     self.sh[:, idx].copy(), self.sh_degree,
                     None if self.lambda_raw is None else self.lambda_raw[idx].copy())

    def planes(self) -> dict:
        out = {"mu_p": self.mu_p, "mu_d": self.mu_d, "l_raw": self.l_raw,
               "opacity_logit": self.opacity_logit, "sh": self.sh}
        if self.lambda_raw is not None:
            out["lambda_raw"] = self.lambda_raw
        return out


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    world_to_cam: np.ndarray  # (3, 4) float64, rows = camera x (right), y (down), z (forward)
    campos: np.ndarray        # (3,) float64
    znear: float = 0.2


@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    cameras: list
    tile_w: int = 16
    tile_h: int = 16
    lambda_opa: float = 0.35
    bg: tuple = (1.0, 1.0, 1.0)
    seed: int = 0


# --------------------------------------------------------------------------
# Cameras
# --------------------------------------------------------------------------

def look_at_camera(campos, width, height, fov_x_deg=50.0, target=(0.0, 0.0, 0.0),
                   up=(0.0, 0.0, 1.0), znear=0.2) -> Camera:
    """Pinhole camera at ``campos`` looking at ``target``; x right, y down, z forward."""
    c = np.asarray(campos, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - c
    f /= np.linalg.norm(f)
    u = np.asarray(up, dtype=np.float64)
    if abs(float(f @ u)) > 0.999:
        u = np.array([0.0, 1.0, 0.0])
    right = np.cross(f, u)
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    rot = np.stack([right, down, f])
    w2c = np.concatenate([rot, (-rot @ c)[:, None]], axis=1)
    fx = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return Camera(int(width), int(height), fx, fx, width / 2.0, height / 2.0, w2c, c, znear)


def ring_cameras(n, width, height, radius=4.0):
    cams = []
    for k in range(n):
        a = 2.0 * math.pi * k / n
        cams.append(look_at_camera((radius * math.cos(a), radius * math.sin(a), 0.0), width, height))
    return cams


def hemisphere_cameras(n, sizes, radius=4.0, min_elev_deg=5.0):
    """Fibonacci points on the upper hemisphere, elevation >= min_elev_deg."""
    zmin = math.sin(math.radians(min_elev_deg))
    golden = math.pi * (3.0 - math.sqrt(5.0))
    cams = []
    for k in range(n):
        z = zmin + (1.0 - zmin) * (k + 0.5) / n
        rxy = math.sqrt(max(0.0, 1.0 - z * z))
        a = golden * k
        pos = (radius * rxy * math.cos(a), radius * rxy * math.sin(a), radius * z)
        w, h = sizes[k]
        cams.append(look_at_camera(pos, w, h))
    return cams


# --------------------------------------------------------------------------
# Scenes
# --------------------------------------------------------------------------

def _unit_vectors(rng, n):
    v = rng.standard_normal((3, n))
    v /= np.linalg.norm(v, axis=0, keepdims=True)
    return v


def _encode_l(l_diag, l_off):
    """Store drawn Cholesky-factor values as raw parameters.

    Input encoding only: the diagonal is kept as its logarithm and each
    off-diagonal value v in (-1, 1) as 2*artanh(v), the pre-image of
    v = 2*sigmoid(raw) - 1.
    """
    raw = np.empty((N_RAW_L, l_diag.shape[1]), dtype=np.float64)
    raw[:6] = np.log(l_diag)
    raw[6:] = 2.0 * np.arctanh(np.clip(l_off, -0.999999, 0.999999))
    return raw


def _scene_common(rng, n, mu_p, pos_sigma, pos_off_sigma, dir_sigma=0.3, dp_sigma=0.02,
                  dd_off_sigma=0.02, sh_degree=3):
    mu_d = _unit_vectors(rng, n)
    l_diag = np.empty((6, n))
    l_diag[:3] = np.exp(rng.normal(math.log(pos_sigma), 0.3, (3, n)))
    l_diag[3:] = np.exp(rng.normal(math.log(dir_sigma), 0.3, (3, n)))
    l_off = np.empty((15, n))
    for k, (i, j) in enumerate(OFFDIAG_ORDER):
        if i < 3:                       # position block L_pp
            s = pos_off_sigma
        elif j < 3:                     # direction-position block L_dp
            s = dp_sigma
        else:                           # direction block L_dd
            s = dd_off_sigma
        l_off[k] = rng.normal(0.0, s, n)
    l_raw = _encode_l(l_diag, l_off)
    logit = rng.normal(0.0, 1.0, n)
    nsh = (sh_degree + 1) ** 2 * 3
    sh = rng.normal(0.0, 0.2, (nsh, n))
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Scene(f32(mu_p), f32(mu_d), f32(l_raw), f32(logit), f32(sh), sh_degree)


def scene_cube(n, seed, sh_degree=3):
    """Config-0 style: positions uniform in [-1,1]^3, position sigma ~0.05."""
    rng = np.random.default_rng(seed)
    mu_p = rng.uniform(-1.0, 1.0, (3, n))
    return _scene_common(rng, n, mu_p, pos_sigma=0.05, pos_off_sigma=0.02, sh_degree=sh_degree)


def scene_shell(n, seed, dp_sigma=0.02, sh_degree=3):
    """Noisy unit-sphere shell, position sigma ~0.01 (all L_pp entries scaled by 0.2
    relative to the cube scene so that the position spread is ~0.01)."""
    rng = np.random.default_rng(seed)
    u = _unit_vectors(rng, n)
    mu_p = u * (1.0 + rng.normal(0.0, 0.01, (1, n)))
    return _scene_common(rng, n, mu_p, pos_sigma=0.01, pos_off_sigma=0.004, dp_sigma=dp_sigma,
                         sh_degree=sh_degree)


def scene_view_dependent(n, seed, dir_sigma=0.15, max_corr=0.8, sh_degree=3):
    """Shell scene whose direction rows are strongly correlated with position.

    Direction row j of L gets L_dp[j,:] = dir_sigma * c_j and
    L_dd[j,j] = dir_sigma * sqrt(1 - |c_j|^2) with |c_j| ~ U[0, max_corr], so
    that with a near-isotropic L_pp the position/direction correlation
    reaches max_corr and each direction component keeps spread dir_sigma.
    """
    rng = np.random.default_rng(seed)
    u = _unit_vectors(rng, n)
    mu_p = u * (1.0 + rng.normal(0.0, 0.01, (1, n)))
    mu_d = _unit_vectors(rng, n)
    l_diag = np.empty((6, n))
    l_diag[:3] = np.exp(rng.normal(math.log(0.01), 0.3, (3, n)))
    l_off = np.zeros((15, n))
    rows_c = []
    for j in range(3):
        c = _unit_vectors(rng, n) * rng.uniform(0.0, max_corr, (1, n))
        rows_c.append(c)
        l_diag[3 + j] = dir_sigma * np.sqrt(1.0 - np.sum(c * c, axis=0))
    for k, (i, j) in enumerate(OFFDIAG_ORDER):
        if i < 3:
            l_off[k] = rng.normal(0.0, 0.002, n)
        elif j < 3:
            l_off[k] = dir_sigma * rows_c[i - 3][j]
    l_raw = _encode_l(l_diag, l_off)
    logit = rng.normal(0.0, 1.0, n)
    sh = rng.normal(0.0, 0.2, ((sh_degree + 1) ** 2 * 3, n))
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Scene(f32(mu_p), f32(mu_d), f32(l_raw), f32(logit), f32(sh), sh_degree)


def perturb(scene: Scene, seed: int) -> Scene:
    """Copy of ``scene`` with small seeded noise: the source of target images."""
    rng = np.random.default_rng(seed)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Scene(
        f32(scene.mu_p + rng.normal(0.0, 0.005, scene.mu_p.shape)),
        scene.mu_d.copy(),
        f32(scene.l_raw + rng.normal(0.0, 0.05, scene.l_raw.shape)),
        f32(scene.opacity_logit + rng.normal(0.0, 0.1, scene.opacity_logit.shape)),
        f32(scene.sh + rng.normal(0.0, 0.05, scene.sh.shape)),
        scene.sh_degree,
        None if scene.lambda_raw is None else scene.lambda_raw.copy())


# pre-sigmoid value of lambda_opa = 0.35, the initial value of section 5.1
LAMBDA_RAW_INIT = -0.6190392084062235


def with_learnable_lambda(scene: Scene, seed: int, spread: float = 0.5) -> Scene:
    """Copy of ``scene`` with a per-Gaussian lambda_opa plane drawn around 0.35."""
    rng = np.random.default_rng(seed)
    out = dataclasses.replace(scene)
    out.lambda_raw = np.ascontiguousarray(LAMBDA_RAW_INIT + rng.normal(0.0, spread, scene.n), dtype=np.float32)
    return out


RES_CHOICES = [(256, 256), (512, 384), (800, 800), (1024, 768)]

CONFIG_NAMES = {
    0: "cube4k_128sq_1view_fwd",
    1: "shell200k_800sq_1view_fwd",
    2: "shell300k_coupled_800sq_8view_fwdbwd",
    3: "shell500k_coupled_64view_mixedres_fwdbwd",
    4: "viewdep2M_1920x1080_4view_fwdbwd",
}


def make_workload(config: int, n_override: int | None = None) -> Workload:
    """The five workloads; ``n_override`` shrinks the scene (same recipe)."""
    seed = CONFIG_SEED_BASE + config
    if config == 0:
        scene = scene_cube(n_override or 4096, seed)
        cams = [look_at_camera((4.0, 0.0, 0.0), 128, 128)]
    elif config == 1:
        scene = scene_shell(n_override or 200_000, seed)
        cams = [look_at_camera((4.0, 0.0, 0.0), 800, 800)]
    elif config == 2:
        scene = scene_shell(n_override or 300_000, seed, dp_sigma=0.1)
        cams = ring_cameras(8, 800, 800)
    elif config == 3:
        scene = scene_shell(n_override or 500_000, seed, dp_sigma=0.1)
        rng = np.random.default_rng(seed + 200)
        sizes = [RES_CHOICES[i] for i in rng.integers(0, len(RES_CHOICES), 64)]
        cams = hemisphere_cameras(64, sizes)
    elif config == 4:
        scene = scene_view_dependent(n_override or 2_000_000, seed)
        cams = ring_cameras(4, 1920, 1080)
    else:
        raise ValueError(f"unknown workload {config}")
    return Workload(CONFIG_NAMES[config], scene, cams, seed=seed)


def scene_volume(n, seed, radius=0.6, sh_degree=3):
    """Volumetric-medium stand-in: positions normally spread in a ball of
    ~radius, position sigma ~0.8x the mean point spacing (so the medium is
    covered), lower opacities (logit ~ N(-1, 1))."""
    rng = np.random.default_rng(seed)
    mu_p = rng.normal(0.0, radius / 1.7, (3, n))
    r = np.linalg.norm(mu_p, axis=0, keepdims=True)
    mu_p = np.where(r > 1.0, mu_p / r, mu_p)
    spacing = (4.0 / 3.0 * math.pi * radius ** 3 / n) ** (1.0 / 3.0)
    sc = _scene_common(rng, n, mu_p, pos_sigma=0.8 * spacing, pos_off_sigma=0.3 * spacing, sh_degree=sh_degree)
    sc.opacity_logit = np.ascontiguousarray(rng.normal(-1.0, 1.0, n), dtype=np.float32)
    return sc


# Point counts and square image sides of the six scenes of the paper's
# Table 2 (forward-only FPS; section 5.2), with the kind of content each
# holds.  The scenes rendered here are synthetic stand-ins of those shapes;
# the last field is the FPS the paper prints for 6DGS (hardware not named).
TABLE2_SHAPES = [
    ("vol6.7k_1408sq", 6660, 1408, "volume", 178.4),
    ("vol12.7k_1408sq", 12657, 1408, "volume", 178.2),
    ("vol17.1k_1024sq", 17133, 1024, "volume", 120.2),
    ("vol10.8k_1536sq", 10762, 1536, "volume", 138.6),
    ("surf175k_1408sq", 174746, 1408, "surface", 34.7),
    ("vol183k_1024sq", 182981, 1024, "volume", 276.8),
]
TABLE2_SEED_BASE = 7000
TABLE2_TEST_VIEWS = 20


def table2_workload(index: int, n_override: int | None = None, views: int = TABLE2_TEST_VIEWS) -> Workload:
    """Inference workload shaped like row ``index`` of Table 2: the scene and
    ``views`` test cameras of that image size on a hemisphere of radius 4."""
    name, n, side, kind, _ = TABLE2_SHAPES[index]
    seed = TABLE2_SEED_BASE + index
    n = n_override or n
    scene = scene_volume(n, seed) if kind == "volume" else scene_shell(n, seed)
    cams = hemisphere_cameras(views, [(side, side)] * views)
    return Workload(name, scene, cams, seed=seed)


def target_seed(config: int) -> int:
    return CONFIG_SEED_BASE + config + 100


def random_grad_images(cameras, seed, scale=1.0):
    """Seeded dL/dI images (one (3,H,W) float32 array per camera)."""
    rng = np.random.default_rng(seed)
    return [np.ascontiguousarray(rng.normal(0.0, scale, (3, c.height, c.width)), dtype=np.float32)
            for c in cameras]
