"""Seeded synthetic scenes and cameras for the Duplex-GS hot path.

This module only draws inputs: cell proxies, the K Gaussians each cell emits,
and pinhole cameras.  It holds none of the renderer's arithmetic (no
projection, binning, blending or spherical-harmonic evaluation), so both the
CUDA path and the CPU oracle can be fed from it without sharing method code.

Scene layout (all float32, structure of arrays, cell-major Gaussians):

    cell_center (N,3)  cell_axes (N,3)  cell_quat (N,4) [w,x,y,z]  cell_v (N,)
    g_mean (G,3)  g_scale (G,3) [linear]  g_quat (G,4) [w,x,y,z]  g_logit (G,)
    g_sh (G,(D+1)^2,3)  with G = N*K; Gaussian g belongs to cell g // K.

The cell parameters are the ellipsoidal proxy of Sec. IV-A (centre x_n,
scales S_n, quaternion Q_n, calibration scalar v_n); each cell emits a fixed
number K of Gaussians (Eq. 1).  Colours are real spherical-harmonic
coefficients of degree D in 0..3; degree 0 is a view-independent colour.

Camera layout (float32[22]): W, H, fx, fy, cx, cy, znear, R (3x3 row-major,
world->view), t (3), eye (3).  View space is x right, y down, +z forward;
pixel (i, j) is sampled at (i + 0.5, j + 0.5).

Draw order inside every generator is fixed and documented so the same seed
always yields the same arrays.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# 1 / Y_00, the inverse of the constant degree-0 real spherical harmonic
# 1/(2 sqrt(pi)).  Used only to turn a drawn base colour u into the DC
# coefficient (u - 0.5) / Y_00, i.e. an input-construction step.
_INV_Y00 = 2.0 * math.sqrt(math.pi)


@dataclass
class Camera:
    W: int
    H: int
    fx: float
    fy: float
    cx: float
    cy: float
    znear: float
    R: np.ndarray  # (3,3) float32, world -> view rotation
    t: np.ndarray  # (3,) float32, world -> view translation
    eye: np.ndarray  # (3,) float32, camera centre in world space

    def as_array(self) -> np.ndarray:
        a = np.zeros(22, dtype=np.float32)
        a[0] = self.W
        a[1] = self.H
        a[2] = self.fx
        a[3] = self.fy
        a[4] = self.cx
        a[5] = self.cy
        a[6] = self.znear
        a[7:16] = np.asarray(self.R, dtype=np.float32).reshape(9)
        a[16:19] = np.asarray(self.t, dtype=np.float32)
        a[19:22] = np.asarray(self.eye, dtype=np.float32)
        return a

    def with_resolution(self, W: int, H: int, fov_y_deg: float = 60.0) -> "Camera":
        return look_at_from_pose(self.R, self.eye, W, H, fov_y_deg, self.znear)


@dataclass
class Scene:
    K: int
    sh_degree: int
    cell_center: np.ndarray
    cell_axes: np.ndarray
    cell_quat: np.ndarray
    cell_v: np.ndarray
    g_mean: np.ndarray
    g_scale: np.ndarray
    g_quat: np.ndarray
    g_logit: np.ndarray
    g_sh: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)
    cell_v_sh: np.ndarray | None = None  # (N, (v_sh_degree+1)^2) view-dependent v_n, or None
    v_sh_degree: int = -1
    neural: dict | None = None  # neural cells: F, H, feat (N,F), offset (G,3), mlp (packed float32)

    @property
    def N(self) -> int:
        return int(self.cell_center.shape[0])

    @property
    def G(self) -> int:
        return int(self.g_mean.shape[0])

    def subset_cells(self, idx) -> "Scene":
        """Scene made of the listed cells (and their K Gaussians each)."""
        idx = np.asarray(idx, dtype=np.int64)
        gidx = (idx[:, None] * self.K + np.arange(self.K)[None, :]).reshape(-1)
        return Scene(self.K, self.sh_degree,
                     self.cell_center[idx].copy(), self.cell_axes[idx].copy(),
                     self.cell_quat[idx].copy(), self.cell_v[idx].copy(),
                     self.g_mean[gidx].copy(), self.g_scale[gidx].copy(),
                     self.g_quat[gidx].copy(), self.g_logit[gidx].copy(),
                     self.g_sh[gidx].copy(), name=self.name + "-subset", meta=dict(self.meta),
                     cell_v_sh=None if self.cell_v_sh is None else self.cell_v_sh[idx].copy(),
                     v_sh_degree=self.v_sh_degree)


# ----------------------------------------------------------------------------
# primitive samplers


def random_unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform rotations: a normalised 4-D standard normal is uniform on S^3."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _rotate_by_quat(q: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Rotate vectors v (n,3) by unit quaternions q (n,4) [w,x,y,z] with the
    vector form of q v q*:  v + 2w (r x v) + 2 r x (r x v),  r = (x,y,z).

    Used only to place Gaussian means inside their cell while drawing inputs.
    """
    w = q[:, :1]
    r = q[:, 1:]
    c1 = np.cross(r, v)
    return v + 2.0 * w * c1 + 2.0 * np.cross(r, c1)


def uniform_in_ball(rng: np.random.Generator, n: int) -> np.ndarray:
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = rng.random(n) ** (1.0 / 3.0)
    return d * r[:, None]


def log_uniform(rng: np.random.Generator, lo: float, hi: float, shape) -> np.ndarray:
    return np.exp(rng.uniform(math.log(lo), math.log(hi), shape))


# ----------------------------------------------------------------------------
# scenes


def make_scene(n_cells: int, K: int, centers_fn, axes_lo: float, axes_hi: float,
               sh_degree: int, seed: int, higher_band_std: float = 0.2,
               name: str = "") -> Scene:
    """Cell proxies plus K Gaussians per cell, drawn in this fixed order:

    1. centres (centers_fn), 2. cell semi-axes log-uniform [axes_lo, axes_hi],
    3. cell quaternions, 4. Gaussian positions uniform in the cell ellipsoid,
    5. Gaussian scales log-normal(mu = log(0.3 * cell axis), sigma = 0.3) per
       axis, 6. Gaussian quaternions, 7. opacity logits N(0,1) (so opacity is
       sigmoid(N(0,1))), 8. base colour u uniform [0,1] -> DC coefficient
       (u - 0.5) / Y_00, 9. higher SH bands N(0, higher_band_std).
    Cell calibration scalars v_n are 1.
    """
    rng = np.random.default_rng(seed)
    N, G = n_cells, n_cells * K
    center = centers_fn(rng, N)
    axes = log_uniform(rng, axes_lo, axes_hi, (N, 3))
    cq = random_unit_quats(rng, N)
    u = uniform_in_ball(rng, G)
    cell_of = np.repeat(np.arange(N), K)
    local = u * axes[cell_of]
    mean = center[cell_of] + _rotate_by_quat(cq[cell_of], local)
    scale = np.exp(rng.normal(np.log(0.3 * axes[cell_of]), 0.3))
    gq = random_unit_quats(rng, G)
    logit = rng.standard_normal(G)
    nco = (sh_degree + 1) ** 2
    sh = np.zeros((G, nco, 3), dtype=np.float32)
    base = rng.random((G, 3))
    sh[:, 0, :] = ((base - 0.5) * _INV_Y00).astype(np.float32)
    if nco > 1:
        sh[:, 1:, :] = rng.standard_normal((G, nco - 1, 3), dtype=np.float32) * np.float32(higher_band_std)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Scene(K=K, sh_degree=sh_degree,
                 cell_center=f32(center), cell_axes=f32(axes), cell_quat=f32(cq),
                 cell_v=np.ones(N, dtype=np.float32),
                 g_mean=f32(mean), g_scale=f32(scale), g_quat=f32(gq),
                 g_logit=f32(logit), g_sh=np.ascontiguousarray(sh), name=name,
                 meta=dict(seed=seed, n_cells=N, K=K))


def with_view_dependent_v(scene: Scene, degree: int = 2, seed: int = 0, base: float = 0.8,
                          band_std: float = 0.15) -> Scene:
    """A copy of `scene` whose calibration v_n is given by real SH
    coefficients of the given degree: DC = base / Y_00 (so v is `base` with
    no view dependence), higher bands N(0, band_std), drawn from `seed`."""
    import dataclasses
    rng = np.random.default_rng(seed)
    nco = (degree + 1) ** 2
    k = np.zeros((scene.N, nco), dtype=np.float32)
    k[:, 0] = np.float32(base * _INV_Y00)
    if nco > 1:
        k[:, 1:] = rng.standard_normal((scene.N, nco - 1), dtype=np.float32) * np.float32(band_std)
    return dataclasses.replace(scene, cell_v_sh=k, v_sh_degree=degree, name=scene.name + f"-vsh{degree}")


def neural_scene(n_cells: int = 2048, K: int = 10, F: int = 32, H: int = 32, seed: int = 0,
                  box: float = 1.0, axes_lo: float = 0.02, axes_hi: float = 0.1) -> Scene:
    """Neural cells: centres uniform in [-box, box]^3, semi-axes log-uniform,
    random unit quaternions, latent features N(0, 1), per-Gaussian offsets
    uniform in the unit ball, and random decoder weights (normal with
    standard deviation 1/sqrt(fan-in); output biases that give a mean opacity
    near tanh(1), colour near 0.5, scale ratios near 0.3 and rotations
    around the identity).  The explicit
    Gaussian arrays are placeholders (zeros): the renderer decodes the
    Gaussians of visible cells per view.  Draw order: centres, axes, cell
    quaternions, features, offsets, weights."""
    rng = np.random.default_rng(seed)
    N, G = n_cells, n_cells * K
    center = rng.uniform(-box, box, (N, 3))
    axes = log_uniform(rng, axes_lo, axes_hi, (N, 3))
    cq = random_unit_quats(rng, N)
    feat = rng.standard_normal((N, F))
    off = uniform_in_ball(rng, G)
    parts = []
    identity = np.tile([1.0, 0.0, 0.0, 0.0], K)
    for n_out, b_out in ((K, 1.0), (3 * K, 0.0), (3 * K, -0.85), (4 * K, identity)):
        W1 = rng.standard_normal((H, F + 4)) / np.sqrt(F + 4)
        b1 = np.zeros(H)
        W2 = rng.standard_normal((n_out, H)) / np.sqrt(H)
        b2 = np.broadcast_to(np.asarray(b_out, dtype=np.float64), (n_out,)).copy()
        parts += [W1.ravel(), b1, W2.ravel(), b2]
    mlp = np.concatenate(parts).astype(np.float32)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Scene(K=K, sh_degree=0, cell_center=f32(center), cell_axes=f32(axes), cell_quat=f32(cq),
                 cell_v=np.ones(N, dtype=np.float32), g_mean=np.zeros((G, 3), np.float32),
                 g_scale=np.zeros((G, 3), np.float32), g_quat=np.zeros((G, 4), np.float32),
                 g_logit=np.zeros(G, np.float32), g_sh=np.zeros((G, 1, 3), np.float32),
                 name=f"neural-{N}x{K}-F{F}H{H}", meta=dict(seed=seed, n_cells=N, K=K),
                 neural=dict(F=F, H=H, feat=f32(feat), offset=f32(off), mlp=mlp))


def _box(lo, hi):
    return lambda rng, n: rng.uniform(lo, hi, (n, 3))


def _ground_plane(rng, n):
    xy = rng.uniform(-200.0, 200.0, (n, 2))
    z = np.abs(rng.normal(0.0, 5.0, n))
    return np.concatenate([xy, z[:, None]], axis=1)


def scene_small(seed: int = 0, sh_degree: int = 0, n_cells: int = 2048, K: int = 8,
                higher_band_std: float = 0.2) -> Scene:
    """2,048 cells x 8 Gaussians in [-1,1]^3, semi-axes log-uniform [0.02, 0.1].

    sh_degree=0 gives the plain-RGB scene; sh_degree=3 keeps the same draws
    for the base colour (as DC) and adds higher bands N(0, 0.2).
    """
    return make_scene(n_cells, K, _box(-1.0, 1.0), 0.02, 0.1, sh_degree, seed,
                      higher_band_std, name=f"small-{n_cells}x{K}-sh{sh_degree}")


def scene_multiscale(seed: int = 0, n_cells: int = 100_000, K: int = 10) -> Scene:
    """100,000 cells x 10 Gaussians in [-10,10]^3, semi-axes log-uniform over
    three decades [0.001, 1], SH degree 3 (the multi-scale workload)."""
    return make_scene(n_cells, K, _box(-10.0, 10.0), 0.001, 1.0, 3, seed,
                      name=f"multiscale-{n_cells}x{K}")


def scene_large(seed: int = 0, n_cells: int = 1_000_000, K: int = 10) -> Scene:
    """1,000,000 cells x 10 Gaussians on a ground-plane-heavy layout
    (x, y uniform [-200,200], z half-normal sigma 5), semi-axes log-uniform
    [0.01, 2], SH degree 3 (the large-scale workload)."""
    return make_scene(n_cells, K, _ground_plane, 0.01, 2.0, 3, seed,
                      name=f"large-{n_cells}x{K}")


# ----------------------------------------------------------------------------
# cameras


def look_at_from_pose(R: np.ndarray, eye: np.ndarray, W: int, H: int,
                      fov_y_deg: float = 60.0, znear: float = 0.2) -> Camera:
    R64 = np.asarray(R, dtype=np.float64)
    eye64 = np.asarray(eye, dtype=np.float64)
    t = -R64 @ eye64
    fy = (H / 2.0) / math.tan(math.radians(fov_y_deg) / 2.0)
    return Camera(W=W, H=H, fx=float(np.float32(fy)), fy=float(np.float32(fy)),
                  cx=W / 2.0, cy=H / 2.0, znear=znear,
                  R=R64.astype(np.float32), t=t.astype(np.float32),
                  eye=eye64.astype(np.float32))


def look_at(eye, target, W: int, H: int, fov_y_deg: float = 60.0,
            up=(0.0, 0.0, 1.0), znear: float = 0.2) -> Camera:
    """Pinhole camera at `eye` looking at `target`; rows of R are the view
    axes (right, down, forward)."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    up = np.asarray(up, dtype=np.float64)
    if abs(float(np.dot(f, up))) > 0.99:
        up = np.array([0.0, 1.0, 0.0])
    r = np.cross(f, up)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    return look_at_from_pose(R, eye, W, H, fov_y_deg, znear)


def sphere_cameras(n: int, radius: float, W: int, H: int, seed0: int = 0,
                   fov_y_deg: float = 60.0) -> list[Camera]:
    """Camera i sits at radius * (unit direction drawn with seed seed0 + i),
    looking at the origin."""
    cams = []
    for i in range(n):
        rng = np.random.default_rng(seed0 + i)
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        cams.append(look_at(radius * d, (0.0, 0.0, 0.0), W, H, fov_y_deg))
    return cams


def street_cameras(n: int, W: int, H: int, seed0: int = 0,
                   fov_y_deg: float = 60.0) -> list[Camera]:
    """Street-level cameras: eye at z = 2 with x, y uniform [-150,150], a
    random yaw and zero pitch (camera i drawn with seed seed0 + i)."""
    cams = []
    for i in range(n):
        rng = np.random.default_rng(seed0 + i)
        x, y = rng.uniform(-150.0, 150.0, 2)
        yaw = rng.uniform(0.0, 2.0 * math.pi)
        eye = np.array([x, y, 2.0])
        tgt = eye + np.array([math.cos(yaw), math.sin(yaw), 0.0])
        cams.append(look_at(eye, tgt, W, H, fov_y_deg))
    return cams


def small_camera(W: int = 256, H: int = 256) -> Camera:
    """The small-scene camera: 60 deg vertical FOV at (0,-3,0) looking at the
    origin with +z up."""
    return look_at((0.0, -3.0, 0.0), (0.0, 0.0, 0.0), W, H, 60.0)


def target_image(n_views: int, H: int, W: int, seed: int = 1234) -> np.ndarray:
    """Seeded L1 target images, float32 [V][3][H][W] uniform [0,1]."""
    rng = np.random.default_rng(seed)
    return rng.random((n_views, 3, H, W), dtype=np.float32)
