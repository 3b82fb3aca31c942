"""Seeded synthetic scenes and cameras for the 4D-GS render path.

This module only draws inputs: canonical Gaussians, HexPlane grids, deformation
MLP weights and pinhole cameras.  It holds none of the method's arithmetic (no
sampling, no MLP, no projection, no compositing), so both the FP64 CPU oracle
and the CUDA path can consume exactly the same arrays.

Every array is float32 (the precision the scene is stored in); both sides read
the same rounded values.

Layouts (shared contract, restated independently by each consumer):
  means          [N][3]           canonical centres X (Sec. 3.1)
  log_scales     [N][3]           s, with scale = exp(s)
  quats          [N][4]           r as (w, x, y, z), not necessarily unit
  opacity_logits [N]              opacity = sigmoid(logit)
  sh             [N][K][3]        K = (deg+1)^2 real-SH coefficients per channel
  planes         flat float32     for level l, plane p in (xy, xz, yz, xt, yt, zt):
                                  [R_b][R_a][h] channels-last, where (a, b) are the
                                  plane's two axes; spatial axes have resolution
                                  res_spatial[l], the time axis res_time
  mlp            flat float32     layers d1, d2, x1, x2, r1, r2, s1, s2; each is
                                  weight [out][in] row-major followed by bias [out]

The distributions follow the workload descriptions of the five benchmark
configurations (tiny 2k-Gaussian scene; 100k D-NeRF-shaped object; 300k
real-scene-shaped box; the serving mix; the 2M stress scene).  The datasets the
paper measures on (D-NeRF, HyperNeRF, Neu3D) are not available, so these
seeded scenes stand in for them.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

PLANE_AXES = ((0, 1), (0, 2), (1, 2), (0, 3), (1, 3), (2, 3))  # xy xz yz xt yt zt; 3 = t
HEAD_OUT = (3, 4, 3)  # delta position, delta rotation, delta log-scale

# Real SH degree-0 constant 1/(2 sqrt(pi)); used only to place DC colours in [0,1].
_SH_C0 = 0.28209479177387814


@dataclasses.dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    sh_degree: int
    aabb_min: Tuple[float, float, float]
    aabb_max: Tuple[float, float, float]
    res_spatial: Tuple[int, ...]
    res_time: int
    feat_dim: int
    planes: np.ndarray
    mlp_width: int
    mlp: np.ndarray
    color_heads: bool = False  # the mlp also holds the colour and opacity heads (App. B)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def n_levels(self) -> int:
        return len(self.res_spatial)

    def copy(self) -> "Scene":
        return dataclasses.replace(
            self, **{f.name: (getattr(self, f.name).copy() if isinstance(getattr(self, f.name), np.ndarray)
                              else getattr(self, f.name)) for f in dataclasses.fields(self)})


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    znear: float
    world_to_cam: np.ndarray  # [4][4] float32 row-major; camera x right, y down, z forward


def plane_shapes(res_spatial: Sequence[int], res_time: int, h: int) -> List[Tuple[int, int, int]]:
    """(R_b, R_a, h) of every plane in packing order: level-major, then xy xz yz xt yt zt."""
    out = []
    for r in res_spatial:
        for a, b in PLANE_AXES:
            ra = r if a < 3 else res_time
            rb = r if b < 3 else res_time
            out.append((rb, ra, h))
    return out


def mlp_layer_shapes(in_dim: int, width: int, color_k: int = 0) -> List[Tuple[int, int]]:
    """(out, in) of the eight linear layers d1 d2 x1 x2 r1 r2 s1 s2, and with
    color_k = K > 0 SH coefficients per channel the colour and opacity heads' four
    (c1 c2 a1 a2: W -> W -> 3K and W -> W -> 1) after them."""
    shapes = [(width, in_dim), (width, width)]
    for o in HEAD_OUT:
        shapes += [(width, width), (o, width)]
    if color_k:
        shapes += [(width, width), (3 * color_k, width), (width, width), (1, width)]
    return shapes


def with_color_heads(scene: Scene, seed: int, std: float = 0.05, bias_std: float = 0.05) -> Scene:
    """A copy of `scene` with colour and opacity heads (App. B) appended to its MLP:
    weights N(0, std), biases N(0, bias_std)."""
    rng = np.random.default_rng(seed)
    width = scene.mlp_width
    k = (scene.sh_degree + 1) ** 2
    parts = [scene.mlp.astype(np.float32)]
    for o, i in mlp_layer_shapes(width, width, k)[8:]:
        parts.append(rng.normal(0.0, std, size=(o, i)).astype(np.float32).ravel())
        parts.append(rng.normal(0.0, bias_std, size=o).astype(np.float32))
    out = scene.copy()
    out.mlp = np.concatenate(parts)
    out.color_heads = True
    return out


def _unit_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    # A normalised 4-D standard normal is uniform on S^3.
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _planes(rng, res_spatial, res_time, h, mean=1.0, std=0.1) -> np.ndarray:
    parts = [rng.normal(mean, std, size=s).astype(np.float32) for s in plane_shapes(res_spatial, res_time, h)]
    return np.concatenate([p.ravel() for p in parts])


def _mlp(rng, in_dim, width, std=0.02, bias_std=0.0) -> np.ndarray:
    parts = []
    for o, i in mlp_layer_shapes(in_dim, width):
        parts.append(rng.normal(0.0, std, size=(o, i)).astype(np.float32).ravel())
        if bias_std > 0:
            parts.append(rng.normal(0.0, bias_std, size=o).astype(np.float32))
        else:
            parts.append(np.zeros(o, np.float32))  # biases are not specified: zero
    return np.concatenate(parts)


def _sh_from_rgb(rng, rgb: np.ndarray, degree: int, rest_std: float) -> np.ndarray:
    k = (degree + 1) ** 2
    sh = np.zeros((rgb.shape[0], k, 3), np.float64)
    sh[:, 0, :] = (rgb - 0.5) / _SH_C0  # DC term so that colour = rgb before view dependence
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, rest_std, size=(rgb.shape[0], k - 1, 3))
    return sh.astype(np.float32)


def make_tiny(seed: int = 0, n: int = 2000, mlp_std: float = 0.02, plane_std: float = 0.1,
              bias_std: float = 0.0) -> Scene:
    """Tiny FP32 scene: N=2000, means U[-1,1]^3, log-scales N(-4,0.5), SH degree 0,
    single-resolution HexPlane (spatial 32, temporal 8, h=16, values N(1,0.1)),
    MLP 16->64->64 with three heads, weights N(0,0.02)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, (n, 3)).astype(np.float32)
    log_scales = rng.normal(-4.0, 0.5, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    opacity = rng.normal(0.0, 1.0, n).astype(np.float32)
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    sh = _sh_from_rgb(rng, rgb, 0, 0.0)
    res_spatial, res_time, h, width = (32,), 8, 16, 64
    planes = _planes(rng, res_spatial, res_time, h, std=plane_std)
    mlp = _mlp(rng, h * len(res_spatial), width, std=mlp_std, bias_std=bias_std)
    return Scene(means, log_scales, quats, opacity, sh, 0, (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0),
                 res_spatial, res_time, h, planes, width, mlp)


def _gmm_points(rng, n, n_comp, centre_lo, centre_hi, std, centre_ok, inside) -> np.ndarray:
    centres = []
    while len(centres) < n_comp:
        c = rng.uniform(centre_lo, centre_hi)
        if centre_ok(c[None])[0]:
            centres.append(c)
    centres = np.array(centres)
    out = np.empty((0, 3))
    while out.shape[0] < n:
        comp = rng.integers(0, n_comp, size=2 * n)
        pts = centres[comp] + rng.normal(0.0, std, (2 * n, 3))
        out = np.concatenate([out, pts[inside(pts)]])
    return out[:n].astype(np.float32)


def make_object(seed: int = 0, n: int = 100_000, res_spatial=(64, 128), res_time: int = 25, h: int = 32,
                width: int = 64, sh_degree: int = 3, log_scale_mean: float = -4.0,
                mlp_std: float = 0.02) -> Scene:
    """D-NeRF-shaped object: N Gaussians from a 32-component isotropic mixture
    (component means uniform in the ball of radius 0.7, std 0.15) restricted to
    the unit sphere; SH degree 3; HexPlane spatial {64,128}, temporal 25, h=32."""
    rng = np.random.default_rng(seed)
    in_ball = lambda p: np.linalg.norm(p, axis=1) <= 1.0
    in_small = lambda p: np.linalg.norm(p, axis=1) <= 0.7
    means = _gmm_points(rng, n, 32, (-0.7,) * 3, (0.7,) * 3, 0.15, in_small, in_ball)
    log_scales = rng.normal(log_scale_mean, 0.5, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    opacity = rng.normal(0.0, 1.0, n).astype(np.float32)
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    sh = _sh_from_rgb(rng, rgb, sh_degree, 0.05)
    planes = _planes(rng, tuple(res_spatial), res_time, h)
    mlp = _mlp(rng, h * len(res_spatial), width, std=mlp_std)
    return Scene(means, log_scales, quats, opacity, sh, sh_degree, (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0),
                 tuple(res_spatial), res_time, h, planes, width, mlp)


def make_room(seed: int = 0, n: int = 300_000, res_spatial=(64, 128), res_time: int = 150, h: int = 32,
              width: int = 64) -> Scene:
    """Real-scene-shaped box: N Gaussians in a 64-cluster mixture spread across a
    6x4x6 box centred on the origin, SH degree 3, temporal resolution 150."""
    rng = np.random.default_rng(seed)
    lo, hi = np.array([-3.0, -2.0, -3.0]), np.array([3.0, 2.0, 3.0])
    inside = lambda p: np.all((p >= lo) & (p <= hi), axis=1)
    means = _gmm_points(rng, n, 64, lo, hi, 0.35, inside, inside)
    log_scales = rng.normal(-3.5, 0.5, (n, 3)).astype(np.float32)
    quats = _unit_quats(rng, n)
    opacity = rng.normal(0.0, 1.0, n).astype(np.float32)
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    sh = _sh_from_rgb(rng, rgb, 3, 0.05)
    planes = _planes(rng, tuple(res_spatial), res_time, h)
    mlp = _mlp(rng, h * len(res_spatial), width)
    return Scene(means, log_scales, quats, opacity, sh, 3, tuple(lo), tuple(hi),
                 tuple(res_spatial), res_time, h, planes, width, mlp)


def make_stress(seed: int = 0, n: int = 2_000_000) -> Scene:
    """Stress scene: N=2M, inflated log-scales N(-2.5,0.5), HexPlane spatial
    {64,128,256}, temporal 300, h=32."""
    return make_object(seed, n, res_spatial=(64, 128, 256), res_time=300, log_scale_mean=-2.5)


def perturb_planes(scene: Scene, seed: int, std: float = 0.01) -> Scene:
    s = scene.copy()
    rng = np.random.default_rng(10_000 + seed)
    s.planes = (s.planes + rng.normal(0.0, std, s.planes.shape)).astype(np.float32)
    return s


# ----------------------------------------------------------------------------- cameras

def look_at(eye, target, up, width, height, fov_deg, znear=0.2) -> Camera:
    """Pinhole camera at `eye` looking at `target`; image x right, y down, z forward."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, np.float64))  # right = forward x up (y points down)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    rot = np.stack([x, y, z])
    m = np.eye(4)
    m[:3, :3] = rot
    m[:3, 3] = -rot @ eye
    f = width / (2.0 * math.tan(math.radians(fov_deg) / 2.0))
    return Camera(width, height, f, f * 1.0, width / 2.0, height / 2.0, znear, m.astype(np.float32))


def tiny_camera(width: int = 128, height: int = 128) -> Camera:
    """Camera at (0,-4,0) looking at the origin along +y, world +z up, 50 deg FOV."""
    return look_at((0.0, -4.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), width, height, 50.0)


def hemisphere_cameras(n: int, radius: float = 4.0, width: int = 800, height: int = 800,
                       fov_deg: float = 50.0, seed: int = 0) -> List[Camera]:
    """Fibonacci-spaced cameras on the upper hemisphere (z >= 0), looking at the origin."""
    rng = np.random.default_rng(seed)
    phase = rng.uniform(0, 2 * math.pi)
    golden = math.pi * (3.0 - math.sqrt(5.0))
    cams = []
    for i in range(n):
        z = (i + 0.5) / n * 0.95
        r = math.sqrt(1.0 - z * z)
        a = phase + golden * i
        eye = (radius * r * math.cos(a), radius * r * math.sin(a), radius * z)
        cams.append(look_at(eye, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0), width, height, fov_deg))
    return cams


def forward_cameras(n: int, width: int = 1352, height: int = 1014, fov_deg: float = 60.0,
                    seed: int = 0) -> List[Camera]:
    """Forward-facing cameras for the box scene: eyes jittered around (0,-5.5,0.3),
    looking towards the box centre."""
    rng = np.random.default_rng(seed)
    cams = []
    for _ in range(n):
        eye = np.array([0.0, -5.5, 0.3]) + rng.uniform(-0.6, 0.6, 3) * np.array([1.0, 0.3, 1.0])
        target = rng.uniform(-0.3, 0.3, 3)
        cams.append(look_at(eye, target, (0.0, 0.0, 1.0), width, height, fov_deg))
    return cams
