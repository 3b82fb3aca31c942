"""FP64 CPU oracle for the 4D-GS render path -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path and
never imports it; it accepts any scene/camera object with the attributes of the
seeded input generator (duck typing), and returns numpy float64 arrays.

The arithmetic lives in ``fs4d_oracle.cpp`` (plain loops in double precision,
each function citing the passage of the paper it follows).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict

import numpy as np

from . import build as _build

_lib = None

F32P = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
F64P = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
I32P = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
I64P = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
U32P = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
U64P = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")


class OrcScene(C.Structure):
    _fields_ = [("n", C.c_int32), ("sh_degree", C.c_int32),
                ("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p),
                ("aabb_min", C.c_double * 3), ("aabb_max", C.c_double * 3),
                ("n_levels", C.c_int32), ("res_spatial", C.c_int32 * 4), ("res_time", C.c_int32),
                ("feat_dim", C.c_int32), ("planes", C.c_void_p), ("mlp_width", C.c_int32),
                ("mlp", C.c_void_p), ("color_heads", C.c_int32)]


class OrcCamera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("znear", C.c_double),
                ("world_to_cam", C.c_double * 16)]


class OrcProjected(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("xy", "conic", "cov2d", "opacity", "rgb", "depth", "radius", "rect",
                                          "margin")]


class OrcGrads(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "planes",
                                          "mlp", "planes_abs", "planes_sens", "xy")]


def lib():
    global _lib
    if _lib is None:
        # FS4D_ORACLE_LIB names another build of fs4d_oracle.cpp; the planted-mistake
        # test uses it to run the pins against copies of the oracle with one error each.
        path = os.environ.get("FS4D_ORACLE_LIB") or _build.build()
        L = C.CDLL(path)
        L.orc_set_threads.argtypes = [C.c_int32]
        L.orc_plane_sample.argtypes = [C.POINTER(OrcScene), C.c_int32, C.c_int32, C.c_double, C.c_double, F64P]
        L.orc_features.argtypes = [C.POINTER(OrcScene), F64P, C.c_int32, C.c_double, F64P]
        L.orc_mlp.argtypes = [C.POINTER(OrcScene), F64P, C.c_int32, F64P]
        L.orc_deform.argtypes = [C.POINTER(OrcScene), C.c_double, F64P, F64P, F64P]
        L.orc_sh_basis.argtypes = [C.c_int32, F64P, F64P]
        L.orc_project.argtypes = [C.POINTER(OrcScene), F64P, F64P, F64P, C.POINTER(OrcCamera), C.c_int32,
                                  C.POINTER(OrcProjected)]
        L.orc_project_appearance.argtypes = [C.POINTER(OrcScene), F64P, F64P, F64P, F64P, F64P,
                                             C.POINTER(OrcCamera), C.c_int32, C.POINTER(OrcProjected)]
        L.orc_appearance.argtypes = [C.POINTER(OrcScene), C.c_double, F64P, F64P]
        L.orc_bin_sort.argtypes = [C.c_int32, U32P, I32P, C.c_int32, C.c_int32, C.c_int64, U64P, U32P, U32P]
        L.orc_bin_sort.restype = C.c_int64
        L.orc_composite.argtypes = [C.c_int32, C.c_int32, C.c_int32, U32P, U32P, F64P, F64P, F64P, F64P, F64P,
                                    F64P, F64P, I32P, F64P]
        L.orc_composite_bruteforce.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, I32P, I32P, F64P,
                                               F64P, F64P, F64P, F64P, F64P, F64P]
        L.orc_pixel_outcomes.argtypes = [C.c_int32, U32P, C.c_double, C.c_double, F64P, F64P, F64P, F64P, F64P,
                                         C.c_double, C.c_double, C.c_int32, C.c_int32, F64P]
        L.orc_pixel_outcomes.restype = C.c_int32
        L.orc_render.argtypes = [C.POINTER(OrcScene), C.POINTER(OrcCamera), C.c_double, C.c_int32, C.c_int32,
                                 F64P, F64P, I32P, F64P]
        L.orc_render.restype = C.c_int64
        L.orc_render_backward.argtypes = [C.POINTER(OrcScene), C.POINTER(OrcCamera), C.c_double, C.c_int32,
                                          C.c_int32, F64P, C.POINTER(OrcGrads)]
        L.orc_render_backward.restype = C.c_int32
        L.orc_l1_loss.argtypes = [C.c_int64, F64P, F64P, C.c_void_p]
        L.orc_l1_loss.restype = C.c_double
        L.orc_tv_loss.argtypes = [C.POINTER(OrcScene), C.c_double, C.c_void_p]
        L.orc_tv_loss.restype = C.c_double
        L.orc_lr.argtypes = [C.c_double, C.c_double, C.c_int64, C.c_int64]
        L.orc_lr.restype = C.c_double
        L.orc_adam_step.argtypes = [C.c_int64, F64P, F64P, F64P, F64P, C.c_double, C.c_double, C.c_double,
                                    C.c_double, C.c_int64]
        L.orc_densify.argtypes = [C.POINTER(OrcScene), F32P, F32P, F32P, C.c_float, C.c_float, C.c_float, C.c_int64,
                                  I64P, I32P, F64P, F64P, F64P, F64P, F64P]
        L.orc_densify.restype = C.c_int64
        _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


class _SceneHandle:
    """Keeps the float32 arrays alive while the C struct points at them."""

    def __init__(self, scene):
        self.arrays = {k: _f32(getattr(scene, k)) for k in ("means", "log_scales", "quats", "opacity_logits",
                                                             "sh", "planes", "mlp")}
        s = OrcScene()
        s.n = int(self.arrays["means"].shape[0])
        s.sh_degree = int(scene.sh_degree)
        for k, v in self.arrays.items():
            setattr(s, k, v.ctypes.data)
        s.aabb_min = (C.c_double * 3)(*[float(v) for v in scene.aabb_min])
        s.aabb_max = (C.c_double * 3)(*[float(v) for v in scene.aabb_max])
        rs = list(scene.res_spatial)
        s.n_levels = len(rs)
        s.res_spatial = (C.c_int32 * 4)(*(rs + [0] * (4 - len(rs))))
        s.res_time = int(scene.res_time)
        s.feat_dim = int(scene.feat_dim)
        s.mlp_width = int(scene.mlp_width)
        s.color_heads = int(bool(getattr(scene, "color_heads", False)))
        self.struct = s
        self.n = s.n
        self.hin = s.feat_dim * s.n_levels
        self.k = (s.sh_degree + 1) ** 2


def _camera(cam) -> OrcCamera:
    c = OrcCamera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy, c.znear = (float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy),
                                       float(cam.znear))
    c.world_to_cam = (C.c_double * 16)(*[float(v) for v in np.asarray(cam.world_to_cam, np.float64).ravel()])
    return c


def plane_sample(scene, level: int, plane: int, ua: float, ub: float) -> np.ndarray:
    h = _SceneHandle(scene)
    out = np.zeros(int(scene.feat_dim), np.float64)
    lib().orc_plane_sample(C.byref(h.struct), level, plane, ua, ub, out)
    return out


def features(scene, xyz: np.ndarray, t: float) -> np.ndarray:
    h = _SceneHandle(scene)
    xyz = np.ascontiguousarray(xyz, np.float64)
    n = xyz.shape[0]
    out = np.zeros((n, h.hin), np.float64)
    lib().orc_features(C.byref(h.struct), xyz, n, float(t), out)
    return out


def mlp(scene, fh: np.ndarray) -> np.ndarray:
    h = _SceneHandle(scene)
    fh = np.ascontiguousarray(fh, np.float64)
    out = np.zeros((fh.shape[0], 10), np.float64)
    lib().orc_mlp(C.byref(h.struct), fh, fh.shape[0], out)
    return out


def deform(scene, t: float):
    """Eq. 6 deformed (means, quats, log_scales), float64."""
    h = _SceneHandle(scene)
    X = np.zeros((h.n, 3)); Q = np.zeros((h.n, 4)); S = np.zeros((h.n, 3))
    lib().orc_deform(C.byref(h.struct), float(t), X, Q, S)
    return X, Q, S


_deform_fn = deform


def sh_basis(degree: int, direction) -> np.ndarray:
    out = np.zeros(16, np.float64)
    lib().orc_sh_basis(int(degree), np.ascontiguousarray(direction, np.float64), out)
    return out[:(degree + 1) ** 2]


def appearance(scene, t: float):
    """App. B: (sh [n][K][3], opacity_logits [n]) after the colour and opacity heads
    at time t (float64; the scene's own values when it has no such heads)."""
    h = _SceneHandle(scene)
    sh = np.zeros((h.n, h.k, 3))
    lg = np.zeros(h.n)
    lib().orc_appearance(C.byref(h.struct), float(t), sh.reshape(-1), lg)
    return sh, lg


def project(scene, cam, means=None, quats=None, log_scales=None, tile: int = 16, sh=None,
            opacity_logits=None) -> Dict[str, np.ndarray]:
    """Eq. 2 / Eq. 3 and the SH colour; sh / opacity_logits (float64, e.g. from
    appearance()) replace the scene's."""
    h = _SceneHandle(scene)
    n = h.n
    X = np.ascontiguousarray(scene.means if means is None else means, np.float64)
    Q = np.ascontiguousarray(scene.quats if quats is None else quats, np.float64)
    S = np.ascontiguousarray(scene.log_scales if log_scales is None else log_scales, np.float64)
    out = dict(xy=np.zeros((n, 2)), conic=np.zeros((n, 3)), cov2d=np.zeros((n, 3)), opacity=np.zeros(n),
               rgb=np.zeros((n, 3)), depth=np.zeros(n), radius=np.zeros(n, np.int32),
               rect=np.zeros((n, 4), np.int32), margin=np.zeros(n))
    P = OrcProjected(**{k: v.ctypes.data for k, v in out.items()})
    cc = _camera(cam)
    if sh is None and opacity_logits is None:
        lib().orc_project(C.byref(h.struct), X, Q, S, C.byref(cc), int(tile), C.byref(P))
    else:
        shd = np.ascontiguousarray(scene.sh if sh is None else sh, np.float64).reshape(-1)
        lgd = np.ascontiguousarray(scene.opacity_logits if opacity_logits is None else opacity_logits, np.float64)
        lib().orc_project_appearance(C.byref(h.struct), X, Q, S, shd, lgd, C.byref(cc), int(tile), C.byref(P))
    return out


def bin_sort(depth_bits: np.ndarray, rect: np.ndarray, tiles_x: int, tiles_y: int):
    """(keys, values, ranges) of the tile binning and (tile, depth, index) sort."""
    depth_bits = np.ascontiguousarray(depth_bits, np.uint32)
    rect = np.ascontiguousarray(rect, np.int32)
    n = depth_bits.shape[0]
    w = np.maximum(rect[:, 2] - rect[:, 0], 0).astype(np.int64)
    hgt = np.maximum(rect[:, 3] - rect[:, 1], 0).astype(np.int64)
    K = int((w * hgt).sum())
    keys = np.zeros(max(K, 1), np.uint64)
    values = np.zeros(max(K, 1), np.uint32)
    ranges = np.zeros(2 * tiles_x * tiles_y, np.uint32)
    k2 = lib().orc_bin_sort(n, depth_bits, rect, tiles_x, tiles_y, K, keys, values, ranges)
    assert k2 == K
    return keys[:K], values[:K], ranges.reshape(tiles_y * tiles_x, 2)


def depth_bits(depth: np.ndarray) -> np.ndarray:
    """float32 bit pattern of each depth: the key decision is taken in float32."""
    return np.ascontiguousarray(depth, np.float64).astype(np.float32).view(np.uint32)


def composite(cam_w: int, cam_h: int, ranges, values, proj, tile: int = 16):
    n_pix = cam_w * cam_h
    img = np.zeros((cam_h, cam_w, 3)); T = np.zeros((cam_h, cam_w)); nc = np.zeros((cam_h, cam_w), np.int32)
    mg = np.zeros((cam_h, cam_w))
    vals = np.ascontiguousarray(values, np.uint32)
    if vals.size == 0:
        vals = np.zeros(1, np.uint32)
    lib().orc_composite(cam_w, cam_h, tile, np.ascontiguousarray(ranges, np.uint32).ravel(), vals,
                        proj["xy"], proj["conic"], proj["opacity"], proj["rgb"], proj["depth"], img, T, nc, mg)
    del n_pix
    return img, T, nc, mg


def composite_bruteforce(cam_w: int, cam_h: int, proj, tile: int = 16):
    n = proj["depth"].shape[0]
    img = np.zeros((cam_h, cam_w, 3)); T = np.zeros((cam_h, cam_w))
    lib().orc_composite_bruteforce(n, cam_w, cam_h, tile, proj["radius"], proj["rect"], proj["xy"],
                                   proj["conic"], proj["opacity"], proj["rgb"], proj["depth"], img, T)
    return img, T


def render(scene, cam, t: float, deform: bool = True, tile: int = 16):
    """Full frame: (image [H][W][3], T_final [H][W], n_contrib [H][W], margin [H][W], K)."""
    h = _SceneHandle(scene)
    cc = _camera(cam)
    H, W = int(cam.height), int(cam.width)
    img = np.zeros((H, W, 3)); T = np.zeros((H, W)); nc = np.zeros((H, W), np.int32); mg = np.zeros((H, W))
    K = lib().orc_render(C.byref(h.struct), C.byref(cc), float(t), int(bool(deform)), int(tile), img, T, nc, mg)
    return img, T, nc, mg, int(K)


def project_composed(scenes, shifts, cam, t: float, deform: bool = True, tile: int = 16):
    """Composition (Sec. 5.4): G' = {G'_1, ..., G'_n}, every scene deformed at t by
    its own field, translated by its shift, and projected; the projected sets are
    concatenated in scene order (Gaussian index = offset of its scene + index)."""
    parts = []
    for scene, sh in zip(scenes, shifts if shifts is not None else [None] * len(scenes)):
        if deform:
            X, Q, S = _deform_fn(scene, t)
        else:
            X = np.array(scene.means, np.float64)
            Q = np.array(scene.quats, np.float64)
            S = np.array(scene.log_scales, np.float64)
        if sh is not None:
            X = X + np.asarray(sh, np.float64)[None, :]
        if deform and getattr(scene, "color_heads", False):
            shd, lgd = appearance(scene, t)
            parts.append(project(scene, cam, X, Q, S, tile=tile, sh=shd, opacity_logits=lgd))
        else:
            parts.append(project(scene, cam, X, Q, S, tile=tile))
    return {k: np.ascontiguousarray(np.concatenate([p[k] for p in parts])) for k in parts[0]}


def composite_projected(proj, cam, tile: int = 16):
    """Bin, sort and composite a projected set: (image, T, n_contrib, margin, values, ranges)."""
    tx, ty = (cam.width + tile - 1) // tile, (cam.height + tile - 1) // tile
    _, vals, ranges = bin_sort(depth_bits(proj["depth"]), proj["rect"], tx, ty)
    img, T, nc, mg = composite(cam.width, cam.height, ranges, vals, proj, tile=tile)
    return img, T, nc, mg, vals, ranges


def unstable_pixels(scene, cam, t: float, deform: bool = True, px_tol: float = 1e-3, margin_tol: float = 1e-5,
                    tile: int = 16):
    """Pixels whose value a float32 implementation may legitimately decide
    differently from this float64 oracle: (a) a blend decision (alpha vs 1/255,
    T vs 1e-4, a depth tie) within margin_tol of its threshold, or (b) a tile whose
    membership in some Gaussian's tile rectangle changes when that Gaussian's
    projected centre moves by up to px_tol pixels or its 3-sigma radius crosses
    the nearest integer.  Returns (mask [H][W] bool, image, T, n_contrib, K)."""
    img, T, nc, mg, K = render(scene, cam, t, deform=deform, tile=tile)
    if deform:
        X, Q, S = _deform_fn(scene, t)
        p = project(scene, cam, X, Q, S, tile=tile)
    else:
        p = project(scene, cam, tile=tile)
    H, W = int(cam.height), int(cam.width)
    ty, tx = (H + tile - 1) // tile, (W + tile - 1) // tile
    bad_tiles = np.zeros(ty * tx, bool)
    bad_tiles[list(uncertain_memberships(p, W, H, px_tol, tile).keys())] = True
    bad_tiles = bad_tiles.reshape(ty, tx)
    mask = np.kron(bad_tiles, np.ones((tile, tile), bool))[:H, :W] | (mg < margin_tol)
    return mask, img, T, nc, K


def pixel_outcomes(lst, px: int, py: int, proj, rel_tol: float = 5e-5, depth_tol: float = 1e-6,
                   max_flip: int = 6):
    """Every colour pixel (px, py)'s blend over the Gaussian list `lst` can take
    when its decisions within rounding of their thresholds (alpha vs 1/255, T vs
    1e-4 within rel_tol relative; blended depths within depth_tol relative) are
    taken either way: array [m][5] of (colour, final T, last contributor), row 0
    the blend as computed, or None when more than max_flip decisions are that
    close."""
    lst = np.ascontiguousarray(lst, np.uint32)
    if lst.size == 0:
        lst = np.zeros(1, np.uint32)
        n = 0
    else:
        n = int(lst.size)
    max_out = 1 << max_flip
    out = np.zeros((max_out, 5))
    m = lib().orc_pixel_outcomes(n, lst, float(px) + 0.5, float(py) + 0.5, proj["xy"], proj["conic"],
                                 proj["opacity"], proj["rgb"], proj["depth"], float(rel_tol), float(depth_tol),
                                 int(max_flip), max_out, out.reshape(-1))
    return None if m < 0 else out[:m]


def uncertain_memberships(proj, width: int, height: int, px_tol: float, tile: int = 16):
    """Tile memberships a float32 projection may decide differently: for every
    Gaussian whose rectangle or radius decision lies within px_tol pixels of its
    integer boundary, the tiles inside some but not all of the rectangles its
    centre (moved by up to px_tol) and its 3-sigma radius (rounded either way)
    give.  Returns {tile index: [Gaussian indices]}."""
    ty, tx = (height + tile - 1) // tile, (width + tile - 1) // tile
    out = {}

    def rect_of(u, v, r):
        x0 = min(tx, max(0, int(np.floor((u - r) / tile))))
        x1 = min(tx, max(0, int(np.floor((u + r) / tile)) + 1))
        y0 = min(ty, max(0, int(np.floor((v - r) / tile))))
        y1 = min(ty, max(0, int(np.floor((v + r) / tile)) + 1))
        return x0, y0, x1, y1

    for g in np.flatnonzero((proj["margin"] < px_tol) & (proj["radius"] > 0)):
        a, b, c = proj["cov2d"][g]
        mid = 0.5 * (a + c)
        r3 = 3.0 * np.sqrt(mid + np.sqrt(max(0.0, mid * mid - (a * c - b * b))))
        radii = {int(np.ceil(r3 - px_tol)), int(np.ceil(r3 + px_tol))}
        u0, v0 = proj["xy"][g]
        cover = np.zeros((ty, tx), int)
        n_cand = 0
        for r in radii:
            for du in (-px_tol, 0.0, px_tol):
                for dv in (-px_tol, 0.0, px_tol):
                    x0, y0, x1, y1 = rect_of(u0 + du, v0 + dv, r)
                    cover[y0:y1, x0:x1] += 1
                    n_cand += 1
        for yy, xx in zip(*np.nonzero((cover > 0) & (cover < n_cand))):
            out.setdefault(int(yy) * tx + int(xx), []).append(int(g))
    return out


def render_backward(scene, cam, t: float, dl_dimage: np.ndarray, deform: bool = True, tile: int = 16,
                    plane_terms: bool = False, xy: bool = False):
    """Gradients of sum(dl_dimage * image) w.r.t. every scene parameter (float64 dict).
    plane_terms: also 'planes_abs', per plane value the sum of the magnitudes of the
    per-Gaussian terms its gradient adds up, and 'planes_sens', the most a unit
    error in every Gaussian's output gradients (dX', dr', ds') can change it.
    xy: also 'xy', the [n][2] gradient of the projected means (pixel units)."""
    h = _SceneHandle(scene)
    cc = _camera(cam)
    g = dict(means=np.zeros((h.n, 3)), log_scales=np.zeros((h.n, 3)), quats=np.zeros((h.n, 4)),
             opacity_logits=np.zeros(h.n), sh=np.zeros((h.n, h.k, 3)),
             planes=np.zeros(h.arrays["planes"].shape[0]), mlp=np.zeros(h.arrays["mlp"].shape[0]))
    if plane_terms:
        g["planes_abs"] = np.zeros(h.arrays["planes"].shape[0])
        g["planes_sens"] = np.zeros(h.arrays["planes"].shape[0])
    if xy:
        g["xy"] = np.zeros((h.n, 2))
    G = OrcGrads(**{k: v.ctypes.data for k, v in g.items()})
    rc = lib().orc_render_backward(C.byref(h.struct), C.byref(cc), float(t), int(bool(deform)), int(tile),
                                   np.ascontiguousarray(dl_dimage, np.float64), C.byref(G))
    if rc != 0:
        raise RuntimeError(f"orc_render_backward failed: {rc}")
    return g


# ----------------------------------------------------------------- training step (Sec. 4.3, App. A)

def l1_loss(image, target):
    """Mean absolute difference over every pixel and channel, and its gradient."""
    a = np.ascontiguousarray(image, np.float64).ravel()
    b = np.ascontiguousarray(target, np.float64).ravel()
    g = np.zeros_like(a)
    loss = lib().orc_l1_loss(a.size, a, b, g.ctypes.data)
    return loss, g.reshape(np.shape(image))


def tv_loss(scene, weight: float):
    """Grid TV loss over the HexPlane planes and its gradient (planes layout)."""
    h = _SceneHandle(scene)
    g = np.zeros(h.arrays["planes"].shape[0])
    loss = lib().orc_tv_loss(C.byref(h.struct), float(weight), g.ctypes.data)
    return loss, g


def lr_at(lr0: float, lr1: float, k: int, total: int) -> float:
    return lib().orc_lr(float(lr0), float(lr1), int(k), int(total))


def adam_step(param, grad, m, v, lr, beta1, beta2, eps, step):
    """In place on float64 arrays: one bias-corrected Adam update."""
    for a in (param, grad, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    lib().orc_adam_step(param.size, param.reshape(-1), grad.reshape(-1), m.reshape(-1), v.reshape(-1), float(lr),
                        float(beta1), float(beta2), float(eps), int(step))


GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh", "planes", "mlp")


def train_step(scene, cam, t: float, target, cfg, state, tile: int = 16):
    """One training step (Sec. 4.3): render the frame, L = |I^ - I| + L_tv, the
    gradient of L by the chain rule of the render (the backward above) plus the TV
    gradient on the planes, then one Adam update per parameter group at the step's
    decayed learning rate (App. A).  cfg: dict with 'lr' {group: (lr0, lr1)} ('sh'
    takes 'sh_dc' for the degree-0 coefficients and 'sh_rest' for the others),
    'total_steps', 'beta1', 'beta2', 'eps', 'tv_weight'.  state: dict with 'step'
    (updates done) and per-group float64 'm', 'v', 'param' (created on the first
    call from the scene).  Returns (l1, tv, gradient dict of this step); the
    updated parameters are in state['param']."""
    if "param" not in state:
        state["param"] = {k: np.array(getattr(scene, k), np.float64) for k in GROUPS}
        state["m"] = {k: np.zeros_like(v) for k, v in state["param"].items()}
        state["v"] = {k: np.zeros_like(v) for k, v in state["param"].items()}
        state["step"] = 0
    cur = scene.copy()
    for k in GROUPS:
        setattr(cur, k, state["param"][k].astype(np.float32))
    img, *_ = render(cur, cam, t, tile=tile)
    l1, dl = l1_loss(img, target)
    g = render_backward(cur, cam, t, dl, tile=tile)
    tv, gtv = tv_loss(cur, cfg["tv_weight"])
    g["planes"] = g["planes"] + gtv
    k = state["step"]
    step = k + 1
    for grp in GROUPS:
        p, m, v, gg = state["param"][grp], state["m"][grp], state["v"][grp], np.ascontiguousarray(g[grp], np.float64)
        if grp == "sh":
            dc = np.zeros(p.shape, bool)
            dc[:, 0, :] = True
            for part, key in ((dc, "sh_dc"), (~dc, "sh_rest")):
                lr = lr_at(*cfg["lr"][key], k, cfg["total_steps"])
                pp, mm, vv = p[part].copy(), m[part].copy(), v[part].copy()
                adam_step(pp, np.ascontiguousarray(gg[part]), mm, vv, lr, cfg["beta1"], cfg["beta2"], cfg["eps"],
                          step)
                p[part], m[part], v[part] = pp, mm, vv
        else:
            lr = lr_at(*cfg["lr"][grp], k, cfg["total_steps"])
            adam_step(p, gg, m, v, lr, cfg["beta1"], cfg["beta2"], cfg["eps"], step)
    state["step"] = step
    return l1, tv, g


# ----------------------------------------------------------------- densification and pruning (App. A)

DENSIFY_KINDS = ("kept", "copy", "first child", "second child")


def densify(scene, grad_sum, visible, normals, grad_threshold: float, split_log_scale: float, prune_logit: float):
    """Adaptive density control on the canonical Gaussians (orc_densify): returns a
    dict with the new float64 arrays (means, log_scales, quats, opacity_logits, sh)
    and, per output Gaussian, 'src' (source index) and 'kind' (0 kept, 1 copy,
    2 / 3 first / second child of a split).  The three decisions are taken in
    float32, on float32 statistics and thresholds."""
    h = _SceneHandle(scene)
    n = h.n
    cap = 2 * n + 1
    k = h.k
    out = dict(src=np.zeros(cap, np.int64), kind=np.zeros(cap, np.int32), means=np.zeros((cap, 3)),
               log_scales=np.zeros((cap, 3)), quats=np.zeros((cap, 4)), opacity_logits=np.zeros(cap),
               sh=np.zeros((cap, k, 3)))
    m = lib().orc_densify(C.byref(h.struct), np.ascontiguousarray(grad_sum, np.float32),
                          np.ascontiguousarray(visible, np.float32),
                          np.ascontiguousarray(normals, np.float32).reshape(-1),
                          np.float32(grad_threshold), np.float32(split_log_scale), np.float32(prune_logit), cap,
                          out["src"], out["kind"], out["means"], out["log_scales"], out["quats"],
                          out["opacity_logits"], out["sh"])
    if m < 0:
        raise RuntimeError("orc_densify: output capacity too small")
    return {key: v[:m] for key, v in out.items()}


def kind() -> str:
    return "oracle"


def default_threads() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
