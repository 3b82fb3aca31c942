"""Python binding of libfs4d.so (include/fs4d.h) -- argument marshalling only.

Every step of the render path runs in the library's CUDA kernels.  PyTorch is
used for device memory (output tensors) and streams.  There is no fallback: if
the library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Optional, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfs4d.so")

FP32, BF16 = 0, 1
BINNING_AUTO, BINNING_SORT, BINNING_BITMAP = 0, 1, 2
STATUS = {0: "FS4D_OK", 1: "FS4D_ERR_INVALID_ARG", 2: "FS4D_ERR_OOM", 3: "FS4D_ERR_CAPACITY",
          4: "FS4D_ERR_CUDA", 5: "FS4D_ERR_TIMEOUT", 6: "FS4D_ERR_NOT_FOUND", 7: "FS4D_ERR_UNIMPLEMENTED",
          8: "FS4D_ERR_CANCELLED", 9: "FS4D_ERR_CORRUPT"}

# Every symbol include/fs4d.h declares (checked by the tests against the .so).
EXPORTS = ("fs4d_create", "fs4d_destroy", "fs4d_last_error", "fs4d_set_stream", "fs4d_check_device_status",
           "fs4d_load_scene", "fs4d_unload_scene", "fs4d_update_scene", "fs4d_scene_bytes", "fs4d_deform", "fs4d_render",
           "fs4d_render_host", "fs4d_render_host_batch", "fs4d_reserve", "fs4d_render_async", "fs4d_render_backward", "fs4d_frame_free",
           "fs4d_frame_pairs", "fs4d_last_pairs", "fs4d_last_launches", "fs4d_set_binning", "fs4d_last_binning", "fs4d_set_stage_timing", "fs4d_stage_times", "fs4d_project",
           "fs4d_bin_sort", "fs4d_sort_pairs", "fs4d_sort_pairs_noalloc", "fs4d_sort_pairs_noalloc_status",
           "fs4d_composite", "fs4d_set_wait_limit", "fs4d_last_bands", "fs4d_set_band_pairs",
           "fs4d_train_create", "fs4d_train_step", "fs4d_train_losses", "fs4d_train_steps_done",
           "fs4d_train_destroy", "fs4d_read_scene", "fs4d_save_scene", "fs4d_load_scene_file",
           "fs4d_backward_times", "fs4d_render_composed", "fs4d_train_read_state", "fs4d_render_backward_stats",
           "fs4d_densify", "fs4d_train_stats", "fs4d_train_densify", "fs4d_check_canaries",
           "fs4d_debug_corrupt_canary")
STAGES = ("deform", "project", "depth_sort", "binning", "sort", "composite")


class Fs4dError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class SceneDesc(C.Structure):
    _fields_ = [("n", C.c_int32), ("sh_degree", C.c_int32), ("means", C.c_void_p), ("log_scales", C.c_void_p),
                ("quats", C.c_void_p), ("opacity_logits", C.c_void_p), ("sh", C.c_void_p),
                ("aabb_min", C.c_float * 3), ("aabb_max", C.c_float * 3), ("n_levels", C.c_int32),
                ("res_spatial", C.c_int32 * 4), ("res_time", C.c_int32), ("feat_dim", C.c_int32),
                ("planes", C.c_void_p), ("mlp_width", C.c_int32), ("mlp", C.c_void_p),
                ("color_heads", C.c_int32)]


class Camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("znear", C.c_float), ("world_to_cam", C.c_float * 16)]


class Projected(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("xy", "conic_opacity", "rgb", "depth", "radius", "rect")]


class TrainConfig(C.Structure):
    _fields_ = [("total_steps", C.c_int32)] + [(k, C.c_float * 2) for k in (
        "lr_means", "lr_log_scales", "lr_quats", "lr_opacity", "lr_sh_dc", "lr_sh_rest", "lr_planes", "lr_mlp")] + [
        ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float), ("tv_weight", C.c_float)]


# Learning rates of the training step: App. A gives the HexPlane (1.6e-3 -> 1.6e-4)
# and the MLP (1.6e-4 -> 1.6e-5); the Gaussian parameters follow the settings of
# 3D Gaussian Splatting that the paper says it follows.
TRAIN_DEFAULTS = dict(lr_means=(1.6e-4, 1.6e-6), lr_log_scales=(5e-3, 5e-3), lr_quats=(1e-3, 1e-3),
                      lr_opacity=(5e-2, 5e-2), lr_sh_dc=(2.5e-3, 2.5e-3), lr_sh_rest=(1.25e-4, 1.25e-4),
                      lr_planes=(1.6e-3, 1.6e-4), lr_mlp=(1.6e-4, 1.6e-5), beta1=0.9, beta2=0.999, eps=1e-15,
                      tv_weight=1e-4)


def train_config(total_steps: int, **kw) -> TrainConfig:
    v = dict(TRAIN_DEFAULTS)
    v.update(kw)
    cfg = TrainConfig()
    cfg.total_steps = int(total_steps)
    for k, x in v.items():
        if k.startswith("lr_"):
            getattr(cfg, k)[0], getattr(cfg, k)[1] = float(x[0]), float(x[1])
        else:
            setattr(cfg, k, float(x))
    return cfg


class Grads(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "planes", "mlp")]


class ViewStats(C.Structure):
    _fields_ = [("grad_norm_sum", C.c_void_p), ("visible", C.c_void_p)]


class DensifyConfig(C.Structure):
    _fields_ = [("grad_threshold", C.c_float), ("split_log_scale", C.c_float), ("prune_logit", C.c_float)]


_libs: Dict[str, object] = {}
LIB_DEBUG_PATH = os.path.join(HERE, "libfs4d_debug.so")


def library(path: str = LIB_PATH):
    """Load libfs4d.so (raises if it is missing: there is no CPU fallback); with
    path=LIB_DEBUG_PATH the FS4D_CHECK_BOUNDS build."""
    if path in _libs:
        return _libs[path]
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() (nvcc, sm_103a)")
    L = C.CDLL(path)
    vp, i32, i64, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_float
    sig = {
        "fs4d_create": [i32, vp, C.POINTER(vp)],
        "fs4d_destroy": [vp],
        "fs4d_set_stream": [vp, vp],
        "fs4d_check_device_status": [vp],
        "fs4d_set_wait_limit": [vp, C.c_uint32],
        "fs4d_load_scene": [vp, C.POINTER(SceneDesc), C.POINTER(i32)],
        "fs4d_unload_scene": [vp, i32],
        "fs4d_update_scene": [vp, i32, C.POINTER(SceneDesc), i32],
        "fs4d_scene_bytes": [vp, i32, i32, i32, f32, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)],
        "fs4d_deform": [vp, i32, i32, vp, i32, vp, vp, vp],
        "fs4d_render": [vp, i32, i32, C.POINTER(Camera), f32, vp, vp, vp, C.POINTER(vp)],
        "fs4d_render_host": [vp, i32, i32, C.POINTER(Camera), f32, vp],
        "fs4d_render_composed": [vp, C.POINTER(i32), C.POINTER(f32), i32, i32, C.POINTER(Camera), f32, vp, vp, vp],
        "fs4d_render_host_batch": [vp, i32, i32, C.POINTER(Camera), C.POINTER(f32), i32, C.POINTER(vp)],
        "fs4d_reserve": [vp, i32, i32, i32, i64],
        "fs4d_render_async": [vp, i32, i32, C.POINTER(Camera), vp, vp, vp],
        "fs4d_render_backward": [vp, vp, vp, C.POINTER(Grads)],
        "fs4d_frame_free": [vp, vp],
        "fs4d_frame_pairs": [vp, C.POINTER(i64)],
        "fs4d_last_pairs": [vp, C.POINTER(i64)],
        "fs4d_last_launches": [vp, C.POINTER(i64)],
        "fs4d_last_bands": [vp, C.POINTER(i32)],
        "fs4d_train_create": [vp, i32, C.POINTER(TrainConfig), C.POINTER(vp)],
        "fs4d_train_step": [vp, i32, C.POINTER(Camera), f32, vp, vp],
        "fs4d_train_losses": [vp, C.POINTER(f32)],
        "fs4d_train_steps_done": [vp, C.POINTER(i64)],
        "fs4d_train_destroy": [vp],
        "fs4d_train_read_state": [vp, i32, vp, vp],
        "fs4d_render_backward_stats": [vp, vp, vp, C.POINTER(Grads), C.POINTER(ViewStats)],
        "fs4d_densify": [vp, i32, C.POINTER(DensifyConfig), C.POINTER(ViewStats), vp, vp, C.POINTER(i64)],
        "fs4d_train_stats": [vp, C.POINTER(ViewStats)],
        "fs4d_train_densify": [vp, C.POINTER(DensifyConfig), vp, C.POINTER(i64)],
        "fs4d_read_scene": [vp, i32, C.POINTER(Grads), i32],
        "fs4d_save_scene": [vp, i32, C.c_char_p],
        "fs4d_load_scene_file": [vp, C.c_char_p, C.POINTER(i32)],
        "fs4d_set_band_pairs": [vp, i64],
        "fs4d_set_binning": [vp, i32],
        "fs4d_last_binning": [vp, C.POINTER(i32)],
        "fs4d_set_stage_timing": [vp, i32],
        "fs4d_stage_times": [vp, C.POINTER(C.c_float)],
        "fs4d_backward_times": [vp, C.POINTER(C.c_float)],
        "fs4d_project": [vp, i32, vp, vp, vp, vp, vp, i32, C.POINTER(Camera), C.POINTER(Projected)],
        "fs4d_bin_sort": [vp, i32, vp, vp, i32, i32, i64, vp, vp, vp, C.POINTER(i64)],
        "fs4d_sort_pairs": [vp, i64, i32, vp, vp],
        "fs4d_composite": [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.fs4d_sort_pairs_noalloc.argtypes = [vp, i64, i32, vp, vp]
    L.fs4d_sort_pairs_noalloc.restype = C.c_int
    L.fs4d_sort_pairs_noalloc_status.argtypes = [vp, vp]
    L.fs4d_sort_pairs_noalloc_status.restype = C.c_int
    L.fs4d_last_error.argtypes = [vp]
    L.fs4d_last_error.restype = C.c_char_p
    for name in ("fs4d_check_canaries", "fs4d_debug_corrupt_canary"):
        getattr(L, name).argtypes = [vp]
        getattr(L, name).restype = C.c_int
    _libs[path] = L
    return L


def camera_struct(cam) -> Camera:
    c = Camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy, c.znear = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy), float(cam.znear)
    c.world_to_cam = (C.c_float * 16)(*[float(v) for v in np.asarray(cam.world_to_cam, np.float32).ravel()])
    return c


def _ptr(t) -> Optional[int]:
    return None if t is None else int(t.data_ptr())


class Context:
    """One fs4d context: a CUDA device and the stream its work is queued on."""

    def __init__(self, device: int = 0, stream=None, lib=None):
        import torch
        self.torch = torch
        self.lib = lib if lib is not None else library()
        self.device = int(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        self._check(self.lib.fs4d_create(self.device, C.c_void_p(self.stream.cuda_stream), C.byref(h)), None)
        self.h = h
        self._scenes: Dict[int, object] = {}
        self._servers = []

    def _check(self, rc: int, h) -> None:
        if rc != 0:
            msg = self.lib.fs4d_last_error(h).decode() if h is not None else ""
            raise Fs4dError(rc, msg)

    def call(self, name: str, *args) -> None:
        self._check(getattr(self.lib, name)(self.h, *args), self.h)

    def close(self) -> None:
        for srv in getattr(self, "_servers", []):
            srv.close()  # a server must stop before its context goes
        if getattr(self, "h", None):
            self.lib.fs4d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream) -> None:
        self.stream = stream
        self.call("fs4d_set_stream", C.c_void_p(stream.cuda_stream))

    def check_device_status(self) -> None:
        self.call("fs4d_check_device_status")

    def set_wait_limit(self, polls: int) -> None:
        """Polls of the look-back waits of later launches (0 = default); a diagnostic."""
        self.call("fs4d_set_wait_limit", int(polls))

    # ------------------------------------------------------------------ scenes
    def load_scene(self, scene) -> int:
        arrs = {k: np.ascontiguousarray(getattr(scene, k), np.float32)
                for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "planes", "mlp")}
        d = SceneDesc()
        d.n = int(arrs["means"].shape[0])
        d.sh_degree = int(scene.sh_degree)
        for k, v in arrs.items():
            setattr(d, k, v.ctypes.data)
        d.aabb_min = (C.c_float * 3)(*map(float, scene.aabb_min))
        d.aabb_max = (C.c_float * 3)(*map(float, scene.aabb_max))
        rs = list(scene.res_spatial)
        d.n_levels = len(rs)
        d.res_spatial = (C.c_int32 * 4)(*(rs + [0] * (4 - len(rs))))
        d.res_time, d.feat_dim, d.mlp_width = int(scene.res_time), int(scene.feat_dim), int(scene.mlp_width)
        d.color_heads = int(bool(getattr(scene, "color_heads", False)))
        sid = C.c_int32()
        self.call("fs4d_load_scene", C.byref(d), C.byref(sid))
        self._scenes[sid.value] = scene
        return sid.value

    def read_scene(self, sid: int) -> Dict[str, np.ndarray]:
        """The scene's current parameters (host float32 arrays of the loaded shapes)."""
        scene = self._scenes[sid]
        out = {k: np.empty(np.shape(getattr(scene, k)), np.float32) for k in PARAMS}
        g = Grads(**{k: v.ctypes.data for k, v in out.items()})
        self.call("fs4d_read_scene", sid, C.byref(g), 0)
        return out

    def save_scene(self, sid: int, path: str) -> None:
        self.call("fs4d_save_scene", sid, os.fsencode(path))

    def load_scene_file(self, path: str, like=None) -> int:
        """Load a scene file; `like` (a scene object of the same shapes) is kept as
        the binding's record of the scene's sizes."""
        sid = C.c_int32()
        self.call("fs4d_load_scene_file", os.fsencode(path), C.byref(sid))
        if like is not None:
            self._scenes[sid.value] = like
        return sid.value

    def unload_scene(self, sid: int) -> None:
        self.call("fs4d_unload_scene", sid)
        self._scenes.pop(sid, None)

    def scene_bytes(self, sid: int, width: int, height: int, pairs_per_gaussian: float) -> Tuple[int, int]:
        r, f = C.c_size_t(), C.c_size_t()
        self.call("fs4d_scene_bytes", sid, width, height, float(pairs_per_gaussian), C.byref(r), C.byref(f))
        return r.value, f.value

    # ------------------------------------------------------------------ path
    def deform(self, sid: int, ts, prec: int = FP32, out=None):
        torch = self.torch
        ts = np.ascontiguousarray(np.atleast_1d(ts), np.float32)
        n = self._scenes[sid].means.shape[0]
        dev = torch.device("cuda", self.device)
        if out is None:
            out = (torch.empty((len(ts), n, 3), device=dev), torch.empty((len(ts), n, 4), device=dev),
                   torch.empty((len(ts), n, 3), device=dev))
        self.call("fs4d_deform", sid, prec, ts.ctypes.data, len(ts), _ptr(out[0]), _ptr(out[1]), _ptr(out[2]))
        return out

    def render(self, sid: int, cam, t: float, prec: int = FP32, image=None, with_aux: bool = False):
        torch = self.torch
        dev = torch.device("cuda", self.device)
        if image is None:
            image = torch.empty((cam.height, cam.width, 3), device=dev)
        T = nc = None
        if with_aux:
            T = torch.empty((cam.height, cam.width), device=dev)
            nc = torch.empty((cam.height, cam.width), device=dev, dtype=torch.int32)
        cs = camera_struct(cam)
        self.call("fs4d_render", sid, prec, C.byref(cs), float(t), _ptr(image), _ptr(T), _ptr(nc), None)
        return (image, T, nc) if with_aux else image

    def render_composed(self, sids, cam, t: float, prec: int = FP32, shifts=None, with_aux: bool = False):
        """One frame of the union of several scenes' deformed Gaussians (composition);
        shifts: [n][3] world translations, or None."""
        torch = self.torch
        dev = torch.device("cuda", self.device)
        image = torch.empty((cam.height, cam.width, 3), device=dev)
        T = nc = None
        if with_aux:
            T = torch.empty((cam.height, cam.width), device=dev)
            nc = torch.empty((cam.height, cam.width), device=dev, dtype=torch.int32)
        ids = (C.c_int32 * len(sids))(*[int(v) for v in sids])
        sh = None
        if shifts is not None:
            flat = np.ascontiguousarray(shifts, np.float32).ravel()
            sh = (C.c_float * flat.size)(*flat.tolist())
        cs = camera_struct(cam)
        self.call("fs4d_render_composed", ids, sh, len(sids), prec, C.byref(cs), float(t), _ptr(image), _ptr(T),
                  _ptr(nc))
        return (image, T, nc) if with_aux else image

    def render_saved(self, sid: int, cam, t: float, prec: int = FP32):
        """Render and keep the forward state for render_backward: (image, frame handle)."""
        torch = self.torch
        image = torch.empty((cam.height, cam.width, 3), device=torch.device("cuda", self.device))
        cs = camera_struct(cam)
        fr = C.c_void_p()
        self.call("fs4d_render", sid, prec, C.byref(cs), float(t), _ptr(image), None, None, C.byref(fr))
        return image, fr

    def render_backward(self, frame, dl_dimage, grads: Dict[str, object], stats=None) -> None:
        """Accumulate d(sum(dl_dimage * image))/d(parameter) into the given device tensors;
        stats = (grad_norm_sum, visible) device tensors [n] also accumulate the
        densification statistics (fs4d_render_backward_stats)."""
        g = Grads(**{k: _ptr(grads.get(k)) for k in ("means", "log_scales", "quats", "opacity_logits", "sh",
                                                       "planes", "mlp")})
        if stats is None:
            self.call("fs4d_render_backward", frame, _ptr(dl_dimage.contiguous()), C.byref(g))
        else:
            vs = ViewStats(_ptr(stats[0]), _ptr(stats[1]))
            self.call("fs4d_render_backward_stats", frame, _ptr(dl_dimage.contiguous()), C.byref(g), C.byref(vs))

    def densify(self, sid: int, stats, normals, grad_threshold: float, split_log_scale: float, prune_logit: float,
                trainer=None) -> int:
        """Densify and prune scene sid (fs4d_densify) from stats = (grad_norm_sum,
        visible) and normals [n][2][3] (device tensors); returns the new number of
        Gaussians.  The binding's record of the scene takes the new parameters."""
        vs = ViewStats(_ptr(stats[0]), _ptr(stats[1]))
        cfg = DensifyConfig(grad_threshold, split_log_scale, prune_logit)
        m = C.c_int64()
        self.call("fs4d_densify", sid, C.byref(cfg), C.byref(vs), _ptr(normals.contiguous()),
                  trainer.h if trainer is not None else None, C.byref(m))
        self._resized(sid, m.value)
        return m.value

    def densify_raw(self, sid: int, stats, normals, grad_threshold: float, split_log_scale: float,
                    prune_logit: float) -> int:
        """fs4d_densify alone: returns the new n and leaves the binding's host
        record of the scene stale (for timing; unload the scene afterwards)."""
        vs = ViewStats(_ptr(stats[0]), _ptr(stats[1]))
        cfg = DensifyConfig(grad_threshold, split_log_scale, prune_logit)
        m = C.c_int64()
        self.call("fs4d_densify", sid, C.byref(cfg), C.byref(vs), _ptr(normals.contiguous()), None, C.byref(m))
        self._scenes[sid] = None
        return m.value

    def _resized(self, sid: int, n: int) -> None:
        """Replace the record of scene sid by a host copy of its parameters at size n."""
        rec = self._scenes[sid].copy()
        k = int(rec.sh.shape[1])
        shapes = {"means": (n, 3), "log_scales": (n, 3), "quats": (n, 4), "opacity_logits": (n,), "sh": (n, k, 3)}
        for key, shp in shapes.items():
            setattr(rec, key, np.empty(shp, np.float32))
        self._scenes[sid] = rec
        for key, v in self.read_scene(sid).items():
            setattr(rec, key, v)

    def frame_free(self, frame) -> None:
        self.call("fs4d_frame_free", frame)

    def update_scene(self, sid: int, params: Dict[str, object]) -> None:
        """Overwrite scene parameters from CUDA tensors (same shapes as loaded)."""
        scene = self._scenes[sid]
        d = SceneDesc()
        d.n = int(scene.means.shape[0])
        d.sh_degree = int(scene.sh_degree)
        keep = []
        for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "planes", "mlp"):
            v = params.get(k)
            if v is not None:
                v = v.detach().contiguous().float()
                keep.append(v)
                setattr(d, k, _ptr(v))
        rs = list(scene.res_spatial)
        d.n_levels = len(rs)
        d.res_spatial = (C.c_int32 * 4)(*(rs + [0] * (4 - len(rs))))
        d.aabb_min = (C.c_float * 3)(*map(float, scene.aabb_min))
        d.aabb_max = (C.c_float * 3)(*map(float, scene.aabb_max))
        d.res_time, d.feat_dim, d.mlp_width = int(scene.res_time), int(scene.feat_dim), int(scene.mlp_width)
        d.color_heads = int(bool(getattr(scene, "color_heads", False)))
        self.call("fs4d_update_scene", sid, C.byref(d), 1)
        del keep

    def render_host(self, sid: int, cam, t: float, prec: int = FP32, out: Optional[np.ndarray] = None):
        if out is None:
            out = np.empty((cam.height, cam.width, 3), np.float32)
        cs = camera_struct(cam)
        self.call("fs4d_render_host", sid, prec, C.byref(cs), float(t), out.ctypes.data)
        return out

    def render_host_batch(self, sid: int, cams, ts, prec: int = FP32, outs=None):
        """Frames (cams[k], ts[k]) into host images outs[k] (numpy float32 [H][W][3]; the
        same array may repeat), each copy overlapped with the next frame's render."""
        n = len(cams)
        if outs is None:
            outs = [np.empty((cams[0].height, cams[0].width, 3), np.float32) for _ in range(n)]
        carr = (Camera * n)(*[camera_struct(cm) for cm in cams])
        tarr = (C.c_float * n)(*[float(t) for t in ts])
        parr = (C.c_void_p * n)(*[o.ctypes.data for o in outs])
        self.call("fs4d_render_host_batch", sid, prec, carr, tarr, n, parr)
        return outs

    def reserve(self, sid: int, width: int, height: int, pair_capacity: int) -> None:
        self.call("fs4d_reserve", sid, width, height, int(pair_capacity))

    def render_async(self, sid: int, shape_cam, d_cam, d_t, image, prec: int = FP32) -> None:
        cs = camera_struct(shape_cam)
        self.call("fs4d_render_async", sid, prec, C.byref(cs), _ptr(d_cam), _ptr(d_t), _ptr(image))

    def set_stage_timing(self, on: bool) -> None:
        self.call("fs4d_set_stage_timing", int(bool(on)))

    def stage_times(self) -> Dict[str, float]:
        ms = (C.c_float * 6)()
        self.call("fs4d_stage_times", ms)
        return dict(zip(STAGES, [float(v) for v in ms]))

    def backward_times(self) -> Dict[str, float]:
        ms = (C.c_float * 4)()
        self.call("fs4d_backward_times", ms)
        return dict(zip(("composite_bwd", "project_bwd", "mlp_planes_bwd", "weight_grads"), [float(v) for v in ms]))

    def last_pairs(self) -> int:
        k = C.c_int64()
        self.call("fs4d_last_pairs", C.byref(k))
        return k.value

    def last_launches(self) -> int:
        """Kernels the last render / render_async call launched."""
        k = C.c_int64()
        self.call("fs4d_last_launches", C.byref(k))
        return k.value

    def last_bands(self) -> int:
        """Bands of tile rows the last frame was rendered in (1 unless it had more
        tile pairs than one pair-sort pass counts)."""
        b = C.c_int32()
        self.call("fs4d_last_bands", C.byref(b))
        return b.value

    def set_band_pairs(self, max_pairs: int) -> None:
        """Most tile pairs one band of a frame may hold (0 = default, 2^30 - 1)."""
        self.call("fs4d_set_band_pairs", int(max_pairs))

    def set_binning(self, mode: int) -> None:
        """BINNING_AUTO (tile bitmap when it fits) or BINNING_SORT (keys + radix sort)."""
        self.call("fs4d_set_binning", int(mode))

    def last_binning(self) -> int:
        """BINNING_BITMAP or BINNING_SORT: how the last frame on this context was binned."""
        m = C.c_int32()
        self.call("fs4d_last_binning", C.byref(m))
        return m.value

    # ------------------------------------------------------------------ stages
    def project(self, means, quats, log_scales, opacity_logits, sh, sh_degree: int, cam):
        torch = self.torch
        n = means.shape[0]
        dev = means.device
        out = dict(xy=torch.empty((n, 2), device=dev), conic_opacity=torch.empty((n, 4), device=dev),
                   rgb=torch.empty((n, 3), device=dev), depth=torch.empty(n, device=dev),
                   radius=torch.empty(n, device=dev, dtype=torch.int32),
                   rect=torch.empty((n, 4), device=dev, dtype=torch.int32))
        p = Projected(**{k: _ptr(v) for k, v in out.items()})
        cs = camera_struct(cam)
        self.call("fs4d_project", n, _ptr(means), _ptr(quats), _ptr(log_scales), _ptr(opacity_logits), _ptr(sh),
                  int(sh_degree), C.byref(cs), C.byref(p))
        return out

    def bin_sort(self, depth, rect, tiles_x: int, tiles_y: int, capacity: int):
        torch = self.torch
        dev = depth.device
        keys = torch.empty(max(capacity, 1), device=dev, dtype=torch.int64)
        vals = torch.empty(max(capacity, 1), device=dev, dtype=torch.int32)
        ranges = torch.empty((tiles_x * tiles_y, 2), device=dev, dtype=torch.int32)
        K = C.c_int64()
        self.call("fs4d_bin_sort", depth.shape[0], _ptr(depth), _ptr(rect), tiles_x, tiles_y, int(capacity),
                  _ptr(keys), _ptr(vals), _ptr(ranges), C.byref(K))
        return keys[:K.value], vals[:K.value], ranges, K.value

    def sort_pairs(self, keys, values, key_bits: int) -> None:
        self.call("fs4d_sort_pairs", keys.shape[0], int(key_bits), _ptr(keys), _ptr(values))

    def composite(self, width: int, height: int, ranges, values, xy, conic_opacity, rgb):
        torch = self.torch
        dev = xy.device
        img = torch.empty((height, width, 3), device=dev)
        T = torch.empty((height, width), device=dev)
        nc = torch.empty((height, width), device=dev, dtype=torch.int32)
        self.call("fs4d_composite", width, height, _ptr(ranges), _ptr(values), _ptr(xy), _ptr(conic_opacity),
                  _ptr(rgb), _ptr(img), _ptr(T), _ptr(nc))
        return img, T, nc


PARAMS = ("means", "log_scales", "quats", "opacity_logits", "sh", "planes", "mlp")


def _render_function():
    import torch

    class RenderFunction(torch.autograd.Function):
        """image = S(M, G + F(G, t)) with the hand-written CUDA backward.

        forward(fs, sid, cam, t, prec, means, log_scales, quats, opacity_logits, sh, planes, mlp)
        copies the parameter tensors into the library's scene, renders, and keeps
        the frame; backward accumulates every parameter gradient with
        fs4d_render_backward.  The backward recomputes the deformation in float32.
        """

        @staticmethod
        def forward(ctx, fs, sid, cam, t, prec, *params):
            fs.update_scene(sid, dict(zip(PARAMS, params)))
            image, frame = fs.render_saved(sid, cam, t, prec)
            ctx.fs, ctx.frame = fs, frame
            ctx.shapes = [(p.shape, p.dtype, p.device) for p in params]
            ctx.needs = ctx.needs_input_grad[5:]
            return image

        @staticmethod
        def backward(ctx, dl_dimage):
            grads = [torch.zeros(s, dtype=d, device=dev) if need else None
                     for (s, d, dev), need in zip(ctx.shapes, ctx.needs)]
            ctx.fs.render_backward(ctx.frame, dl_dimage, dict(zip(PARAMS, grads)))
            ctx.fs.frame_free(ctx.frame)
            ctx.frame = None
            return (None, None, None, None, None, *grads)

    return RenderFunction


_RF = None


def render_differentiable(fs: "Context", sid: int, cam, t: float, params: Dict[str, object], prec: int = FP32):
    """Differentiable render: params maps means/log_scales/quats/opacity_logits/sh/
    planes/mlp to CUDA float32 tensors (requires_grad as needed)."""
    global _RF
    if _RF is None:
        _RF = _render_function()
    return _RF.apply(fs, sid, cam, float(t), prec, *[params[k] for k in PARAMS])


# ---------------------------------------------------------------------- serving

class ServerConfig(C.Structure):
    _fields_ = [("max_inflight", C.c_int32), ("max_batch", C.c_int32), ("hbm_budget_bytes", C.c_int64),
                ("pairs_per_gaussian", C.c_float)]


class Request(C.Structure):
    _fields_ = [("scene", C.c_int32), ("prec", C.c_int32), ("cam", Camera), ("t", C.c_float), ("out", C.c_void_p),
                ("out_on_device", C.c_int32)]


class Completion(C.Structure):
    _fields_ = [("ticket", C.c_uint64), ("status", C.c_int32), ("slot", C.c_int32), ("pairs", C.c_int64),
                ("submit_ms", C.c_double), ("start_ms", C.c_double), ("done_ms", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64), ("retried", C.c_int64),
                ("batches", C.c_int64), ("deformed", C.c_int64), ("slots", C.c_int32),
                ("max_concurrent", C.c_int32), ("slot_bytes", C.c_int64), ("peak_slot_bytes", C.c_int64)]


class Trainer:
    """The on-device training step of a loaded scene (fs4d_train_*)."""

    def __init__(self, ctx: "Context", sid: int, total_steps: int, **cfg):
        self.ctx = ctx
        self.lib = ctx.lib
        self.cfg = train_config(total_steps, **cfg)
        h = C.c_void_p()
        ctx.call("fs4d_train_create", sid, C.byref(self.cfg), C.byref(h))
        self.h = h
        self.sid = sid

    def step(self, cam, t: float, target, prec: int = FP32, losses=None) -> None:
        cs = camera_struct(cam)
        st = self.lib.fs4d_train_step(self.h, int(prec), C.byref(cs), float(t), _ptr(target.contiguous()),
                                      _ptr(losses))
        if st != 0:
            raise Fs4dError(st, self.lib.fs4d_last_error(self.ctx.h).decode())

    def losses(self) -> Tuple[float, float]:
        out = (C.c_float * 2)()
        st = self.lib.fs4d_train_losses(self.h, out)
        if st != 0:
            raise Fs4dError(st, "train_losses")
        return float(out[0]), float(out[1])

    def steps_done(self) -> int:
        k = C.c_int64()
        self.lib.fs4d_train_steps_done(self.h, C.byref(k))
        return k.value

    def read_state(self, group: int):
        """Adam moments (m, v) of parameter group `group` (0 means .. 6 mlp) as host arrays."""
        names = ("means", "log_scales", "quats", "opacity_logits", "sh", "planes", "mlp")
        rec = self.ctx._scenes[self.sid]
        size = int(np.prod(np.shape(getattr(rec, names[group]))))
        m, v = np.empty(size, np.float32), np.empty(size, np.float32)
        st = self.lib.fs4d_train_read_state(self.h, int(group), m.ctypes.data, v.ctypes.data)
        if st != 0:
            raise Fs4dError(st, self.lib.fs4d_last_error(self.ctx.h).decode())
        return m, v

    def stats(self):
        """The densification statistics accumulated by the steps: (grad_norm_sum, visible), device tensors."""
        import torch
        n = int(self.ctx._scenes[self.sid].means.shape[0])
        g = torch.empty(n, dtype=torch.float32, device="cuda")
        vis = torch.empty(n, dtype=torch.float32, device="cuda")
        vs = ViewStats(_ptr(g), _ptr(vis))
        st = self.lib.fs4d_train_stats(self.h, C.byref(vs))
        if st != 0:
            raise Fs4dError(st, self.lib.fs4d_last_error(self.ctx.h).decode())
        return g, vis

    def densify(self, normals, grad_threshold: float, split_log_scale: float, prune_logit: float) -> int:
        """fs4d_train_densify with the trainer's own statistics; returns the new n."""
        cfg = DensifyConfig(grad_threshold, split_log_scale, prune_logit)
        m = C.c_int64()
        st = self.lib.fs4d_train_densify(self.h, C.byref(cfg), _ptr(normals.contiguous()), C.byref(m))
        if st != 0:
            raise Fs4dError(st, self.lib.fs4d_last_error(self.ctx.h).decode())
        self.ctx._resized(self.sid, m.value)
        return m.value

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.fs4d_train_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SERVER_EXPORTS = ("fs4d_server_create", "fs4d_server_submit", "fs4d_server_submit_batch", "fs4d_server_cancel",
                  "fs4d_server_poll",
                  "fs4d_server_drain", "fs4d_server_stats_get", "fs4d_server_destroy")
EXPORTS = EXPORTS + SERVER_EXPORTS


def _server_sigs(L):
    vp = C.c_void_p
    sig = {"fs4d_server_create": [vp, C.POINTER(ServerConfig), C.POINTER(vp)],
           "fs4d_server_submit": [vp, C.POINTER(Request), C.POINTER(C.c_uint64)],
           "fs4d_server_submit_batch": [vp, C.POINTER(Request), C.c_int32, C.POINTER(C.c_uint64)],
           "fs4d_server_cancel": [vp, C.c_uint64],
           "fs4d_server_poll": [vp, C.POINTER(Completion), C.c_int32, C.POINTER(C.c_int32)],
           "fs4d_server_drain": [vp],
           "fs4d_server_stats_get": [vp, C.POINTER(ServerStats)],
           "fs4d_server_destroy": [vp]}
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int


class Server:
    """Continuous-batching render server on a Context (native scheduler thread)."""

    def __init__(self, ctx: Context, max_inflight: int = 8, max_batch: int = 8, hbm_budget_bytes: int = 16 << 30,
                 pairs_per_gaussian: float = 16.0):
        self.ctx = ctx
        self.lib = ctx.lib
        _server_sigs(self.lib)
        cfg = ServerConfig(max_inflight, max_batch, hbm_budget_bytes, pairs_per_gaussian)
        h = C.c_void_p()
        ctx.call("fs4d_server_create", C.byref(cfg), C.byref(h))
        self.h = h
        self._keep: Dict[int, object] = {}
        ctx._servers.append(self)

    def _check(self, rc: int) -> None:
        if rc != 0:
            raise Fs4dError(rc, "server call failed")

    def submit(self, sid: int, cam, t: float, out, prec: int = FP32) -> int:
        """Queue a frame; out is a CUDA tensor (device output) or a numpy array (host output)."""
        r = Request()
        r.scene, r.prec, r.cam, r.t = sid, prec, camera_struct(cam), float(t)
        if hasattr(out, "data_ptr"):
            r.out, r.out_on_device = out.data_ptr(), 1
        else:
            r.out, r.out_on_device = out.ctypes.data, 0
        tk = C.c_uint64()
        self._check(self.lib.fs4d_server_submit(self.h, C.byref(r), C.byref(tk)))
        self._keep[tk.value] = out
        return tk.value

    def _request(self, sid, cam, t, out, prec) -> Request:
        r = Request()
        r.scene, r.prec, r.cam, r.t = sid, prec, camera_struct(cam), float(t)
        if hasattr(out, "data_ptr"):
            r.out, r.out_on_device = out.data_ptr(), 1
        else:
            r.out, r.out_on_device = out.ctypes.data, 0
        return r

    def submit_batch(self, items):
        """items: list of (sid, cam, t, out, prec); queued together.  Returns tickets."""
        arr = (Request * len(items))(*[self._request(*it) for it in items])
        tks = (C.c_uint64 * len(items))()
        self._check(self.lib.fs4d_server_submit_batch(self.h, arr, len(items), tks))
        for tk, it in zip(tks, items):
            self._keep[tk] = it[3]
        return list(tks)

    def cancel(self, ticket: int) -> bool:
        return self.lib.fs4d_server_cancel(self.h, C.c_uint64(ticket)) == 0

    def poll(self, max_n: int = 256):
        buf = (Completion * max_n)()
        n = C.c_int32()
        self._check(self.lib.fs4d_server_poll(self.h, buf, max_n, C.byref(n)))
        out = []
        for i in range(n.value):
            c = buf[i]
            self._keep.pop(c.ticket, None)
            out.append(dict(ticket=c.ticket, status=c.status, slot=c.slot, pairs=c.pairs, submit_ms=c.submit_ms,
                            start_ms=c.start_ms, done_ms=c.done_ms))
        return out

    def drain(self) -> None:
        self._check(self.lib.fs4d_server_drain(self.h))

    def stats(self) -> Dict[str, int]:
        s = ServerStats()
        self._check(self.lib.fs4d_server_stats_get(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.fs4d_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
