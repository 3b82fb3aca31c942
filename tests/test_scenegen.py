"""The seeded synthetic inputs follow their stated recipes (the shapes and value
distributions of the workloads the paper measures on), and are deterministic
per seed.  Statistical checks use bounds many standard errors wide."""
import math

import numpy as np
import pytest

from paper_2310_08528_gb300 import scenegen as sg

SH_C0 = 0.5 / math.sqrt(math.pi)


def _layer_blocks(s):
    hin = s.feat_dim * s.n_levels
    off, out = 0, []
    for o, i in sg.mlp_layer_shapes(hin, s.mlp_width):
        out.append((s.mlp[off:off + o * i], s.mlp[off + o * i:off + o * i + o]))
        off += o * i + o
    assert off == s.mlp.size
    return out


def _check_common(s, n, deg, res_spatial, res_time, h, log_scale_mean, mlp_std):
    K = (deg + 1) ** 2
    assert s.means.shape == (n, 3) and s.log_scales.shape == (n, 3) and s.quats.shape == (n, 4)
    assert s.opacity_logits.shape == (n,) and s.sh.shape == (n, K, 3) and s.sh_degree == deg
    for a in (s.means, s.log_scales, s.quats, s.opacity_logits, s.sh, s.planes, s.mlp):
        assert a.dtype == np.float32
    assert tuple(s.res_spatial) == tuple(res_spatial) and s.res_time == res_time and s.feat_dim == h
    assert s.planes.size == sum(int(np.prod(x)) for x in sg.plane_shapes(res_spatial, res_time, h))
    assert abs(s.log_scales.mean() - log_scale_mean) < 5 * 0.5 / math.sqrt(3 * n)  # 5 standard errors
    assert abs(s.log_scales.std() - 0.5) < 0.02
    assert np.allclose(np.linalg.norm(s.quats.astype(np.float64), axis=1), 1.0, atol=1e-6)
    assert abs(s.opacity_logits.mean()) < 5.0 / math.sqrt(n) + 0.01 and abs(s.opacity_logits.std() - 1.0) < 0.05
    colour = 0.5 + SH_C0 * s.sh[:, 0, :].astype(np.float64)  # the DC colour, drawn U[0,1]
    assert colour.min() > -1e-5 and colour.max() < 1 + 1e-5
    assert abs(colour.mean() - 0.5) < 0.02
    assert abs(s.planes.mean() - 1.0) < 0.01 and abs(s.planes.std() - 0.1) < 0.01
    for w, b in _layer_blocks(s):
        assert not b.any()  # biases are not specified: zero
    w0 = _layer_blocks(s)[0][0]
    assert abs(w0.std() - mlp_std) < 0.15 * mlp_std


def test_tiny_scene_recipe():
    s = sg.make_tiny(0)
    _check_common(s, 2000, 0, (32,), 8, 16, -4.0, 0.02)
    assert s.means.min() >= -1.0 and s.means.max() <= 1.0
    assert abs(s.means.mean()) < 0.05
    assert s.aabb_min == (-1.0, -1.0, -1.0) and s.aabb_max == (1.0, 1.0, 1.0)


def test_object_scene_recipe():
    s = sg.make_object(0, n=20000)
    _check_common(s, 20000, 3, (64, 128), 25, 32, -4.0, 0.02)
    assert (np.linalg.norm(s.means.astype(np.float64), axis=1) <= 1.0 + 1e-6).all()
    rest = s.sh[:, 1:, :]
    assert abs(rest.std() - 0.05) < 0.005 and abs(rest.mean()) < 0.005
    assert s.feat_dim * s.n_levels == 64 and s.mlp_width == 64


def test_room_and_stress_recipes():
    r = sg.make_room(0, n=6000)
    _check_common(r, 6000, 3, (64, 128), 150, 32, -3.5, 0.02)
    lo, hi = np.array(r.aabb_min), np.array(r.aabb_max)
    assert np.allclose(hi - lo, [6.0, 4.0, 6.0])
    assert (r.means >= lo).all() and (r.means <= hi).all()
    st = sg.make_stress(0, n=6000)
    _check_common(st, 6000, 3, (64, 128, 256), 300, 32, -2.5, 0.02)


def test_hemisphere_cameras_look_at_the_origin():
    cams = sg.hemisphere_cameras(50, width=800, height=800, seed=0)
    assert len(cams) == 50
    for c in cams:
        M = np.asarray(c.world_to_cam, np.float64)
        R, t = M[:3, :3], M[:3, 3]
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-6)
        eye = -R.T @ t
        assert abs(np.linalg.norm(eye) - 4.0) < 1e-5 and eye[2] >= 0.0
        p = R @ np.zeros(3) + t  # the origin: on the optical axis, 4 ahead
        assert abs(p[0]) < 1e-5 and abs(p[1]) < 1e-5 and abs(p[2] - 4.0) < 1e-5
        assert c.fx == pytest.approx(800 / (2 * math.tan(math.radians(25.0))))
        assert (c.cx, c.cy) == (400.0, 400.0)
        assert R[1] @ np.array([0.0, 0.0, 1.0]) <= 1e-6  # world up maps to image up (y down)


def test_generators_are_deterministic_per_seed():
    a, b, c = sg.make_tiny(3), sg.make_tiny(3), sg.make_tiny(4)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "planes", "mlp"):
        assert np.array_equal(getattr(a, k), getattr(b, k))
        assert not np.array_equal(getattr(a, k), getattr(c, k))
    ca = sg.hemisphere_cameras(5, seed=2)
    cb = sg.hemisphere_cameras(5, seed=2)
    assert all(np.array_equal(x.world_to_cam, y.world_to_cam) for x, y in zip(ca, cb))
