"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a closed form,
an independent library routine (scipy), a special case that reduces to a
simpler model, or a brute-force restatement.  None needs a GPU.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2310_08528_gb300 import scenegen as sg


def one_gaussian_scene(mean=(0.0, 0.0, 0.0), log_scale=(-3.0, -3.0, -3.0), quat=(1.0, 0.0, 0.0, 0.0),
                       logit=0.3, dc=(0.0, 0.0, 0.0), extra=()):
    base = sg.make_tiny(0, n=1 + len(extra))
    rows = [(mean, log_scale, quat, logit, dc)] + list(extra)
    base.means = np.array([r[0] for r in rows], np.float32)
    base.log_scales = np.array([r[1] for r in rows], np.float32)
    base.quats = np.array([r[2] for r in rows], np.float32)
    base.opacity_logits = np.array([r[3] for r in rows], np.float32)
    base.sh = np.array([[r[4]] for r in rows], np.float32)
    return base


def centred_camera(w=128, h=128):
    cam = sg.tiny_camera(w, h)
    cam.cx, cam.cy = w / 2 + 0.5, h / 2 + 0.5  # the origin projects onto pixel centre (w/2, h/2)
    return cam


def sigmoid(x):
    return 1.0 / (1.0 + math.exp(-x))


# --------------------------------------------------------------------- Eq. 1 / Eq. 4 closed forms

def test_single_gaussian_at_pixel_centre_closed_form():
    """Eq. 1 at the mean is 1 and Eq. 4 has one term: pixel = colour * min(0.99, sigmoid(o))."""
    for logit in (-1.0, 0.3, 6.0):  # the last one hits the 0.99 clamp
        s = one_gaussian_scene(logit=logit)
        img, T, nc, _, K = oracle.render(s, centred_camera(), 0.5, deform=False)
        o = sigmoid(float(np.float32(logit)))
        a = min(0.99, o)
        assert img[64, 64] == pytest.approx([0.5 * a] * 3, abs=1e-15)
        assert T[64, 64] == pytest.approx(1.0 - a, abs=1e-15)
        assert nc[64, 64] == 1


def test_single_gaussian_neighbour_closed_form():
    """Neighbouring pixel: alpha = o * exp(-d^2 / (2 var)), var = (f s / z)^2 + 0.3 (Eq. 3 on the axis)."""
    ls = -3.0
    s = one_gaussian_scene(log_scale=(ls, ls, ls), logit=0.0)
    cam = centred_camera()
    img, *_ = oracle.render(s, cam, 0.5, deform=False)
    var = (cam.fx * math.exp(float(np.float32(ls))) / 4.0) ** 2 + 0.3
    for d in (1, 2, 3):
        a = 0.5 * math.exp(-0.5 * d * d / var)
        want = 0.5 * a if a >= 1 / 255 else 0.0
        assert img[64, 64 + d, 0] == pytest.approx(want, rel=1e-12, abs=1e-15)
        assert img[64 + d, 64, 0] == pytest.approx(want, rel=1e-12, abs=1e-15)


def test_front_to_back_order_and_stop_rule():
    """Eq. 4 read as prod_{j<i}(1 - a_j): two opaque Gaussians give 0.99 c1 + 0.01*0.99 c2;
    a third would take T to 1e-6 < 1e-4 and is not blended."""
    c1, c2, c3 = 0.3, -0.2, 0.4  # DC coefficients; colours 0.5 + Y0 * dc
    y0 = 0.5 / math.sqrt(math.pi)
    extra = [((0.0, 0.5, 0.0), (-3.0,) * 3, (1.0, 0, 0, 0), 9.0, (c2,) * 3),
             ((0.0, 1.0, 0.0), (-3.0,) * 3, (1.0, 0, 0, 0), 9.0, (c3,) * 3)]
    s = one_gaussian_scene(logit=9.0, dc=(c1,) * 3, extra=extra)
    img, T, nc, _, _ = oracle.render(s, centred_camera(), 0.5, deform=False)
    col1 = 0.5 + y0 * float(np.float32(c1))
    col2 = 0.5 + y0 * float(np.float32(c2))
    assert img[64, 64, 0] == pytest.approx(0.99 * col1 + 0.01 * 0.99 * col2, rel=1e-12)
    assert T[64, 64] == pytest.approx(0.01 * 0.01, rel=1e-12)
    assert nc[64, 64] == 2


# --------------------------------------------------------------------- Eq. 2 / Eq. 3 closed forms

def test_ewa_covariance_axis_aligned():
    """On the optical axis J = diag(f/z): Sigma' = diag(f^2 s_x^2 / z^2, f^2 s_z^2 / z^2) + 0.3 I
    (camera x = world x, camera y = -world z for the tiny camera)."""
    ls = (-3.0, -2.5, -2.0)
    s = one_gaussian_scene(log_scale=ls)
    cam = centred_camera()
    p = oracle.project(s, cam)
    sx, sy, sz = [math.exp(float(np.float32(v))) for v in ls]
    z = 4.0
    assert p["cov2d"][0] == pytest.approx([cam.fx ** 2 * sx ** 2 / z ** 2 + 0.3, 0.0,
                                           cam.fy ** 2 * sz ** 2 / z ** 2 + 0.3], rel=1e-12, abs=1e-12)
    assert p["depth"][0] == pytest.approx(z)
    assert p["xy"][0] == pytest.approx([64.5, 64.5])


def test_ewa_covariance_rotated_against_scipy_rotation():
    """Rotation about the world y axis (the viewing axis) mixes image x and y; the
    expected covariance uses scipy's quaternion-to-matrix, not the oracle's."""
    from scipy.spatial.transform import Rotation
    ang = 0.7
    q = (math.cos(ang / 2), 0.0, math.sin(ang / 2), 0.0)  # w x y z
    ls = (-3.0, -2.6, -2.2)
    s = one_gaussian_scene(log_scale=ls, quat=q)
    cam = centred_camera()
    p = oracle.project(s, cam)
    qf = np.array(q, np.float32).astype(np.float64)
    R = Rotation.from_quat([qf[1], qf[2], qf[3], qf[0]]).as_matrix()
    S = np.diag(np.exp(np.array(ls, np.float32).astype(np.float64)))
    sig = R @ S @ S @ R.T
    W = np.asarray(cam.world_to_cam, np.float64)[:3, :3]
    J = np.array([[cam.fx / 4.0, 0, 0], [0, cam.fy / 4.0, 0]])  # on-axis Jacobian
    want = J @ W @ sig @ W.T @ J.T + 0.3 * np.eye(2)
    assert p["cov2d"][0] == pytest.approx([want[0, 0], want[0, 1], want[1, 1]], rel=1e-10, abs=1e-12)
    assert abs(want[0, 1]) > 1.0  # the off-diagonal term is really exercised
    det = want[0, 0] * want[1, 1] - want[0, 1] ** 2
    assert p["conic"][0] == pytest.approx([want[1, 1] / det, -want[0, 1] / det, want[0, 0] / det], rel=1e-10)
    lam = np.linalg.eigvalsh(want).max()
    assert p["radius"][0] == math.ceil(3 * math.sqrt(lam))


def _scipy_sigma(quat_wxyz, log_scale):
    """Sigma = R S S^T R^T (Eq. 2) with R from scipy's rotation of the normalised quaternion."""
    from scipy.spatial.transform import Rotation
    q = np.array(quat_wxyz, np.float32).astype(np.float64)
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy takes (x, y, z, w), normalises
    S = np.diag(np.exp(np.array(log_scale, np.float32).astype(np.float64)))
    return R @ S @ S @ R.T


def test_ewa_covariance_general_unnormalised_quaternion():
    """A rotation with all four quaternion components non-zero, stored with norm 1.7
    (Eq. 6 adds dr to r and the rotation uses r / |r|), against scipy's rotation."""
    q = tuple(1.7 * v / math.sqrt(0.8 ** 2 + 0.3 ** 2 + 0.4 ** 2 + 0.5 ** 2) for v in (0.8, 0.3, -0.4, 0.5))
    ls = (-3.1, -2.4, -2.7)
    s = one_gaussian_scene(log_scale=ls, quat=q)
    cam = centred_camera()
    p = oracle.project(s, cam)
    W = np.asarray(cam.world_to_cam, np.float64)[:3, :3]
    J = np.array([[cam.fx / 4.0, 0, 0], [0, cam.fy / 4.0, 0]])
    want = J @ W @ _scipy_sigma(q, ls) @ W.T @ J.T + 0.3 * np.eye(2)
    assert abs(want[0, 1]) > 0.5
    assert p["cov2d"][0] == pytest.approx([want[0, 0], want[0, 1], want[1, 1]], rel=1e-9, abs=1e-12)
    assert p["radius"][0] == math.ceil(3 * math.sqrt(np.linalg.eigvalsh(want).max()))


def test_ewa_covariance_off_axis_jacobian():
    """Off the optical axis the Jacobian of the perspective map (Eq. 3's J) has the
    third column (-f p_x / p_z^2, -f p_y / p_z^2) at the camera-space mean p."""
    mean, q, ls = (0.5, 0.3, -0.4), (0.9, -0.2, 0.3, 0.25), (-2.9, -2.3, -3.2)
    s = one_gaussian_scene(mean=mean, log_scale=ls, quat=q)
    cam = sg.tiny_camera()
    out = oracle.project(s, cam)
    M = np.asarray(cam.world_to_cam, np.float64)
    W = M[:3, :3]
    p = W @ np.array(mean, np.float32).astype(np.float64) + M[:3, 3]
    assert abs(p[0] / p[2]) > 0.1 and abs(p[1] / p[2]) > 0.05  # off axis, inside the guard band
    J = np.array([[cam.fx / p[2], 0, -cam.fx * p[0] / p[2] ** 2],
                  [0, cam.fy / p[2], -cam.fy * p[1] / p[2] ** 2]])
    want = J @ W @ _scipy_sigma(q, ls) @ W.T @ J.T + 0.3 * np.eye(2)
    assert out["cov2d"][0] == pytest.approx([want[0, 0], want[0, 1], want[1, 1]], rel=1e-9, abs=1e-12)
    assert out["xy"][0] == pytest.approx([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy],
                                         rel=1e-12)
    assert out["depth"][0] == pytest.approx(p[2], rel=1e-12)


def test_ewa_jacobian_guard_band():
    """Far off the optical axis the Jacobian uses p_x/p_z and p_y/p_z clamped to
    +-1.3 tan(fov/2) (the guard band read from differentiable splatting; the mean
    itself is not clamped).  The covariance is written even when the rectangle
    falls outside the image."""
    mean, q, ls = (3.2, 0.6, -2.9), (0.8, 0.3, -0.1, 0.5), (-2.5, -2.1, -2.8)
    s = one_gaussian_scene(mean=mean, log_scale=ls, quat=q)
    cam = sg.tiny_camera()
    out = oracle.project(s, cam)
    M = np.asarray(cam.world_to_cam, np.float64)
    W = M[:3, :3]
    p = W @ np.array(mean, np.float32).astype(np.float64) + M[:3, 3]
    lim_x, lim_y = 1.3 * cam.width / (2 * cam.fx), 1.3 * cam.height / (2 * cam.fy)
    assert abs(p[0] / p[2]) > lim_x and abs(p[1] / p[2]) > lim_y  # both ratios are clamped
    rx, ry = np.clip(p[0] / p[2], -lim_x, lim_x), np.clip(p[1] / p[2], -lim_y, lim_y)
    J = np.array([[cam.fx / p[2], 0, -cam.fx * rx / p[2]], [0, cam.fy / p[2], -cam.fy * ry / p[2]]])
    want = J @ W @ _scipy_sigma(q, ls) @ W.T @ J.T + 0.3 * np.eye(2)
    assert out["cov2d"][0] == pytest.approx([want[0, 0], want[0, 1], want[1, 1]], rel=1e-9, abs=1e-12)
    assert out["xy"][0] == pytest.approx([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy],
                                         rel=1e-12)


def test_single_anisotropic_gaussian_image_closed_form():
    """Eq. 1 with a full 2-D covariance: every pixel is colour * alpha with
    alpha = min(0.99, o exp(-1/2 d^T Sigma'^-1 d)), d from the projected mean to the
    pixel centre, and 0 where alpha < 1/255.  With o < 255^-1 e^4.5 nothing beyond
    the 3-sigma tile rectangle could pass the 1/255 test, so the whole image is fixed."""
    q, ls, logit = (0.9, 0.1, 0.4, 0.1), (-2.0, -3.2, -3.0), -1.2
    s = one_gaussian_scene(log_scale=ls, quat=q, logit=logit)
    cam = centred_camera()
    img, T, nc, _, _ = oracle.render(s, cam, 0.5, deform=False)
    W = np.asarray(cam.world_to_cam, np.float64)[:3, :3]
    J = np.array([[cam.fx / 4.0, 0, 0], [0, cam.fy / 4.0, 0]])
    cov = J @ W @ _scipy_sigma(q, ls) @ W.T @ J.T + 0.3 * np.eye(2)
    assert abs(cov[0, 1]) > 0.3 * math.sqrt(cov[0, 0] * cov[1, 1])
    conic = np.linalg.inv(cov)
    o = sigmoid(float(np.float32(logit)))
    assert o * math.exp(-4.5) < 1 / 255
    ys, xs = np.mgrid[0:128, 0:128]
    dx, dy = xs + 0.5 - 64.5, ys + 0.5 - 64.5
    q2 = conic[0, 0] * dx * dx + 2 * conic[0, 1] * dx * dy + conic[1, 1] * dy * dy
    alpha = np.minimum(0.99, o * np.exp(-0.5 * q2))
    keep = alpha >= 1 / 255
    near = np.abs(alpha - 1 / 255) < 1e-9
    want = np.where(keep, 0.5 * alpha, 0.0)
    assert keep.sum() > 50
    assert np.allclose(img[~near, 0], want[~near], rtol=1e-10, atol=1e-14)
    assert np.array_equal(nc[~near], keep[~near].astype(nc.dtype))


def test_projection_of_offaxis_mean_and_rect():
    s = one_gaussian_scene(mean=(0.4, 0.0, -0.2), log_scale=(-3.0,) * 3)
    cam = sg.tiny_camera()
    p = oracle.project(s, cam)
    X = np.array([0.4, 0.0, -0.2], np.float32).astype(np.float64)
    u = cam.fx * X[0] / 4.0 + cam.cx
    v = cam.fy * (-X[2]) / 4.0 + cam.cy
    assert p["xy"][0] == pytest.approx([u, v], rel=1e-12)
    r = p["radius"][0]
    assert p["rect"][0].tolist() == [math.floor((u - r) / 16), math.floor((v - r) / 16),
                                     math.floor((u + r) / 16) + 1, math.floor((v + r) / 16) + 1]


def test_cull_behind_near_plane():
    s = one_gaussian_scene(mean=(0.0, -3.9, 0.0))  # 0.1 in front of the camera, znear = 0.2
    p = oracle.project(s, sg.tiny_camera())
    assert p["radius"][0] == 0 and p["rect"][0].tolist() == [0, 0, 0, 0]


# --------------------------------------------------------------------- SH colour

def test_sh_basis_against_scipy():
    """Real SH basis (no Condon-Shortley phase) built from scipy's complex harmonics."""
    from scipy.special import sph_harm_y
    rng = np.random.default_rng(1)
    for _ in range(20):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        want = []
        for l in range(4):
            for m in range(-l, l + 1):
                Y = sph_harm_y(l, abs(m), theta, phi)
                if m > 0:
                    want.append(float(math.sqrt(2) * (-1) ** m * Y.real))
                elif m < 0:
                    want.append(float(math.sqrt(2) * (-1) ** m * Y.imag))
                else:
                    want.append(float(Y.real))
        assert oracle.sh_basis(3, d) == pytest.approx(want, abs=1e-12)


def test_sh_colour_is_view_dependent_and_clamped():
    s = sg.make_object(0, n=64, res_spatial=(8,), res_time=4, h=8)
    cam = sg.hemisphere_cameras(1, width=64, height=64)[0]
    p = oracle.project(s, cam)
    vis = p["radius"] > 0
    assert vis.sum() > 10
    assert (p["rgb"][vis] >= 0).all()
    # colour = max(0, 0.5 + sum_k Y_k(dir) c_k), dir from the camera centre to the mean
    W = np.asarray(cam.world_to_cam, np.float64)
    campos = -W[:3, :3].T @ W[:3, 3]
    g = int(np.flatnonzero(vis)[0])
    d = s.means[g].astype(np.float64) - campos
    d /= np.linalg.norm(d)
    Y = oracle.sh_basis(3, d)
    want = np.maximum(0.0, 0.5 + Y @ s.sh[g].astype(np.float64))
    assert p["rgb"][g] == pytest.approx(want, rel=1e-12)


# --------------------------------------------------------------------- Eq. 5 HexPlane

def test_bilinear_matches_scipy_regular_grid():
    """interp of Eq. 5 is corner-aligned bilinear; compare with scipy's RegularGridInterpolator."""
    from scipy.interpolate import RegularGridInterpolator
    s = sg.make_tiny(3)
    shapes = sg.plane_shapes(s.res_spatial, s.res_time, s.feat_dim)
    offs = np.cumsum([0] + [int(np.prod(sh)) for sh in shapes])
    rng = np.random.default_rng(0)
    for p in range(6):
        rb, ra, h = shapes[p]
        grid = s.planes[offs[p]:offs[p + 1]].reshape(rb, ra, h).astype(np.float64)
        f = RegularGridInterpolator((np.linspace(-1, 1, rb), np.linspace(-1, 1, ra)), grid)
        for _ in range(10):
            ua, ub = rng.uniform(-1, 1, 2)
            assert oracle.plane_sample(s, 0, p, ua, ub) == pytest.approx(f([ub, ua])[0], rel=1e-12, abs=1e-14)
        # vertices return the stored value; outside the box clamps to the border
        assert oracle.plane_sample(s, 0, p, -1.0, 1.0) == pytest.approx(grid[rb - 1, 0], abs=0)
        assert oracle.plane_sample(s, 0, p, -3.0, 7.0) == pytest.approx(grid[rb - 1, 0], abs=0)
        assert oracle.plane_sample(s, 0, p, 1.0, -1.0) == pytest.approx(grid[0, ra - 1], abs=0)


def test_bilinear_on_2x2_grids_by_hand():
    """The smallest grid (R = 2 on every axis): the four stored corners weighted by
    (1-a)(1-b), a(1-b), (1-a)b, ab with a = (u_a+1)/2, b = (u_b+1)/2 (corner-aligned)."""
    s = sg.make_tiny(9, n=4)
    s.res_spatial, s.res_time, s.feat_dim = (2,), 2, 4
    rng = np.random.default_rng(9)
    s.planes = rng.normal(1.0, 0.3, 6 * 2 * 2 * 4).astype(np.float32)
    for p in range(6):
        g = s.planes[16 * p:16 * (p + 1)].reshape(2, 2, 4).astype(np.float64)  # [b][a][h]
        for ua, ub in ((-1.0, -1.0), (1.0, 1.0), (0.3, -0.6), (-0.9, 0.95), (0.0, 0.0)):
            a, b = (ua + 1) / 2, (ub + 1) / 2
            want = (1 - a) * (1 - b) * g[0, 0] + a * (1 - b) * g[0, 1] + (1 - a) * b * g[1, 0] + a * b * g[1, 1]
            assert oracle.plane_sample(s, 0, p, ua, ub) == pytest.approx(want, rel=1e-14, abs=1e-15)


def test_hadamard_of_constant_planes_is_v_to_the_sixth():
    s = sg.make_object(0, n=50, res_spatial=(8, 16), res_time=5, h=8)
    shapes = sg.plane_shapes(s.res_spatial, s.res_time, s.feat_dim)
    rng = np.random.default_rng(2)
    v = rng.uniform(0.5, 1.5, (2, 8)).astype(np.float32)  # per level, per channel
    parts = []
    for i, sh in enumerate(shapes):
        parts.append(np.broadcast_to(v[i // 6], sh).ravel())
    s.planes = np.concatenate(parts).astype(np.float32)
    fh = oracle.features(s, s.means.astype(np.float64), 0.3)
    want = np.concatenate([v[0].astype(np.float64) ** 6, v[1].astype(np.float64) ** 6])
    assert np.allclose(fh, want[None, :], rtol=1e-13, atol=0)


def test_features_concat_levels_and_time_axis():
    """Each level's block of f_h depends on its own planes only, and only the
    xt/yt/zt planes see the time coordinate."""
    s = sg.make_object(0, n=30, res_spatial=(8, 16), res_time=5, h=4)
    X = s.means.astype(np.float64)
    a = oracle.features(s, X, 0.2)
    shapes = sg.plane_shapes(s.res_spatial, s.res_time, s.feat_dim)
    sizes = [int(np.prod(x)) for x in shapes]
    s2 = s.copy()
    lvl1 = sum(sizes[:6])
    s2.planes[lvl1:] *= 2.0  # scale every plane of level 1 by 2 -> level-1 features x 2^6
    b = oracle.features(s2, X, 0.2)
    assert np.allclose(b[:, :4], a[:, :4], rtol=0, atol=0)
    assert np.allclose(b[:, 4:], 64.0 * a[:, 4:], rtol=1e-13)
    # make the time planes constant in t: features no longer depend on t
    s3 = s.copy()
    off = 0
    for i, (rb, ra, h) in enumerate(shapes):
        if i % 6 >= 3:
            blk = s3.planes[off:off + rb * ra * h].reshape(rb, ra, h)
            blk[:] = blk[:1]
        off += rb * ra * h
    assert np.allclose(oracle.features(s3, X, 0.1), oracle.features(s3, X, 0.9), rtol=1e-13)
    assert not np.allclose(oracle.features(s, X, 0.1), oracle.features(s, X, 0.9))


def test_features_of_bilinear_planes_closed_form():
    """Planes filled with bilinear functions of their own two grid coordinates are
    reproduced exactly by corner-aligned interpolation, so Eq. 5 has a closed form:
    f_l[c] = prod over the six planes of (k0 + k1 u_a + k2 u_b + k3 u_a u_b) at the
    normalised coordinates u = 2 (x - box_min) / (box_max - box_min) - 1 and
    tau = 2 t - 1.  This fixes the axis pair each plane reads (xy xz yz xt yt zt),
    the box and time normalisation and the level blocks.  Vertex coordinates and
    coefficients are dyadic, so the float32 plane values hold them exactly."""
    axes = [(0, 1), (0, 2), (1, 2), (0, 3), (1, 3), (2, 3)]
    s = sg.make_tiny(0, n=8)
    s.res_spatial, s.res_time, s.feat_dim = (5, 9), 5, 3
    lo, hi = np.array([0.0, -2.0, 1.0]), np.array([4.0, 2.0, 1.5])
    s.aabb_min, s.aabb_max = tuple(lo), tuple(hi)
    rng = np.random.default_rng(11)
    coef = rng.integers(-3, 4, (2, 6, 4, 3)) / 8.0   # level, plane, (1, u_a, u_b, u_a u_b), channel
    coef[:, :, 0, :] = rng.integers(6, 11, (2, 6, 3)) / 8.0
    parts = []
    for i, (rb, ra, h) in enumerate(sg.plane_shapes(s.res_spatial, s.res_time, s.feat_dim)):
        c = coef[i // 6, i % 6]
        ua = np.linspace(-1, 1, ra)[None, :, None]
        ub = np.linspace(-1, 1, rb)[:, None, None]
        parts.append((c[0] + c[1] * ua + c[2] * ub + c[3] * ua * ub).astype(np.float32).ravel())
    s.planes = np.concatenate(parts)
    X = lo + (hi - lo) * rng.uniform(0.02, 0.98, (40, 3))
    for t in (0.0, 0.37, 1.0):
        u = np.concatenate([2 * (X - lo) / (hi - lo) - 1, np.full((len(X), 1), 2 * t - 1)], 1)
        want = np.ones((len(X), 2, 3))
        for lvl in range(2):
            for p, (a, b) in enumerate(axes):
                c = coef[lvl, p]
                ua, ub = u[:, a:a + 1], u[:, b:b + 1]
                want[:, lvl] *= c[0] + c[1] * ua + c[2] * ub + c[3] * ua * ub
        assert oracle.features(s, X, t) == pytest.approx(want.reshape(len(X), 6), rel=1e-12, abs=1e-14)


# --------------------------------------------------------------------- MLP heads (Sec. 4.2)

def _layers(s):
    hin = s.feat_dim * s.n_levels
    out, off = [], 0
    for o, i in sg.mlp_layer_shapes(hin, s.mlp_width):
        out.append((off, o, i))
        off += o * i + o
    return out


def test_mlp_hand_built_network():
    """A network wired by hand: dX_1 = 6 * relu(f_h[5]), dr_0 = 2 relu(f_h[5]) + 0.25,
    ds_2 = -relu(f_h[5]); every other output is its bias."""
    s = sg.make_tiny(0)
    L = _layers(s)
    m = np.zeros_like(s.mlp)

    def W(k, o, i, v):
        off, O, I = L[k]
        m[off + o * I + i] = v

    def B(k, o, v):
        off, O, I = L[k]
        m[off + O * I + o] = v

    W(0, 0, 5, 1.0); W(1, 0, 0, 1.0)
    W(2, 0, 0, 2.0); W(3, 1, 0, 3.0)                    # x head
    W(4, 3, 0, 1.0); W(5, 0, 3, 2.0); B(5, 0, 0.25)     # r head
    W(6, 7, 0, 1.0); W(7, 2, 7, -1.0); B(7, 0, 0.5)     # s head
    s.mlp = m
    fh = np.random.default_rng(0).normal(size=(40, 16))
    d = oracle.mlp(s, fh)
    r = np.maximum(fh[:, 5], 0)
    want = np.zeros((40, 10))
    want[:, 1] = 6 * r
    want[:, 3] = 2 * r + 0.25
    want[:, 7] = 0.5
    want[:, 9] = -r
    assert np.array_equal(d, want)


def test_mlp_against_torch_linear_layers():
    torch = pytest.importorskip("torch")
    s = sg.make_tiny(1, mlp_std=0.3, bias_std=0.1)
    L = _layers(s)
    lins = []
    for off, o, i in L:
        lin = torch.nn.Linear(i, o).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(s.mlp[off:off + o * i].reshape(o, i).astype(np.float64)))
            lin.bias.copy_(torch.from_numpy(s.mlp[off + o * i:off + o * i + o].astype(np.float64)))
        lins.append(lin)
    fh = np.random.default_rng(1).normal(size=(25, 16))
    x = torch.from_numpy(fh)
    relu = torch.relu
    fd = relu(lins[1](relu(lins[0](x))))
    outs = [lins[3 + 2 * h](relu(lins[2 + 2 * h](fd))) for h in range(3)]
    want = torch.cat(outs, 1).detach().numpy()
    assert oracle.mlp(s, fh) == pytest.approx(want, rel=1e-12, abs=1e-14)


# --------------------------------------------------------------------- App. B: colour and opacity heads

def _color_layers(s):
    """(offset, out, in) of the colour and opacity heads c1 c2 a1 a2 after the 8 layers."""
    k = (s.sh_degree + 1) ** 2
    shapes = sg.mlp_layer_shapes(s.feat_dim * s.n_levels, s.mlp_width, k)
    off, out = 0, []
    for o, i in shapes:
        out.append((off, o, i))
        off += o * i + o
    assert off == s.mlp.size
    return out[8:]


def test_color_heads_against_torch_linear_layers():
    """dC = phi_C(f_d) and dalpha = phi_alpha(f_d) (App. B) with torch.nn.Linear
    layers on the oracle's features: C' = C + dC (the 3K outputs in the [K][3]
    layout), logit' = logit + dalpha."""
    torch = pytest.importorskip("torch")
    s = sg.with_color_heads(sg.make_object(3, n=30, res_spatial=(6, 8), res_time=4, h=16, mlp_std=0.2), 4, std=0.2)
    lins = []
    for off, o, i in _layers(s) + _color_layers(s):
        lin = torch.nn.Linear(i, o).double()
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(s.mlp[off:off + o * i].reshape(o, i).astype(np.float64)))
            lin.bias.copy_(torch.from_numpy(s.mlp[off + o * i:off + o * i + o].astype(np.float64)))
        lins.append(lin)
    t = 0.6
    x = torch.from_numpy(oracle.features(s, s.means.astype(np.float64), t))
    relu = torch.relu
    fd = relu(lins[1](relu(lins[0](x))))
    dc = lins[9](relu(lins[8](fd))).detach().numpy().reshape(s.n, -1, 3)
    da = lins[11](relu(lins[10](fd))).detach().numpy()[:, 0]
    sh, lg = oracle.appearance(s, t)
    assert sh == pytest.approx(s.sh.astype(np.float64) + dc, rel=1e-12, abs=1e-14)
    assert lg == pytest.approx(s.opacity_logits.astype(np.float64) + da, rel=1e-12, abs=1e-14)
    assert np.abs(dc).max() > 1e-3 and np.abs(da).max() > 1e-3


def test_color_heads_zero_layers_change_nothing():
    """Colour and opacity heads with all weights and biases 0 render exactly the scene without them."""
    s = sg.make_tiny(5, n=300, mlp_std=0.2)
    c = sg.with_color_heads(s, 1)
    for off, o, i in _color_layers(c):
        c.mlp[off:off + o * i + o] = 0.0
    a, Ta, na, _, _ = oracle.render(s, sg.tiny_camera(), 0.4)
    b, Tb, nb, _, _ = oracle.render(c, sg.tiny_camera(), 0.4)
    assert np.array_equal(a, b) and np.array_equal(Ta, Tb) and np.array_equal(na, nb)


def test_color_heads_output_bias_is_a_constant_shift():
    """Only the output biases non-zero: every Gaussian's SH coefficients move by the
    colour head's bias and its opacity logit by the opacity head's, so the frame is
    the frame of the scene shifted that way without heads."""
    s = sg.make_object(2, n=400, res_spatial=(6, 8), res_time=4, h=16, mlp_std=0.1)
    c = sg.with_color_heads(s, 3)
    (o1, n1, i1), (o2, n2, i2), (o3, n3, i3), (o4, n4, i4) = _color_layers(c)
    for off, o, i in _color_layers(c):
        c.mlp[off:off + o * i] = 0.0
    beta = c.mlp[o2 + n2 * i2:o2 + n2 * i2 + n2].astype(np.float64)
    gamma = float(c.mlp[o4 + n4 * i4])
    sh, lg = oracle.appearance(c, 0.5)
    assert np.array_equal(sh, s.sh.astype(np.float64) + beta.reshape(-1, 3)[None])
    assert np.array_equal(lg, s.opacity_logits.astype(np.float64) + gamma)
    shifted = s.copy()
    shifted.sh = (s.sh.astype(np.float64) + beta.reshape(-1, 3)[None]).astype(np.float32)
    shifted.opacity_logits = (s.opacity_logits.astype(np.float64) + gamma).astype(np.float32)
    cam = sg.hemisphere_cameras(2, width=96, height=80, seed=1)[0]
    X, Q, S = oracle.deform(c, 0.5)
    p_heads = oracle.project(c, cam, X, Q, S, sh=sh, opacity_logits=lg)
    p_shift = oracle.project(shifted, cam, X, Q, S, sh=shifted.sh.astype(np.float64),
                             opacity_logits=shifted.opacity_logits.astype(np.float64))
    np.testing.assert_allclose(p_heads["rgb"], p_shift["rgb"], rtol=0, atol=1e-6)
    np.testing.assert_allclose(p_heads["opacity"], p_shift["opacity"], rtol=1e-6)
    img_c, *_ = oracle.render(c, cam, 0.5)
    img_s, *_ = oracle.render(shifted, cam, 0.5)
    np.testing.assert_allclose(img_c, img_s, atol=2e-6)


def test_deform_is_eq6_addition():
    s = sg.make_tiny(2, mlp_std=0.3)
    X, Q, S = oracle.deform(s, 0.7)
    d = oracle.mlp(s, oracle.features(s, s.means.astype(np.float64), 0.7))
    assert np.allclose(X - s.means, d[:, :3], rtol=0, atol=1e-15)
    assert np.allclose(Q - s.quats, d[:, 3:7], rtol=0, atol=1e-15)
    assert np.allclose(S - s.log_scales, d[:, 7:], rtol=0, atol=1e-15)
    assert np.abs(d).max() > 1e-3


# --------------------------------------------------------------------- special case (b)

def test_zero_heads_reduce_to_static_3dgs():
    """Zeroing the head output layers gives dG = 0, so the 4D render equals the
    static render of the canonical Gaussians (the warm-up mode of Sec. 4.3)."""
    s = sg.make_tiny(4, mlp_std=0.3)
    L = _layers(s)
    for k in (3, 5, 7):
        off, o, i = L[k]
        s.mlp[off:off + o * i + o] = 0.0
    X, Q, S = oracle.deform(s, 0.3)
    assert np.array_equal(X, s.means.astype(np.float64))
    assert np.array_equal(Q, s.quats.astype(np.float64))
    cam = sg.tiny_camera()
    a = oracle.render(s, cam, 0.3, deform=True)
    b = oracle.render(s, cam, 0.3, deform=False)
    assert np.array_equal(a[0], b[0]) and a[4] == b[4]


def test_zero_planes_reduce_to_static_3dgs():
    s = sg.make_tiny(5, mlp_std=0.3)
    s.planes[:] = 0.0
    cam = sg.tiny_camera()
    a = oracle.render(s, cam, 0.8, deform=True)
    b = oracle.render(s, cam, 0.8, deform=False)
    assert np.array_equal(a[0], b[0])


# --------------------------------------------------------------------- tiling, sort, ranges (c)

def test_tiled_equals_bruteforce_per_pixel():
    for seed in range(3):
        s = sg.make_tiny(seed)
        cam = sg.tiny_camera()
        X, Q, S = oracle.deform(s, 0.5)
        p = oracle.project(s, cam, X, Q, S)
        keys, vals, ranges = oracle.bin_sort(oracle.depth_bits(p["depth"]), p["rect"], 8, 8)
        img, T, nc, _ = oracle.composite(128, 128, ranges, vals, p)
        img_bf, T_bf = oracle.composite_bruteforce(128, 128, p)
        assert np.array_equal(img, img_bf) and np.array_equal(T, T_bf)
        img_r, *_ = oracle.render(s, cam, 0.5)
        assert np.array_equal(img, img_r)


def test_bin_sort_against_numpy_lexsort():
    rng = np.random.default_rng(7)
    n, tx, ty = 3000, 13, 9
    depth = rng.uniform(0.5, 9.0, n).astype(np.float32)
    depth[::17] = depth[5]  # ties: broken by Gaussian index
    x0 = rng.integers(0, tx, n); y0 = rng.integers(0, ty, n)
    rect = np.stack([x0, y0, np.minimum(tx, x0 + rng.integers(0, 4, n)),
                     np.minimum(ty, y0 + rng.integers(0, 4, n))], 1).astype(np.int32)
    bits = depth.view(np.uint32)
    keys, vals, ranges = oracle.bin_sort(bits, rect, tx, ty)
    tiles, gids = [], []
    for g in range(n):
        for yy in range(rect[g, 1], rect[g, 3]):
            for xx in range(rect[g, 0], rect[g, 2]):
                tiles.append(yy * tx + xx); gids.append(g)
    tiles, gids = np.array(tiles, np.int64), np.array(gids, np.int64)
    order = np.lexsort((gids, depth[gids], tiles))
    assert np.array_equal(vals, gids[order].astype(np.uint32))
    assert np.array_equal(keys, ((tiles[order].astype(np.uint64) << np.uint64(32)) | bits[gids[order]]))
    counts = np.bincount(tiles, minlength=tx * ty)
    assert (ranges[:, 1] - ranges[:, 0]).sum() == len(tiles)
    nz = counts > 0
    assert np.array_equal((ranges[:, 1] - ranges[:, 0])[nz], counts[nz])
    assert np.array_equal(ranges[nz, 0], np.cumsum(counts)[nz] - counts[nz])


# --------------------------------------------------------------------- transmittance (d)

def test_transmittance_invariants():
    s = sg.make_tiny(6)
    cam = sg.tiny_camera()
    X, Q, S = oracle.deform(s, 0.5)
    p = oracle.project(s, cam, X, Q, S)
    _, vals, ranges = oracle.bin_sort(oracle.depth_bits(p["depth"]), p["rect"], 8, 8)
    img, T, nc, _ = oracle.composite(128, 128, ranges, vals, p)
    assert (T >= 1e-4).all() and (T <= 1.0).all()
    lens = (ranges[:, 1] - ranges[:, 0]).reshape(8, 8)
    assert (nc <= np.kron(lens, np.ones((16, 16), np.int64))).all()
    assert (img >= 0).all() and (img <= p["rgb"].max() + 1e-12).all()
    # T over prefixes of each tile's list is non-increasing
    prev = np.ones((128, 128))
    for k in range(0, int(lens.max()) + 1, 7):
        r2 = ranges.copy()
        r2[:, 1] = np.minimum(r2[:, 1], r2[:, 0] + k)
        _, Tk, _, _ = oracle.composite(128, 128, r2, vals, p)
        assert (Tk <= prev + 1e-15).all()
        prev = Tk
    assert np.array_equal(prev, T) or k < lens.max()


def test_image_is_convex_combination_bound():
    """sum_i a_i prod_{j<i}(1-a_j) = 1 - T_final, so each channel <= (1 - T) * max colour."""
    s = sg.make_tiny(8)
    img, T, *_ = oracle.render(s, sg.tiny_camera(), 0.5)
    p = oracle.project(s, sg.tiny_camera(), *oracle.deform(s, 0.5))
    assert (img <= (1.0 - T)[..., None] * p["rgb"].max(0)[None, None, :] + 1e-12).all()


def test_unstable_pixels_flags_threshold_decisions_only():
    """The pixels a float32 implementation may decide differently are those whose
    alpha lies within the margin of 1/255 (or T of 1e-4, or a depth tie, or a tile
    edge); with one Gaussian placed so that a neighbour's alpha is 1/255 to 1e-7,
    that pixel and no pixel far from every threshold is flagged."""
    ls, d = -3.0, 3
    cam = centred_camera()
    var = (cam.fx * math.exp(float(np.float32(ls))) / 4.0) ** 2 + 0.3
    o = (1 / 255) * (1 + 1e-7) / math.exp(-0.5 * d * d / var)
    s = one_gaussian_scene(log_scale=(ls,) * 3, logit=math.log(o / (1 - o)))
    mask, img, T, nc, _ = oracle.unstable_pixels(s, cam, 0.5, deform=False)
    assert mask[64, 64 + d] and mask[64 + d, 64]
    assert not mask[64, 64] and not mask[64, 64 + 1] and not mask[10, 10]
    assert mask.sum() < 0.01 * mask.size


# --------------------------------------------------------------------- per-pixel outcomes (parity support)

def _proj(rows):
    """Projected Gaussians (u, v, conic a, b, c, opacity, rgb, depth) as the oracle's dict."""
    r = np.array(rows, np.float64)
    return dict(xy=np.ascontiguousarray(r[:, 0:2]), conic=np.ascontiguousarray(r[:, 2:5]),
                opacity=np.ascontiguousarray(r[:, 5]), rgb=np.ascontiguousarray(r[:, 6:9]),
                depth=np.ascontiguousarray(r[:, 9]))


def test_pixel_outcomes_single_term_closed_form():
    """One Gaussian centred on the pixel, far from every threshold: the only
    outcome is colour * min(0.99, o), T = 1 - alpha, one contributor (Eq. 4)."""
    p = _proj([(10.5, 7.5, 0.2, 0.0, 0.2, 0.6, 0.3, 0.5, 0.9, 2.0)])
    out = oracle.pixel_outcomes([0], 10, 7, p)
    assert out.shape == (1, 5)
    np.testing.assert_allclose(out[0, :3], 0.6 * np.array([0.3, 0.5, 0.9]), rtol=0, atol=1e-15)
    assert out[0, 3] == pytest.approx(0.4, abs=1e-15) and out[0, 4] == 1


def test_pixel_outcomes_alpha_at_skip_threshold_both_ways():
    """alpha = (1/255)(1 + 1e-7): the term is blended, and the outcome with it
    skipped (black, T = 1, no contributor) is listed too."""
    d = 2.0
    a = (1 / 255) * (1 + 1e-7)
    o = a / math.exp(-0.5 * 0.5 * d * d)
    p = _proj([(10.5 + d, 7.5, 0.5, 0.0, 0.5, o, 1.0, 0.2, 0.4, 2.0)])
    out = oracle.pixel_outcomes([0], 10, 7, p)
    assert out.shape == (2, 5)
    np.testing.assert_allclose(out[0, :3], a * np.array([1.0, 0.2, 0.4]), rtol=1e-12)
    assert out[0, 4] == 1 and out[0, 3] == pytest.approx(1 - a, rel=1e-12)
    np.testing.assert_array_equal(out[1], [0, 0, 0, 1, 0])
    # far from the threshold: one outcome only
    assert oracle.pixel_outcomes([0], 10, 7, _proj([(10.5 + d, 7.5, 0.5, 0.0, 0.5, 10 * o, 1, 1, 1, 2.0)])
                                 ).shape == (1, 5)


def test_pixel_outcomes_depth_tie_both_orders():
    """Two blended terms at equal depth: both front-to-back orders are outcomes,
    c1 a1 + c2 a2 (1 - a1) and c2 a2 + c1 a1 (1 - a2)."""
    a1, a2 = 0.5, 0.3
    c1, c2 = np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.0])
    p = _proj([(3.5, 3.5, 0.1, 0.0, 0.1, a1, *c1, 5.0), (3.5, 3.5, 0.1, 0.0, 0.1, a2, *c2, 5.0)])
    out = oracle.pixel_outcomes([0, 1], 3, 3, p)
    assert out.shape == (2, 5)
    np.testing.assert_allclose(out[0, :3], c1 * a1 + c2 * a2 * (1 - a1), atol=1e-15)
    np.testing.assert_allclose(out[1, :3], c2 * a2 + c1 * a1 * (1 - a2), atol=1e-15)
    assert out[0, 3] == pytest.approx(out[1, 3], abs=1e-15)  # T does not depend on the order
    # well-separated depths: one order only
    p2 = _proj([(3.5, 3.5, 0.1, 0.0, 0.1, a1, *c1, 5.0), (3.5, 3.5, 0.1, 0.0, 0.1, a2, *c2, 5.1)])
    assert oracle.pixel_outcomes([0, 1], 3, 3, p2).shape == (1, 5)


def test_pixel_outcomes_transmittance_stop_both_ways():
    """T after two terms is 1e-4 (1 + 1e-6): the second term is blended; the
    outcome that stops before it (the stop rule of Eq. 4's reading) is listed too."""
    a1 = 0.99
    a2 = 1.0 - 1e-2 * (1 + 1e-6)
    c1, c2 = np.array([0.2, 0.4, 0.6]), np.array([1.0, 1.0, 1.0])
    p = _proj([(0.5, 0.5, 0.1, 0.0, 0.1, 1.0, *c1, 1.0), (0.5, 0.5, 0.1, 0.0, 0.1, a2, *c2, 2.0)])
    out = oracle.pixel_outcomes([0, 1], 0, 0, p)
    assert out.shape == (2, 5)
    np.testing.assert_allclose(out[0, :3], c1 * a1 + c2 * a2 * (1 - a1), rtol=1e-12)
    assert out[0, 4] == 2
    np.testing.assert_allclose(out[1, :3], c1 * a1, rtol=1e-12)
    assert out[1, 4] == 1 and out[1, 3] == pytest.approx(1 - a1, rel=1e-12)


def test_pixel_outcomes_identical_terms_decide_alike():
    """Two identical terms (a Gaussian and its densification copy) at the skip
    threshold: both are blended or both skipped -- two outcomes, not four -- and
    their equal depths form no order decision (swapping them changes nothing)."""
    d = 2.0
    a = (1 / 255) * (1 + 1e-7)
    o = a / math.exp(-0.5 * 0.5 * d * d)
    g = (10.5 + d, 7.5, 0.5, 0.0, 0.5, o, 1.0, 0.2, 0.4, 2.0)
    out = oracle.pixel_outcomes([0, 1], 10, 7, _proj([g, g]))
    assert out.shape == (2, 5)
    np.testing.assert_allclose(out[0, :3], (a + a * (1 - a)) * np.array([1.0, 0.2, 0.4]), rtol=1e-12)
    assert out[0, 4] == 2
    np.testing.assert_array_equal(out[1], [0, 0, 0, 1, 0])
    # the same two terms with one colour changed are two decisions again
    h = g[:6] + (0.5, 0.2, 0.4) + g[9:]
    assert oracle.pixel_outcomes([0, 1], 10, 7, _proj([g, h])).shape[0] > 2


def test_pixel_outcomes_limit_on_flips():
    """More near-threshold decisions than max_flip: not enumerated (None)."""
    rows = [(0.5, 0.5, 0.1, 0.0, 0.1, 0.2, 1 - 0.1 * k, 1, 1, 3.0) for k in range(4)]  # three depth ties
    assert oracle.pixel_outcomes([0, 1, 2, 3], 0, 0, _proj(rows), max_flip=2) is None
    assert oracle.pixel_outcomes([0, 1, 2, 3], 0, 0, _proj(rows), max_flip=3).shape == (8, 5)


# --------------------------------------------------------------------- training step (Sec. 4.3, App. A)

def test_l1_loss_closed_form():
    img = np.array([[0.5, 0.2, 0.9], [0.1, 0.1, 0.4]])
    tgt = np.array([[0.4, 0.2, 1.0], [0.3, 0.0, 0.4]])
    loss, g = oracle.l1_loss(img, tgt)
    assert loss == pytest.approx((0.1 + 0 + 0.1 + 0.2 + 0.1 + 0) / 6, abs=1e-15)
    np.testing.assert_array_equal(g * 6, [[1, 0, -1], [-1, 1, 0]])


def _plane_scene(fill):
    """A scene whose every plane value is fill(level, plane, b, a, c)."""
    s = sg.make_object(0, n=10, res_spatial=(4, 6), res_time=5, h=16)
    out = []
    for lvl, R in enumerate(s.res_spatial):
        for p, (ax, bx) in enumerate([(0, 1), (0, 2), (1, 2), (0, 3), (1, 3), (2, 3)]):
            Ra = R if ax < 3 else s.res_time
            Rb = R if bx < 3 else s.res_time
            b, a, c = np.meshgrid(np.arange(Rb), np.arange(Ra), np.arange(s.feat_dim), indexing="ij")
            out.append(fill(lvl, p, b, a, c).astype(np.float32).ravel())
    s.planes = np.concatenate(out)
    return s


def test_tv_loss_of_linear_planes_closed_form():
    """P = alpha a + beta b (+ any per-channel offset): every neighbour difference
    along a is alpha and along b is beta, so each plane adds alpha^2 + beta^2; 12
    planes in all; the gradient vanishes at interior cells."""
    al, be = 0.25, -0.5
    s = _plane_scene(lambda lvl, p, b, a, c: al * a + be * b + 0.0625 * c)  # exact in float32
    loss, g = oracle.tv_loss(s, 0.3)
    assert loss == pytest.approx(0.3 * 12 * (al ** 2 + be ** 2), rel=1e-12)
    P0 = s.res_spatial[0]
    h = s.feat_dim
    g0 = g[:P0 * P0 * h].reshape(P0, P0, h)     # level 0, plane xy
    np.testing.assert_allclose(g0[1:-1, 1:-1], 0.0, atol=1e-15)
    # a corner cell (b=0, a=0): -2 alpha / n_a - 2 beta / n_b per channel, times the weight
    na, nb = P0 * (P0 - 1) * h, (P0 - 1) * P0 * h
    np.testing.assert_allclose(g0[0, 0], 0.3 * (-2 * al / na - 2 * be / nb), rtol=1e-12)


def test_tv_loss_of_checkerboard_planes_closed_form():
    """P = (-1)^(a+b): every neighbour difference is +-2 (squared 4), so each plane
    adds 8; an interior cell's gradient is w * 8 P (1/n_a + 1/n_b) per channel."""
    s = _plane_scene(lambda lvl, p, b, a, c: (-1.0) ** (a + b))
    loss, g = oracle.tv_loss(s, 1.0)
    assert loss == pytest.approx(12 * 8.0, rel=1e-12)
    P0, h = s.res_spatial[0], s.feat_dim
    na, nb = P0 * (P0 - 1) * h, (P0 - 1) * P0 * h
    g0 = g[:P0 * P0 * h].reshape(P0, P0, h)
    np.testing.assert_allclose(g0[1, 2], 8.0 * (-1.0) ** 3 * (1 / na + 1 / nb), rtol=1e-12)


def test_tv_gradient_matches_central_differences():
    s = _plane_scene(lambda lvl, p, b, a, c: np.sin(0.7 * a + 1.3 * b + 0.1 * c + p + lvl))
    _, g = oracle.tv_loss(s, 0.7)
    rng = np.random.default_rng(0)
    for i in rng.choice(s.planes.size, 12, replace=False):
        x0 = s.planes[i]
        h = 2.0 ** -10
        s.planes[i] = x0 + h
        lp, _ = oracle.tv_loss(s, 0.7)
        s.planes[i] = x0 - h
        lm, _ = oracle.tv_loss(s, 0.7)
        s.planes[i] = x0
        assert (lp - lm) / (2 * h) == pytest.approx(g[i], rel=1e-6, abs=1e-12)


def test_lr_schedule_endpoints_and_geometric_midpoint():
    assert oracle.lr_at(1.6e-3, 1.6e-4, 0, 1000) == pytest.approx(1.6e-3, rel=1e-15)
    assert oracle.lr_at(1.6e-3, 1.6e-4, 1000, 1000) == pytest.approx(1.6e-4, rel=1e-13)
    assert oracle.lr_at(1.6e-3, 1.6e-4, 5000, 1000) == pytest.approx(1.6e-4, rel=1e-13)
    assert oracle.lr_at(1.6e-3, 1.6e-4, 500, 1000) == pytest.approx(math.sqrt(1.6e-3 * 1.6e-4), rel=1e-13)


def test_adam_against_torch_optim_adam():
    """Three bias-corrected Adam steps against torch.optim.Adam; the first step
    moves each parameter by lr * g / (|g| + eps)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    p = rng.normal(size=50)
    grads = [rng.normal(size=50) for _ in range(3)]
    tp = torch.tensor(p.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-15)
    m, v = np.zeros(50), np.zeros(50)
    q = p.copy()
    for k, g in enumerate(grads):
        oracle.adam_step(q, g.copy(), m, v, 1e-2, 0.9, 0.999, 1e-15, k + 1)
        if k == 0:
            np.testing.assert_allclose(p - q, 1e-2 * g / (np.abs(g) + 1e-15), rtol=1e-12)
        tp.grad = torch.tensor(g)
        opt.step()
    np.testing.assert_allclose(q, tp.detach().numpy(), rtol=1e-12, atol=1e-15)


# --------------------------------------------------------------------- composition (Sec. 5.4)

def test_composition_of_one_scene_is_its_render():
    s = sg.make_tiny(2, n=400, mlp_std=0.2)
    cam = sg.tiny_camera()
    p = oracle.project_composed([s], None, cam, 0.4)
    img, T, nc, *_ = oracle.composite_projected(p, cam)
    want, Tw, ncw, _, _ = oracle.render(s, cam, 0.4)
    np.testing.assert_array_equal(img, want)
    np.testing.assert_array_equal(nc, ncw)


def test_composition_of_static_scenes_is_the_render_of_their_union():
    """With zero head output layers no Gaussian moves, so composing two scenes is
    the static render of one scene holding both sets of Gaussians (the second
    translated by its shift)."""
    a = sg.make_tiny(3, n=300, mlp_std=0.2)
    b = sg.make_tiny(4, n=250, mlp_std=0.2)
    shapes = sg.mlp_layer_shapes(16, 64)
    for s in (a, b):
        off = 0
        for k, (o, i) in enumerate(shapes):
            if k in (3, 5, 7):
                s.mlp[off:off + o * i + o] = 0.0
            off += o * i + o
    b.means = (np.round(b.means * 1024) / 1024).astype(np.float32)  # b.means + shift exact in float32
    shift = np.array([0.25, -0.125, 0.0625])
    p = oracle.project_composed([a, b], [np.zeros(3), shift], cam := sg.tiny_camera(), 0.7)
    img, T, nc, *_ = oracle.composite_projected(p, cam)
    u = a.copy()
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        extra = getattr(b, k) + (shift.astype(np.float32) if k == "means" else 0)
        setattr(u, k, np.concatenate([getattr(a, k), extra]).astype(np.float32))
    want, Tw, ncw, _, _ = oracle.render(u, cam, 0.7, deform=False)
    np.testing.assert_array_equal(img, want)
    np.testing.assert_array_equal(nc, ncw)


def test_composition_with_a_scene_out_of_view_is_the_scene_alone():
    a = sg.make_tiny(5, n=300, mlp_std=0.2)
    b = sg.make_tiny(6, n=300, mlp_std=0.2)
    cam = sg.tiny_camera()
    p = oracle.project_composed([a, b], [np.zeros(3), np.array([0.0, -50.0, 0.0])], cam, 0.5)  # behind the camera
    img, *_ = oracle.composite_projected(p, cam)
    want, *_ = oracle.render(a, cam, 0.5)
    np.testing.assert_array_equal(img, want)
