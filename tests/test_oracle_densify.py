"""Pins of the oracle's densification and pruning (App. A, which keeps the
adaptive density control of 3D Gaussian splatting) and of the view-space
gradient it accumulates, each against something other than the oracle itself:
a case worked by hand, the child positions by hand and through scipy's
rotations, the distribution of many children against the covariance of Eq. 2,
and the gradient of the projected means against central differences of the
oracle's own compositing.  None needs a GPU.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2310_08528_gb300 import scenegen as sg

LN16 = math.log(1.6)


def scene_of(rows, degree=0):
    """rows: (mean, log_scale, quat (w, x, y, z), opacity logit)."""
    s = sg.make_tiny(0, n=len(rows))
    s.means = np.array([r[0] for r in rows], np.float32)
    s.log_scales = np.array([r[1] for r in rows], np.float32)
    s.quats = np.array([r[2] for r in rows], np.float32)
    s.opacity_logits = np.array([r[3] for r in rows], np.float32)
    rng = np.random.default_rng(7)
    s.sh = rng.normal(size=(len(rows), (degree + 1) ** 2, 3)).astype(np.float32)
    s.sh_degree = degree
    return s


def test_densify_case_by_hand():
    """Six Gaussians, one of each kind of decision; the output order is the kept
    Gaussians, then the copies, then the first and the second children."""
    big, small = (-1.0, -2.0, -1.5), (-4.0, -4.5, -4.0)
    rows = [((0.1, 0.0, 0.0), small, (1, 0, 0, 0), 1.0),   # 0: low gradient -> kept
            ((0.2, 0.0, 0.0), small, (1, 0, 0, 0), 1.0),   # 1: high gradient, small -> kept + copy
            ((0.3, 0.0, 0.0), big, (0.9, 0.1, 0.2, 0.3), 1.0),  # 2: high gradient, large -> two children
            ((0.4, 0.0, 0.0), big, (1, 0, 0, 0), -6.0),    # 3: transparent -> removed, children too
            ((0.5, 0.0, 0.0), small, (1, 0, 0, 0), 1.0),   # 4: never visible -> kept
            ((0.6, 0.0, 0.0), small, (1, 0, 0, 0), 1.0)]   # 5: mean gradient exactly at the threshold -> copy
    s = scene_of(rows, degree=1)
    grad_sum = np.array([0.001, 0.5, 0.9, 0.9, 0.0, 0.75], np.float32)
    visible = np.array([2, 2, 3, 1, 0, 3], np.float32)      # means 5e-4, .25, .3, .9, 0, .25
    normals = np.random.default_rng(3).normal(size=(6, 2, 3)).astype(np.float32)
    d = oracle.densify(s, grad_sum, visible, normals, grad_threshold=0.25, split_log_scale=-3.0,
                       prune_logit=math.log(0.005 / 0.995))
    assert list(d["src"]) == [0, 1, 4, 5, 1, 5, 2, 2]
    assert list(d["kind"]) == [0, 0, 0, 0, 1, 1, 2, 3]
    for o, i in enumerate(d["src"]):
        assert np.array_equal(d["quats"][o], s.quats[i].astype(np.float64))
        assert d["opacity_logits"][o] == float(s.opacity_logits[i])
        assert np.array_equal(d["sh"][o], s.sh[i].astype(np.float64))
        if d["kind"][o] < 2:  # kept and copied Gaussians are unchanged
            assert np.array_equal(d["means"][o], s.means[i].astype(np.float64))
            assert np.array_equal(d["log_scales"][o], s.log_scales[i].astype(np.float64))
        else:                 # children: the scales divided by 1.6
            assert d["log_scales"][o] == pytest.approx(s.log_scales[i].astype(np.float64) - LN16, abs=1e-15)


def test_densify_nothing_selected_keeps_everything_in_order():
    s = sg.make_tiny(1, n=50)
    z = np.zeros(50, np.float32)
    d = oracle.densify(s, z, z, np.zeros((50, 2, 3), np.float32), 1e-3, -3.0, -1e9)
    assert list(d["src"]) == list(range(50)) and not d["kind"].any()
    assert np.array_equal(d["means"], s.means.astype(np.float64))


def test_split_children_identity_rotation_by_hand():
    """With r = (1, 0, 0, 0) a child sits at mu + exp(s) * z, componentwise."""
    mu, ls = (0.25, -0.5, 1.0), (-1.0, -2.0, -0.5)
    s = scene_of([(mu, ls, (1, 0, 0, 0), 0.0)])
    z = np.array([[[0.5, -1.25, 2.0], [-0.75, 0.3, -1.5]]], np.float32)
    d = oracle.densify(s, np.array([1.0], np.float32), np.array([1.0], np.float32), z, 0.5, -3.0, -1e9)
    assert list(d["kind"]) == [2, 3]
    for c in range(2):
        for k in range(3):
            want = float(np.float32(mu[k])) + math.exp(float(np.float32(ls[k]))) * float(z[0, c, k])
            assert d["means"][c, k] == pytest.approx(want, rel=1e-14, abs=1e-15)


def test_split_children_rotated_match_scipy():
    """A general (unnormalised) quaternion: child = mu + R(r / |r|) (exp(s) * z), with R
    from scipy's rotation (scalar-last quaternion)."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(11)
    rows = [(tuple(rng.normal(size=3)), tuple(rng.uniform(-2.5, -0.5, size=3)), tuple(rng.normal(size=4) * 1.7),
             1.0) for _ in range(20)]
    s = scene_of(rows)
    z = rng.normal(size=(20, 2, 3)).astype(np.float32)
    ones = np.ones(20, np.float32)
    d = oracle.densify(s, ones, ones, z, 0.5, -3.0, -1e9)
    assert len(d["src"]) == 40
    for o in range(40):
        i, c = int(d["src"][o]), int(d["kind"][o]) - 2
        w, x, y, zz = (float(v) for v in s.quats[i])
        R = Rot.from_quat([x, y, zz, w]).as_matrix()
        want = s.means[i].astype(np.float64) + R @ (np.exp(s.log_scales[i].astype(np.float64)) * z[i, c])
        assert np.allclose(d["means"][o], want, rtol=1e-12, atol=1e-13)


def test_split_children_are_drawn_from_the_gaussian():
    """Children of many copies of one Gaussian: sample mean mu and sample covariance
    R S S^T R^T (Eq. 2), within the sampling error."""
    n = 20000
    q = np.array([0.8, -0.3, 0.4, 0.2])
    q /= np.linalg.norm(q)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    mu, ls = np.array([0.3, -0.2, 0.1]), np.array([-1.0, -2.0, -1.5])
    s = scene_of([(tuple(mu), tuple(ls), tuple(q), 2.0)] * n)
    normals = np.random.default_rng(5).normal(size=(n, 2, 3)).astype(np.float32)
    ones = np.ones(n, np.float32)
    d = oracle.densify(s, ones, ones, normals, 0.5, -3.0, -1e9)
    X = d["means"]
    assert X.shape == (2 * n, 3)
    S = np.diag(np.exp(s.log_scales[0].astype(np.float64)))
    cov = R @ S @ S @ R.T
    m = X.mean(0)
    se = np.sqrt(np.diag(cov) / (2 * n))
    assert np.all(np.abs(m - s.means[0]) < 5 * se)
    emp = np.cov(X.T)
    assert np.linalg.norm(emp - cov) <= 0.03 * np.linalg.norm(cov)


def test_projected_mean_gradient_matches_central_differences():
    """d(sum dL/dI * I)/d(projected mean) from the backward equals central
    differences of the oracle's compositing with one projected mean moved."""
    s = sg.make_tiny(2, n=60)
    s.log_scales = (s.log_scales + 1.5).astype(np.float32)  # larger footprints: more pixels per Gaussian
    cam = sg.tiny_camera(64, 64)
    rng = np.random.default_rng(0)
    dl = rng.normal(size=(64, 64, 3))
    g = oracle.render_backward(s, cam, 0.5, dl, deform=False, xy=True)["xy"]
    p = oracle.project(s, cam)
    visible = np.flatnonzero(p["radius"] > 0)
    assert len(visible) >= 20
    h = 1e-6
    worst = 0.0
    for gi in visible[:25]:
        for a in range(2):
            vals = []
            for sgn in (1, -1):
                q = {k: v.copy() for k, v in p.items()}
                q["xy"][gi, a] += sgn * h
                img = oracle.composite_projected(q, cam)[0]
                vals.append(float((dl * img).sum()))
            fd = (vals[0] - vals[1]) / (2 * h)
            scale = max(1e-6, abs(g[gi, a]))
            worst = max(worst, abs(fd - g[gi, a]) / scale)
    assert worst < 1e-5, worst
