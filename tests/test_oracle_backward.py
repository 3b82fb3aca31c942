"""The oracle's analytic backward against central finite differences of its own
FP64 forward (the gradient of L = sum(dL/dI * I) with respect to every scene
parameter).  Steps are powers of two, so the float32 scene values are perturbed
exactly.  A parameter whose +-h evaluations straddle a discrete decision of the
method (a tile-rectangle edge, the 1/255 skip, the transmittance stop, a ReLU
kink) has no derivative there; such samples are rare and are counted."""
import numpy as np
import pytest

import oracle
from paper_2310_08528_gb300 import scenegen as sg

H = 2.0 ** -13
GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh", "planes", "mlp")


def small_scene(seed, deg=0):
    if deg == 0:
        s = sg.make_tiny(seed, n=48, mlp_std=0.15, bias_std=0.05)
    else:
        s = sg.make_object(seed, n=48, res_spatial=(6, 8), res_time=4, h=16, mlp_std=0.15)
    # pull the Gaussians towards the view so that most of them are visible
    s.means *= 0.8
    s.log_scales += 1.2
    return s


def camera(w=40, h=36):
    cam = sg.tiny_camera(w, h)
    cam.fx = cam.fy = 40.0
    return cam


def loss(scene, cam, t, dl, deform=True):
    img, *_ = oracle.render(scene, cam, t, deform=deform)
    return float(np.sum(img * dl))


def fd_check(scene, cam, t, dl, deform, rng, per_group=14):
    g = oracle.render_backward(scene, cam, t, dl, deform=deform)
    rows = []
    for name in GROUPS:
        arr = getattr(scene, name)
        flat = arr.reshape(-1)
        ga = g[name].reshape(-1)
        nz = np.flatnonzero(np.abs(ga) > 1e-9)
        pick = list(rng.choice(nz, size=min(per_group, len(nz)), replace=False)) if len(nz) else []
        pick += list(rng.integers(0, flat.size, 3))
        for i in pick:
            x0 = flat[i]
            flat[i] = np.float32(x0 + H)
            lp = loss(scene, cam, t, dl, deform)
            flat[i] = np.float32(x0 - H)
            lm = loss(scene, cam, t, dl, deform)
            flat[i] = x0
            fd = (lp - lm) / (2 * H)
            rows.append((name, int(i), float(ga[i]), fd))
    return g, rows


def _assert_rows(rows, rel=1e-4, max_bad_frac=0.05):
    scale = max(abs(r[2]) for r in rows)
    bad = [r for r in rows if abs(r[2] - r[3]) > rel * max(abs(r[2]), abs(r[3])) + 1e-7 * scale]
    assert len(bad) <= max_bad_frac * len(rows), bad[:10]
    for name in GROUPS:
        assert any(r[0] == name and abs(r[2]) > 0 for r in rows), f"no non-zero gradient checked for {name}"


@pytest.mark.parametrize("seed,deg", [(0, 0), (1, 3)])
def test_backward_matches_central_differences(seed, deg):
    s = small_scene(seed, deg)
    cam = camera()
    rng = np.random.default_rng(seed)
    dl = rng.normal(size=(cam.height, cam.width, 3))
    _, rows = fd_check(s, cam, 0.4, dl, True, rng)
    _assert_rows(rows)


def test_backward_static_mode_has_no_field_gradient():
    s = small_scene(2)
    cam = camera()
    rng = np.random.default_rng(2)
    dl = rng.normal(size=(cam.height, cam.width, 3))
    g = oracle.render_backward(s, cam, 0.5, dl, deform=False)
    assert not g["planes"].any() and not g["mlp"].any()
    assert np.abs(g["means"]).max() > 0 and np.abs(g["opacity_logits"]).max() > 0
    _, rows = fd_check(s, cam, 0.5, dl, False, rng, per_group=8)
    rows = [r for r in rows if r[0] not in ("planes", "mlp")]
    scale = max(abs(r[2]) for r in rows)
    bad = [r for r in rows if abs(r[2] - r[3]) > 1e-4 * max(abs(r[2]), abs(r[3])) + 1e-7 * scale]
    assert len(bad) <= 0.05 * len(rows), bad


def test_backward_is_linear_in_dl_dimage():
    s = small_scene(3)
    cam = camera()
    rng = np.random.default_rng(3)
    d1 = rng.normal(size=(cam.height, cam.width, 3))
    d2 = rng.normal(size=(cam.height, cam.width, 3))
    g1 = oracle.render_backward(s, cam, 0.3, d1)
    g2 = oracle.render_backward(s, cam, 0.3, d2)
    g12 = oracle.render_backward(s, cam, 0.3, 2.0 * d1 - d2)
    for k in GROUPS:
        assert np.allclose(g12[k], 2.0 * g1[k] - g2[k], rtol=1e-9, atol=1e-12)
