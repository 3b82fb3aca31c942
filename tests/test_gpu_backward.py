"""GPU backward (fs4d_render_backward, through the C ABI) against the FP64
oracle's analytic gradient and against FP64 central finite differences.

Bar, element by element: |g_gpu - g_ref| <= 1e-3 |g_ref| + 1e-5 max |g_ref| of
the parameter group, and 1e-3 relative for every element above 1% of the
group's largest; plane values, whose gradients sum one term per Gaussian that
samples them, add 1e-3 of the sum of those terms' magnitudes (each term within
1e-3) and the most that the per-Gaussian groups' allowed error (the floor)
can change them through the MLP (|J|^T, from the oracle).  The floor covers elements that are float32 sums of up to ~1e4
per-pixel terms of either sign cancelling to near zero: their rounding error
(~sqrt(n) 2^-24 of the terms' absolute sum, and the float32 forward values'
~1e-6 relative error times that sum) is relative to the terms, not to the sum;
it is also the bound on the GPU's own run-to-run variation (summation order).
Pixels whose forward contains a discrete decision within float32 rounding of
its threshold (oracle.unstable_pixels) get dL/dI = 0, since the gradient is not
defined across such a decision.
"""
import numpy as np
import pytest

import oracle
from paper_2310_08528_gb300 import scenegen as sg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2310_08528_gb300 import fs4d  # noqa: E402

GROUPS = fs4d.PARAMS
REL = 1e-3


@pytest.fixture(scope="module")
def ctx():
    c = fs4d.Context(0)
    yield c
    c.close()


def small_scene(seed, deg=0, n=48):
    if deg == 0:
        s = sg.make_tiny(seed, n=n, mlp_std=0.15, bias_std=0.05)
    else:
        s = sg.make_object(seed, n=n, res_spatial=(6, 8), res_time=4, h=16, mlp_std=0.15)
    s.means *= 0.8
    s.log_scales += 1.2
    return s


def small_camera(w=40, h=36):
    cam = sg.tiny_camera(w, h)
    cam.fx = cam.fy = 40.0
    return cam


def gpu_grads(ctx, s, cam, t, dl, prec=fs4d.FP32):
    sid = ctx.load_scene(s)
    img, frame = ctx.render_saved(sid, cam, t, prec)
    shapes = {k: getattr(s, k).shape for k in GROUPS}
    g = {k: torch.zeros(shapes[k], device="cuda") for k in GROUPS}
    ctx.render_backward(frame, torch.from_numpy(dl.astype(np.float32)).cuda(), g)
    ctx.frame_free(frame)
    torch.cuda.synchronize()
    ctx.unload_scene(sid)
    return img.cpu().numpy(), {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}


def masked_dl(s, cam, t, seed):
    rng = np.random.default_rng(seed)
    dl = rng.normal(size=(cam.height, cam.width, 3))
    unstable, *_ = oracle.unstable_pixels(s, cam, t)
    dl[unstable] = 0.0
    return dl


def check_groups(g, ref, rel=REL, floor=1e-5):
    """Element-wise: |g - ref| <= rel |ref| + floor max|ref| per parameter group,
    and |g - ref| <= rel |ref| where |ref| > 1% of the group's max.  A plane value's
    gradient sums one term per Gaussian that samples it (thousands at a time row
    of the temporal planes, of either sign): its bound is rel times the sum of the
    terms' magnitudes (ref['planes_abs'], from the oracle) -- each term within
    rel -- and the 1%-of-max rule applies where the sum is not dominated by
    cancellation (|ref| >= 10% of that magnitude)."""
    worst = {}
    for k in GROUPS:
        scale = np.abs(ref[k]).max()
        assert scale > 0, k
        err = np.abs(g[k] - ref[k])
        bound = rel * np.abs(ref[k]) + floor * scale
        big = np.abs(ref[k]) > 1e-2 * scale
        if k == "planes" and "planes_abs" in ref:
            # each Gaussian's output gradients (dX', dr', ds') carry the float32 error the
            # per-Gaussian groups are allowed (floor x their largest gradient); its effect
            # on a plane value is at most that error times planes_sens
            eps = floor * max(np.abs(ref[q]).max() for q in ("means", "quats", "log_scales"))
            bound = bound + rel * ref["planes_abs"] + eps * ref["planes_sens"]
            big &= (np.abs(ref[k]) >= 0.1 * ref["planes_abs"]) & (rel * np.abs(ref[k]) >= eps * ref["planes_sens"])
        worst_rel = float((err[big] / np.abs(ref[k][big])).max()) if big.any() else 0.0
        worst[k] = worst_rel
        print(f"{k:15s} max|ref| {scale:.3e}  max err/bound {float((err / bound).max()):.3f}  "
              f"worst rel (|ref| > 1% of max) {worst_rel:.2e}")
        assert (err <= bound).all(), (k, float((err / bound).max()))
        assert worst_rel <= rel, (k, worst_rel)
    return worst


@pytest.mark.parametrize("seed,deg", [(0, 0), (1, 3), (4, 0)])
def test_backward_matches_oracle_small(ctx, seed, deg):
    s = small_scene(seed, deg)
    cam = small_camera()
    dl = masked_dl(s, cam, 0.4, seed)
    _, g = gpu_grads(ctx, s, cam, 0.4, dl)
    ref = oracle.render_backward(s, cam, 0.4, dl, plane_terms=True)
    check_groups(g, ref)


def test_backward_matches_oracle_tiny_scene(ctx):
    """N=2000 at 128x128, several tiles per Gaussian and many per tile."""
    s = sg.make_tiny(0, mlp_std=0.1)
    cam = sg.tiny_camera()
    dl = masked_dl(s, cam, 0.5, 7)
    _, g = gpu_grads(ctx, s, cam, 0.5, dl)
    ref = oracle.render_backward(s, cam, 0.5, dl, plane_terms=True)
    check_groups(g, ref)


def test_backward_matches_central_differences(ctx):
    """GPU gradient against FP64 central differences of the oracle forward.  A
    sample counts where the loss is smooth over [x - h, x + h]: its central
    differences at h and h/2 agree to 1e-4 (no decision flips in between); every
    such sample must pass, and every group must have at least four."""
    s = small_scene(2, deg=3)
    cam = small_camera()
    t = 0.6
    dl = masked_dl(s, cam, t, 2)
    _, g = gpu_grads(ctx, s, cam, t, dl)
    h = 2.0 ** -12
    rng = np.random.default_rng(5)

    def loss():
        return float(np.sum(oracle.render(s, cam, t)[0] * dl))

    def central(flat, i, step):
        x0 = flat[i]
        flat[i] = np.float32(x0 + step)
        lp = loss()
        flat[i] = np.float32(x0 - step)
        lm = loss()
        flat[i] = x0
        return (lp - lm) / (np.float64(np.float32(x0 + step)) - np.float64(np.float32(x0 - step)))

    for k in GROUPS:
        flat = getattr(s, k).reshape(-1)
        gk = g[k].reshape(-1)
        idx = np.flatnonzero(np.abs(gk) > 1e-3 * np.abs(gk).max())
        checked = 0
        for i in rng.permutation(idx)[:24]:
            fd = central(flat, i, h)
            fd2 = central(flat, i, h / 2)
            if abs(fd - fd2) > 1e-4 * max(abs(fd), abs(fd2)) + 1e-9 * np.abs(gk).max():
                continue  # a decision flips inside [x - h, x + h]: no derivative to compare
            assert abs(fd2 - gk[i]) <= REL * abs(fd2) + 1e-6 * np.abs(gk).max(), (k, int(i), fd2, gk[i])
            checked += 1
            if checked == 8:
                break
        print(f"{k}: {checked} central-difference samples")
        assert checked >= 4, k


def test_autograd_function_matches_direct_call(ctx):
    s = small_scene(3)
    cam = small_camera()
    sid = ctx.load_scene(s)
    params = {k: torch.from_numpy(np.ascontiguousarray(getattr(s, k))).cuda().requires_grad_(True) for k in GROUPS}
    dl = masked_dl(s, cam, 0.3, 3)
    img = fs4d.render_differentiable(ctx, sid, cam, 0.3, params)
    loss = (img * torch.from_numpy(dl.astype(np.float32)).cuda()).sum()
    loss.backward()
    ref = oracle.render_backward(s, cam, 0.3, dl, plane_terms=True)
    check_groups({k: params[k].grad.cpu().numpy().astype(np.float64) for k in GROUPS}, ref)
    # the update path: a parameter change reaches the render
    with torch.no_grad():
        params["opacity_logits"] -= 3.0
    img2 = fs4d.render_differentiable(ctx, sid, cam, 0.3, params)
    assert float(img2.detach().sum()) < float(img.detach().sum())
    ctx.unload_scene(sid)


def test_backward_matches_oracle_object_256(ctx):
    """20k Gaussians (SH 3, two HexPlane levels) at 256x256: many Gaussians per
    tile and tiles per Gaussian, plane cells shared by many Gaussians."""
    s = sg.make_object(5, n=20000, mlp_std=0.05)
    cam = sg.hemisphere_cameras(4, width=256, height=256, seed=1)[2]
    oracle.set_threads(oracle.default_threads())
    rng = np.random.default_rng(11)
    dl = rng.normal(size=(256, 256, 3))
    dl[oracle.unstable_pixels(s, cam, 0.4, px_tol=5e-4, margin_tol=5e-5)[0]] = 0.0
    _, g = gpu_grads(ctx, s, cam, 0.4, dl)
    ref = oracle.render_backward(s, cam, 0.4, dl, plane_terms=True)
    check_groups(g, ref)


def test_backward_matches_oracle_object_800(ctx):
    """The full-size training view: 100k Gaussians at 800x800 (the bench's
    backward workload), every element of every gradient group."""
    s = sg.make_object(0)
    cam = sg.hemisphere_cameras(50, seed=0)[7]
    oracle.set_threads(oracle.default_threads())
    rng = np.random.default_rng(12)
    dl = rng.normal(size=(800, 800, 3))
    dl[oracle.unstable_pixels(s, cam, 0.35, px_tol=2e-4, margin_tol=5e-5)[0]] = 0.0
    _, g = gpu_grads(ctx, s, cam, 0.35, dl)
    ref = oracle.render_backward(s, cam, 0.35, dl, plane_terms=True)
    check_groups(g, ref)


def test_backward_repeatable(ctx):
    """Two backward passes agree to float32 reassociation (per-pixel contributions
    are summed in shared memory in arrival order; plane cells use atomics)."""
    s = sg.make_tiny(5, mlp_std=0.1)
    cam = sg.tiny_camera()
    dl = np.random.default_rng(9).normal(size=(128, 128, 3))
    _, g1 = gpu_grads(ctx, s, cam, 0.5, dl)
    _, g2 = gpu_grads(ctx, s, cam, 0.5, dl)
    for k in GROUPS:
        assert np.abs(g1[k] - g2[k]).max() <= 1e-5 * np.abs(g1[k]).max(), k
