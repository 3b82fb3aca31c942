"""Densification and pruning (App. A) on the GPU, through the C ABI, against the
FP64 oracle.

* The statistics (fs4d_render_backward_stats): per Gaussian, the norm of the
  gradient of the loss with respect to its projected mean and whether it was
  visible, against the oracle's backward, with the backward's element-wise bar.
* fs4d_densify on identical float32 inputs (statistics and normal draws written
  by the test): which Gaussians are kept, copied, split or removed, and the
  output order, are integer results and must match exactly; kept and copied
  parameters are bit-exact copies; children's positions (mu + R S z, float32 on
  the GPU) within float32 rounding of the oracle's.  With zero draws (children
  on their parents' means, so both sides hold the same scene) the densified
  scene renders like the oracle's render of the oracle's densified scene (every
  pixel, so the rebuilt deformation work order is a permutation).
* The trainer's optimiser state follows the Gaussians: kept ones keep their
  Adam moments, new ones start at zero, the statistics restart at zero, and a
  trainer that was not passed refuses to step.
"""
import math

import numpy as np
import pytest

import oracle
import parity
from paper_2310_08528_gb300 import scenegen as sg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2310_08528_gb300 import fs4d  # noqa: E402

ARRAYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


@pytest.fixture(scope="module")
def ctx():
    c = fs4d.Context(0)
    yield c
    c.close()


def test_view_stats_match_oracle(ctx):
    s = sg.make_tiny(3, n=600, mlp_std=0.15, bias_std=0.05)
    s.log_scales += 1.0
    cam = sg.tiny_camera(96, 80)
    t = 0.3
    rng = np.random.default_rng(1)
    dl = rng.normal(size=(cam.height, cam.width, 3))
    unstable, *_ = oracle.unstable_pixels(s, cam, t)
    dl[unstable] = 0.0  # no gradient across a decision within float32 rounding of its threshold
    sid = ctx.load_scene(s)
    try:
        _, frame = ctx.render_saved(sid, cam, t)
        gs = torch.zeros(s.n, device="cuda")
        vis = torch.zeros(s.n, device="cuda")
        dlt = torch.from_numpy(dl.astype(np.float32)).cuda()
        ctx.render_backward(frame, dlt, {}, stats=(gs, vis))
        ctx.render_backward(frame, dlt, {}, stats=(gs, vis))  # accumulates
        ctx.frame_free(frame)
        torch.cuda.synchronize()
    finally:
        ctx.unload_scene(sid)
    gs, vis = gs.cpu().numpy().astype(np.float64), vis.cpu().numpy()
    ref = oracle.render_backward(s, cam, t, dl, xy=True)["xy"]
    X, Q, S = oracle.deform(s, t)
    radius = oracle.project(s, cam, X, Q, S)["radius"]
    want_vis = 2.0 * (radius > 0)
    assert np.array_equal(vis, want_vis)
    want = 2.0 * np.sqrt((ref ** 2).sum(1))
    scale = want.max()
    err = np.abs(gs - want)
    print(f"visible {int((radius > 0).sum())}/{s.n}; max |ref| {scale:.3e}, max err / bound "
          f"{float((err / (1e-3 * want + 1e-5 * scale)).max()):.3f}")
    assert (err <= 1e-3 * want + 1e-5 * scale).all()


def _inputs(s, seed):
    rng = np.random.default_rng(seed)
    gsum = rng.exponential(1.0, s.n).astype(np.float32)
    vis = rng.integers(0, 4, s.n).astype(np.float32)
    normals = rng.normal(size=(s.n, 2, 3)).astype(np.float32)
    smax = s.log_scales.max(1)
    avg = np.where(vis > 0, gsum / np.maximum(vis, 1), 0)
    thr = float(np.float32(np.quantile(avg, 0.6)))
    split = float(np.float32(np.quantile(smax, 0.5)))
    prune = float(np.float32(np.quantile(s.opacity_logits, 0.15)))
    return gsum, vis, normals, thr, split, prune


def _compare(got, d, s):
    kind, src = d["kind"], d["src"]
    assert got["means"].shape[0] == len(kind)
    parent = kind < 2
    for k in ("quats", "opacity_logits", "sh"):
        assert np.array_equal(got[k].astype(np.float64), d[k]), k
    for k in ("means", "log_scales"):
        assert np.array_equal(got[k][parent].astype(np.float64), d[k][parent]), k
    child = ~parent
    if child.any():
        mu = np.abs(s.means[src[child]]).max(1)
        off = np.abs(d["means"][child] - s.means[src[child]]).max(1)
        tol = 2e-6 * (mu + off)[:, None] + 1e-7
        assert (np.abs(got["means"][child] - d["means"][child]) <= tol).all()
        assert np.abs(got["log_scales"][child] - d["log_scales"][child]).max() <= 1e-6


@pytest.mark.parametrize("n,degree", [(3000, 0), (100_000, 3)])
def test_densify_matches_oracle(ctx, n, degree):
    if degree == 0:
        s = sg.make_tiny(5, n=n)
    else:
        s = sg.make_object(0, n=n)
    gsum, vis, normals, thr, split, prune = _inputs(s, n)
    d = oracle.densify(s, gsum, vis, normals, thr, split, prune)
    counts = np.bincount(d["kind"], minlength=4)
    print(f"n {n}: kept {counts[0]}, copies {counts[1]}, split {counts[2]} (removed "
          f"{n - counts[0] - counts[2]})")
    assert counts.min() > 0
    stats = (torch.from_numpy(gsum).cuda(), torch.from_numpy(vis).cuda())
    sid = ctx.load_scene(s)
    try:
        m = ctx.densify(sid, stats, torch.from_numpy(normals).cuda(), thr, split, prune)
        assert m == len(d["src"])
        _compare(ctx.read_scene(sid), d, s)
    finally:
        ctx.unload_scene(sid)
    # with zero draws the children sit exactly on their parents' means on both sides,
    # so the GPU's densified scene is the oracle's (up to the rounding of the log-scales'
    # shift) and its frame must match the oracle's frame of it pixel by pixel; this also
    # checks the rebuilt deformation work order
    zero = np.zeros_like(normals)
    d = oracle.densify(s, gsum, vis, zero, thr, split, prune)
    sid = ctx.load_scene(s)
    try:
        m = ctx.densify(sid, stats, torch.from_numpy(zero).cuda(), thr, split, prune)
        assert m == len(d["src"])
        got = ctx.read_scene(sid)
        _compare(got, d, s)
        assert np.array_equal(got["means"].astype(np.float64), d["means"])
        dense = s.copy()
        for k in ARRAYS:
            setattr(dense, k, np.ascontiguousarray(d[k], np.float32))
        cam = sg.hemisphere_cameras(3, width=160, height=120, seed=3)[1] if degree else sg.tiny_camera(128, 128)
        img, T, nc = ctx.render(sid, cam, 0.4, with_aux=True)
        fr = parity.oracle_frame(dense, cam, 0.4)
        st = parity.check_frame(img.cpu().numpy(), fr, T.cpu().numpy(), nc.cpu().numpy(), tol=1e-4, px_tol=5e-4)
        assert st["unresolved"] == 0
    finally:
        ctx.unload_scene(sid)


def test_densify_refuses_to_remove_everything(ctx):
    s = sg.make_tiny(6, n=500)
    sid = ctx.load_scene(s)
    try:
        z = torch.zeros(s.n, device="cuda")
        normals = torch.zeros((s.n, 2, 3), device="cuda")
        before = ctx.render(sid, sg.tiny_camera(), 0.5).clone()
        with pytest.raises(fs4d.Fs4dError) as e:
            ctx.densify(sid, (z, z), normals, 1.0, 0.0, 1e9)
        assert e.value.status == 1
        after = ctx.render(sid, sg.tiny_camera(), 0.5)
        assert torch.equal(before, after)
    finally:
        ctx.unload_scene(sid)


def test_trainer_state_follows_the_gaussians(ctx):
    s = sg.make_tiny(7, n=1500, mlp_std=0.1)
    s.log_scales += 0.8
    cam = sg.tiny_camera(96, 96)
    sid = ctx.load_scene(s)
    sid_t = ctx.load_scene(sg.perturb_planes(s, 0, std=0.05))
    target = ctx.render(sid_t, cam, 0.5).clone()
    ctx.unload_scene(sid_t)
    tr = fs4d.Trainer(ctx, sid, 10)
    other = fs4d.Trainer(ctx, sid, 10)
    try:
        for _ in range(2):
            tr.step(cam, 0.5, target)
        g, vis = tr.stats()
        torch.cuda.synchronize()
        assert float(vis.max().item()) == 2.0 and float(g.max().item()) > 0
        params = ctx.read_scene(sid)
        before = {k: tr.read_state(q) for q, k in enumerate(ARRAYS)}
        n = s.n
        logits = params["opacity_logits"]
        smax = params["log_scales"].max(1)
        prune = float(np.float32(np.quantile(logits, 0.2)))
        split = float(np.float32(np.quantile(smax, 0.5)))
        # threshold 0: every Gaussian is selected (the mean gradient of an unseen one is 0)
        normals = torch.from_numpy(np.random.default_rng(2).normal(size=(n, 2, 3)).astype(np.float32)).cuda()
        m = tr.densify(normals, 0.0, split, prune)
        keep = logits >= np.float32(prune)
        large = smax > np.float32(split)
        kept = np.flatnonzero(keep & ~large)
        copies = np.flatnonzero(keep & ~large)
        split_ix = np.flatnonzero(keep & large)
        assert m == len(kept) + len(copies) + 2 * len(split_ix)
        after = ctx.read_scene(sid)
        assert np.array_equal(after["opacity_logits"][:len(kept)], logits[kept])
        for q, k in enumerate(ARRAYS):
            width = int(np.prod(params[k].shape[1:]))
            mm, vv = tr.read_state(q)
            mm, vv = mm.reshape(m, width), vv.reshape(m, width)
            bm, bv = (x.reshape(n, width) for x in before[k])
            assert np.array_equal(mm[:len(kept)], bm[kept]) and np.array_equal(vv[:len(kept)], bv[kept]), k
            assert not mm[len(kept):].any() and not vv[len(kept):].any(), k
        g2, vis2 = tr.stats()
        torch.cuda.synchronize()
        assert g2.shape[0] == m and not g2.any() and not vis2.any()
        tr.step(cam, 0.5, target)  # the densified scene trains on
        l1, _ = tr.losses()
        assert math.isfinite(l1)
        with pytest.raises(fs4d.Fs4dError) as e:
            other.step(cam, 0.5, target)
        assert e.value.status == 1
    finally:
        other.close()
        tr.close()
        ctx.unload_scene(sid)
