"""Frames with more tile pairs than one pair-sort pass counts, rendered in bands
of tile rows, and the stress workload at full size: 2M Gaussians with inflated
log-scales N(-2.5, 0.5), HexPlane {64,128,256} x 300 x 32, rendered at
1920x1080 (about 1.3e9 tile pairs) and 3840x2160 (about 5e9), and 16 timestamps
deformed in one launch.

At full size the oracle checks sampled outputs one by one: pixels (each against
the oracle's outcomes for its tile list, built from the oracle's projection of
all 2M Gaussians), the pair count (the sum of the oracle's tile rectangles), and
sampled Gaussians of the batched deformation.
"""
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

IMG_TOL = 1e-4


@pytest.fixture(scope="module")
def ctx():
    c = fs4d.Context(0)
    yield c
    c.close()


def test_banded_frame_matches_oracle(ctx):
    """A frame limited to a quarter of its pairs per band: rendered in bands (a
    second frame of the same size starts with bands directly), every pixel, T and
    last contributor against the oracle; a frame saved for the backward must fit
    one band."""
    s = sg.make_object(3, n=30000, log_scale_mean=-3.0)
    cam = sg.hemisphere_cameras(3, width=333, height=517, seed=2)[1]
    sid = ctx.load_scene(s)
    try:
        ctx.render(sid, cam, 0.4)
        K = ctx.last_pairs()
        assert ctx.last_bands() == 1
        ctx.set_band_pairs(K // 6)
        img, T, nc = ctx.render(sid, cam, 0.4, with_aux=True)
        bands = ctx.last_bands()
        Kb = ctx.last_pairs()
        print(f"pairs {K}, limit {K // 6} per band: {bands} bands, {Kb} pairs in all")
        assert bands >= 6
        assert abs(Kb - K) <= 1e-4 * K + 16
        img2, T2, nc2 = ctx.render(sid, cam, 0.4, with_aux=True)  # bands from the start
        assert ctx.last_bands() == bands
        assert torch.equal(img, img2) and torch.equal(T, T2) and torch.equal(nc, nc2)
        ctx.set_stage_timing(True)
        ctx.render(sid, cam, 0.4)
        st = ctx.stage_times()
        ctx.set_stage_timing(False)
        assert all(v > 0 for v in st.values()), st
        with pytest.raises(fs4d.Fs4dError) as e:
            ctx.render_saved(sid, cam, 0.4)
        assert e.value.status == 3
        # a frame after the banded one reports its own stage times, not the bands' sums
        ctx.set_stage_timing(True)
        ctx.render(sid, cam, 0.4)
        st = ctx.stage_times()
        ctx.set_band_pairs(0)
        shape = fs4d.camera_struct(cam)
        d_cam = torch.from_numpy(np.frombuffer(bytes(shape), dtype=np.float32).copy()).cuda()
        d_t = torch.full((1,), 0.4, device="cuda")
        ctx.reserve(sid, cam.width, cam.height, K + 4096)
        ctx.render_async(sid, cam, d_cam, d_t, torch.empty((cam.height, cam.width, 3), device="cuda"))
        st1 = ctx.stage_times()
        ctx.set_stage_timing(False)
        assert st1 != st and all(v >= 0 for v in st1.values()), (st, st1)
        fr = parity.oracle_frame(s, cam, 0.4)
        stt = parity.check_frame(img.cpu().numpy(), fr, T.cpu().numpy(), nc.cpu().numpy(), tol=IMG_TOL,
                                 px_tol=5e-4)
        assert stt["unresolved"] == 0
        assert stt["other_outcome_frac"] <= 5e-3
    finally:
        ctx.set_band_pairs(0)
        ctx.unload_scene(sid)


# ------------------------------------------------------------------ the stress workload at full size

@pytest.fixture(scope="module")
def stress(ctx):
    s = sg.make_stress(0)
    sid = ctx.load_scene(s)
    oracle.set_threads(oracle.default_threads())
    t = 0.5
    X, Q, S = oracle.deform(s, t)
    yield s, sid, t, (X, Q, S)
    ctx.unload_scene(sid)


def _sampled_pixels(rng, proj, dbits, W, H, n_tiles=40, per_tile=3, tile=16):
    tx, ty = (W + tile - 1) // tile, (H + tile - 1) // tile
    r = proj["rect"]
    cover = np.zeros((ty + 1, tx + 1), np.int64)  # 2-D difference array of the rectangles
    np.add.at(cover, (r[:, 1], r[:, 0]), 1)
    np.add.at(cover, (r[:, 1], r[:, 2]), -1)
    np.add.at(cover, (r[:, 3], r[:, 0]), -1)
    np.add.at(cover, (r[:, 3], r[:, 2]), 1)
    counts = cover.cumsum(0).cumsum(1)[:ty, :tx].ravel()
    tiles = rng.choice(np.flatnonzero(counts > 0), size=n_tiles, replace=False)
    out = []
    for t_id in tiles:
        x0, y0 = (t_id % tx) * tile, (t_id // tx) * tile
        for _ in range(per_tile):
            px = int(min(W - 1, x0 + rng.integers(0, tile)))
            py = int(min(H - 1, y0 + rng.integers(0, tile)))
            out.append((int(t_id), px, py))
    return out, int(counts.sum())


@pytest.mark.parametrize("w,h", [(1920, 1080), (3840, 2160)])
def test_stress_frame_sampled_pixels_match_oracle(ctx, stress, w, h):
    s, sid, t, (X, Q, S) = stress
    cam = sg.hemisphere_cameras(4, width=w, height=h, seed=7)[1]
    img = ctx.render(sid, cam, t, fs4d.FP32)
    bf = ctx.render(sid, cam, t, fs4d.BF16)
    torch.cuda.synchronize()
    img, bf = img.cpu().numpy(), bf.cpu().numpy()
    K, bands = ctx.last_pairs(), ctx.last_bands()
    p = oracle.project(s, cam, X, Q, S)
    dbits = oracle.depth_bits(p["depth"])
    rng = np.random.default_rng(w)
    pix, K_o = _sampled_pixels(rng, p, dbits, w, h)
    print(f"{w}x{h}: {K} tile pairs in {bands} bands (oracle {K_o})")
    assert bands >= 2
    assert abs(K - K_o) <= 1e-4 * K_o
    tx = (w + 15) // 16
    members = oracle.uncertain_memberships(p, w, h, 5e-4)
    lists = {}
    bad = 0
    sq_err, n_bf = 0.0, 0
    for t_id, px, py in pix:
        if t_id not in lists:
            lists[t_id] = parity.tile_list(p, dbits, tx, t_id)
        base = lists[t_id]
        gs = members.get(t_id, [])[:4]
        if not parity.pixel_matches(img[py, px], px, py, base, gs, p, dbits, IMG_TOL, 5e-5, 1e-6):
            bad += 1
        want = oracle.pixel_outcomes(base, px, py, p, 0.0, 0.0)[0, :3]  # the blend as computed
        sq_err += float(((bf[py, px] - want) ** 2).sum())
        n_bf += 3
    psnr = 10 * np.log10(1.0 / max(sq_err / n_bf, 1e-30))
    print(f"{len(pix)} sampled pixels: {bad} match no oracle outcome; BF16 PSNR on them {psnr:.1f} dB")
    assert bad == 0
    assert psnr >= 50.0


def test_stress_batched_deform_sampled_gaussians_match_oracle(ctx, stress):
    """16 timestamps in one launch, FP32 and BF16, on 2000 sampled Gaussians."""
    s, sid, _, _ = stress
    ts = np.linspace(0.0, 1.0, 16)
    rng = np.random.default_rng(4)
    idx = np.sort(rng.choice(s.n, size=2000, replace=False))
    sub = s.copy()
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        setattr(sub, k, np.ascontiguousarray(getattr(s, k)[idx]))
    for prec, rel in ((fs4d.FP32, 2e-5), (fs4d.BF16, 5e-2)):
        m, q, ls = ctx.deform(sid, ts, prec)
        torch.cuda.synchronize()
        for k in (0, 7, 15):
            Xo, Qo, So = oracle.deform(sub, float(ts[k]))
            got = [m[k].cpu().numpy()[idx], q[k].cpu().numpy()[idx], ls[k].cpu().numpy()[idx]]
            scale = max(float(np.abs(Xo - sub.means).max()), float(np.abs(Qo - sub.quats).max()),
                        float(np.abs(So - sub.log_scales).max()))
            tol = rel * (max(1.0, scale) if prec == fs4d.FP32 else scale) + 1e-6
            errs = [float(np.abs(a - b).max()) for a, b in zip(got, (Xo, Qo, So))]
            print(f"prec {prec} t={ts[k]:.3f}: max|dX| {errs[0]:.2e} |dr| {errs[1]:.2e} |ds| {errs[2]:.2e} "
                  f"(tol {tol:.2e})")
            assert max(errs) <= tol
        del m, q, ls
