"""Colour and opacity deformation (App. B: C' = C + phi_C(f_d), logit' = logit +
phi_alpha(f_d)) on the GPU, through the C ABI, against the FP64 oracle.

* FP32 frames, every pixel, against the oracle's frame of the same scene with the
  heads (its per-pixel outcome enumeration), for a degree-0 and a degree-3 scene;
* BF16 frames (f_d from the tensor-core deformation, both heads as two tcgen05
  GEMMs per 128 Gaussians): PSNR, for SH degrees 0 to 3 (3K = 3, 12, 27, 48
  outputs of the colour head);
* heads with all weights and biases 0 give bit-identical frames to the scene
  without them, and composition with a scene that has heads matches the oracle;
* what such scenes do not support fails loudly: the backward and the trainer
  (FS4D_ERR_UNIMPLEMENTED), and serving requests complete with that status;
* the scene file keeps the heads.
"""
import os

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

UNIMPLEMENTED = 7


@pytest.fixture(scope="module")
def ctx():
    c = fs4d.Context(0)
    yield c
    c.close()


def _scenes():
    tiny = sg.with_color_heads(sg.make_tiny(21, n=3000, mlp_std=0.1), 1, std=0.1)
    obj = sg.with_color_heads(sg.make_object(22, n=40000, mlp_std=0.05), 2, std=0.05)
    return [(tiny, sg.tiny_camera(128, 128)), (obj, sg.hemisphere_cameras(3, width=320, height=240, seed=4)[2])]


@pytest.mark.parametrize("which", [0, 1])
def test_color_heads_frame_matches_oracle(ctx, which):
    s, cam = _scenes()[which]
    sid = ctx.load_scene(s)
    try:
        img, T, nc = ctx.render(sid, cam, 0.35, fs4d.FP32, with_aux=True)
        culled = ctx.render(sid, cam, 0.35, fs4d.FP32)
        bf = ctx.render(sid, cam, 0.35, fs4d.BF16)
        torch.cuda.synchronize()
        assert torch.equal(img, culled)
        oracle.set_threads(oracle.default_threads())
        fr = parity.oracle_frame(s, cam, 0.35)
        # the heads move the colours and opacities visibly
        plain = s.copy()
        plain.color_heads = False
        plain.mlp = plain.mlp[:sum(o * i + o for o, i in sg.mlp_layer_shapes(s.feat_dim * s.n_levels,
                                                                            s.mlp_width))].copy()
        base_img, *_ = oracle.render(plain, cam, 0.35)
        moved = float(np.abs(fr["img"] - base_img).max())
        print(f"heads move the frame by up to {moved:.3f}")
        assert moved > 1e-2
        st = parity.check_frame(img.cpu().numpy(), fr, T.cpu().numpy(), nc.cpu().numpy(), tol=1e-4, px_tol=5e-4)
        assert st["unresolved"] == 0
        assert st["other_outcome_frac"] <= 5e-3
        mse = float(np.mean((bf.cpu().numpy() - fr["img"]) ** 2))
        psnr = 10 * np.log10(1.0 / max(mse, 1e-30))
        print(f"BF16 with colour heads: PSNR {psnr:.1f} dB")
        assert psnr >= 50.0
    finally:
        ctx.unload_scene(sid)


@pytest.mark.parametrize("degree", [1, 2])
def test_color_heads_other_sh_degrees(ctx, degree):
    """SH degrees 1 and 2 (colour heads of 12 and 27 outputs: the rows of 27 are
    not 16-byte aligned): FP32 every pixel, BF16 by PSNR, against the oracle."""
    s = sg.with_color_heads(sg.make_object(30 + degree, n=6000, sh_degree=degree, mlp_std=0.05), degree, std=0.08)
    cam = sg.hemisphere_cameras(3, width=160, height=144, seed=degree)[0]
    sid = ctx.load_scene(s)
    try:
        img, T, nc = ctx.render(sid, cam, 0.55, fs4d.FP32, with_aux=True)
        bf = ctx.render(sid, cam, 0.55, fs4d.BF16)
        torch.cuda.synchronize()
        oracle.set_threads(oracle.default_threads())
        fr = parity.oracle_frame(s, cam, 0.55)
        st = parity.check_frame(img.cpu().numpy(), fr, T.cpu().numpy(), nc.cpu().numpy(), tol=1e-4, px_tol=5e-4)
        assert st["unresolved"] == 0
        mse = float(np.mean((bf.cpu().numpy() - fr["img"]) ** 2))
        psnr = 10 * np.log10(1.0 / max(mse, 1e-30))
        print(f"degree {degree}, BF16 with colour heads: PSNR {psnr:.1f} dB")
        assert psnr >= 50.0
    finally:
        ctx.unload_scene(sid)


def test_zero_heads_are_bit_identical_to_no_heads(ctx):
    s = sg.make_object(23, n=20000, mlp_std=0.05)
    c = sg.with_color_heads(s, 5)
    n8 = sum(o * i + o for o, i in sg.mlp_layer_shapes(s.feat_dim * s.n_levels, s.mlp_width))
    c.mlp[n8:] = 0.0
    cam = sg.hemisphere_cameras(3, width=256, height=192, seed=6)[0]
    a, b = ctx.load_scene(s), ctx.load_scene(c)
    try:
        for prec in (fs4d.FP32, fs4d.BF16):
            x = ctx.render(a, cam, 0.6, prec)
            y = ctx.render(b, cam, 0.6, prec)
            torch.cuda.synchronize()
            assert torch.equal(x, y)
    finally:
        ctx.unload_scene(a)
        ctx.unload_scene(b)


def test_composition_with_color_heads_matches_oracle(ctx):
    scenes = [sg.with_color_heads(sg.make_object(24, n=12000, mlp_std=0.05), 7, std=0.08),
              sg.make_tiny(25, n=2000, mlp_std=0.05)]
    shifts = np.array([[0.0, 0.0, 0.0], [0.5, -0.2, 0.1]])
    sids = [ctx.load_scene(x) for x in scenes]
    cam = sg.hemisphere_cameras(3, width=240, height=200, seed=8)[1]
    try:
        img, T, nc = ctx.render_composed(sids, cam, 0.45, fs4d.FP32, shifts=shifts, with_aux=True)
        torch.cuda.synchronize()
        fr = parity.oracle_frame_composed(scenes, shifts, cam, 0.45)
        st = parity.check_frame(img.cpu().numpy(), fr, T.cpu().numpy(), nc.cpu().numpy(), tol=1e-4, rel_tol=2e-4,
                                px_tol=5e-4)
        assert st["unresolved"] == 0
    finally:
        for sid in sids:
            ctx.unload_scene(sid)


def test_composition_with_color_heads_bf16(ctx):
    """BF16 composition of two scenes with heads and one without; the first has 60
    Gaussians, so its f_d tile image (16 KB) runs past its share of the f_d buffer
    into the next scene's, which the next deformation writes only after the first
    scene's heads have read it.  PSNR against the oracle's composed frame."""
    scenes = [sg.with_color_heads(sg.make_tiny(26, n=60, mlp_std=0.05), 8, std=0.08),
              sg.with_color_heads(sg.make_tiny(27, n=4000, mlp_std=0.05), 9, std=0.08),
              sg.make_tiny(28, n=2000, mlp_std=0.05)]
    shifts = np.array([[0.0, 0.0, 0.0], [0.3, 0.1, -0.1], [-0.4, 0.2, 0.1]])
    sids = [ctx.load_scene(x) for x in scenes]
    cam = sg.tiny_camera(160, 128)
    try:
        bf = ctx.render_composed(sids, cam, 0.45, fs4d.BF16, shifts=shifts).cpu().numpy()
        oracle.set_threads(oracle.default_threads())
        fr = parity.oracle_frame_composed(scenes, shifts, cam, 0.45)
        mse = float(np.mean((bf - fr["img"]) ** 2))
        psnr = 10 * np.log10(1.0 / max(mse, 1e-30))
        print(f"composed BF16 with colour heads: PSNR {psnr:.1f} dB")
        assert psnr >= 45.0
    finally:
        for sid in sids:
            ctx.unload_scene(sid)


def test_unsupported_calls_fail_loudly(ctx, tmp_path):
    s, cam = _scenes()[0]
    sid = ctx.load_scene(s)
    try:
        _, frame = ctx.render_saved(sid, cam, 0.5)
        with pytest.raises(fs4d.Fs4dError) as e:
            ctx.render_backward(frame, torch.zeros((cam.height, cam.width, 3), device="cuda"), {})
        assert e.value.status == UNIMPLEMENTED
        ctx.frame_free(frame)
        with pytest.raises(fs4d.Fs4dError) as e:
            fs4d.Trainer(ctx, sid, 10)
        assert e.value.status == UNIMPLEMENTED
        srv = fs4d.Server(ctx, max_inflight=1, max_batch=1)
        try:
            out = torch.zeros((cam.height, cam.width, 3), device="cuda")
            tk = srv.submit(sid, cam, 0.5, out)
            srv.drain()
            done = {c["ticket"]: c for c in srv.poll(16)}
            assert done[tk]["status"] == UNIMPLEMENTED
        finally:
            srv.close()
        # the scene file keeps the heads: the reloaded scene renders the same frame
        path = os.path.join(str(tmp_path), "heads.fs4d")
        ctx.save_scene(sid, path)
        sid2 = ctx.load_scene_file(path, like=s)
        try:
            a = ctx.render(sid, cam, 0.5)
            b = ctx.render(sid2, cam, 0.5)
            torch.cuda.synchronize()
            assert torch.equal(a, b)
        finally:
            ctx.unload_scene(sid2)
    finally:
        ctx.unload_scene(sid)
