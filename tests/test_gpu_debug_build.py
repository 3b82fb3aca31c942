"""The bounds-checking debug build (FS4D_CHECK_BOUNDS, libfs4d_debug.so): every
device buffer the library allocates carries canary bytes after its end.  A
workout of the library's paths -- bitmap and sort binning, culled and full lists,
bands, the backward, a training step, densification, colour heads, composition --
must leave every canary intact, and the check must notice a canary that was
overwritten.  The release build reports the check as not built.
"""
import numpy as np
import pytest

from paper_2310_08528_gb300 import scenegen as sg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2310_08528_gb300 import build, fs4d  # noqa: E402

CORRUPT, UNIMPLEMENTED = 9, 7


def test_release_build_has_no_canaries():
    ctx = fs4d.Context(0)
    try:
        assert ctx.lib.fs4d_check_canaries(ctx.h) == UNIMPLEMENTED
    finally:
        ctx.close()


def test_every_path_leaves_the_canaries_intact():
    lib = fs4d.library(build.build(debug=True))
    ctx = fs4d.Context(0, lib=lib)
    try:
        s = sg.make_object(31, n=30000, mlp_std=0.05)
        sid = ctx.load_scene(s)
        cam = sg.hemisphere_cameras(3, width=333, height=517, seed=2)[1]
        for prec in (fs4d.FP32, fs4d.BF16):
            ctx.render(sid, cam, 0.4, prec)
            ctx.render(sid, cam, 0.4, prec, with_aux=True)
        ctx.set_binning(fs4d.BINNING_SORT)
        ctx.render(sid, cam, 0.4)
        ctx.render(sid, cam, 0.4, with_aux=True)
        ctx.set_binning(fs4d.BINNING_AUTO)
        ctx.render(sid, cam, 0.4)
        ctx.set_band_pairs(max(1, ctx.last_pairs() // 4))
        ctx.render(sid, cam, 0.4)
        ctx.set_band_pairs(0)
        ctx.render_host(sid, cam, 0.4)
        # backward, a training step, densification
        _, frame = ctx.render_saved(sid, cam, 0.4)
        g = {k: torch.zeros(np.shape(getattr(s, k)), device="cuda") for k in fs4d.PARAMS}
        ctx.render_backward(frame, torch.randn((cam.height, cam.width, 3), device="cuda"), g)
        ctx.frame_free(frame)
        target = ctx.render(sid, cam, 0.5).clone()
        tr = fs4d.Trainer(ctx, sid, 10)
        tr.step(cam, 0.4, target)
        normals = torch.randn((s.n, 2, 3), device="cuda")
        tr.densify(normals, 0.0, float(np.quantile(s.log_scales.max(1), 0.5)),
                   float(np.quantile(s.opacity_logits, 0.2)))
        tr.step(cam, 0.4, target)
        tr.close()
        # colour heads and composition
        c = sg.with_color_heads(sg.make_tiny(32, n=3000, mlp_std=0.1), 3)
        cid = ctx.load_scene(c)
        ctx.render(cid, sg.tiny_camera(), 0.3)
        ctx.render(cid, sg.tiny_camera(), 0.3, fs4d.BF16)
        ctx.render_composed([sid, cid], cam, 0.4, shifts=np.array([[0, 0, 0], [0.4, 0.1, 0.0]]))
        torch.cuda.synchronize()
        rc = lib.fs4d_check_canaries(ctx.h)
        assert rc == 0, lib.fs4d_last_error(ctx.h).decode()
        # the check notices an overwritten canary
        assert lib.fs4d_debug_corrupt_canary(ctx.h) == 0
        assert lib.fs4d_check_canaries(ctx.h) == CORRUPT
        ctx.unload_scene(cid)
        ctx.unload_scene(sid)
    finally:
        ctx.close()
