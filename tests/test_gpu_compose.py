"""Composition and tracking (Sec. 5.4) on the GPU against the FP64 oracle.

Composition renders G' = {G'_1, ..., G'_n}: every scene deformed by its own field,
translated, and the union binned, sorted and composited in one frame
(fs4d_render_composed); every pixel, T and last contributor must match the
oracle's composed frame or one of its near-threshold outcomes.  Tracking follows
Gaussians over time: the deformed means of 64 timestamps from one batched
fs4d_deform launch against the oracle's deformation at each timestamp.
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


@pytest.fixture(scope="module")
def ctx():
    c = fs4d.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("w,h", [(320, 240), (800, 800)])
def test_composed_frame_matches_oracle(ctx, w, h):
    scenes = [sg.make_object(11, n=20000, mlp_std=0.1),
              sg.make_tiny(12, n=3000, mlp_std=0.1),
              sg.make_object(13, n=9000, res_spatial=(16, 32, 64), res_time=9, h=16, mlp_std=0.1)]
    shifts = np.array([[0.0, 0.0, 0.0], [0.6, -0.3, 0.2], [-0.7, 0.4, -0.1]])
    sids = [ctx.load_scene(s) for s in scenes]
    cam = sg.hemisphere_cameras(3, width=w, height=h, seed=9)[1]
    try:
        img, T, nc = ctx.render_composed(sids, cam, 0.45, fs4d.FP32, shifts=shifts, with_aux=True)
        torch.cuda.synchronize()
        oracle.set_threads(oracle.default_threads())
        fr = parity.oracle_frame_composed(scenes, shifts, cam, 0.45)
        assert abs(ctx.last_pairs() - fr["K"]) <= 1e-4 * fr["K"]
        # three deformation fields and translated scenes: decisions within 2e-4 of their
        # threshold may go either way
        st = parity.check_frame(img.cpu().numpy(), fr, T.cpu().numpy(), nc.cpu().numpy(), tol=1e-4, rel_tol=2e-4,
                                px_tol=5e-4)
        assert st["unresolved"] == 0
        assert st["other_outcome_frac"] <= 5e-3
        # the composed frame with BF16 deformation: PSNR against the oracle.  These
        # scenes' MLP weights (std 0.1, five times the object workload's) make
        # deltas and their BF16 rounding larger; the bar is 45 dB here
        bf = ctx.render_composed(sids, cam, 0.45, fs4d.BF16, shifts=shifts).cpu().numpy()
        mse = float(np.mean((bf - fr["img"]) ** 2))
        print(f"composed BF16 PSNR {10 * np.log10(1 / mse):.1f} dB")
        assert 10 * np.log10(1 / mse) >= 45.0
        # one scene alone through the composed call is that scene's frame
        one = ctx.render_composed(sids[:1], cam, 0.45, fs4d.FP32)
        assert torch.equal(one, ctx.render(sids[0], cam, 0.45, fs4d.FP32))
    finally:
        for sid in sids:
            ctx.unload_scene(sid)


@pytest.mark.parametrize("prec,rel", [(fs4d.FP32, 2e-5), (fs4d.BF16, 5e-2)])
def test_tracking_trajectories_match_oracle(ctx, prec, rel):
    """Trajectories X'(t) of 500 Gaussians over 64 timestamps in [0, 1] from one
    batched launch (the tracking of Sec. 5.4), against the oracle at every t."""
    s = sg.make_object(14, n=500, mlp_std=0.2)
    sid = ctx.load_scene(s)
    ts = np.linspace(0.0, 1.0, 64)
    try:
        m, q, ls = ctx.deform(sid, ts, prec)
        torch.cuda.synchronize()
        traj = m.cpu().numpy()  # [64][500][3]
        ref = np.stack([oracle.deform(s, float(t))[0] for t in ts])
        motion = np.abs(ref - s.means[None]).max()
        assert motion > 1e-3  # the Gaussians really move
        err = np.abs(traj - ref).max()
        tol = rel * (max(1.0, motion) if prec == fs4d.FP32 else motion) + 1e-6
        print(f"trajectories: max motion {motion:.3e}, max |dX| {err:.2e} (tol {tol:.2e})")
        assert err <= tol
    finally:
        ctx.unload_scene(sid)
