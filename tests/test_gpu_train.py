"""The on-device training step (fs4d_train_step, Sec. 4.3 loss, App. A schedules)
against the FP64 oracle's training step (oracle.train_step), and the scene
read-back, file save and load.

Three steps on a small scene against a target whose every pixel differs from the
render by at least 0.05 (so that the L1 gradient's signs are decided): the L1
and TV losses of each step, and every parameter after the three updates.  An
element whose gradient is above 1% of its group's largest at every step has a
gradient the GPU reproduces to ~2e-3 (the backward's element-wise bound), and
its update must match to 1e-2 relative plus float32 rounding of the parameter;
every other element's update (Adam moves at most a few learning rates per step
whatever the gradient) must stay within that bound.
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
CFG = dict(lr_means=(1e-3, 1e-4), lr_log_scales=(2e-3, 1e-3), lr_quats=(1e-3, 5e-4), lr_opacity=(1e-2, 5e-3),
           lr_sh_dc=(2e-3, 1e-3), lr_sh_rest=(1e-3, 5e-4), lr_planes=(1.6e-3, 1.6e-4), lr_mlp=(1.6e-4, 1.6e-5),
           beta1=0.9, beta2=0.999, eps=1e-15, tv_weight=0.05)
STEPS = 3


@pytest.fixture(scope="module")
def ctx():
    c = fs4d.Context(0)
    yield c
    c.close()


def _scene_and_view():
    s = sg.make_object(1, n=400, res_spatial=(6, 8), res_time=4, h=16, mlp_std=0.15)
    s.means *= 0.8
    s.log_scales += 1.5
    cam = sg.tiny_camera(48, 40)
    cam.fx = cam.fy = 48.0
    return s, cam


def _oracle_cfg():
    lr = {k[3:]: v for k, v in CFG.items() if k.startswith("lr_")}
    lr["opacity_logits"] = lr.pop("opacity")
    return {"lr": lr, "total_steps": STEPS, "beta1": CFG["beta1"], "beta2": CFG["beta2"], "eps": CFG["eps"],
            "tv_weight": CFG["tv_weight"]}


def test_train_steps_match_oracle(ctx):
    s, cam = _scene_and_view()
    t = 0.3
    img0, *_ = oracle.render(s, cam, t)
    rng = np.random.default_rng(3)
    target = np.clip(img0 + 0.05 * np.where(rng.uniform(size=img0.shape) < 0.5, -1.0, 1.0), -1, 2)
    sid = ctx.load_scene(s)
    tr = fs4d.Trainer(ctx, sid, STEPS, **CFG)
    d_target = torch.from_numpy(target.astype(np.float32)).cuda()
    state = {}
    ocfg = _oracle_cfg()
    grads = []
    try:
        for k in range(STEPS):
            losses = torch.zeros(2, device="cuda")
            tr.step(cam, t, d_target, fs4d.FP32, losses)
            l1, tv, g = oracle.train_step(s, cam, t, target, ocfg, state)
            grads.append(g)
            gl1, gtv = (float(v) for v in losses.cpu())
            print(f"step {k}: L1 {gl1:.7f} (oracle {l1:.7f})  TV {gtv:.7e} (oracle {tv:.7e})")
            assert abs(gl1 - l1) <= 1e-5 * l1 + 1e-6
            assert abs(gtv - tv) <= 1e-4 * tv + 1e-9
        assert tr.steps_done() == STEPS
        got = ctx.read_scene(sid)
        lr_sum = 0.0
        for k in range(STEPS):
            lr_sum += max(oracle.lr_at(*v, k, STEPS) for kk, v in CFG.items() if kk.startswith("lr_"))
        for grp in GROUPS:
            p0 = np.asarray(getattr(s, grp), np.float64)
            d_gpu = got[grp].astype(np.float64) - p0
            d_ref = state["param"][grp] - p0
            decided = np.ones(p0.shape, bool)
            for g in grads:
                decided &= np.abs(g[grp]) > 1e-2 * np.abs(g[grp]).max()
            ulp = 4 * np.spacing(np.abs(p0).astype(np.float32)).astype(np.float64)
            err = np.abs(d_gpu - d_ref)
            ok_decided = err <= 1e-2 * np.abs(d_ref) + ulp
            ok_rest = err <= 2 * 3 * lr_sum + ulp
            print(f"{grp:15s} decided {decided.sum():6d}/{decided.size}  worst decided err/|d_ref| "
                  f"{float((err[decided] / np.maximum(np.abs(d_ref[decided]), 1e-30)).max()) if decided.any() else 0:.2e}")
            assert decided.sum() > 0, grp
            assert ok_decided[decided].all(), grp
            assert ok_rest.all(), grp
    finally:
        tr.close()
        ctx.unload_scene(sid)


def test_trained_scene_renders_like_a_fresh_load(ctx, tmp_path):
    """After training steps the device refreshes the derived copies (BF16 planes,
    transposed MLP, tensor-core operands): frames of the trained scene equal, bit
    for bit, frames of a scene freshly loaded from its read-back parameters, in
    both precisions; a saved scene file loads back to the same parameters, and a
    damaged file is rejected."""
    s, cam = _scene_and_view()
    sid = ctx.load_scene(s)
    tr = fs4d.Trainer(ctx, sid, 10, **CFG)
    target = torch.rand((cam.height, cam.width, 3), device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    try:
        for k in range(4):
            tr.step(cam, 0.1 * k, target, fs4d.BF16 if k % 2 else fs4d.FP32)
        l1, tv = tr.losses()
        assert np.isfinite(l1) and np.isfinite(tv)
        got = ctx.read_scene(sid)
        fresh = s.copy()
        for k, v in got.items():
            setattr(fresh, k, v)
        assert not np.array_equal(got["planes"], s.planes) and not np.array_equal(got["mlp"], s.mlp)
        sid2 = ctx.load_scene(fresh)
        path = str(tmp_path / "scene.fs4d")
        ctx.save_scene(sid, path)
        sid3 = ctx.load_scene_file(path, like=s)
        try:
            for prec in (fs4d.FP32, fs4d.BF16):
                for t in (0.2, 0.7):
                    a = ctx.render(sid, cam, t, prec)
                    b = ctx.render(sid2, cam, t, prec)
                    c3 = ctx.render(sid3, cam, t, prec)
                    assert torch.equal(a, b) and torch.equal(a, c3)
            back = ctx.read_scene(sid3)
            for k in GROUPS:
                assert np.array_equal(back[k], got[k]), k
        finally:
            ctx.unload_scene(sid2)
            ctx.unload_scene(sid3)
        raw = bytearray(open(path, "rb").read())
        raw[100] ^= 0xFF
        bad = str(tmp_path / "bad.fs4d")
        open(bad, "wb").write(bytes(raw))
        with pytest.raises(fs4d.Fs4dError) as e:
            ctx.load_scene_file(bad)
        assert e.value.status == 1
    finally:
        tr.close()
        ctx.unload_scene(sid)
