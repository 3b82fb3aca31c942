"""GPU parity of the forward render path against the FP64 oracle, through the C ABI.

Tolerances (float32 path): deformed Gaussians within 2e-5 of their scale;
projection outputs within 1e-5 relative; tile keys, sorted values and ranges
bit-exact on identical inputs; every pixel of a frame within 1e-4 max-abs per
channel of the oracle's frame, or of one of the outcomes the oracle enumerates
for that pixel when one of its decisions (alpha vs 1/255, T vs 1e-4, a depth
tie, a tile-rectangle edge) lies within float32 rounding of its threshold.  No
pixel is excluded; the pixels that took another outcome are counted.
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


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def test_library_exports_every_declared_symbol():
    lib = fs4d.library()
    for name in fs4d.EXPORTS:
        assert hasattr(lib, name), name


# ------------------------------------------------------------------ deformation (Eq. 5, Eq. 6)

def deform_tol(s, X, Q, S):
    """float32 tolerance of the deformed outputs: four chained length-64 dot
    products accumulate ~4 * 64 * 2^-24 ~ 1.5e-5 of the output scale; the bound
    is 2e-5 of max(1, max |delta|)."""
    d = max(1.0, float(np.abs(X - s.means).max()), float(np.abs(Q - s.quats).max()),
            float(np.abs(S - s.log_scales).max()))
    return 2e-5 * d


def _check_deform(s, m, q, ls, X, Q, S):
    tol = deform_tol(s, X, Q, S)
    assert np.abs(m.cpu().numpy() - X).max() <= tol
    assert np.abs(q.cpu().numpy() - Q).max() <= tol
    assert np.abs(ls.cpu().numpy() - S).max() <= tol


@pytest.mark.parametrize("maker", [
    lambda: sg.make_tiny(0, mlp_std=0.3),
    lambda: sg.make_tiny(1, n=4099, mlp_std=0.3, bias_std=0.05),
    lambda: sg.make_object(2, n=5000, mlp_std=0.15),
    lambda: sg.make_object(3, n=3001, res_spatial=(16, 32, 64), res_time=9, mlp_std=0.15),
])
def test_deform_fp32_matches_oracle(ctx, maker):
    s = maker()
    sid = ctx.load_scene(s)
    ts = [0.0, 0.37, 1.0]
    m, q, ls = ctx.deform(sid, ts, fs4d.FP32)
    torch.cuda.synchronize()
    for i, t in enumerate(ts):
        X, Q, S = oracle.deform(s, t)
        assert np.abs(X - s.means).max() > 1e-4  # the deformation is really non-trivial
        _check_deform(s, m[i], q[i], ls[i], X, Q, S)
    ctx.unload_scene(sid)


def test_deform_outside_box_clamps(ctx):
    s = sg.make_tiny(4, n=300, mlp_std=0.3)
    s.means[:100] *= 1.7  # outside [-1,1]^3: border clamping
    sid = ctx.load_scene(s)
    m, q, ls = ctx.deform(sid, [0.5, -0.2, 1.3], fs4d.FP32)
    for i, t in enumerate([0.5, -0.2, 1.3]):
        X, Q, S = oracle.deform(s, t)
        _check_deform(s, m[i], q[i], ls[i], X, Q, S)
    ctx.unload_scene(sid)


# ------------------------------------------------------------------ projection (Eq. 2, Eq. 3)

@pytest.mark.parametrize("deg,seed", [(0, 0), (3, 1)])
def test_project_matches_oracle(ctx, deg, seed):
    if deg == 0:
        s = sg.make_tiny(seed)
        cam = sg.tiny_camera()
    else:
        s = sg.make_object(seed, n=20000, res_spatial=(8,), res_time=4, h=16)
        cam = sg.hemisphere_cameras(3, width=800, height=800, seed=seed)[1]
    p = ctx.project(dev(s.means), dev(s.quats), dev(s.log_scales), dev(s.opacity_logits), dev(s.sh), s.sh_degree,
                    cam)
    torch.cuda.synchronize()
    o = oracle.project(s, cam)
    vis = o["radius"] > 0
    # a rect/radius decision within 1e-4 px of its integer boundary may round
    # either way in float32; such Gaussians are ~2.5e-4 of a uniform scene
    safe = o["margin"] > 1e-4
    gr = p["radius"].cpu().numpy()
    grect = p["rect"].cpu().numpy()
    assert vis.sum() > 0.5 * s.n
    assert np.array_equal(gr[safe], o["radius"][safe])
    assert np.array_equal(grect[safe], o["rect"][safe])
    assert (~safe).mean() <= 2e-3
    both = vis & (gr > 0)
    rel = lambda a, b: np.abs(a - b) / np.maximum(np.abs(b), 1.0)
    assert rel(p["xy"].cpu().numpy()[both], o["xy"][both]).max() <= 1e-5
    co = p["conic_opacity"].cpu().numpy()
    scale = np.abs(o["conic"][both]).max(1, keepdims=True)
    assert (np.abs(co[both, :3] - o["conic"][both]) / scale).max() <= 1e-5
    assert np.abs(co[:, 3] - o["opacity"]).max() <= 1e-6
    assert rel(p["depth"].cpu().numpy(), o["depth"]).max() <= 1e-6
    assert np.abs(p["rgb"].cpu().numpy()[both] - o["rgb"][both]).max() <= 1e-5


# ------------------------------------------------------------------ binning + sort + ranges (bit-exact)

def _random_bins(rng, n, tx, ty, max_w=4, tie_every=17):
    depth = rng.uniform(0.3, 20.0, n).astype(np.float32)
    if n > 5 and tie_every:
        depth[::tie_every] = depth[5]
    x0 = rng.integers(0, tx, n)
    y0 = rng.integers(0, ty, n)
    rect = np.stack([x0, y0, np.minimum(tx, x0 + rng.integers(0, max_w + 1, n)),
                     np.minimum(ty, y0 + rng.integers(0, max_w + 1, n))], 1).astype(np.int32)
    return depth, rect


BITMAP_MAX = 256 << 20


def _expect_binning(mode, n, tx, ty):
    """The binning a frame of n Gaussians over tx x ty tiles gets under `mode`."""
    fits = tx * ty * ((n + 127) // 128) * 16 <= BITMAP_MAX
    return fs4d.BINNING_BITMAP if mode == fs4d.BINNING_AUTO and fits else fs4d.BINNING_SORT


@pytest.fixture(params=[fs4d.BINNING_AUTO, fs4d.BINNING_SORT], ids=["auto", "sort"])
def binning(ctx, request):
    ctx.set_binning(request.param)
    yield request.param
    ctx.set_binning(fs4d.BINNING_AUTO)


@pytest.mark.parametrize("n,tx,ty", [(1, 1, 1), (7, 3, 2), (2047, 8, 8), (2049, 50, 50), (40000, 50, 50),
                                     (3001, 200, 100),     # more tiles than the per-CTA shared-memory counts
                                     (150001, 240, 135)])  # bitmap above its size limit: sort binning
def test_bin_sort_bit_exact(ctx, binning, n, tx, ty):
    rng = np.random.default_rng(n)
    depth, rect = _random_bins(rng, n, tx, ty)
    keys_o, vals_o, ranges_o = oracle.bin_sort(depth.view(np.uint32), rect, tx, ty)
    K = len(keys_o)
    keys, vals, ranges, Kg = ctx.bin_sort(dev(depth), dev(rect), tx, ty, K + 100)
    torch.cuda.synchronize()
    assert ctx.last_binning() == _expect_binning(binning, n, tx, ty)
    assert Kg == K
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), keys_o)
    assert np.array_equal(vals.cpu().numpy().view(np.uint32), vals_o)
    assert np.array_equal(ranges.cpu().numpy().view(np.uint32), ranges_o)


@pytest.mark.parametrize("n,tx,ty,max_w", [(30000, 4, 4, 4),     # tiles of ~7k pairs: the long-tile sort
                                           (60000, 2, 2, 2),     # tiles of ~30k: chunk sort + merges
                                           (50000, 40, 3, 3)])   # one hot tile among short ones
def test_bin_sort_dense_tiles_bit_exact(ctx, binning, n, tx, ty, max_w):
    rng = np.random.default_rng(n + tx)
    depth, rect = _random_bins(rng, n, tx, ty, max_w=max_w, tie_every=7)
    if tx == 40:  # half of the Gaussians on tile 0 only (several merge rounds, odd last run)
        rect[: n // 2] = (0, 0, 1, 1)
    keys_o, vals_o, ranges_o = oracle.bin_sort(depth.view(np.uint32), rect, tx, ty)
    lens = ranges_o[1::2].astype(np.int64) - ranges_o[0::2]
    assert lens.max() > 2048
    K = len(keys_o)
    keys, vals, ranges, Kg = ctx.bin_sort(dev(depth), dev(rect), tx, ty, K)
    torch.cuda.synchronize()
    assert ctx.last_binning() == _expect_binning(binning, n, tx, ty)
    assert Kg == K
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), keys_o)
    assert np.array_equal(vals.cpu().numpy().view(np.uint32), vals_o)
    assert np.array_equal(ranges.cpu().numpy().view(np.uint32), ranges_o)


def test_bin_sort_empty_and_capacity(ctx, binning):
    depth = np.ones(10, np.float32)
    rect = np.zeros((10, 4), np.int32)  # every Gaussian culled
    keys, vals, ranges, K = ctx.bin_sort(dev(depth), dev(rect), 4, 4, 16)
    assert K == 0 and int(ranges.abs().sum()) == 0
    rect[:, 2:] = 4  # 16 tiles each -> 160 pairs
    with pytest.raises(fs4d.Fs4dError) as e:
        ctx.bin_sort(dev(depth), dev(rect), 4, 4, 100)
    assert e.value.status == 3
    # the overflowed call leaves no state behind (the tile bitmap is cleared)
    depth = np.random.default_rng(3).uniform(1, 2, 10).astype(np.float32)
    rect[5:] = (1, 1, 3, 2)
    keys_o, vals_o, ranges_o = oracle.bin_sort(depth.view(np.uint32), rect, 4, 4)
    keys, vals, ranges, K = ctx.bin_sort(dev(depth), dev(rect), 4, 4, 200)
    torch.cuda.synchronize()
    assert K == len(keys_o)
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), keys_o)
    assert np.array_equal(vals.cpu().numpy().view(np.uint32), vals_o)
    assert np.array_equal(ranges.cpu().numpy().view(np.uint32), ranges_o)


@pytest.mark.parametrize("n,bits", [(1, 8), (4095, 12), (4097, 33), (100000, 44), (262145, 64), (30000, 1),
                                    (17, 3), (50001, 24), (100000, 32), (131072, 32), (131073, 32),
                                    ((1 << 19) + 1, 20),     # above 2^19 keys: the persistent, prefetching pass
                                    (3 * (1 << 20) + 7, 64)])
def test_sort_pairs_matches_stable_numpy(ctx, n, bits):
    rng = np.random.default_rng(bits)
    # bits above key_bits are not part of the key: they travel along and do not order
    keys = rng.integers(0, 2 ** 63, n, dtype=np.uint64) | (rng.integers(0, 2, n, dtype=np.uint64) << np.uint64(63))
    keys[::5] = keys[min(1, n - 1)]  # ties keep input order
    low = keys & np.uint64((1 << bits) - 1) if bits < 64 else keys
    vals = np.arange(n, dtype=np.uint32)
    tk = dev(keys.view(np.int64))
    tv = dev(vals.view(np.int32))
    ctx.sort_pairs(tk, tv, bits)
    order = np.argsort(low, kind="stable")
    assert np.array_equal(tk.cpu().numpy().view(np.uint64), keys[order])
    assert np.array_equal(tv.cpu().numpy().view(np.uint32), vals[order])


@pytest.mark.parametrize("binning", ["auto", "sort"])
def test_last_launches_counts_the_frame_kernels(ctx, binning):
    """fs4d_last_launches: deform, project, the depth sort in one launch (its 1024-key
    partitions all fit at once), then mark, tile scan, extract (bitmap) or emission,
    tile scan and the pair-sort passes on the tile bits (sort), then composite."""
    s = sg.make_tiny(41, n=3000)
    cam = sg.tiny_camera(200, 136)
    sid = ctx.load_scene(s)
    try:
        ctx.set_binning(fs4d.BINNING_SORT if binning == "sort" else fs4d.BINNING_AUTO)
        ctx.render(sid, cam, 0.5)
        torch.cuda.synchronize()
        tiles = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
        passes = (int(np.ceil(np.log2(tiles))) + 7) // 8
        want = 7 if ctx.last_binning() == fs4d.BINNING_BITMAP else 6 + passes
        assert ctx.last_launches() == want
    finally:
        ctx.set_binning(fs4d.BINNING_AUTO)
        ctx.unload_scene(sid)


@pytest.mark.parametrize("n", [5, 100000, 131072])
def test_sort_depth_keys_and_constant_digits(ctx, n):
    """Depth-like keys (float32 bits of depths in [2, 4): the top byte is the same
    for every key, so that pass moves nothing), all-equal keys (every pass keeps
    the order) and bits above 32 that travel with the keys."""
    rng = np.random.default_rng(n)
    depth = rng.uniform(2.0, 4.0, n).astype(np.float32)
    depth[::7] = depth[0]
    hi = rng.integers(0, 2 ** 31, n, dtype=np.uint64) << np.uint64(32)
    for keys in (depth.view(np.uint32).astype(np.uint64) | hi, np.full(n, 0xABCD00001234, np.uint64)):
        vals = rng.permutation(n).astype(np.uint32)
        tk = dev(keys.view(np.int64))
        tv = dev(vals.view(np.int32))
        ctx.sort_pairs(tk, tv, 32)
        order = np.argsort(keys & np.uint64(0xFFFFFFFF), kind="stable")
        assert np.array_equal(tk.cpu().numpy().view(np.uint64), keys[order])
        assert np.array_equal(tv.cpu().numpy().view(np.uint32), vals[order])


# ------------------------------------------------------------------ compositing (Eq. 4)

@pytest.mark.parametrize("seed", [0, 1])
def test_composite_matches_oracle_on_same_inputs(ctx, seed):
    s = sg.make_tiny(seed)
    cam = sg.tiny_camera(144, 120)  # ragged: 9 x 8 tiles, last row partial
    o = oracle.project(s, cam)
    # the float32 values the kernel sees are also the oracle's inputs
    p32 = {k: (v.astype(np.float32).astype(np.float64) if v.dtype == np.float64 else v) for k, v in o.items()}
    _, vals, ranges = oracle.bin_sort(oracle.depth_bits(p32["depth"]), o["rect"], 9, 8)
    img_o, T_o, nc_o, mg = oracle.composite(144, 120, ranges, vals, p32)
    co = np.concatenate([p32["conic"], p32["opacity"][:, None]], 1)
    img, T, nc = ctx.composite(144, 120, dev(ranges.view(np.int32)), dev(vals.view(np.int32)),
                               dev(p32["xy"].astype(np.float32)), dev(co.astype(np.float32)),
                               dev(p32["rgb"].astype(np.float32)))
    torch.cuda.synchronize()
    fr = dict(img=img_o, T=T_o, nc=nc_o, margin=mg, proj=p32, values=vals, ranges=ranges,
              dbits=oracle.depth_bits(p32["depth"]), tx=9, tile=16)
    # same float32 inputs: only the blend's own rounding can flip a decision
    st = parity.check_frame(img.cpu().numpy(), fr, T.cpu().numpy(), nc.cpu().numpy(), tol=1e-5, rel_tol=1e-5,
                            px_tol=0.0)
    assert st["unresolved"] == 0 and st["other_outcome"] == 0


# ------------------------------------------------------------------ full frame

def _gpu_rects(ctx, sid, s, cam, t):
    """The GPU's own tile rectangles and radii of the frame at t: fs4d_deform (FP32)
    then fs4d_project, the kernels the frame runs on the same inputs."""
    m, q, ls = ctx.deform(sid, [t], fs4d.FP32)
    p = ctx.project(m[0], q[0], ls[0], dev(s.opacity_logits), dev(s.sh), s.sh_degree, cam)
    torch.cuda.synchronize()
    return p["rect"].cpu().numpy(), p["radius"].cpu().numpy()


def _rect_decisions(ctx, sid, s, cam, t, fr, px_tol):
    """Every tile rectangle the GPU decides differently from the oracle must be a
    decision within px_tol of its boundary in the oracle; the frame's pair count
    is the sum of the GPU rectangles' areas.  Returns the number that differ."""
    rect, radius = _gpu_rects(ctx, sid, s, cam, t)
    ro = fr["proj"]["rect"]
    diff = np.any(rect != ro, axis=1)
    assert (fr["proj"]["margin"][diff] < px_tol).all()
    area = (np.maximum(rect[:, 2] - rect[:, 0], 0) * np.maximum(rect[:, 3] - rect[:, 1], 0)).sum()
    assert int(area) == ctx.last_pairs()
    print(f"tile rectangles decided differently: {int(diff.sum())} of {s.n}")
    return int(diff.sum())


@pytest.mark.parametrize("seed,std", [(0, 0.1), (1, 0.1), (2, 0.05), (3, 0.02)])
def test_render_fp32_tiny_matches_oracle(ctx, seed, std):
    """Every pixel, its final transmittance and its last contributor against the
    oracle (1e-4); at these seeds the GPU takes every decision as the oracle does."""
    s = sg.make_tiny(seed, mlp_std=std)
    cam = sg.tiny_camera()
    sid = ctx.load_scene(s)
    img, T, nc = ctx.render(sid, cam, 0.5, fs4d.FP32, with_aux=True)
    torch.cuda.synchronize()
    fr = parity.oracle_frame(s, cam, 0.5)
    st = parity.check_frame(img.cpu().numpy(), fr, T.cpu().numpy(), nc.cpu().numpy(), tol=IMG_TOL,
                            px_tol=1e-3)
    assert st["unresolved"] == 0
    assert st["other_outcome"] == 0
    assert _rect_decisions(ctx, sid, s, cam, 0.5, fr, 1e-3) == 0
    ctx.unload_scene(sid)


def test_render_static_special_case(ctx):
    """Zero head output layers: dG = 0 and the frame is the static 3D-GS render."""
    s = sg.make_tiny(3, mlp_std=0.1)
    shapes = sg.mlp_layer_shapes(16, 64)
    off = 0
    for k, (o, i) in enumerate(shapes):
        if k in (3, 5, 7):
            s.mlp[off:off + o * i + o] = 0.0
        off += o * i + o
    cam = sg.tiny_camera()
    sid = ctx.load_scene(s)
    img = ctx.render(sid, cam, 0.9, fs4d.FP32).cpu().numpy()
    st = parity.check_frame(img, parity.oracle_frame(s, cam, 0.9, deform=False), tol=IMG_TOL, px_tol=1e-3)
    assert st["unresolved"] == 0 and st["other_outcome"] == 0
    ctx.unload_scene(sid)


@pytest.mark.parametrize("ci,t", [(7, 0.35), (31, 0.9)])
def test_render_object_800_matches_oracle(ctx, ci, t):
    """The 100k-Gaussian 800x800 object frame, every pixel against the oracle.
    At 800 px one float32 ulp of a pixel coordinate is 6e-5 px, which moves alpha
    by up to ~|grad power| * 6e-5 ~ 3e-5 relative: decisions within 5e-5 of their
    threshold, and tile rectangles within 2e-4 px of an integer boundary, may go
    either way; such a pixel must equal one of the oracle's outcomes for it."""
    s = sg.make_object(0)
    cam = sg.hemisphere_cameras(50, seed=0)[ci]
    sid = ctx.load_scene(s)
    img = ctx.render(sid, cam, t, fs4d.FP32).cpu().numpy()
    oracle.set_threads(oracle.default_threads())
    fr = parity.oracle_frame(s, cam, t)
    K_gpu = ctx.last_pairs()
    st = parity.check_frame(img, fr, tol=IMG_TOL, rel_tol=5e-5, px_tol=2e-4)
    assert st["unresolved"] == 0
    assert st["other_outcome_frac"] <= 5e-3
    assert abs(K_gpu - fr["K"]) <= 1e-4 * fr["K"]
    n_diff = _rect_decisions(ctx, sid, s, cam, t, fr, 2e-4)
    assert n_diff <= 1e-3 * s.n
    ctx.unload_scene(sid)


def test_render_host_equals_device(ctx):
    s = sg.make_tiny(5, mlp_std=0.3)
    cam = sg.tiny_camera(200, 150)
    sid = ctx.load_scene(s)
    a = ctx.render(sid, cam, 0.2).cpu().numpy()
    b = ctx.render_host(sid, cam, 0.2)
    assert np.array_equal(a, b)
    ctx.unload_scene(sid)


def test_render_host_first_frame_regrows_capacity():
    """A fresh context has no pair capacity: its first host-buffer frame overflows,
    is rendered again with the capacity grown, and equals the device render."""
    c = fs4d.Context(0)
    try:
        s = sg.make_tiny(8, mlp_std=0.3)
        cam = sg.tiny_camera(160, 96)
        sid = c.load_scene(s)
        b = c.render_host(sid, cam, 0.7)
        assert c.last_pairs() > 0
        a = c.render(sid, cam, 0.7).cpu().numpy()
        assert np.array_equal(a, b)
    finally:
        c.close()


@pytest.mark.parametrize("fresh", [True, False])
def test_render_host_batch_equals_single_frames(ctx, fresh):
    """The batched host render (two device image slots, copies overlapped with the
    next frame) gives each frame's image exactly; on a fresh context the first
    frames overflow the empty pair capacity and are rendered again."""
    c = fs4d.Context(0) if fresh else ctx
    try:
        s = sg.make_object(9, n=20000)
        sid = c.load_scene(s)
        cams = sg.hemisphere_cameras(5, width=200, height=136, seed=4)
        ts = [0.1, 0.9, 0.3, 0.5, 0.7]
        for prec in (fs4d.FP32, fs4d.BF16):
            got = c.render_host_batch(sid, cams, ts, prec)
            for cam, t, g in zip(cams, ts, got):
                assert np.array_equal(g, c.render_host(sid, cam, t, prec))
            # one destination for every frame: the last frame's image
            one = np.zeros((136, 200, 3), np.float32)
            c.render_host_batch(sid, cams, ts, prec, [one] * len(cams))
            assert np.array_equal(one, got[-1])
        c.unload_scene(sid)
    finally:
        if fresh:
            c.close()


def test_render_async_and_graph_replay_equal_sync(ctx):
    s = sg.make_tiny(6, mlp_std=0.3)
    cams = [sg.tiny_camera(), sg.hemisphere_cameras(4, width=128, height=128, seed=3)[2]]
    sid = ctx.load_scene(s)
    ctx.reserve(sid, 128, 128, 200000)
    d_cam = torch.empty(23, dtype=torch.float32, device="cuda")
    d_t = torch.empty(1, dtype=torch.float32, device="cuda")
    out = torch.empty((128, 128, 3), device="cuda")

    def set_view(cam, t):
        cs = fs4d.camera_struct(cam)
        raw = np.frombuffer(bytes(cs), dtype=np.float32).copy()
        d_cam.copy_(torch.from_numpy(raw))
        d_t.fill_(t)

    set_view(cams[0], 0.4)
    ctx.render_async(sid, cams[0], d_cam, d_t, out)
    ref = ctx.render(sid, cams[0], 0.4)
    assert torch.equal(out, ref)
    # capture once, replay for another view
    stream = torch.cuda.Stream()
    ctx.set_stream(stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        ctx.render_async(sid, cams[0], d_cam, d_t, out)  # warm-up outside capture
        stream.synchronize()
        with torch.cuda.graph(g, stream=stream):
            ctx.render_async(sid, cams[0], d_cam, d_t, out)
    ctx.set_stream(torch.cuda.current_stream())
    set_view(cams[1], 0.8)
    g.replay()
    torch.cuda.synchronize()
    ref = ctx.render(sid, cams[1], 0.8)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    ctx.check_device_status()
    ctx.unload_scene(sid)


def test_capacity_overflow_sets_status_not_fault(ctx, binning):
    """A frame with more tile pairs than the reserved capacity must report, not
    fault, and leave nothing behind (the tile bitmap is cleared)."""
    s = sg.make_tiny(7)
    cam = sg.tiny_camera()
    sid = ctx.load_scene(s)
    ctx.reserve(sid, 128, 128, 4096)
    K = oracle.render(s, cam, 0.5)[4]
    assert K > 4096
    ctx._scenes[sid] = s
    d_cam = torch.from_numpy(np.frombuffer(bytes(fs4d.camera_struct(cam)), dtype=np.float32).copy()).cuda()
    d_t = torch.full((1,), 0.5, device="cuda")
    out = torch.zeros((128, 128, 3), device="cuda")
    # shrink the reservation to below K: the frame must report, not fault
    ctx.call("fs4d_reserve", sid, 128, 128, 1000)
    ctx.render_async(sid, cam, d_cam, d_t, out)
    with pytest.raises(fs4d.Fs4dError) as e:
        ctx.check_device_status()
    assert e.value.status == 3
    assert ctx.last_binning() == _expect_binning(binning, s.n, 8, 8)
    ctx.check_device_status()  # cleared
    # nothing of the overflowed frame stays behind: the next one is exact
    ctx.call("fs4d_reserve", sid, 128, 128, 2 * K)
    ctx.render_async(sid, cam, d_cam, d_t, out)
    ref = ctx.render(sid, cam, 0.5)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    ctx.check_device_status()
    ctx.unload_scene(sid)


@pytest.mark.parametrize("prec", [fs4d.FP32, fs4d.BF16])
@pytest.mark.parametrize("w,h", [(800, 800), (333, 517)])
def test_bitmap_and_sort_binning_render_identical_images(ctx, prec, w, h):
    """Both binnings give the same per-tile lists, so the images are bit-identical
    (Sec. 3.1: per-tile depth order), also for ragged tile grids and views whose
    Gaussians leave the image."""
    s = sg.make_object(4, n=30011)
    sid = ctx.load_scene(s)
    cams = sg.hemisphere_cameras(3, width=w, height=h, seed=5)
    try:
        for i, cam in enumerate(cams):
            ctx.set_binning(fs4d.BINNING_SORT)
            a = ctx.render(sid, cam, 0.3 * i, prec=prec, with_aux=True)
            assert ctx.last_binning() == fs4d.BINNING_SORT
            ctx.set_binning(fs4d.BINNING_AUTO)
            b = ctx.render(sid, cam, 0.3 * i, prec=prec, with_aux=True)
            assert ctx.last_binning() == fs4d.BINNING_BITMAP
            torch.cuda.synchronize()
            for x, y in zip(a, b):  # image, final transmittance, last contributor
                assert torch.equal(x, y)
    finally:
        ctx.set_binning(fs4d.BINNING_AUTO)
        ctx.unload_scene(sid)


@pytest.mark.parametrize("prec", [fs4d.FP32, fs4d.BF16])
@pytest.mark.parametrize("binning", ["auto", "sort"])
def test_culled_tile_lists_render_identical_images(ctx, prec, binning):
    """Frames that report no list positions leave out of each tile's list the
    Gaussians whose ellipse {alpha >= 1/255} reaches none of the tile's pixel
    centres (the bitmap binning in its marks, the sort binning in its emission);
    no pixel would blend them, so the image is bit-identical to the frame over the
    full rectangles (a frame with last-contributor output), on the 800x800 object,
    a ragged frame, and through the host call; both report the rectangles' pairs."""
    s = sg.make_object(0)
    sid = ctx.load_scene(s)
    ctx.set_binning(fs4d.BINNING_SORT if binning == "sort" else fs4d.BINNING_AUTO)
    try:
        for cam in (sg.hemisphere_cameras(50, width=800, height=800)[7],
                    sg.hemisphere_cameras(3, width=333, height=517, seed=2)[1]):
            full, _, _ = ctx.render(sid, cam, 0.35, prec=prec, with_aux=True)
            k_full = ctx.last_pairs()
            culled = ctx.render(sid, cam, 0.35, prec=prec)
            k_culled = ctx.last_pairs()
            host = ctx.render_host(sid, cam, 0.35, prec=prec)
            torch.cuda.synchronize()
            assert torch.equal(full, culled)
            assert np.array_equal(full.cpu().numpy(), host)
            assert k_full == k_culled
    finally:
        ctx.set_binning(fs4d.BINNING_AUTO)
        ctx.unload_scene(sid)


# ------------------------------------------------------------------ BF16 tensor-core path

def bf16_tol(s, X, Q, S):
    """BF16 keeps 8 significant bits (unit roundoff 2^-9 ~ 2e-3).  Planes, every
    layer input and every weight are rounded once: ~6 roundings into f_h and ~2
    per layer over 4 layers, so the deltas carry a relative error of a few 1e-2
    of their scale; the bound is 5e-2 of max |delta| (+1e-6)."""
    d = max(float(np.abs(X - s.means).max()), float(np.abs(Q - s.quats).max()), float(np.abs(S - s.log_scales).max()))
    return 5e-2 * d + 1e-6


@pytest.mark.parametrize("maker", [
    lambda: sg.make_tiny(0, mlp_std=0.1),
    lambda: sg.make_tiny(1, n=129, mlp_std=0.1, bias_std=0.05),
    lambda: sg.make_object(2, n=5000, mlp_std=0.1),
    lambda: sg.make_object(3, n=3001, res_spatial=(16, 32, 64), res_time=9, mlp_std=0.1),
])
def test_deform_bf16_matches_oracle(ctx, maker):
    s = maker()
    sid = ctx.load_scene(s)
    ts = [0.0, 0.61]
    m, q, ls = ctx.deform(sid, ts, fs4d.BF16)
    torch.cuda.synchronize()
    for i, t in enumerate(ts):
        X, Q, S = oracle.deform(s, t)
        tol = bf16_tol(s, X, Q, S)
        errs = [np.abs(m[i].cpu().numpy() - X).max(), np.abs(q[i].cpu().numpy() - Q).max(),
                np.abs(ls[i].cpu().numpy() - S).max()]
        print(f"bf16 deform t={t}: max|dX|={errs[0]:.2e} max|dr|={errs[1]:.2e} max|ds|={errs[2]:.2e} tol={tol:.2e}")
        assert max(errs) <= tol
    ctx.unload_scene(sid)


def psnr(a, b):
    mse = float(np.mean((a - b) ** 2))
    return float("inf") if mse == 0 else 10.0 * np.log10(1.0 / mse)


def test_render_bf16_psnr_object_800(ctx):
    """BF16 MLP/planes on tcgen05: image PSNR against the FP64 oracle >= 50 dB."""
    s = sg.make_object(0)
    sid = ctx.load_scene(s)
    oracle.set_threads(oracle.default_threads())
    for ci, t in ((7, 0.35), (31, 0.9)):
        cam = sg.hemisphere_cameras(50, seed=0)[ci]
        img = ctx.render(sid, cam, t, fs4d.BF16).cpu().numpy()
        want, *_ = oracle.render(s, cam, t)
        p = psnr(img, want)
        print(f"bf16 frame cam {ci} t={t}: PSNR {p:.1f} dB, max abs {np.abs(img - want).max():.2e}")
        assert p >= 50.0
    ctx.unload_scene(sid)


def test_render_bf16_tiny_psnr(ctx):
    s = sg.make_tiny(2, mlp_std=0.1)
    cam = sg.tiny_camera()
    sid = ctx.load_scene(s)
    img = ctx.render(sid, cam, 0.5, fs4d.BF16).cpu().numpy()
    want, *_ = oracle.render(s, cam, 0.5)
    assert psnr(img, want) >= 50.0
    ctx.unload_scene(sid)
