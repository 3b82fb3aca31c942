"""Continuous-batching server (fs4d_server_*, through the C ABI).

The central check: a request's image is the same when it is served alone and
when it is served in a mix of other scenes, resolutions and precisions that
overlap on the device.  The frame path is deterministic, so the bar is bit
equality (and equality with the single-frame fs4d_render)."""
import numpy as np
import pytest

from paper_2310_08528_gb300 import scenegen as sg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2310_08528_gb300 import fs4d  # noqa: E402

OK, CAPACITY, NOT_FOUND, CANCELLED = 0, 3, 6, 8


@pytest.fixture(scope="module")
def world():
    ctx = fs4d.Context(0)
    scenes = [ctx.load_scene(sg.make_tiny(0, mlp_std=0.1)),
              ctx.load_scene(sg.make_object(1, n=20000, mlp_std=0.05)),
              ctx.load_scene(sg.make_object(2, n=12000, res_spatial=(16, 32, 64), res_time=9, mlp_std=0.05))]
    yield ctx, scenes
    ctx.close()


def cam_for(scene_idx, w, h, k):
    if scene_idx == 0:
        return sg.tiny_camera(w, h)
    return sg.hemisphere_cameras(8, width=w, height=h, seed=scene_idx)[k % 8]


@pytest.fixture
def server(world):
    made = []

    def make(**kw):
        srv = fs4d.Server(world[0], **kw)
        made.append(srv)
        return srv

    yield make
    for srv in made:
        srv.close()
    

def wait_all(srv, tickets):
    srv.drain()
    done = {c["ticket"]: c for c in srv.poll(1024)}
    assert set(tickets) <= set(done), "missing completions"
    return done


def test_alone_equals_mix(world, server):
    ctx, scenes = world
    srv = server(max_inflight=4, max_batch=4)
    probes = [(1, 256, 192, 3, 0.3, fs4d.FP32), (2, 200, 200, 5, 0.7, fs4d.BF16), (0, 128, 128, 0, 0.5, fs4d.FP32)]
    alone = []
    for si, w, h, k, t, p in probes:
        out = torch.zeros((h, w, 3), device="cuda")
        tk = srv.submit(scenes[si], cam_for(si, w, h, k), t, out, p)
        d = wait_all(srv, [tk])
        assert d[tk]["status"] == OK
        alone.append(out)
    # the same requests inside a mix of 24 others that overlap on the device
    rng = np.random.default_rng(0)
    mix, outs, tickets = [], [], []
    for j in range(24):
        si = int(rng.integers(0, 3))
        w, h = [(128, 128), (256, 192), (200, 200), (320, 240)][int(rng.integers(0, 4))]
        mix.append((si, w, h, int(rng.integers(0, 8)), float(rng.uniform()), [fs4d.FP32, fs4d.BF16][j % 2]))
    for pos, pr in zip((3, 11, 19), probes):
        mix.insert(pos, pr)
    # half submitted one by one while frames run, half queued as one group
    items = []
    for j, (si, w, h, k, t, p) in enumerate(mix):
        out = torch.zeros((h, w, 3), device="cuda")
        outs.append(out)
        items.append((scenes[si], cam_for(si, w, h, k), t, out, p))
    for it in items[:13]:
        tickets.append(srv.submit(*it))
    tickets += srv.submit_batch(items[13:])
    d = wait_all(srv, tickets)
    assert all(d[tk]["status"] == OK for tk in tickets)
    for pos, ref in zip((3, 11, 19), alone):
        assert torch.equal(outs[pos], ref)
    # and equal to the single-frame call
    for (si, w, h, k, t, p), ref in zip(probes, alone):
        direct = ctx.render(scenes[si], cam_for(si, w, h, k), t, p)
        torch.cuda.synchronize()
        assert torch.equal(direct, ref)
    st = srv.stats()
    print("serving stats:", st)
    assert st["batches"] < st["deformed"]  # requests of one scene shared a deformation launch
    assert st["max_concurrent"] > 1        # frames of several requests were on the GPU together


@pytest.mark.parametrize("binning", ["sort", "auto"])
def test_capacity_overflow_is_retried(world, server, binning):
    """A frame whose pairs overflow the slot's first capacity guess is re-run with
    a larger one (either binning), and gives the reference image."""
    ctx, scenes = world
    ctx.set_binning(fs4d.BINNING_SORT if binning == "sort" else fs4d.BINNING_AUTO)
    try:
        srv = server(max_inflight=2, max_batch=2, pairs_per_gaussian=0.01)
        cam = cam_for(1, 256, 256, 2)
        out = torch.zeros((256, 256, 3), device="cuda")
        tk = srv.submit(scenes[1], cam, 0.4, out)
        d = wait_all(srv, [tk])
        assert d[tk]["status"] == OK
        assert srv.stats()["retried"] >= 1
        ref = ctx.render(scenes[1], cam, 0.4)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    finally:
        ctx.set_binning(fs4d.BINNING_AUTO)


def test_admission_respects_the_device_memory_budget(world, server):
    ctx, scenes = world
    srv = server(max_inflight=8, max_batch=8, hbm_budget_bytes=12 << 20, pairs_per_gaussian=8.0)
    outs, tickets = [], []
    for k in range(6):
        out = torch.zeros((320, 240, 3), device="cuda")
        tickets.append(srv.submit(scenes[1], cam_for(1, 240, 320, k), 0.1 * k, out))
        outs.append(out)
    d = wait_all(srv, tickets)
    assert all(d[tk]["status"] == OK for tk in tickets)
    st = srv.stats()
    assert st["peak_slot_bytes"] <= 12 << 20
    assert st["max_concurrent"] == 1  # only one slot fits the budget


def test_unknown_scene_and_cancel(world, server):
    ctx, scenes = world
    srv = server(max_inflight=1, max_batch=1)
    bad = srv.submit(9999, cam_for(0, 64, 64, 0), 0.5, torch.zeros((64, 64, 3), device="cuda"))
    tickets = [srv.submit(scenes[1], cam_for(1, 320, 240, k), 0.5, torch.zeros((240, 320, 3), device="cuda"))
               for k in range(6)]
    cancelled = srv.cancel(tickets[-1])
    d = wait_all(srv, [bad] + tickets)
    assert d[bad]["status"] == NOT_FOUND
    assert d[tickets[-1]]["status"] == (CANCELLED if cancelled else OK)
    assert all(d[tk]["status"] == OK for tk in tickets[:-1])


def test_unload_while_queued(world, server):
    ctx, _ = world
    sid = ctx.load_scene(sg.make_object(5, n=8000, mlp_std=0.05))
    srv = server(max_inflight=1, max_batch=1)
    tickets = [srv.submit(sid, cam_for(1, 256, 256, k), 0.5, torch.zeros((256, 256, 3), device="cuda"))
               for k in range(8)]
    ctx.unload_scene(sid)  # waits for in-flight frames; queued ones fail cleanly
    late = srv.submit(sid, cam_for(1, 64, 64, 0), 0.5, torch.zeros((64, 64, 3), device="cuda"))
    d = wait_all(srv, tickets + [late])
    assert all(d[tk]["status"] in (OK, NOT_FOUND) for tk in tickets)
    assert d[late]["status"] == NOT_FOUND


def test_host_output_equals_device_output(world, server):
    ctx, scenes = world
    srv = server(max_inflight=2, max_batch=2)
    cam = cam_for(2, 200, 150, 1)
    dev = torch.zeros((150, 200, 3), device="cuda")
    host = torch.zeros((150, 200, 3)).pin_memory().numpy()
    t1 = srv.submit(scenes[2], cam, 0.25, dev)
    t2 = srv.submit(scenes[2], cam, 0.25, host)
    d = wait_all(srv, [t1, t2])
    assert d[t1]["status"] == OK and d[t2]["status"] == OK
    assert np.array_equal(dev.cpu().numpy(), host)


def test_served_frame_matches_oracle():
    """A request served at a benchmark resolution (the 100k-Gaussian object at
    800x800), in a mix with other requests, against the FP64 oracle: every pixel
    equals the oracle's frame or one of its near-threshold outcomes."""
    import oracle
    import parity
    ctx = fs4d.Context(0)
    try:
        s = sg.make_object(0)
        sid = ctx.load_scene(s)
        other = ctx.load_scene(sg.make_object(5, n=30000))
        srv = fs4d.Server(ctx, max_inflight=4, max_batch=4)
        cam = sg.hemisphere_cameras(50, seed=0)[7]
        out = torch.zeros((800, 800, 3), device="cuda")
        others = [torch.zeros((400, 400, 3), device="cuda") for _ in range(6)]
        tickets = [srv.submit(other, sg.hemisphere_cameras(6, width=400, height=400, seed=3)[k], 0.1 * k, o,
                              fs4d.BF16 if k % 2 else fs4d.FP32) for k, o in enumerate(others)]
        tk = srv.submit(sid, cam, 0.35, out, fs4d.FP32)
        done = wait_all(srv, tickets + [tk])
        assert done[tk]["status"] == OK
        srv.close()
        oracle.set_threads(oracle.default_threads())
        st = parity.check_frame(out.cpu().numpy(), parity.oracle_frame(s, cam, 0.35), tol=1e-4, rel_tol=5e-5,
                                px_tol=2e-4)
        assert st["unresolved"] == 0
        assert st["other_outcome_frac"] <= 5e-3
    finally:
        ctx.close()
