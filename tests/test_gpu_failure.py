"""Failure detection on the GPU without a fault: a bounded device-side wait that
gives up sets the context's status word, fs4d_check_device_status reports
FS4D_ERR_TIMEOUT, and the context keeps working.

The wait is made to give up by lowering the context's look-back poll limit
(fs4d_set_wait_limit) to one poll, so that radix-sort partitions stop waiting
for predecessors that are still running.  Their output is then wrong, but the
scatter is bounds-checked, so every access stays inside the buffers; the sort
reads and writes only its own key/value buffers (no index it produces is used
to address memory), which is why the sort, and not a frame, is the test case.
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

TIMEOUT = 5


def _pairs(n, seed):
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 2 ** 63, n, dtype=np.uint64)
    return keys, np.arange(n, dtype=np.uint32)


def test_sort_wait_timeout_is_reported_and_the_context_recovers():
    ctx = fs4d.Context(0)
    try:
        keys, vals = _pairs(4_000_000, 1)
        hit = False
        ctx.set_wait_limit(1)
        try:
            for _ in range(8):
                tk = torch.from_numpy(keys.view(np.int64)).cuda()
                tv = torch.from_numpy(vals.view(np.int32)).cuda()
                ctx.sort_pairs(tk, tv, 64)  # queued; the outcome is in the status word
                try:
                    ctx.check_device_status()
                except fs4d.Fs4dError as e:
                    assert e.status == TIMEOUT
                    hit = True
                    break
        finally:
            ctx.set_wait_limit(0)
        assert hit, "no look-back wait gave up at a limit of one poll"
        ctx.check_device_status()  # read and cleared: nothing pending
        # the default limit again: the sort is exact ...
        tk = torch.from_numpy(keys.view(np.int64)).cuda()
        tv = torch.from_numpy(vals.view(np.int32)).cuda()
        ctx.sort_pairs(tk, tv, 64)
        ctx.check_device_status()
        order = np.argsort(keys, kind="stable")
        assert np.array_equal(tk.cpu().numpy().view(np.uint64), keys[order])
        assert np.array_equal(tv.cpu().numpy().view(np.uint32), vals[order])
        # ... and so is a frame, against the oracle
        s = sg.make_tiny(0, mlp_std=0.1)
        cam = sg.tiny_camera()
        sid = ctx.load_scene(s)
        img = ctx.render(sid, cam, 0.5, fs4d.FP32).cpu().numpy()
        ctx.check_device_status()
        st = parity.check_frame(img, parity.oracle_frame(s, cam, 0.5), tol=1e-4, px_tol=1e-3)
        assert st["unresolved"] == 0
        ctx.unload_scene(sid)
    finally:
        ctx.close()
