"""The allocation-free sort entry point, through the C ABI.

fs4d_sort_pairs_noalloc exists for callers that must not let the library
allocate device memory -- an application that owns the whole device-memory
budget, or a latency-critical loop where cudaMalloc/cudaFree (which can
synchronise the device) are not allowed.  It keeps its work area in a fixed
device array instead.  This test checks that it sorts exactly like the regular
fs4d_sort_pairs (sorting is integer work, so the comparison is bit-exact) on
calls in a row, up to the size limit with every key bit sorted, that its status
word (fs4d_sort_pairs_noalloc_status) reports no bounded wait that gave up, and
that it rejects a size above its limit.

This file is collected last on purpose, so that a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2310_08528_gb300 import fs4d  # noqa: E402

CAPACITY = 3


def _pairs(seed, n, bits):
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 2 ** 63, n, dtype=np.uint64)
    keys &= np.uint64((1 << bits) - 1) if bits < 64 else np.uint64(2 ** 64 - 1)
    keys[::7] = keys[3]  # equal keys must keep their input order
    return keys, np.arange(n, dtype=np.uint32)


def test_noalloc_sort_matches_regular_sort_twice():
    lib = fs4d.library()
    ctx = fs4d.Context(0)
    stream = torch.cuda.current_stream()
    # calls in a row with different sizes and key widths: a later call must not
    # see anything an earlier one left in the shared work area; the last one
    # fills the work area (the size limit, 8 passes of 256 large partitions)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for seed, n, bits in ((1, 300_001, 44), (2, 70_000, 33), (3, 1 << 20, 64)):
        keys, vals = _pairs(seed, n, bits)
        ref_k = torch.from_numpy(keys.view(np.int64)).cuda()
        ref_v = torch.from_numpy(vals.view(np.int32)).cuda()
        ctx.sort_pairs(ref_k, ref_v, bits)
        got_k = torch.from_numpy(keys.view(np.int64)).cuda()
        got_v = torch.from_numpy(vals.view(np.int32)).cuda()
        rc = lib.fs4d_sort_pairs_noalloc(ctypes.c_void_p(stream.cuda_stream), n, bits,
                                         ctypes.c_void_p(got_k.data_ptr()), ctypes.c_void_p(got_v.data_ptr()))
        assert rc == 0
        assert lib.fs4d_sort_pairs_noalloc_status(ctypes.c_void_p(stream.cuda_stream),
                                                  ctypes.c_void_p(status.data_ptr())) == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(got_k, ref_k)
        assert torch.equal(got_v, ref_v)
        order = np.argsort(keys, kind="stable")
        assert np.array_equal(got_v.cpu().numpy().view(np.uint32), vals[order])
    ctx.close()


def test_noalloc_sort_rejects_sizes_above_its_limit():
    lib = fs4d.library()
    too_many = (1 << 20) + 1  # FS4D_NOALLOC_MAX_PAIRS + 1
    rc = lib.fs4d_sort_pairs_noalloc(None, too_many, 32, ctypes.c_void_p(16), ctypes.c_void_p(16))
    assert rc == CAPACITY  # rejected before any launch: the dummy pointers are never touched
