"""The no-allocation overlap count, called through the C ABI.

hpmc_count_overlaps_noalloc is for callers that cannot allocate device memory
where they need an overlap check (inside a custom memory pool or a callback
that must not touch the allocator, while a tool records work, or in an
embedder that owns all device memory).  It takes the caller's device arrays
and keeps its cell list in a fixed array of the library.  This test checks,
on two calls in a row, that it counts the same pairs as the allocating entry
point hpmc_check_overlaps (integer counts: exact equality), and that sizes
beyond its fixed limit are refused.  The file is named so that pytest runs
it after every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1509_04692_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
hpmc = pytest.importorskip("paper_1509_04692_gb300.hpmc")


def _entry():
    lib = hpmc.lib()
    f = lib.hpmc_count_overlaps_noalloc
    dp = ctypes.POINTER(ctypes.c_double)
    f.argtypes = [dp, dp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def _noalloc_count(s, pos, ori):
    f = _entry()
    box = np.ascontiguousarray(s.L, dtype=np.float64)
    verts = np.ascontiguousarray(s.verts, dtype=np.float64)
    p = torch.from_numpy(np.ascontiguousarray(pos)).cuda()
    o = torch.from_numpy(np.ascontiguousarray(ori)).cuda()
    out = torch.full((1,), 12345, dtype=torch.int64, device="cuda")   # must be overwritten
    stream = torch.cuda.current_stream()
    rc = f(box.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
           verts.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), verts.shape[0], pos.shape[0],
           p.data_ptr(), o.data_ptr(), out.data_ptr(), stream.cuda_stream)
    assert rc == 0, hpmc.lib().hpmc_strerror(rc)
    stream.synchronize()
    return int(out.item())


def _allocating_count(s, pos, ori):
    b = hpmc.Batch.single(2, s.verts, s.L, pos, ori, s.seed)
    n = b.check_overlaps()
    b.close()
    return n


def test_noalloc_matches_check_overlaps_on_two_calls():
    s = inputs.pentagon_system(3000, 0.55, seed=21)
    # call 1: a valid configuration after some sweeps (no overlaps)
    b = hpmc.from_system(s)
    b.sweep(30)
    pos, ori, _ = b.get_state()
    b.close()
    want1 = _allocating_count(s, pos, ori)
    got1 = _noalloc_count(s, pos, ori)
    assert want1 == 0 and got1 == want1
    # call 2: plant overlaps; the fixed scratch still holds call 1's cell list
    pos2 = pos.copy()
    pos2[1] = pos2[0]
    pos2[5] = np.mod(pos2[4] + np.array([0.25, 0.1]), s.L)
    pos2[9] = np.mod(pos2[8] + np.array([0.0, 0.3]), s.L)
    want2 = _allocating_count(s, pos2, ori)
    got2 = _noalloc_count(s, pos2, ori)
    assert want2 >= 3 and got2 == want2


def test_noalloc_refuses_sizes_beyond_its_scratch():
    f = _entry()
    s = inputs.pentagon_system(1000, 0.5, seed=3)
    box = np.ascontiguousarray(s.L, dtype=np.float64)
    verts = np.ascontiguousarray(s.verts, dtype=np.float64)
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = f(box.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
           verts.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 5, 65537,
           dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), None)
    assert rc == -9
    big = np.array([600.0, 600.0])          # 600 x 600 cells > 65536
    rc = f(big.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
           verts.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 5, 10,
           dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), None)
    assert rc == -9
