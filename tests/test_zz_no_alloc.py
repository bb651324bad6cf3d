"""The no-allocation overlap count, called through the C ABI.

hpmc_count_overlaps_noalloc is for callers that cannot allocate device memory
where they need an overlap check (inside a custom memory pool or a callback
that must not touch the allocator, while a tool records work, or in an
embedder that owns all device memory).  It takes the caller's device arrays
and keeps its cell list in a fixed array of the library.  This test checks,
on two calls in a row, that it counts the same pairs as an O(N^2) count with
the oracle's overlap test and as the allocating entry point
hpmc_check_overlaps (integer counts: exact equality), with pairs planted
across the periodic x and y boundaries and the corner, and that sizes beyond
its fixed limit are refused.  The file is named so that pytest runs it after
every other test.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs
from tests.paircount import oracle_pair_count, plant_wrap_pairs

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


def test_noalloc_matches_the_oracle_pair_count_on_two_calls():
    s = inputs.pentagon_system(3000, 0.55, seed=21)
    ref = orc.OracleSystem(2, s.L, s.verts)
    # call 1: a valid configuration after some sweeps (no overlaps)
    b = hpmc.from_system(s)
    b.sweep(30)
    pos, ori, _ = b.get_state()
    b.close()
    assert oracle_pair_count(ref, pos, ori) == 0
    assert _allocating_count(s, pos, ori) == 0
    assert _noalloc_count(s, pos, ori) == 0
    # call 2: pairs planted across the x wrap, the y wrap and the corner; the
    # fixed scratch still holds call 1's cell list
    pos2 = plant_wrap_pairs(pos, s.L, seed=1)
    pos2[41] = pos2[40]                     # and two coincident centres
    want2 = oracle_pair_count(ref, pos2, ori)
    assert want2 >= 3
    assert _allocating_count(s, pos2, ori) == want2
    assert _noalloc_count(s, pos2, ori) == want2


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
    # 600 x 600 cells > 65536; and a box so large that its cell count does
    # not fit an int (refused before any conversion)
    for side in (600.0, 1e12):
        big = np.array([side, side])
        rc = f(big.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
               verts.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 5, 10,
               dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), None)
        assert rc == -9
