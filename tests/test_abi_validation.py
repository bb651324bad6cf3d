"""Host-side argument checks of the C ABI, which run before any CUDA call
(so they are exercised here without a GPU), and the loud failure of a valid
call on a machine without a usable GPU (no CPU fallback)."""
import ctypes

import numpy as np
import pytest

from paper_1509_04692_gb300 import hpmc, inputs

INVALID, BOX_SMALL, CUDA = -1, -2, -5


def _create(dim=2, verts=None, N=4, L=10.0, pos=None, orient=None, d=0.1, a=0.1, nselect=4, w_min=0.0):
    rng = np.random.default_rng(0)
    if verts is None:
        verts = inputs.regular_polygon(5, 0.5) if dim == 2 else inputs.cube(1.0)
    if pos is None:
        pos = rng.uniform(0.0, L, (N, dim))
    if orient is None:
        orient = np.tile([1.0, 0.0] if dim == 2 else [1.0, 0.0, 0.0, 0.0], (len(pos), 1))
    return hpmc.Batch.single(dim, verts, L, pos, orient, 42, d=d, a=a, nselect=nselect, w_min=w_min)


def _code(**kw):
    with pytest.raises(hpmc.HPMCError) as e:
        _create(**kw)
    return e.value.code


def test_shapes_are_checked():
    assert _code(dim=2, verts=np.array([[0.0, 0.0], [1.0, 0.0]])) == INVALID          # fewer than 3
    assert _code(dim=2, verts=inputs.regular_polygon(17, 0.5)) == INVALID              # more than 16
    assert _code(dim=3, verts=np.zeros((3, 3)) + [[1, 0, 0], [0, 1, 0], [0, 0, 1]]) == INVALID
    bad = inputs.regular_polygon(5, 0.5).copy()
    bad[2, 0] = np.nan
    assert _code(dim=2, verts=bad) == INVALID
    assert _code(dim=2, verts=np.array(-0.5)) == INVALID                             # disk radius


def test_moves_and_cell_floor_are_checked():
    assert _code(d=-0.1) == INVALID
    assert _code(a=3.2) == INVALID
    assert _code(nselect=0) == INVALID
    assert _code(nselect=70000) == INVALID
    assert _code(w_min=-1.0) == INVALID
    assert _code(w_min=float("nan")) == INVALID


def test_configurations_and_boxes_are_checked():
    assert _code(pos=np.array([[1.0, 1.0], [10.5, 2.0]])) == INVALID                # outside [0, L)
    assert _code(pos=np.array([[1.0, 1.0], [np.nan, 2.0]])) == INVALID
    assert _code(orient=np.array([[1.0, 0.0], [0.8, 0.0]]), pos=np.array([[1.0, 1.0], [3.0, 2.0]])) == INVALID
    assert _code(L=3.5) == BOX_SMALL                                               # 3 cells of 2R = 1
    assert _code(L=10.0, w_min=3.0) == BOX_SMALL                                   # 3 cells of >= 3
    assert _code(dim=3, L=3.0) == BOX_SMALL


def test_grid_limits_are_checked_before_any_allocation():
    # cell and particle indices are 32-bit: at most 65536 cells per axis and
    # 2^31 - 1 cells per replica and per batch, counted in 64 bits
    assert _code(L=70000.0) == INVALID                                            # 70000 cells per axis
    assert _code(L=65536.5, w_min=1.0) == INVALID                                 # 65536^2 = 2^32 cells
    assert _code(L=46342.5, w_min=1.0) == INVALID                                 # 46342^2 > 2^31 - 1
    assert _code(dim=3, L=4000.0) == INVALID                                      # 2308^3 cubes' cells
    assert _code(dim=3, L=3000.0, w_min=2.0) == INVALID                           # 1500^3
    rng = np.random.default_rng(1)
    reps = [dict(box=40000.0, pos=rng.uniform(0, 40000.0, (4, 2)), orient=np.tile([1.0, 0.0], (4, 1)),
                 seed=42 + r) for r in range(2)]                                  # 2 x 1.6e9 cells
    with pytest.raises(hpmc.HPMCError) as e:
        hpmc.Batch(2, inputs.regular_polygon(5, 0.5), reps, w_min=1.0)
    assert e.value.code == INVALID


def test_null_handles_and_pointers():
    lib = hpmc.lib()
    null = ctypes.c_void_p()
    assert lib.hpmc_sweep(null, 1, None) == INVALID
    assert lib.hpmc_sweep_graph(null, 2, None) == INVALID
    assert lib.hpmc_set_moves(null, -1, 0.1, 0.1, 4) == INVALID
    assert lib.hpmc_set_precision(null, 1) == INVALID
    assert lib.hpmc_set_group_size(null, 8, 2) == INVALID
    assert lib.hpmc_set_cell_width_min(null, 1.0) == INVALID
    assert lib.hpmc_destroy(null) == INVALID
    assert lib.hpmc_batch_create(2, None, 0, 0.0, 0, None, None) == INVALID
    o64 = np.zeros(1, dtype=np.int32)
    ip = ctypes.POINTER(ctypes.c_int32)
    assert lib.hpmc_pair_test(2, None, 5, 1, None, None, None, o64.ctypes.data_as(ip),
                              o64.ctypes.data_as(ip)) == INVALID
    assert lib.hpmc_pair_test_warp3d(None, 8, 1, None, None, None, o64.ctypes.data_as(ip),
                                     o64.ctypes.data_as(ip)) == INVALID


def test_a_valid_call_fails_loudly_without_a_gpu():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(hpmc.HPMCError) as e:
        _create(N=4)
    assert e.value.code == CUDA


def test_binding_checks_array_sizes_before_the_library_reads_them():
    # a handle-less batch of two replicas (3 and 5 disks): the checks raise
    # before any call into the library, which would read or write exactly
    # N * dim (N * 2 | 4) doubles through the pointers
    b = object.__new__(hpmc.Batch)
    b.h, b.dim, b.qd, b.N, b.R = None, 2, 2, [3, 5], 2
    with pytest.raises(ValueError):
        b.set_state(np.zeros((2, 2)), np.zeros((3, 2)), r=0)          # too few positions
    with pytest.raises(ValueError):
        b.set_state(np.zeros((5, 2)), np.zeros((3, 2)), r=0)          # replica 0 holds 3
    with pytest.raises(ValueError):
        b.set_state(np.zeros((5, 2)), np.zeros((5, 4)), r=1)          # 2D orientations: 2 values
    p, o = np.zeros((8, 2)), np.zeros((8, 2))
    with pytest.raises(ValueError):
        b.run_host(p[:7], o, 1, np.zeros((8, 2)), np.zeros((8, 2)))    # inputs of every replica
    with pytest.raises(ValueError):
        b.run_host(p, o, 1, np.zeros((8, 2), np.float32), np.zeros((8, 2)))
    with pytest.raises(ValueError):
        b.run_host(p, o, 1, np.zeros((2, 8)).T, np.zeros((8, 2)))      # not C-contiguous
    ro = np.zeros((8, 2))
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        b.run_host(p, o, 1, np.zeros((8, 2)), ro)
    with pytest.raises(ValueError):
        b.sdf(0.05, 10, hist=np.zeros(9, dtype=np.uint64))
    with pytest.raises(ValueError):
        b.sdf(0.05, 10, hist=np.zeros(10, dtype=np.int64))


def test_binding_checks_pair_and_replica_arrays():
    v = inputs.regular_polygon(5, 0.5)
    with pytest.raises(ValueError):
        hpmc.pair_test(2, v, np.zeros((4, 2)), np.zeros((3, 2)), np.zeros((4, 2)))
    with pytest.raises(ValueError):
        hpmc.pair_test_warp3d(inputs.cube(1.0), np.zeros((4, 3)), np.zeros((4, 4)), np.zeros((4, 2)))
    with pytest.raises(ValueError):                                   # 4 positions, 3 orientations
        _create(N=4, orient=np.tile([1.0, 0.0], (3, 1)))
