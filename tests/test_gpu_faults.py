"""Failure paths made on the host (no GPU fault is ever provoked): every
device allocation of batch creation, of the volume move and of the MSD
tracker is made to fail in turn; each failure returns HPMC_ERR_OOM, leaves
no handle behind, and the library keeps working afterwards (the run then
matches the oracle bit for bit)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs

pytestmark = pytest.mark.gpu

hpmc = pytest.importorskip("paper_1509_04692_gb300.hpmc")
OOM = -4


def test_every_creation_allocation_failure_is_reported():
    s = inputs.pentagon_system(300, 0.5, 51, d=0.1, a=0.2)
    failures = 0
    for n in range(200):
        hpmc.debug_fail_alloc(n)
        try:
            b = hpmc.from_system(s)
        except hpmc.HPMCError as e:
            assert e.code == OOM
            failures += 1
            continue
        b.close()
        break
    hpmc.debug_fail_alloc(-1)
    assert failures > 10                       # creation makes that many allocations
    b = hpmc.from_system(s)
    b.sweep(10)
    o = orc.OracleSystem(2, s.L, s.verts)
    o.set_moves(s.d, s.a, s.nselect, s.seed)
    p, q = s.pos.copy(), s.orient.copy()
    o.sweep(p, q, 0, 10)
    assert np.array_equal(b.get_state()[0], p)
    b.close()


def test_lazy_allocations_fail_cleanly():
    s = inputs.disk_system(400, 0.5, 52, d=0.1)
    b = hpmc.from_system(s)
    hpmc.debug_fail_alloc(0)
    with pytest.raises(hpmc.HPMCError) as e:
        b.msd_reset()
    assert e.value.code == OOM
    hpmc.debug_fail_alloc(0)
    with pytest.raises(hpmc.HPMCError) as e:
        b.box_move(5.0, 0.5)
    assert e.value.code == OOM
    hpmc.debug_fail_alloc(-1)
    b.msd_reset()                                # now allocates and works
    b.sweep(5)
    b.msd_update()
    assert b.msd() > 0.0
    L0 = b.box()
    b.box_move(5.0, 0.5)
    assert b.check_overlaps() == 0 and b.box().shape == L0.shape
    b.close()


def test_failed_grid_growth_keeps_the_old_grid():
    # a finer cell grid needs larger cell arrays; when one of their three
    # allocations fails, the call reports OOM and the old grid stays in force
    # on host and device alike (the run matches the oracle on that grid)
    s = inputs.pentagon_system(700, 0.5, 53, d=0.12, a=0.15, w_min=1.7)
    b = hpmc.from_system(s)
    nc = b.geometry()["nc"][0]
    for n in range(3):
        hpmc.debug_fail_alloc(n)
        with pytest.raises(hpmc.HPMCError) as e:
            b.set_cell_width_min(0.0)
        assert e.value.code == OOM
        assert b.geometry()["nc"][0] == nc
    hpmc.debug_fail_alloc(-1)
    b.sweep(12, graph=True)
    c = b.counters()
    p, q, _ = b.get_state()
    o = orc.OracleSystem(2, s.L, s.verts, w_min=1.7)
    o.set_moves(s.d, s.a, s.nselect, s.seed)
    rp, rq = s.pos.copy(), s.orient.copy()
    rc = o.sweep(rp, rq, 0, 12)
    assert (c["accept"], c["reject_overlap"], c["reject_boundary"]) == tuple(int(x) for x in rc[:3])
    assert np.array_equal(p, rp) and np.array_equal(q, rq)
    b.set_cell_width_min(0.0)                     # and the growth itself works
    assert b.geometry()["nc"][0] > nc
    b.close()


def test_select_table_allocation_failure_is_reported():
    # the latency-regime kernels allocate their select table at the first
    # sweep after the configuration change; a failure there is OOM from the
    # sweep call, and the next sweep allocates and runs normally
    s = inputs.pentagon_system(500, 0.5, 54, d=0.12, a=0.15)
    b = hpmc.from_system(s)
    b.set_group_size(32, 2)
    hpmc.debug_fail_alloc(0)
    with pytest.raises(hpmc.HPMCError) as e:
        b.sweep(3)
    assert e.value.code == OOM
    hpmc.debug_fail_alloc(-1)
    b.sweep(6)
    c = b.counters()
    p, q, sw = b.get_state()
    b.close()
    assert sw == 6
    o = orc.OracleSystem(2, s.L, s.verts)
    o.set_moves(s.d, s.a, s.nselect, s.seed)
    rp, rq = s.pos.copy(), s.orient.copy()
    rc = o.sweep(rp, rq, 0, 6)
    assert (c["accept"], c["reject_overlap"], c["reject_boundary"]) == tuple(int(x) for x in rc[:3])
    assert np.array_equal(p, rp) and np.array_equal(q, rq)
