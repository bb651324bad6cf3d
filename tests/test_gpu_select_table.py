"""The latency-regime kernels (8 or more lanes per cell) take every select's
pick and move deltas from a table that a separate kernel fills for each
sweep, alongside the cell-list rebuild.  These cases change what that table
must hold while a run goes on -- the number of selects per cell, the cell
grid under volume moves, replicas with different select counts -- and check
the trajectories against the oracle bit for bit."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs

pytestmark = pytest.mark.gpu

hpmc = pytest.importorskip("paper_1509_04692_gb300.hpmc")
F64, F32 = 0, 1


def _oracle(s):
    o = orc.OracleSystem(s.dim, s.L, s.verts, w_min=s.w_min)
    o.set_moves(s.d, s.a, s.nselect, s.seed)
    return o


def _same(p, q, rp, rq):
    bad = np.nonzero(np.any(p != rp, axis=1) | np.any(q != rq, axis=1))[0]
    assert bad.size == 0, f"{bad.size} particles differ, first {bad[:5]}"


@pytest.mark.parametrize("lanes", [8, 32])
@pytest.mark.parametrize("mode", [F64, F32])
def test_nselect_grows_mid_run(lanes, mode):
    # 4 selects, then 11, then 37 (more selects than lanes: several chunks)
    s = inputs.pentagon_system(900, 0.55, 31, d=0.12, a=0.2)
    o = _oracle(s)
    p, q = s.pos.copy(), s.orient.copy()
    b = hpmc.from_system(s)
    b.set_precision(mode)
    b.set_group_size(lanes, 2)
    sw = 0
    for nsel, n in [(4, 6), (11, 4), (37, 3)]:
        o.set_moves(s.d, s.a, nsel, s.seed)
        b.set_moves(s.d, s.a, nsel)
        o.sweep(p, q, sw, n)
        b.sweep(n, graph=True)
        sw += n
    c = b.counters()
    gp, gq, gsw = b.get_state()
    b.close()
    assert gsw == sw
    _same(gp, gq, p, q)
    assert c["moves"] > 0


@pytest.mark.parametrize("lanes", [16, 32])
def test_volume_moves_change_the_grid_under_the_table(lanes):
    # w_min just below L / 24: the first compression drops the grid to 22
    # cells, expansions bring it back (the table is regrown, never shrunk)
    s = inputs.disk_system(512, 0.60, 21, d=0.12, w_min=1.0782)
    o = _oracle(s)
    p, q = s.pos.copy(), s.orient.copy()
    b = hpmc.from_system(s)
    b.set_group_size(lanes, 2)
    acc_o, acc_g, nc_seen, sw, m = [], [], set(), 0, 0
    for _ in range(20):
        o.sweep(p, q, sw, 2)
        b.sweep(2, graph=True)
        sw += 2
        for _ in range(4):
            acc_o.append(o.box_move(p, q, 30.0, 0.4, m))
            acc_g.append(int(b.box_move(30.0, 0.4)))
            nc_seen.add(int(o.geometry()["nc"][0]))
            m += 1
    gp, gq, _ = b.get_state()
    box = b.box()
    b.close()
    assert acc_g == acc_o and 0 < sum(acc_o) < len(acc_o)
    assert len(nc_seen) > 1
    assert np.array_equal(box, o.box)
    _same(gp, gq, p, q)


def test_replicas_with_different_select_counts_2d():
    spec = [(300, 0.45, 42, 1), (777, 0.62, 43, 4), (256, 0.70, 44, 9), (500, 0.40, 45, 33)]
    systems = [inputs.pentagon_system(N, phi, seed, nselect=ns) for N, phi, seed, ns in spec]
    b = hpmc.from_systems(systems)
    b.set_group_size(16, 4)
    b.sweep(9, graph=True)
    b.sweep(3)                                      # direct launches too
    for r, s in enumerate(systems):
        o = _oracle(s)
        p, q = s.pos.copy(), s.orient.copy()
        rc = o.sweep(p, q, 0, 12)
        c = b.counters(r)
        assert (c["accept"], c["reject_overlap"], c["reject_boundary"]) == tuple(int(x) for x in rc[:3])
        gp, gq, sw = b.get_state(r)
        assert sw == 12
        _same(gp, gq, p, q)
    b.close()


@pytest.mark.parametrize("mode", [F64, F32])
def test_replicas_with_different_select_counts_3d(mode):
    spec = [(216, 0.40, 21, 2), (343, 0.45, 22, 4), (512, 0.30, 23, 10)]
    systems = [inputs.cube_system(N, phi, seed, d=0.1, a=0.1, nselect=ns) for N, phi, seed, ns in spec]
    b = hpmc.from_systems(systems)
    b.set_precision(mode)
    b.set_group_size(8, 2)
    b.sweep(8, graph=True)
    for r, s in enumerate(systems):
        o = _oracle(s)
        p, q = s.pos.copy(), s.orient.copy()
        rc = o.sweep(p, q, 0, 8)
        c = b.counters(r)
        assert (c["accept"], c["reject_overlap"], c["reject_boundary"]) == tuple(int(x) for x in rc[:3])
        gp, gq, _ = b.get_state(r)
        _same(gp, gq, p, q)
    b.close()


def test_switching_regimes_keeps_the_trajectory():
    # throughput regime (no table), latency regime (table), and back
    s = inputs.pentagon_system(1024, 0.58, 12, d=0.15, a=0.15)
    o = _oracle(s)
    p, q = s.pos.copy(), s.orient.copy()
    o.sweep(p, q, 0, 12)
    b = hpmc.from_system(s)
    for lanes, n in [(2, 4), (32, 4), (1, 2), (8, 2)]:
        b.set_group_size(lanes, 4 if lanes < 8 else 2)
        b.sweep(n, graph=n >= 2)
    gp, gq, sw = b.get_state()
    b.close()
    assert sw == 12
    _same(gp, gq, p, q)


@pytest.mark.parametrize("lanes", [4, 16])
def test_cell_width_floor_set_after_creation(lanes):
    # created on the paper's minimal grid, then switched to a coarser floor:
    # the trajectory is the oracle's on the coarser grid from then on
    s = inputs.pentagon_system(1200, 0.5, 41, d=0.12, a=0.15)
    b = hpmc.from_system(s)
    b.set_group_size(lanes, 2 if lanes >= 8 else 4)
    nc0 = b.geometry()["nc"][0]
    b.set_cell_width_min(1.7)
    g = b.geometry()
    o = orc.OracleSystem(2, s.L, s.verts, w_min=1.7)
    assert g["nc"][0] < nc0 and g["nc"][0] == o.geometry()["nc"][0]
    o.set_moves(s.d, s.a, s.nselect, s.seed)
    p, q = s.pos.copy(), s.orient.copy()
    rc = o.sweep(p, q, 0, 12)
    b.sweep(12, graph=True)
    c = b.counters()
    assert (c["accept"], c["reject_overlap"], c["reject_boundary"]) == tuple(int(x) for x in rc[:3])
    gp, gq, _ = b.get_state()
    _same(gp, gq, p, q)
    # a floor leaving fewer than 4 cells is refused and the grid kept
    with pytest.raises(hpmc.HPMCError) as e:
        b.set_cell_width_min(s.L[0] / 3.0)
    assert e.value.code == -2
    assert b.geometry()["nc"][0] == g["nc"][0]
    b.close()
