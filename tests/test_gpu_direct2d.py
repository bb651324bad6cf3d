"""GPU parity of the 2D direct set kernel (lanes_per_cell = 0: one lane per
active cell, neighbours read through L1, unreachable stencil columns and
rows skipped) against the CPU oracle, bit for bit: small and ragged grids,
cells much wider than the circumdiameter (where the skipping acts), many
selects (beyond the select table), disks, replica batches, volume moves that
change the grid, and every block shape; and the same kernel's plain FP64
form on the ragged, wide-cell, disk and batch cases."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs
from tests.test_oracle_sweep import load_rsa_start

pytestmark = pytest.mark.gpu

hpmc = pytest.importorskip("paper_1509_04692_gb300.hpmc")
F64, F32 = 0, 1
DIRECT = 0


def _oracle(s, n, sweep0=0, pos=None, ori=None):
    o = orc.OracleSystem(2, s.L, s.verts if s.verts is not None else None, w_min=s.w_min)
    o.set_moves(s.d, s.a, s.nselect, s.seed)
    p = (s.pos if pos is None else pos).copy()
    q = (s.orient if ori is None else ori).copy()
    c = o.sweep(p, q, sweep0, n)
    return p, q, [int(x) for x in c[:3]]


def _gpu(s, n, warps=4, graph=False, prec=F32):
    b = hpmc.from_system(s)
    b.set_precision(prec)
    b.set_group_size(DIRECT, warps)
    b.sweep(n, graph=graph)
    c = b.counters()
    p, q, sw = b.get_state()
    ov = b.check_overlaps()
    b.close()
    assert sw == n and ov == 0
    return p, q, [c["accept"], c["reject_overlap"], c["reject_boundary"]], c


def _same(got, ref, what=""):
    assert got[2] == ref[2], (what, got[2], ref[2])
    bad = np.nonzero(np.any(got[0] != ref[0], axis=1) | np.any(got[1] != ref[1], axis=1))[0]
    assert bad.size == 0, f"{what}: {bad.size} particles differ, first {bad[:5]}"


def _rsa():
    pos, ori, L = load_rsa_start()
    return inputs.System(name="rsa1024", dim=2, verts=inputs.regular_polygon(5, 0.5), L=np.array([L, L]),
                         pos=pos, orient=ori, phi=0.5, seed=42)


@pytest.mark.parametrize("warps", [1, 2, 4, 8])
def test_direct_rsa1024_every_block_shape(warps):
    s = _rsa()
    _same(_gpu(s, 20, warps=warps), _oracle(s, 20), f"warps {warps}")


def test_direct_block_shape_limit():
    s = _rsa()
    b = hpmc.from_system(s)
    with pytest.raises(hpmc.HPMCError):
        b.set_group_size(DIRECT, 16)
    b.close()


def test_direct_fluid4096_graph():
    s = inputs.fluid4096(42)
    got = _gpu(s, 300, graph=True)
    _same(got, _oracle(s, 300))
    assert got[3]["fp64_rechecks"] < 1e-3 * got[3]["overlap_checks"] + 50


@pytest.mark.parametrize("N, w_min", [(65536, 1.99), (40000, 2.6), (20000, 3.3)])
def test_direct_wide_cells_skip_unreachable_layers(N, w_min):
    # cells from twice to more than three times the circumdiameter: most
    # trials reach only some of the stencil's columns and rows
    s = inputs.large2d(42, N=N)
    s.w_min = w_min
    got = _gpu(s, 60, graph=True)
    _same(got, _oracle(s, 60), f"N {N} w_min {w_min}")


@pytest.mark.parametrize("case", ["small_box", "dense_aligned", "dilute", "heptagon", "triangle", "odd_N"])
def test_direct_edge_cases(case):
    if case == "small_box":        # 4 x 4 cells, wrap on every side
        s = inputs.pentagon_system(12, 0.30, seed=3, d=0.3, a=0.5)
    elif case == "dense_aligned":
        s = inputs.pentagon_system(2000, 0.70, seed=4, d=0.05, a=0.05)
    elif case == "dilute":         # mostly empty cells
        s = inputs.pentagon_system(300, 0.02, seed=5, d=0.4, a=1.0)
    elif case in ("heptagon", "triangle"):
        v = inputs.regular_polygon(7 if case == "heptagon" else 3, 0.5)
        base = inputs.pentagon_system(900, 0.35, seed=8)
        s = inputs.System(name=case, dim=2, verts=v, L=base.L, pos=base.pos, orient=base.orient, phi=0.0, seed=9)
    else:                          # ragged rows, 3 selects
        s = inputs.pentagon_system(1237, 0.45, seed=10, nselect=3)
    _same(_gpu(s, 30), _oracle(s, 30), case)


def test_direct_more_selects_than_the_table():
    # the table holds up to 8 selects of a cell; later ones are computed in
    # the kernel
    s = inputs.pentagon_system(900, 0.55, 31, d=0.12, a=0.2)
    o = orc.OracleSystem(2, s.L, s.verts)
    p, q = s.pos.copy(), s.orient.copy()
    b = hpmc.from_system(s)
    b.set_group_size(DIRECT, 4)
    sw = 0
    for nsel, n in [(4, 6), (11, 4), (37, 3), (2, 5)]:
        o.set_moves(s.d, s.a, nsel, s.seed)
        b.set_moves(s.d, s.a, nsel)
        o.sweep(p, q, sw, n)
        b.sweep(n, graph=True)
        sw += n
    gp, gq, gsw = b.get_state()
    b.close()
    assert gsw == sw
    assert np.array_equal(gp, p) and np.array_equal(gq, q)


def test_direct_disks():
    s = inputs.disk_system(1024, 0.60, 5, d=0.12, w_min=1.06)
    o = orc.OracleSystem(2, s.L, 0.5, w_min=s.w_min)
    o.set_moves(s.d, s.a, s.nselect, s.seed)
    p, q = s.pos.copy(), s.orient.copy()
    rc = o.sweep(p, q, 0, 30)
    b = hpmc.from_system(s)
    b.set_group_size(DIRECT, 2)
    b.sweep(30, graph=True)
    c = b.counters()
    gp, gq, _ = b.get_state()
    b.close()
    assert [c["accept"], c["reject_overlap"], c["reject_boundary"]] == [int(x) for x in rc[:3]]
    assert np.array_equal(gp, p) and np.array_equal(gq, q)


def test_direct_replica_batch():
    systems = [inputs.pentagon_system(N, phi, seed, gen_seed=seed)
               for N, phi, seed in [(300, 0.45, 42), (777, 0.62, 43), (256, 0.70, 44), (5000, 0.40, 45)]]
    b = hpmc.from_systems(systems)
    b.set_group_size(DIRECT, 4)
    b.sweep(25, graph=True)
    for r, s in enumerate(systems):
        p, q, sw = b.get_state(r)
        c = b.counters(r)
        ref = _oracle(s, 25)
        assert sw == 25
        _same((p, q, [c["accept"], c["reject_overlap"], c["reject_boundary"]]), ref, f"replica {r}")
    b.close()


def test_direct_volume_moves_change_the_grid():
    s = inputs.disk_system(512, 0.60, 21, d=0.12, w_min=1.0782)
    o = orc.OracleSystem(2, s.L, 0.5, w_min=s.w_min)
    o.set_moves(s.d, s.a, s.nselect, s.seed)
    p, q = s.pos.copy(), s.orient.copy()
    b = hpmc.from_system(s)
    b.set_group_size(DIRECT, 2)
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
    b.close()
    assert acc_g == acc_o and 0 < sum(acc_o) < len(acc_o) and len(nc_seen) > 1
    assert np.array_equal(gp, p) and np.array_equal(gq, q)


# ---- the plain FP64 form of the direct kernel

@pytest.mark.parametrize("warps", [1, 8])
def test_direct_fp64_rsa1024(warps):
    s = _rsa()
    _same(_gpu(s, 20, warps=warps, prec=F64), _oracle(s, 20), f"FP64 warps {warps}")


@pytest.mark.parametrize("case", ["small_box", "dilute", "heptagon", "odd_N", "wide_cells"])
def test_direct_fp64_cases(case):
    if case == "small_box":
        s = inputs.pentagon_system(12, 0.30, seed=3, d=0.3, a=0.5)
    elif case == "dilute":
        s = inputs.pentagon_system(300, 0.02, seed=5, d=0.4, a=1.0)
    elif case == "heptagon":
        base = inputs.pentagon_system(900, 0.35, seed=8)
        s = inputs.System(name=case, dim=2, verts=inputs.regular_polygon(7, 0.5), L=base.L, pos=base.pos,
                          orient=base.orient, phi=0.0, seed=9)
    elif case == "odd_N":
        s = inputs.pentagon_system(1237, 0.45, seed=10, nselect=3)
    else:
        s = inputs.large2d(42, N=40000)
        s.w_min = 2.6
    got = _gpu(s, 30, graph=True, prec=F64)
    _same(got, _oracle(s, 30), f"FP64 {case}")
    assert got[3]["fp64_rechecks"] == 0


def test_direct_fp64_disks_and_batch():
    s = inputs.disk_system(1024, 0.60, 5, d=0.12, w_min=1.06)
    o = orc.OracleSystem(2, s.L, 0.5, w_min=s.w_min)
    o.set_moves(s.d, s.a, s.nselect, s.seed)
    p, q = s.pos.copy(), s.orient.copy()
    rc = o.sweep(p, q, 0, 30)
    _same(_gpu(s, 30, warps=2, prec=F64), (p, q, [int(x) for x in rc[:3]]), "FP64 disks")
    systems = [inputs.pentagon_system(N, phi, seed, gen_seed=seed)
               for N, phi, seed in [(300, 0.45, 42), (777, 0.62, 43), (5000, 0.40, 45)]]
    b = hpmc.from_systems(systems)
    b.set_precision(F64)
    b.set_group_size(DIRECT, 4)
    b.sweep(25, graph=True)
    for r, sr in enumerate(systems):
        p, q, sw = b.get_state(r)
        c = b.counters(r)
        assert sw == 25
        _same((p, q, [c["accept"], c["reject_overlap"], c["reject_boundary"]]), _oracle(sr, 25), f"FP64 replica {r}")
    b.close()
