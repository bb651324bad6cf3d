"""GPU parity of the 2D checkerboard sweep against the CPU oracle.

The CUDA path (through the C ABI) and the oracle run the same seeded input;
positions, orientations (FP64) and the accept / reject counters must agree
bit for bit, in both precision modes and for every lanes-per-cell choice."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs
from tests.paircount import oracle_pair_count, plant_wrap_pairs
from tests.test_oracle_sweep import load_rsa_start

pytestmark = pytest.mark.gpu

hpmc = pytest.importorskip("paper_1509_04692_gb300.hpmc")
F64, F32 = 0, 1


def oracle_run(s, n, sweep0=0):
    ref = orc.OracleSystem(2, s.L, s.verts, w_min=s.w_min)
    ref.set_moves(s.d, s.a, s.nselect, s.seed)
    pos, ori = s.pos.copy(), s.orient.copy()
    c = ref.sweep(pos, ori, sweep0, n)
    return pos, ori, [int(x) for x in c[:3]]


def gpu_run(s, n, mode=F32, lanes=4, warps=4, graph=False):
    b = hpmc.from_system(s)
    b.set_precision(mode)
    b.set_group_size(lanes, warps)
    b.sweep(n, graph=graph)
    c = b.counters()
    p, o, sw = b.get_state()
    b.close()
    assert sw == n
    return p, o, [c["accept"], c["reject_overlap"], c["reject_boundary"]], c


def rsa_system():
    pos, ori, L = load_rsa_start()
    v = inputs.regular_polygon(5, 0.5)
    return inputs.System(name="rsa1024", dim=2, verts=v, L=np.array([L, L]), pos=pos, orient=ori,
                         phi=0.5, seed=42, d=0.1, a=0.1, nselect=4)


def assert_same(a, b):
    pa, oa, ca = a[:3]
    pb, ob, cb = b[:3]
    assert ca == cb, (ca, cb)
    bad = np.nonzero(np.any(pa != pb, axis=1) | np.any(oa != ob, axis=1))[0]
    assert bad.size == 0, f"{bad.size} particles differ, first {bad[:5]}"


@pytest.mark.parametrize("mode", [F64, F32])
def test_rsa1024_first_sweeps(mode):
    s = rsa_system()
    for n in (1, 3):
        assert_same(gpu_run(s, n, mode), oracle_run(s, n))


@pytest.mark.parametrize("mode", [F64, F32])
def test_rsa1024_1000_sweeps_bit_exact(mode):
    s = rsa_system()
    ref = oracle_run(s, 1000)
    got = gpu_run(s, 1000, mode, graph=True)
    assert_same(got, ref)
    assert got[3]["moves"] == sum(ref[2])


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
def test_every_group_size_same_trajectory(lanes):
    s = rsa_system()
    ref = oracle_run(s, 20)
    assert_same(gpu_run(s, 20, F32, lanes=lanes, warps=2), ref)
    # (kernels with up to 4 lanes per cell take blocks of at most 6 warps)
    assert_same(gpu_run(s, 20, F64, lanes=lanes, warps=8 if lanes >= 8 else 6), ref)
    with pytest.raises(hpmc.HPMCError):
        gpu_run(s, 1, F32, lanes=lanes, warps=16 if lanes >= 8 else 8)


def test_fluid_4096_phi060_prefix():
    s = inputs.pentagon_system(4096, 0.60, seed=42)
    ref = oracle_run(s, 200)
    got = gpu_run(s, 200, F32, graph=True)
    assert_same(got, ref)
    assert_same(gpu_run(s, 200, F64), ref)
    # the filter must rarely need FP64
    assert got[3]["fp64_rechecks"] < 1e-3 * got[3]["overlap_checks"] + 50


@pytest.mark.parametrize("case", ["small_box", "dense_aligned", "dilute", "big_cells", "heptagon",
                                  "triangle", "odd_N"])
def test_edge_cases(case):
    if case == "small_box":        # 4 x 4 cells, wrap on every side
        s = inputs.pentagon_system(12, 0.30, seed=3, d=0.3, a=0.5)
    elif case == "dense_aligned":  # beyond random-orientation lattice reach
        s = inputs.pentagon_system(2000, 0.70, seed=4, d=0.05, a=0.05)
    elif case == "dilute":         # mostly empty cells
        s = inputs.pentagon_system(300, 0.02, seed=5, d=0.4, a=1.0)
    elif case == "big_cells":      # many particles per cell (cell width floor)
        s = inputs.pentagon_system(3000, 0.55, seed=6)
        s.w_min = 3.3
    elif case in ("heptagon", "triangle"):
        nvx = 7 if case == "heptagon" else 3
        v = inputs.regular_polygon(nvx, 0.5)
        base = inputs.pentagon_system(900, 0.35, seed=8)
        s = inputs.System(name=case, dim=2, verts=v, L=base.L, pos=base.pos, orient=base.orient,
                          phi=0.0, seed=9)
    else:                          # N not filling the lattice, ragged rows
        s = inputs.pentagon_system(1237, 0.45, seed=10, nselect=3)
    ref = oracle_run(s, 30)
    for mode in (F64, F32):
        assert_same(gpu_run(s, 30, mode), ref)


def test_checkpoint_resume_and_determinism():
    s = rsa_system()
    b = hpmc.from_system(s)
    b.sweep(7)
    p7, o7, sw = b.get_state()
    assert sw == 7
    b.sweep(5)
    p12, o12, _ = b.get_state()
    b.set_state(p7, o7, 7)
    b.sweep(5)
    q12, r12, sw = b.get_state()
    assert sw == 12
    assert np.array_equal(p12, q12) and np.array_equal(o12, r12)
    b.close()
    # same seed, same bytes; another seed, another trajectory
    a1 = gpu_run(s, 15)
    a2 = gpu_run(s, 15)
    assert np.array_equal(a1[0], a2[0])
    s.seed = 43
    a3 = gpu_run(s, 15)
    assert not np.array_equal(a1[0], a3[0])


def test_overlap_check_counts_pairs():
    s = rsa_system()
    b = hpmc.from_system(s)
    assert b.check_overlaps() == 0
    b.sweep(50)
    assert b.check_overlaps() == 0
    p, o, sw = b.get_state()
    # plant overlapping pairs, across the periodic boundaries too; the count
    # equals the O(N^2) count with the oracle's overlap test
    p = plant_wrap_pairs(p, s.L, seed=2)
    p[41] = p[40]
    b.set_state(p, o, sw)
    want = oracle_pair_count(orc.OracleSystem(2, s.L, s.verts), p, o)
    assert want >= 3
    assert b.check_overlaps() == want
    b.close()


def test_batched_replicas_match_independent_oracle_runs():
    systems = [inputs.pentagon_system(N, phi, seed, gen_seed=seed)
               for N, phi, seed in [(300, 0.45, 42), (777, 0.62, 43), (256, 0.70, 44), (1500, 0.40, 45)]]
    b = hpmc.from_systems(systems)
    b.sweep(25, graph=True)
    for r, s in enumerate(systems):
        p, o, sw = b.get_state(r)
        ref = oracle_run(s, 25)
        c = b.counters(r)
        assert sw == 25
        assert_same((p, o, [c["accept"], c["reject_overlap"], c["reject_boundary"]]), ref)
    b.close()


def test_errors_are_reported_not_trapped():
    s = rsa_system()
    with pytest.raises(hpmc.HPMCError) as e:
        hpmc.Batch.single(2, s.verts, [3.0, 3.0], s.pos[:2] * 0.0, s.orient[:2], 1)
    assert e.value.code == -2
    with pytest.raises(hpmc.HPMCError):
        hpmc.Batch.single(2, s.verts[::-1], s.L, s.pos, s.orient, 1)     # clockwise
    bad = s.pos.copy()
    bad[0, 0] = np.nan
    with pytest.raises(hpmc.HPMCError):
        hpmc.Batch.single(2, s.verts, s.L, bad, s.orient, 1)
    b = hpmc.from_system(s)
    with pytest.raises(hpmc.HPMCError):
        b.set_moves(-1.0, 0.1, 4)
    with pytest.raises(hpmc.HPMCError):
        b.set_group_size(3)
    b.close()
