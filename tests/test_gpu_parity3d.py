"""GPU parity of the 3D checkerboard sweep (convex polyhedra, GJK) against
the CPU oracle: positions, quaternions (FP64) and accept / reject counters
bit for bit, in both precision modes and for every lanes-per-cell choice."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs

pytestmark = pytest.mark.gpu

hpmc = pytest.importorskip("paper_1509_04692_gb300.hpmc")
F64, F32 = 0, 1


def oracle_run(s, n, sweep0=0):
    ref = orc.OracleSystem(3, s.L, s.verts, w_min=s.w_min)
    ref.set_moves(s.d, s.a, s.nselect, s.seed)
    pos, ori = s.pos.copy(), s.orient.copy()
    c = ref.sweep(pos, ori, sweep0, n)
    return pos, ori, [int(x) for x in c[:3]], int(c[3])


def gpu_run(s, n, mode=F32, lanes=4, warps=2, graph=False):
    b = hpmc.from_system(s)
    b.set_precision(mode)
    b.set_group_size(lanes, warps)
    b.sweep(n, graph=graph)
    c = b.counters()
    p, o, sw = b.get_state()
    ov = b.check_overlaps()
    b.close()
    assert sw == n
    return p, o, [c["accept"], c["reject_overlap"], c["reject_boundary"]], c, ov


def assert_same(got, ref):
    pa, oa, ca = got[:3]
    pb, ob, cb = ref[:3]
    assert ca == cb, (ca, cb)
    bad = np.nonzero(np.any(pa != pb, axis=1) | np.any(oa != ob, axis=1))[0]
    assert bad.size == 0, f"{bad.size} particles differ, first {bad[:5]}"


def cubes(N, phi=0.5, seed=7, d=0.1, a=0.1):
    return inputs.cube_system(N, phi, seed=seed, d=d, a=a)


@pytest.mark.parametrize("mode", [F64, F32])
def test_cubes_512_bit_exact(mode):
    s = cubes(512, d=0.15, a=0.3)
    ref = oracle_run(s, 40)
    got = gpu_run(s, 40, mode)
    assert_same(got, ref)
    # (which pairs are evaluated depends on the early-exit order, so only
    # decisions are compared; the GJK cap is never reached here anyway)
    assert got[3]["gjk_cap"] == 0 and ref[3] == 0
    assert got[4] == 0


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
def test_every_group_size_same_trajectory_3d(lanes):
    s = cubes(1000, phi=0.45, seed=9, d=0.12, a=0.25)
    ref = oracle_run(s, 10)
    assert_same(gpu_run(s, 10, F32, lanes=lanes, warps=2), ref)


def test_cubes_32768_phi050_prefix():
    # the 32768-cube system at volume fraction 0.50 (22^3 cells)
    s = cubes(32768, phi=0.50, seed=11, d=0.1, a=0.1)
    ref = oracle_run(s, 8)
    got = gpu_run(s, 8, F32, graph=True)
    assert_same(got, ref)
    assert_same(gpu_run(s, 8, F64), ref)


def test_general_polyhedron_generic_path():
    # an irregular convex polyhedron (not 8 vertices: generic kernel)
    rng = np.random.default_rng(3)
    p = rng.normal(size=(12, 3))
    v = 0.5 * p / np.linalg.norm(p, axis=1)[:, None]
    base = cubes(343, phi=0.25, seed=5)
    s = inputs.System(name="poly12", dim=3, verts=v, L=base.L, pos=base.pos, orient=base.orient,
                      phi=0.0, seed=13, d=0.2, a=0.5)
    ref = oracle_run(s, 15)
    for mode in (F64, F32):
        assert_same(gpu_run(s, 15, mode), ref)


def test_batched_3d_replicas():
    systems = [cubes(N, phi, seed) for N, phi, seed in [(216, 0.40, 21), (512, 0.50, 22), (343, 0.30, 23)]]
    b = hpmc.from_systems(systems)
    b.set_group_size(4, 2)
    b.sweep(12, graph=True)
    for r, s in enumerate(systems):
        p, o, sw = b.get_state(r)
        c = b.counters(r)
        ref = oracle_run(s, 12)
        assert_same((p, o, [c["accept"], c["reject_overlap"], c["reject_boundary"]]), ref)
    b.close()


@pytest.mark.parametrize("mode", [F64, F32])
def test_dodecahedra_32000_phi050(mode):
    # 32000 regular dodecahedra (20 vertices: generic kernel) at volume
    # fraction 0.50 from the aligned FCC start, with the tuned move sizes
    s = inputs.dodecahedra32000(42)
    ref = oracle_run(s, 4)
    got = gpu_run(s, 4, mode, lanes=32, warps=4, graph=True)
    assert_same(got, ref)
    assert got[4] == 0


def test_cubes_32768_tuned_moves():
    # the benchmark's cube system and move sizes, graph-replayed as timed
    s = inputs.cubes32768(42)
    ref = oracle_run(s, 6)
    assert_same(gpu_run(s, 6, F32, lanes=32, warps=4, graph=True), ref)
