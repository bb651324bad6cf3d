"""The seeded synthetic workloads follow their stated recipes: sizes,
densities, move sizes and ranges, overlap-free starts, unit orientations,
and determinism under a seed (the same arrays every time, other arrays for
another seed).  The inputs module holds no method arithmetic; these checks
use numpy, the brute-force pair test and the oracle's geometry rule."""
import numpy as np

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs
from tests import bruteforce as bf

A_P = inputs.polygon_area(inputs.regular_polygon(5, 0.5))


def test_pentagon_systems_density_range_and_start():
    for N, phi in [(400, 0.45), (600, 0.62), (500, 0.68)]:
        s = inputs.pentagon_system(N, phi, 7)
        assert s.pos.shape == (N, 2) and s.orient.shape == (N, 2)
        assert abs(N * A_P / (s.L[0] * s.L[1]) - phi) < 1e-12
        assert np.all(s.pos >= 0.0) and np.all(s.pos < s.L)
        assert np.allclose(np.hypot(s.orient[:, 0], s.orient[:, 1]), 1.0, atol=1e-12)
        assert bf.pairwise_overlaps_2d(s.verts, s.L[0], s.pos, s.orient) == []
    a, b, c = (inputs.pentagon_system(300, 0.5, sd) for sd in (9, 9, 10))
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.orient, b.orient)
    assert not np.array_equal(a.orient, c.orient)


def test_benchmark_workload_parameters():
    f = inputs.fluid4096(42)
    assert f.N == 4096 and f.phi == 0.60 and f.d == f.a == 0.165 and f.nselect == 4
    assert abs(4096 * A_P / f.L[0] ** 2 - 0.60) < 1e-12
    g = orc.OracleSystem(2, f.L, f.verts).geometry()
    assert tuple(g["nc"]) == (62, 62)                        # 961 active cells a set
    # the 2^24 system: geometry from its box alone (no 16.8 M-particle arrays)
    L = inputs.box_length(inputs.LARGE2D_N, A_P, 0.60, 2)
    assert abs(L - 4076.876) < 1e-3
    g = orc.OracleSystem(2, [L, L], f.verts, w_min=inputs.LARGE2D_W_MIN).geometry()
    assert tuple(g["nc"]) == (2048, 2048)


def test_replica_batch_recipe():
    params = inputs.replica_params(512)
    Ns = np.array([p[0] for p in params])
    phis = np.array([p[1] for p in params])
    assert Ns.min() >= 256 and Ns.max() <= 8192 and phis.min() >= 0.40 and phis.max() <= 0.70
    assert [p[2] for p in params] == [42 + r for r in range(512)]
    assert params == inputs.replica_params(512)              # seeded
    assert Ns.std() > 1500 and phis.std() > 0.06              # spread over the ranges
    # the batch as built (the densities of a shorter batch differ: all N are
    # drawn before all densities); a few small members: overlap-free starts
    systems = inputs.replica_systems(512)
    assert sum(x.N for x in systems) == int(Ns.sum())
    for r in range(512):
        assert systems[r].N == Ns[r] and abs(systems[r].N * A_P / systems[r].L[0] ** 2 - phis[r]) < 1e-12
    small = [r for r, (N, phi, _) in enumerate(params) if N < 700][:3]
    for r in small:
        s = systems[r]
        assert abs(s.N * A_P / s.L[0] ** 2 - params[r][1]) < 1e-12
        assert bf.pairwise_overlaps_2d(s.verts, s.L[0], s.pos, s.orient) == []


def test_cube_and_disk_starts():
    c = inputs.cube_system(512, 0.45, 3)
    assert abs(c.N / c.L[0] ** 3 - 0.45) < 1e-12
    assert np.allclose(c.orient, [1.0, 0.0, 0.0, 0.0])       # aligned start
    d = c.pos[:, None, :] - c.pos[None, :, :]
    d -= c.L[0] * np.round(d / c.L[0])
    sep = np.max(np.abs(d), axis=2) + np.eye(c.N) * 10
    assert sep.min() >= 1.0                                   # aligned unit cubes apart
    k = inputs.cubes32768(42)
    assert k.N == 32768 and k.d == k.a == 0.0817
    s = inputs.disk_system(900, 0.65, 4)
    d = s.pos[:, None, :] - s.pos[None, :, :]
    d -= s.L[0] * np.round(d / s.L[0])
    r = np.hypot(d[..., 0], d[..., 1]) + np.eye(s.N) * 10
    assert r.min() >= 1.0 and abs(s.N * np.pi / 4 / s.L[0] ** 2 - 0.65) < 1e-12


def test_cube_replica_batch_recipe():
    params = inputs.cube_replica_params()
    Ns = np.array([p[0] for p in params])
    phis = np.array([p[1] for p in params])
    assert len(params) == 32 and Ns.min() >= 2048 and Ns.max() <= 16384
    assert phis.min() >= 0.40 and phis.max() <= 0.55
    assert [p[2] for p in params] == [1000 + r for r in range(32)]
    assert params == inputs.cube_replica_params()            # seeded
    systems = inputs.cube_replica_systems()
    for s, (N, phi, _) in zip(systems, params):
        assert s.N == N and abs(N / s.L[0] ** 3 - phi) < 1e-12 and s.notes["spacing"] >= 1.0
        assert s.d == s.a == inputs.CUBES32768_D and s.nselect == 4
        assert np.allclose(s.orient, [1.0, 0.0, 0.0, 0.0])   # aligned cubes, spacing >= edge
        assert tuple(orc.OracleSystem(3, s.L, s.verts).geometry()["nc"]) >= (4, 4, 4)


def test_tiny_lattices_are_overlap_free():
    # a handful of sites in a small box: the lattice search must count the
    # distance between rows two apart (same column) too
    for N, phi, seed in [(3, 0.05, 2), (7, 0.1, 1), (12, 0.30, 3), (30, 0.30, 3), (60, 0.5, 4)]:
        s = inputs.pentagon_system(N, phi, seed)
        assert s.notes["site_distance"] >= 1.0
        assert bf.pairwise_overlaps_2d(s.verts, s.L[0], s.pos, s.orient) == []
