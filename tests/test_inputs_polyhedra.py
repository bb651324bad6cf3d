"""The polyhedron input generators give overlap-free starts (checked with the
oracle's overlap test on every pair closer than the circumdiameter) and the
shapes they claim."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs

spatial = pytest.importorskip("scipy.spatial")


def _overlapping_pairs(s):
    L = float(s.L[0])
    R = inputs.circumradius(s.verts)
    tree = spatial.cKDTree(np.mod(s.pos, L), boxsize=L)
    pairs = np.array(sorted(tree.query_pairs(2.0 * R)))
    D = s.pos[pairs[:, 1]] - s.pos[pairs[:, 0]]
    D -= L * np.round(D / L)
    o = orc.OracleSystem(3, s.L, s.verts)
    ov = o.overlap(D, s.orient[pairs[:, 0]], s.orient[pairs[:, 1]])
    return int(ov.sum()), len(pairs)


def test_dodecahedron_shape():
    v = inputs.dodecahedron(1.0)
    assert v.shape == (20, 3)
    hull = spatial.ConvexHull(v)
    assert abs(hull.volume - 1.0) < 1e-12
    r = np.linalg.norm(v, axis=1)
    assert np.allclose(r, r[0])                          # all on the circumsphere
    # 30 equal edges: the shortest vertex distances
    dist = np.linalg.norm(v[:, None] - v[None], axis=2)
    e = np.sort(dist[np.triu_indices(20, 1)])
    assert np.allclose(e[:30], e[0]) and e[30] > 1.5 * e[0]


def test_dodecahedra_fcc_start_is_overlap_free():
    s = inputs.dodecahedron_system(n=20, phi=0.50, seed=42)
    assert s.N == 32000
    assert abs(s.N * 1.0 / s.L[0] ** 3 - 0.50) < 1e-12
    n_ov, n_pairs = _overlapping_pairs(s)
    assert n_pairs > 12 * s.N // 2 - 1                   # every FCC neighbour is a candidate
    assert n_ov == 0


def test_cube_start_is_overlap_free():
    s = inputs.cubes32768(42)
    n_ov, n_pairs = _overlapping_pairs(s)
    assert n_pairs > 0 and n_ov == 0
