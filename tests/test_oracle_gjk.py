"""Pins of the oracle's 3D overlap contract (boolean GJK on the Minkowski
difference in A's frame, Eq. 2) against the 15-axis box test and an
independent edge-clipping brute force."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs
from tests import bruteforce as bf


def _rand_quat(rng, n):
    q = rng.normal(size=(n, 4))
    return q / np.linalg.norm(q, axis=1)[:, None]


def _rand_dirs(rng, n):
    u = rng.normal(size=(n, 3))
    return u / np.linalg.norm(u, axis=1)[:, None]


def _sys(v, L=30.0):
    return orc.OracleSystem(3, [L, L, L], v)


def test_gjk_cubes_vs_sat15_random():
    rng = np.random.default_rng(1)
    v = inputs.cube(1.0)
    s = _sys(v)
    n = 40000
    R = np.sqrt(3) / 2
    D = _rand_dirs(rng, n) * (2 * R * 1.02 * rng.uniform(0, 1, n) ** (1 / 3))[:, None]
    qA, qB = _rand_quat(rng, n), _rand_quat(rng, n)
    got = s.overlap(D, qA, qB).astype(bool)
    gap = bf.sat15_boxes(np.array([0.5, 0.5, 0.5]), D, qA, qB)
    sure_sep = gap > 1e-9
    sure_ov = gap < -1e-9
    assert not np.any(got & sure_sep)
    assert not np.any(~got & sure_ov)
    assert sure_sep.sum() > 5000 and sure_ov.sum() > 5000


def test_gjk_cubes_vs_sat15_near_contact():
    rng = np.random.default_rng(2)
    v = inputs.cube(1.0)
    s = _sys(v)
    n = 20000
    u = _rand_dirs(rng, n)
    qA, qB = _rand_quat(rng, n), _rand_quat(rng, n)
    lo = np.zeros(n)
    hi = np.full(n, 2.0)
    h = np.array([0.5, 0.5, 0.5])
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        ov = bf.sat15_boxes(h, u * mid[:, None], qA, qB) < 0
        lo = np.where(ov, mid, lo)
        hi = np.where(ov, hi, mid)
    off = rng.choice([-1, 1], n) * 10.0 ** rng.uniform(-7, -3, n)
    D = u * (0.5 * (lo + hi) + off)[:, None]
    got = s.overlap(D, qA, qB).astype(bool)
    gap = bf.sat15_boxes(h, D, qA, qB)
    sure_sep = gap > 1e-10
    sure_ov = gap < -1e-10
    assert not np.any(got & sure_sep)
    assert not np.any(~got & sure_ov)
    assert (sure_sep | sure_ov).mean() > 0.99


def test_gjk_aligned_cubes_faces_edges_corners():
    v = inputs.cube(1.0)
    s = _sys(v)
    I = np.array([[1.0, 0.0, 0.0, 0.0]])
    for D, want in [([1.0, 0, 0], 1), ([1.0 + 2 ** -40, 0, 0], 0), ([0, 0, -1.0], 1),
                    ([1.0, 1.0, 0], 1), ([1.0, 1.0 + 2 ** -40, 0], 0), ([1, 1, 1.0], 1),
                    ([0.5, 0.5, 0.5], 1), ([0, 0, 0], 1), ([3.0, 0, 0], 0),
                    ([1 + 2 ** -40, 1 + 2 ** -40, 1 + 2 ** -40], 0)]:
        assert s.overlap(np.array([D]), I, I)[0] == want, D


@pytest.mark.parametrize("shape", ["octahedron", "tetrahedron", "prism", "random"])
def test_gjk_general_polyhedra_vs_clipping(shape):
    rng = np.random.default_rng(hash(shape) % 1000)
    if shape == "octahedron":
        v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float) * 0.6
    elif shape == "tetrahedron":
        v = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float) * 0.4
    elif shape == "prism":
        t = np.array([[0.0, 0.5], [-0.433, -0.25], [0.433, -0.25]])
        v = np.array([[x, y, z] for z in (-0.4, 0.4) for x, y in t])
    else:
        p = rng.normal(size=(14, 3))
        v = 0.5 * p / np.linalg.norm(p, axis=1)[:, None]
    s = _sys(v)
    n = 4000
    R = np.sqrt((v ** 2).sum(1)).max()
    D = _rand_dirs(rng, n) * (2 * R * 1.02 * rng.uniform(0, 1, n) ** (1 / 3))[:, None]
    qA, qB = _rand_quat(rng, n), _rand_quat(rng, n)
    got = s.overlap(D, qA, qB).astype(bool)
    sure_ov, sure_sep = bf.classify_3d(v, D, qA, qB, eps=1e-8)
    assert not np.any(got & sure_sep)
    assert not np.any(~got & sure_ov)
    assert sure_ov.sum() > 300 and sure_sep.sum() > 300


def test_gjk_iteration_counts():
    # the oracle reports the GJK's support evaluations after the first (the
    # GPU pair tests compare them): the verdict is the same with or without
    # the count; every count lies in 1..33 (33 = cap reached); two aligned
    # cubes far apart along an axis separate at the first test; spheres run
    # no GJK
    rng = np.random.default_rng(7)
    s = _sys(inputs.cube(1.0))
    n = 5000
    D = _rand_dirs(rng, n) * rng.uniform(0.0, 2.0, n)[:, None]
    qA, qB = _rand_quat(rng, n), _rand_quat(rng, n)
    ov, it = s.overlap(D, qA, qB, iters=True)
    assert np.array_equal(ov, s.overlap(D, qA, qB))
    assert it.min() >= 1 and it.max() <= 33
    I = np.tile([1.0, 0, 0, 0], (3, 1))
    far = np.array([[3.0, 0, 0], [0, -2.5, 0], [0, 0, 1.2]])
    ov, it = s.overlap(far, I, I, iters=True)
    assert not ov.any() and np.all(it == 1)
    sph = orc.OracleSystem(3, [30.0] * 3, 0.5)
    ov, it = sph.overlap(D, qA, qB, iters=True)
    assert np.array_equal(ov, (np.linalg.norm(D, axis=1) <= 1.0).astype(np.int32)) and not it.any()


def _contact_dirs(rng, n):
    u = _rand_dirs(rng, n)
    q = _rand_quat(rng, 2 * n)
    return u, q[:n], q[n:]


def test_gjk_answers_separated_beyond_a_micro_gap():
    # What the FP32 filter's separation certificate relies on: the contract's
    # GJK answers "separated" for every pair farther apart than a small gap.
    # Just outside contact it is conservative -- a cap or a degenerate simplex
    # counts as overlap, and for unit cubes separated pairs up to ~2e-7 apart
    # can read "overlap" (that is the contract, which the GPU re-check
    # reproduces) -- but the certificate proves a gap of at least |n|_1 times
    # its FP32 error bound, ~6e-5 for the 32768-cube system, so it only acts
    # where this test shows the contract to be exact.  Classifiers: the 15-axis
    # test on cubes enlarged by 1 + eps (disjoint enlarged cubes are more than
    # eps apart; every pair more than sqrt(3) eps apart qualifies) and, for
    # dodecahedra, the clipping brute force on shapes scaled by 1 + eps.
    eps = 1e-6
    rng = np.random.default_rng(8)
    s = _sys(inputs.cube(1.0))
    h = np.array([0.5, 0.5, 0.5])
    n_sep = 0
    for _ in range(4):
        n = 250000
        u, qA, qB = _contact_dirs(rng, n)
        tstar = bf.sat15_exit(h, u, qA, qB)          # contact distance along u
        D = u * (tstar + 10.0 ** rng.uniform(-7.5, -3, n))[:, None]
        sep = bf.sat15_boxes(h * (1 + eps), D, qA, qB) > 1e-13
        got = s.overlap(D, qA, qB).astype(bool)
        assert not np.any(got & sep), np.nonzero(got & sep)[0][:5]
        n_sep += int(sep.sum())
    assert n_sep > 500000
    v = inputs.dodecahedron(1.0)
    s = _sys(v)
    n = 20000
    u, qA, qB = _contact_dirs(rng, n)
    R = np.sqrt((v ** 2).sum(1)).max()
    lo, hi = np.zeros(n), np.full(n, 2 * R * 1.001)
    for _ in range(50):
        mid = 0.5 * (lo + hi)
        ov = s.overlap(u * mid[:, None], qA, qB).astype(bool)
        lo, hi = np.where(ov, mid, lo), np.where(ov, hi, mid)
    D = u * (hi + 10.0 ** rng.uniform(-7, -3, n))[:, None]
    _, sep = bf.classify_3d(v, D, qA, qB, eps=eps)
    got = s.overlap(D, qA, qB).astype(bool)
    assert not np.any(got & sep)
    assert sep.sum() > 10000
