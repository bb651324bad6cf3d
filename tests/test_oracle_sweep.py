"""Pins of the oracle's checkerboard sweep as a whole (Sec. 2.1, 2.2.1,
2.5.1-2.5.2): invariants, closed forms and the stationary law."""
import os

import numpy as np
from scipy import stats

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs
from tests import bruteforce as bf

GOLD = os.path.join(os.path.dirname(__file__), "golden", "rsa_pentagons_N1024_phi050_seed42.txt")


def load_rsa_start():
    rows = []
    header = None
    for line in open(GOLD):
        if line.startswith("#"):
            if " L=" in line:
                header = line
            continue
        rows.append([float.fromhex(t) for t in line.split()])
    a = np.array(rows)
    L = float.fromhex(header.split("L=")[1].split(",")[0])
    return a[:, :2].copy(), a[:, 2:].copy(), L


def test_rsa_fixture_is_overlap_free():
    pos, ori, L = load_rsa_start()
    v = inputs.regular_polygon(5, 0.5)
    assert pos.shape == (1024, 2)
    assert abs(1024 * inputs.polygon_area(v) / L ** 2 - 0.50) < 1e-12
    assert bf.pairwise_overlaps_2d(v, L, pos, ori) == []


def _nonempty_cells(s, pos, sweep):
    start, _, _ = s.build_cells(pos, s.grid_shift(sweep))
    return int(np.count_nonzero(np.diff(start.astype(np.int64))))


def test_sweeps_keep_config_valid_and_count_every_move():
    pos, ori, L = load_rsa_start()
    v = inputs.regular_polygon(5, 0.5)
    s = orc.OracleSystem(2, [L, L], v)
    s.set_moves(0.1, 0.1, 4, 42)
    total = np.zeros(4, np.uint64)
    for sw in range(6):
        ne = _nonempty_cells(s, pos, sw)
        c = s.sweep(pos, ori, sw, 1)
        assert int(c[0] + c[1] + c[2]) == 4 * ne
        total += c
        assert ((pos >= 0) & (pos < L)).all()
        assert np.abs(np.hypot(ori[:, 0], ori[:, 1]) - 1).max() < 1e-14
        assert bf.pairwise_overlaps_2d(v, L, pos, ori) == []
    assert total[0] > 0 and total[1] > 0 and total[2] > 0


def test_checkpoint_resume_is_bit_identical_and_seed_matters():
    pos0, ori0, L = load_rsa_start()
    s = orc.OracleSystem(2, [L, L], inputs.regular_polygon(5, 0.5))
    s.set_moves(0.1, 0.1, 4, 42)
    pa, oa = pos0.copy(), ori0.copy()
    ca = s.sweep(pa, oa, 0, 20)
    pb, ob = pos0.copy(), ori0.copy()
    cb = s.sweep(pb, ob, 0, 8) + s.sweep(pb, ob, 8, 12)
    assert np.array_equal(pa, pb) and np.array_equal(oa, ob) and np.array_equal(ca, cb)
    s.set_moves(0.1, 0.1, 4, 43)
    pc, oc = pos0.copy(), ori0.copy()
    s.sweep(pc, oc, 0, 20)
    assert not np.array_equal(pa, pc)


def test_ideal_gas_boundary_rejection_closed_form():
    # vanishing shapes: no overlaps, every rejection is a boundary rejection,
    # and with positions uniform inside each cell the in-cell probability of
    # a uniform step in [-d, d) is prod_axes (1 - d / (2 w)).
    v = inputs.regular_polygon(5, 1e-4)
    L = 40.0
    s = orc.OracleSystem(2, [L, L], v, w_min=1.0)
    d = 0.3
    s.set_moves(d, 0.5, 4, 11)
    rng = np.random.default_rng(0)
    N = 3000
    pos = rng.uniform(0, L, (N, 2))
    th = rng.uniform(0, 2 * np.pi, N)
    ori = np.stack([np.cos(th), np.sin(th)], 1)
    c = s.sweep(pos, ori, 0, 40)
    moves = int(c[0] + c[1] + c[2])
    assert c[1] == 0
    w = s.geometry()["w"]
    p_in = np.prod(1 - d / (2 * w))
    rate = c[2] / moves
    sigma = np.sqrt(p_in * (1 - p_in) / moves)
    assert abs(rate - (1 - p_in)) < 5 * sigma, (rate, 1 - p_in, sigma)
    # stationary law of the ideal gas: uniform positions and angles
    h, _, _ = np.histogram2d(pos[:, 0], pos[:, 1], bins=10, range=[[0, L], [0, L]])
    assert stats.chisquare(h.ravel()).pvalue > 1e-4
    ang = np.arctan2(ori[:, 1], ori[:, 0])
    assert stats.kstest((ang + np.pi) / (2 * np.pi), "uniform").pvalue > 1e-4


def test_ideal_gas_boundary_rejection_closed_form_3d():
    # the same in 3D (vanishing cubes, eight sets): in-cell probability
    # (1 - d / (2 w))^3, and the uniform law stays stationary -- positions,
    # and orientations uniform on the unit quaternions, whose components have
    # the marginal density (2 / pi) sqrt(1 - x^2)
    L = 20.0
    s = orc.OracleSystem(3, [L, L, L], inputs.cube(1e-4), w_min=1.0)
    d = 0.3
    s.set_moves(d, 0.5, 4, 12)
    rng = np.random.default_rng(1)
    N = 3000
    pos = rng.uniform(0, L, (N, 3))
    q = rng.normal(size=(N, 4))
    ori = q / np.linalg.norm(q, axis=1)[:, None]
    c = s.sweep(pos, ori, 0, 40)
    moves = int(c[0] + c[1] + c[2])
    assert c[1] == 0
    w = s.geometry()["w"]
    assert len(w) == 3 and np.all(w == 1.0)
    p_in = np.prod(1 - d / (2 * w))
    rate = c[2] / moves
    sigma = np.sqrt(p_in * (1 - p_in) / moves)
    assert abs(rate - (1 - p_in)) < 5 * sigma, (rate, 1 - p_in, sigma)
    h, _ = np.histogramdd(pos, bins=5, range=[[0, L]] * 3)
    assert stats.chisquare(h.ravel()).pvalue > 1e-4
    assert np.allclose(np.linalg.norm(ori, axis=1), 1.0, atol=1e-14)

    def cdf(x):
        return 0.5 + (x * np.sqrt(1 - x * x) + np.arcsin(x)) / np.pi

    for k in range(4):
        assert stats.kstest(ori[:, k], cdf).pvalue > 1e-4, k


def test_two_pentagon_pair_distance_law():
    # Two hard pentagons in a small periodic box: the chain's stationary law is
    # uniform over non-overlapping configurations.  Compare the distribution
    # of the minimum-image centre distance with rejection sampling that uses
    # the independent brute-force predicate.
    v = inputs.regular_polygon(5, 0.5)
    L = 4.2
    s = orc.OracleSystem(2, [L, L], v)
    s.set_moves(0.35, 0.8, 2, 5)
    pos = np.array([[0.5, 0.5], [2.6, 2.6]])
    ori = np.array([[1.0, 0.0], [0.0, 1.0]])
    samples = []
    for k in range(30000):
        s.sweep(pos, ori, k, 1)
        if k >= 200 and k % 6 == 0:
            D = pos[1] - pos[0]
            D -= L * np.round(D / L)
            samples.append(np.hypot(*D))
    chain = np.array(samples)
    rng = np.random.default_rng(9)
    M = 200000
    D = rng.uniform(-L / 2, L / 2, (M, 2))
    ta, tb = rng.uniform(0, 2 * np.pi, M), rng.uniform(0, 2 * np.pi, M)
    zA = np.stack([np.cos(ta), np.sin(ta)], 1)
    zB = np.stack([np.cos(tb), np.sin(tb)], 1)
    r = np.hypot(D[:, 0], D[:, 1])
    keep = np.ones(M, bool)
    near = r <= 1.0
    sure_ov, sure_sep = bf.classify_2d(v, D[near], zA[near], zB[near], eps=0.0)
    keep[np.nonzero(near)[0][sure_ov]] = False
    ref = r[keep]
    res = stats.ks_2samp(chain, ref)
    assert res.pvalue > 1e-3, res


def test_one_particle_chain_carries_no_current():
    # Detailed balance.  With a single particle exactly one checkerboard set
    # acts in a sweep (the set of its cell), after a random grid shift that
    # does not depend on the state; each such update is reversible for the
    # uniform measure (symmetric proposals, in-cell rejection symmetric
    # between x and x'), and so is their mixture.  A reversible chain carries
    # no net probability current across any cut, so the net number of
    # crossings of the x, y and angle bin boundaries (forward minus
    # backward) stays within noise of zero.  A bias of 0.005 in x per sweep
    # (under 2% of the step) reads z = 5.3 here, a rotation bias of 0.01 rad
    # per sweep z = 4.6; the unbiased chain |z| < 0.4.
    v = inputs.regular_polygon(5, 0.5)
    L = 4.4                                         # 4 x 4 cells
    s = orc.OracleSystem(2, [L, L], v)
    s.set_moves(0.35, 0.6, 4, 2024)
    pos = np.array([[1.3, 2.9]])
    ori = np.array([[1.0, 0.0]])
    nb, na = 8, 4

    def bins(p, o):
        ix = min(int(p[0, 0] / L * nb), nb - 1)
        iy = min(int(p[0, 1] / L * nb), nb - 1)
        ia = min(int((np.arctan2(o[0, 1], o[0, 0]) + np.pi) / (2 * np.pi) * na), na - 1)
        return ix, iy, ia

    s.sweep(pos, ori, 0, 200)                       # burn-in
    a = bins(pos, ori)
    current, crossings = np.zeros(3), np.zeros(3)
    for sw in range(200, 150200):
        s.sweep(pos, ori, sw, 1)
        b = bins(pos, ori)
        for k, m in enumerate((nb, nb, na)):
            step = (b[k] - a[k]) % m
            if step == 1:
                current[k] += 1
                crossings[k] += 1
            elif step == m - 1:
                current[k] -= 1
                crossings[k] += 1
        a = b
    assert np.all(crossings > 20000)
    z = current / np.sqrt(crossings)
    assert np.all(np.abs(z) < 4.0), (z, crossings)


def _cube_chain_currents(n, drift_x=0.0, drift_rot=0.0):
    # one cube in a 4 x 4 x 4 cell box; net signed bin crossings of x, y, z
    # (16 bins) and of psi = atan2(q3, q0) (8 bins; a jump of exactly half a
    # turn has no direction and is left out), each divided by the square root
    # of its crossings.  The optional drift composes every sweep with a
    # translation along x and a body rotation about z (which advances psi by
    # drift_rot exactly): a chain that is not reversible.
    L = 7.3
    s = orc.OracleSystem(3, [L, L, L], inputs.cube(1.0))
    s.set_moves(0.6, 0.8, 4, 2024)
    pos = np.array([[1.3, 2.9, 5.1]])
    ori = np.array([[1.0, 0.0, 0.0, 0.0]])
    nb, na = 16, 8
    cb, sb = np.cos(drift_rot), np.sin(drift_rot)

    def bins():
        b = [min(int(pos[0, k] / L * nb), nb - 1) for k in range(3)]
        return b + [min(int((np.arctan2(ori[0, 3], ori[0, 0]) + np.pi) / (2 * np.pi) * na), na - 1)]

    s.sweep(pos, ori, 0, 200)                       # burn-in
    a = bins()
    current, crossings = np.zeros(4), np.zeros(4)
    for sw in range(200, 200 + n):
        s.sweep(pos, ori, sw, 1)
        if drift_x:
            pos[0, 0] = (pos[0, 0] + drift_x) % L
        if drift_rot:
            q0, q1, q2, q3 = ori[0]
            ori[0] = [q0 * cb - q3 * sb, q1 * cb + q2 * sb, q2 * cb - q1 * sb, q3 * cb + q0 * sb]
        b = bins()
        for k, m in enumerate((nb, nb, nb, na)):
            step = (b[k] - a[k]) % m
            if 2 * step == m:
                continue
            if step > m // 2:
                step -= m
            current[k] += step
            crossings[k] += abs(step)
        a = b
    return current / np.sqrt(crossings), crossings


def test_one_particle_chain_carries_no_current_3d():
    # Detailed balance of the 3D sweep (eight sets, quaternion steps q dq with
    # dq and its inverse equally likely), by the argument of the 2D test.
    # The unbiased chain reads |z| < 2 on all four statistics; composed with
    # a drift of 0.005 along x and 0.01 rad about the body z axis per sweep
    # (about 1% of the step and of the rotation range) it reads z_x = 5.6 and
    # z_psi = 9.9.
    z, crossings = _cube_chain_currents(300000)
    assert np.all(crossings > 150000)
    assert np.all(np.abs(z) < 4.0), (z, crossings)
    zd, _ = _cube_chain_currents(300000, 0.005, 0.01)
    assert zd[0] > 4.0 and zd[3] > 4.0, zd
