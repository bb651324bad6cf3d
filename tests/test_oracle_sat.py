"""Pins of the oracle's 2D overlap contract (separating axes in A's frame,
Sec. 2.3) against an independent brute-force edge-crossing/containment test."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs
from tests import bruteforce as bf


def _sys(verts, L=20.0):
    return orc.OracleSystem(2, [L, L], verts)


def _rand_pairs(rng, n, R, rmax_factor=1.05):
    ang = rng.uniform(0, 2 * np.pi, n)
    r = 2 * R * rmax_factor * np.sqrt(rng.uniform(0, 1, n))
    D = np.stack([r * np.cos(ang), r * np.sin(ang)], 1)
    ta = rng.uniform(0, 2 * np.pi, n)
    tb = rng.uniform(0, 2 * np.pi, n)
    zA = np.stack([np.cos(ta), np.sin(ta)], 1)
    zB = np.stack([np.cos(tb), np.sin(tb)], 1)
    return D, zA, zB


def _near_contact(rng, verts, n):
    """Pairs placed at the brute-force contact distance along a random
    direction (bisection), then pushed in/out by 1e-7..1e-3."""
    R = inputs.circumradius(verts)
    ang = rng.uniform(0, 2 * np.pi, n)
    u = np.stack([np.cos(ang), np.sin(ang)], 1)
    ta = rng.uniform(0, 2 * np.pi, n)
    tb = rng.uniform(0, 2 * np.pi, n)
    zA = np.stack([np.cos(ta), np.sin(ta)], 1)
    zB = np.stack([np.cos(tb), np.sin(tb)], 1)
    lo = np.zeros(n)
    hi = np.full(n, 2 * R * 1.001)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        ov, _ = bf.classify_2d(verts, u * mid[:, None], zA, zB, eps=0.0)
        lo = np.where(ov, mid, lo)
        hi = np.where(ov, hi, mid)
    contact = 0.5 * (lo + hi)
    off = rng.choice([-1, 1], n) * 10.0 ** rng.uniform(-7, -3, n)
    return u * (contact + off)[:, None], zA, zB


@pytest.mark.parametrize("nv", [3, 4, 5, 7])
def test_sat_matches_bruteforce_random(nv):
    rng = np.random.default_rng(100 + nv)
    v = inputs.regular_polygon(nv, 0.5)
    s = _sys(v)
    D, zA, zB = _rand_pairs(rng, 40000, 0.5)
    got = s.overlap(D, zA, zB).astype(bool)
    sure_ov, sure_sep = bf.classify_2d(v, D, zA, zB)
    assert not np.any(got & sure_sep)
    assert not np.any(~got & sure_ov)
    assert sure_ov.sum() > 5000 and sure_sep.sum() > 5000


def test_sat_matches_bruteforce_near_contact_pentagon():
    rng = np.random.default_rng(7)
    v = inputs.regular_polygon(5, 0.5)
    s = _sys(v)
    D, zA, zB = _near_contact(rng, v, 20000)
    got = s.overlap(D, zA, zB).astype(bool)
    sure_ov, sure_sep = bf.classify_2d(v, D, zA, zB, eps=1e-11)
    assert not np.any(got & sure_sep)
    assert not np.any(~got & sure_ov)
    assert (sure_ov | sure_sep).mean() > 0.99


def test_sat_irregular_convex_polygon():
    rng = np.random.default_rng(11)
    th = np.sort(rng.uniform(0, 2 * np.pi, 9))
    rad = rng.uniform(0.3, 0.5, 9)
    pts = np.stack([rad * np.cos(th), rad * np.sin(th)], 1)
    # convex hull (monotone chain) to get a convex CCW polygon
    P = sorted(map(tuple, pts))

    def cross(o, a, b):
        return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])
    lower, upper = [], []
    for p in P:
        while len(lower) >= 2 and cross(lower[-2], lower[-1], p) <= 0:
            lower.pop()
        lower.append(p)
    for p in reversed(P):
        while len(upper) >= 2 and cross(upper[-2], upper[-1], p) <= 0:
            upper.pop()
        upper.append(p)
    hull = np.array(lower[:-1] + upper[:-1])
    s = _sys(hull)
    D, zA, zB = _rand_pairs(rng, 30000, inputs.circumradius(hull))
    got = s.overlap(D, zA, zB).astype(bool)
    sure_ov, sure_sep = bf.classify_2d(hull, D, zA, zB)
    assert not np.any(got & sure_sep)
    assert not np.any(~got & sure_ov)


def test_sat_touching_squares_is_overlap():
    v = np.array([[-0.5, -0.5], [0.5, -0.5], [0.5, 0.5], [-0.5, 0.5]])
    s = _sys(v)
    I = np.array([[1.0, 0.0]])
    # face-to-face contact at exactly distance 1: touching counts as overlap
    assert s.overlap(np.array([[1.0, 0.0]]), I, I)[0] == 1
    assert s.overlap(np.array([[1.0 + 2.0 ** -40, 0.0]]), I, I)[0] == 0
    assert s.overlap(np.array([[0.0, -1.0]]), I, I)[0] == 1
    assert s.overlap(np.array([[0.0, 0.0]]), I, I)[0] == 1
    # corner-to-corner along the diagonal
    assert s.overlap(np.array([[1.0, 1.0]]), I, I)[0] == 1
    assert s.overlap(np.array([[1.0, 1.0 + 2.0 ** -40]]), I, I)[0] == 0


def test_sat_rotation_and_swap_invariance():
    rng = np.random.default_rng(3)
    v = inputs.regular_polygon(5, 0.5)
    s = _sys(v)
    D, zA, zB = _rand_pairs(rng, 20000, 0.5)
    base = s.overlap(D, zA, zB)
    sure_ov, sure_sep = bf.classify_2d(v, D, zA, zB, eps=1e-6)
    clear = sure_ov | sure_sep
    # swapping the roles of A and B
    sw = s.overlap(-D, zB, zA)
    assert np.array_equal(base[clear], sw[clear])
    # a common rotation of the whole pair
    phi = 0.7
    c, sn = np.cos(phi), np.sin(phi)
    Dr = np.stack([c * D[:, 0] - sn * D[:, 1], sn * D[:, 0] + c * D[:, 1]], 1)

    def rot(z):
        return np.stack([c * z[:, 0] - sn * z[:, 1], sn * z[:, 0] + c * z[:, 1]], 1)
    rr = s.overlap(Dr, rot(zA), rot(zB))
    assert np.array_equal(base[clear], rr[clear])
