"""Pin of the oracle's single trial move: the exact acceptance probability of
one move of a pentagon next to another, in a 4 x 4-cell box.

Sec. 2.1 defines one Metropolis step for hard particles: a random trial
move (translation and rotation) is accepted iff the moved particle overlaps
nothing; Sec. 2.5.2 adds the checkerboard rule that a trial leaving its
active cell is rejected.  With the readings of the move distribution
(translation uniform in [-d, d)^2, rotation by the Cayley angle 2 atan t
with t uniform in [-tan(a/2), tan(a/2))) and of the grid shift (uniform in
[0, w)^2 per sweep), the probability that particle A's one trial of a sweep
is accepted is

    P = E_t E_delta [ p_x(delta_x) p_y(delta_y) 1{A moved by (delta, t) misses B} ]

where p_x, p_y are the probabilities over the shift that the trial stays in
A's cell.  The overlap region in delta is a Minkowski sum, (r_B - r_A) +
B (-) A_t (the convex hull of the pairwise vertex differences), so the inner
integral is exact: the piecewise bilinear p_x p_y integrated over the box
minus that polygon (clipped polygons, a degree-2 exact triangle rule).  The
outer integral over t uses composite Gauss-Legendre.  None of this uses the
oracle's separating-axis test, its proposal code or its cell rule.

The oracle side: many single sweeps from the same configuration (nselect =
1), each with its own sweep index and so its own shift and move; a sweep is
counted when A's row is even and B's row differs, so that A's set (2 py +
px, py = 0) runs before B's (py = 1) and B has not moved when A's trial is
decided; A is then alone in its cell and is the particle picked.
"""
import numpy as np

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs
from tests import bruteforce as bf

L = 5.0                      # 4 cells of width 1.25 per axis (floor(5 / 1.0) = 5, made even)
W = 1.25
RA = np.array([2.0, 3.0])
RB = np.array([2.3, 2.2])
THA, THB = 0.2, 1.0
D_MOVE, A_MOVE = 0.3, 0.8
SEED = 12345
N_SWEEPS = 10_000_000


def _rot(th, v):
    c, s = np.cos(th), np.sin(th)
    return np.stack([c * v[:, 0] - s * v[:, 1], s * v[:, 0] + c * v[:, 1]], -1)


def _hull(pts):
    """Convex hull, counter-clockwise (monotone chain)."""
    p = sorted(map(tuple, pts))

    def half(seq):
        h = []
        for q in seq:
            while len(h) >= 2 and ((h[-1][0] - h[-2][0]) * (q[1] - h[-2][1]) -
                                   (h[-1][1] - h[-2][1]) * (q[0] - h[-2][0])) <= 0:
                h.pop()
            h.append(q)
        return h
    lo, up = half(p), half(reversed(p))
    return np.array(lo[:-1] + up[:-1])


def _clip(poly, axis, bound, keep_below):
    """Sutherland-Hodgman against x_axis <= bound (keep_below) or >= bound."""
    out = []
    n = len(poly)
    for i in range(n):
        P, Q = poly[i], poly[(i + 1) % n]
        inP = P[axis] <= bound if keep_below else P[axis] >= bound
        inQ = Q[axis] <= bound if keep_below else Q[axis] >= bound
        if inP:
            out.append(P)
        if inP != inQ:
            t = (bound - P[axis]) / (Q[axis] - P[axis])
            out.append(P + t * (Q - P))
    return out


def _integrate_bilinear(poly, f, g):
    """Integral of f(x) g(y) (f, g affine) over a convex polygon: triangle
    fan, edge-midpoint rule (exact for polynomials of degree 2)."""
    tot = 0.0
    for i in range(1, len(poly) - 1):
        a, b, c = poly[0], poly[i], poly[i + 1]
        area = 0.5 * abs((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]))
        h = sum(f((p[0] + q[0]) / 2) * g((p[1] + q[1]) / 2) for p, q in ((a, b), (b, c), (c, a)))
        tot += area * h / 3.0
    return tot


def _weights(d):
    """In-cell probabilities over the shift, each affine on [-d, 0] and
    [0, d].  x: no condition on s_x, A's in-cell coordinate u uniform on
    [0, w): p = 1 - |delta| / w.  y: the counted sweeps have s_y in [0, 0.5]
    (A in row 2, B in row 1), A's in-cell coordinate u = 0.5 - s_y uniform on
    [0, 0.5]: p = 1 + delta / 0.5 below zero (u >= -delta), 1 above (u +
    delta <= 0.8 < w)."""
    px = {(-d, 0.0): lambda x: 1.0 + x / W, (0.0, d): lambda x: 1.0 - x / W}
    py = {(-d, 0.0): lambda y: 1.0 + y / 0.5, (0.0, d): lambda y: 1.0}
    return px, py


def _integral_over(poly, px, py):
    tot = 0.0
    for (x0, x1), f in px.items():
        for (y0, y1), g in py.items():
            q = [np.asarray(v, dtype=float) for v in poly]
            for axis, bnd, below in ((0, x1, True), (0, x0, False), (1, y1, True), (1, y0, False)):
                q = _clip(q, axis, bnd, below)
                if len(q) < 3:
                    break
            if len(q) >= 3:
                tot += _integrate_bilinear(q, f, g)
    return tot


def exact_acceptance(angle_of_t=lambda t: 2.0 * np.arctan(t), px=None, py=None, panels=120, nodes=8):
    verts = inputs.regular_polygon(5, 0.5)
    d = D_MOVE
    tau = np.tan(0.5 * A_MOVE)
    wpx, wpy = _weights(d)
    px = px or wpx
    py = py or wpy
    box = [np.array(p) for p in ((-d, -d), (d, -d), (d, d), (-d, d))]
    i_box = _integral_over(box, px, py)
    B = _rot(THB, verts)
    xg, wg = np.polynomial.legendre.leggauss(nodes)
    edges = np.linspace(-tau, tau, panels + 1)
    acc = 0.0
    for t0, t1 in zip(edges[:-1], edges[1:]):
        for x, wq in zip(xg, wg):
            t = 0.5 * (t1 - t0) * x + 0.5 * (t1 + t0)
            A = _rot(THA + angle_of_t(t), verts)
            M = _hull((B[None, :, :] - A[:, None, :]).reshape(-1, 2)) + (RB - RA)
            inner = (i_box - _integral_over(list(M), px, py)) / (4 * d * d)
            acc += 0.5 * (t1 - t0) * wq * inner
    return acc / (2 * tau)


def _cell_row(y, s):
    v = y - s
    v = np.where(v < 0, v + L, v)
    i = (v * (4 / L)).astype(np.int64)
    return np.minimum(i, 3)


def test_one_move_acceptance_equals_the_exact_integral():
    verts = inputs.regular_polygon(5, 0.5)
    zA = np.array([np.cos(THA), np.sin(THA)])
    zB = np.array([np.cos(THB), np.sin(THB)])
    # the starting pair does not overlap (brute-force polygon predicate)
    sure_ov, sure_sep = bf.classify_2d(verts, (RB - RA)[None], zA[None], zB[None], eps=1e-6)
    assert sure_sep[0]
    ref = orc.OracleSystem(2, L, verts)
    g = ref.geometry()
    assert tuple(g["nc"]) == (4, 4) and abs(g["w"][0] - W) < 1e-15
    ref.set_moves(D_MOVE, A_MOVE, 1, SEED)
    pos = np.array([RA, RB])
    ori = np.array([zA, zB])
    moved, shifts = ref.sweep_repeats(pos, ori, 0, N_SWEEPS)
    sy = shifts[:, 1]
    rowA, rowB = _cell_row(RA[1], sy), _cell_row(RB[1], sy)
    counted = (rowA % 2 == 0) & (rowB != rowA)
    # the counted sweeps are those with s_y in [0, 0.5] (A in row 2, B in row 1)
    assert np.array_equal(counted, sy <= 0.5)
    n = int(counted.sum())
    freq = moved[counted, 0].mean()
    P = exact_acceptance()
    sigma = np.sqrt(P * (1 - P) / n)
    assert n > 3_500_000
    assert abs(freq - P) < 4.5 * sigma, (freq, P, sigma, n)
    # the pin tells plausible misreadings apart: a rotation by atan t instead
    # of 2 atan t, no in-cell rule, and the in-cell rule without the shift's
    # conditioning on A's row each move P by many sigma
    px_free = {(-D_MOVE, D_MOVE): lambda x: 1.0}
    py_free = {(-D_MOVE, D_MOVE): lambda y: 1.0}
    py_uncond = {(-D_MOVE, 0.0): lambda y: 1.0 + y / W, (0.0, D_MOVE): lambda y: 1.0 - y / W}
    for alt in (exact_acceptance(angle_of_t=np.arctan),
                exact_acceptance(px=px_free, py=py_free),
                exact_acceptance(py=py_uncond)):
        assert abs(alt - P) > 12 * sigma, (alt, P, sigma)


def test_exact_integral_limits():
    # with B far away nothing overlaps: P is the in-cell probability alone,
    # (2d - d^2/w)(2d - d^2) / (4 d^2) for the weights above (closed form)
    global RB
    keep = RB
    try:
        RB = np.array([4.9, 0.1])
        d = D_MOVE
        want = (2 * d - d * d / W) * (2 * d - d * d) / (4 * d * d)
        assert abs(exact_acceptance(panels=4, nodes=4) - want) < 1e-12
    finally:
        RB = keep
