"""Independent brute-force overlap predicates used to pin the oracle.

None of this shares code with the oracle or the CUDA library.  The methods
are deliberately different from the separating-axis / GJK contract:

* 2D: two convex polygons overlap iff an edge of one properly crosses an edge
  of the other, or a vertex of one lies inside the other (orientation tests).
* 3D: two convex polyhedra overlap iff some edge of one, clipped against the
  facet half-spaces of the other (Cyrus-Beck), keeps a non-empty piece.
  Facets come from a brute-force hull over all vertex triples.
* 3D boxes: the 15-axis separating-axis test of Gottschalk et al. (OBBTree).

Near contact the answer is ill-conditioned, so every predicate is evaluated
on shapes shrunk and grown by a relative ``eps`` about their centres: a pair
is "sure overlap" when the shrunk shapes overlap, "sure separated" when the
grown shapes do not, and "ambiguous" otherwise.
"""
from __future__ import annotations

import itertools

import numpy as np


# --------------------------------------------------------------------- 2D
def rot2(z):
    """(n,2) unit complex -> (n,2,2) rotation matrices."""
    c, s = z[:, 0], z[:, 1]
    return np.stack([np.stack([c, -s], -1), np.stack([s, c], -1)], -2)


def _orient(p, q, r):
    return (q[..., 0] - p[..., 0]) * (r[..., 1] - p[..., 1]) - (q[..., 1] - p[..., 1]) * (r[..., 0] - p[..., 0])


def _poly_world(verts, z, t, scale):
    # (n, nv, 2)
    R = rot2(z)
    v = verts[None, :, :] * scale
    return np.einsum("nij,nvj->nvi", R, np.broadcast_to(v, (z.shape[0],) + verts.shape)) + t[:, None, :]


def _bf_overlap_2d(PA, PB):
    A0 = PA
    A1 = np.roll(PA, -1, axis=1)
    B0 = PB
    B1 = np.roll(PB, -1, axis=1)
    # edge-edge proper crossings, (n, na, nb)
    a0 = A0[:, :, None, :]
    a1 = A1[:, :, None, :]
    b0 = B0[:, None, :, :]
    b1 = B1[:, None, :, :]
    o1 = _orient(a0, a1, b0)
    o2 = _orient(a0, a1, b1)
    o3 = _orient(b0, b1, a0)
    o4 = _orient(b0, b1, a1)
    cross = ((o1 * o2) < 0) & ((o3 * o4) < 0)
    hit = cross.any(axis=(1, 2))
    # vertex of A inside B (B counter-clockwise): left of every edge
    inB = (_orient(b0, b1, PA[:, :, None, :]) > 0).all(axis=2).any(axis=1)
    inA = (_orient(A0[:, None, :, :], A1[:, None, :, :], PB[:, :, None, :]) > 0).all(axis=2).any(axis=1)
    return hit | inB | inA


def classify_2d(verts, D, zA, zB, eps=1e-9):
    """Return (sure_overlap, sure_separated) boolean arrays for pairs with
    A at the origin (orientation zA) and B at D (orientation zB)."""
    n = D.shape[0]
    zero = np.zeros((n, 2))
    ov_small = _bf_overlap_2d(_poly_world(verts, zA, zero, 1 - eps), _poly_world(verts, zB, D, 1 - eps))
    ov_big = _bf_overlap_2d(_poly_world(verts, zA, zero, 1 + eps), _poly_world(verts, zB, D, 1 + eps))
    return ov_small, ~ov_big


def pairwise_overlaps_2d(verts, L, pos, ori, eps=0.0):
    """All overlapping pairs (i<j) of a periodic 2D configuration, O(N^2)."""
    N = pos.shape[0]
    R = np.sqrt((verts ** 2).sum(1)).max()
    bad = []
    for i in range(N - 1):
        D = pos[i + 1:] - pos[i]
        D -= L * np.round(D / L)
        close = np.nonzero((D ** 2).sum(1) <= (2 * R) ** 2 * (1 + 1e-12))[0]
        if close.size == 0:
            continue
        zA = np.repeat(ori[i:i + 1], close.size, axis=0)
        sure_ov, sure_sep = classify_2d(verts, D[close], zA, ori[i + 1:][close], eps=max(eps, 1e-12))
        for c in close[~sure_sep]:
            bad.append((i, i + 1 + int(c)))
    return bad


# --------------------------------------------------------------------- 3D
def quat_to_mat(q):
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    n = w * w + x * x + y * y + z * z
    s = 2.0 / n
    return np.stack([
        np.stack([1 - s * (y * y + z * z), s * (x * y - w * z), s * (x * z + w * y)], -1),
        np.stack([s * (x * y + w * z), 1 - s * (x * x + z * z), s * (y * z - w * x)], -1),
        np.stack([s * (x * z - w * y), s * (y * z + w * x), 1 - s * (x * x + y * y)], -1),
    ], -2)


def hull_facets(verts, tol=1e-12):
    """Facet planes (n, c) with n.x <= c inside, of the convex hull of verts."""
    nv = verts.shape[0]
    planes = []
    for i, j, k in itertools.combinations(range(nv), 3):
        nrm = np.cross(verts[j] - verts[i], verts[k] - verts[i])
        ln = np.linalg.norm(nrm)
        if ln < 1e-14:
            continue
        nrm = nrm / ln
        c = nrm @ verts[i]
        side = verts @ nrm - c
        if (side <= tol).all():
            planes.append((nrm, c))
        elif (side >= -tol).all():
            planes.append((-nrm, -c))
    uniq = []
    for nrm, c in planes:
        if not any(np.allclose(nrm, u[0]) and abs(c - u[1]) < 1e-9 for u in uniq):
            uniq.append((nrm, c))
    return np.array([u[0] for u in uniq]), np.array([u[1] for u in uniq])


def hull_edges(verts, normals, offsets, tol=1e-9):
    on = np.abs(verts @ normals.T - offsets[None, :]) < tol  # (nv, nf)
    edges = []
    for i, j in itertools.combinations(range(verts.shape[0]), 2):
        if (on[i] & on[j]).sum() >= 2:
            edges.append((i, j))
    return np.array(edges)


def _clip_any(P0, P1, nrm, off):
    """Do segments P0->P1 (n, e, 3) keep a piece inside {x: nrm.x <= off}?"""
    d = P1 - P0
    a = np.einsum("nek,nfk->nef", P0, nrm)                    # n.P0
    b = np.einsum("nek,nfk->nef", d, nrm)                     # n.d
    rhs = off[:, None, :] - a                                  # need b t <= rhs
    t0 = np.zeros(a.shape[:2])
    t1 = np.ones(a.shape[:2])
    with np.errstate(divide="ignore", invalid="ignore"):
        tt = rhs / b
    pos = b > 0
    neg = b < 0
    zer = ~(pos | neg)
    t1 = np.minimum(t1, np.where(pos, tt, np.inf).min(axis=2))
    t0 = np.maximum(t0, np.where(neg, tt, -np.inf).max(axis=2))
    infeasible = (zer & (rhs < 0)).any(axis=2)
    return ((t0 <= t1) & ~infeasible).any(axis=1)


def _bf_overlap_3d(verts, normals, offsets, edges, qA, qB, D, scale):
    n = D.shape[0]
    RA = quat_to_mat(qA)
    RB = quat_to_mat(qB)
    v = verts * scale
    VA = np.einsum("nij,vj->nvi", RA, v)
    VB = np.einsum("nij,vj->nvi", RB, v) + D[:, None, :]
    nA = np.einsum("nij,fj->nfi", RA, normals)
    nB = np.einsum("nij,fj->nfi", RB, normals)
    oA = np.broadcast_to(offsets * scale, (n, offsets.size))
    oB = oA + np.einsum("nfi,ni->nf", nB, D)
    e0, e1 = edges[:, 0], edges[:, 1]
    hitA = _clip_any(VA[:, e0], VA[:, e1], nB, oB)
    hitB = _clip_any(VB[:, e0], VB[:, e1], nA, oA)
    return hitA | hitB


def classify_3d(verts, D, qA, qB, eps=1e-9):
    normals, offsets = hull_facets(verts)
    edges = hull_edges(verts, normals, offsets)
    ov_small = _bf_overlap_3d(verts, normals, offsets, edges, qA, qB, D, 1 - eps)
    ov_big = _bf_overlap_3d(verts, normals, offsets, edges, qA, qB, D, 1 + eps)
    return ov_small, ~ov_big


def sat15_exit(h, u, qA, qB):
    """Distance along the unit directions u at which two boxes (half-extents
    h) stop overlapping: the set of overlapping offsets is the intersection of
    the 15 slabs |D.L| <= ra + rb (L a unit test axis), so the ray t u leaves
    it at the smallest (ra + rb) / |u.L|."""
    RA = quat_to_mat(qA)
    RB = quat_to_mat(qB)
    A = np.swapaxes(RA, 1, 2)
    B = np.swapaxes(RB, 1, 2)
    axes = [A[:, i] for i in range(3)] + [B[:, j] for j in range(3)]
    axes += [np.cross(A[:, i], B[:, j]) for i in range(3) for j in range(3)]
    t = np.full(u.shape[0], np.inf)
    for L_ in axes:
        ln = np.linalg.norm(L_, axis=1)
        ok = ln > 1e-12
        Ln = np.where(ok[:, None], L_ / np.where(ok, ln, 1.0)[:, None], 0.0)
        ra = sum(h[i] * np.abs(np.einsum("nk,nk->n", A[:, i], Ln)) for i in range(3))
        rb = sum(h[j] * np.abs(np.einsum("nk,nk->n", B[:, j], Ln)) for j in range(3))
        c = np.abs(np.einsum("nk,nk->n", u, Ln))
        hit = ok & (c > 0)
        t = np.minimum(t, np.where(hit, (ra + rb) / np.where(hit, c, 1.0), np.inf))
    return t


def sat15_boxes(h, D, qA, qB):
    """Signed separation proxy of two boxes (half-extents h) by the 15-axis
    test: > 0 separated, < 0 overlapping (per-axis gap over |axis|)."""
    RA = quat_to_mat(qA)
    RB = quat_to_mat(qB)
    A = np.swapaxes(RA, 1, 2)  # rows = box axes in world
    B = np.swapaxes(RB, 1, 2)
    axes = [A[:, i] for i in range(3)] + [B[:, j] for j in range(3)]
    axes += [np.cross(A[:, i], B[:, j]) for i in range(3) for j in range(3)]
    best = np.full(D.shape[0], -np.inf)
    for L_ in axes:
        ln = np.linalg.norm(L_, axis=1)
        ok = ln > 1e-12
        Ln = np.where(ok[:, None], L_ / np.where(ok, ln, 1.0)[:, None], 0.0)
        ra = sum(h[i] * np.abs(np.einsum("nk,nk->n", A[:, i], Ln)) for i in range(3))
        rb = sum(h[j] * np.abs(np.einsum("nk,nk->n", B[:, j], Ln)) for j in range(3))
        gap = np.abs(np.einsum("nk,nk->n", D, Ln)) - ra - rb
        best = np.where(ok, np.maximum(best, gap), best)
    return best
