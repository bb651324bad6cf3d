"""O(N^2) overlap-pair count of a configuration with the oracle's FP64
contract test (test infrastructure).

Every unordered pair (i < j) is taken once: D = minimum image of
r_j - r_i (per axis: D - L when D > L/2, D + L when D < -L/2), culled when
|D|^2 exceeds the circumdiameter squared, otherwise decided by the oracle's
overlap test D(r_i, q_i; r_j, q_j) (Sec. 2.1: a configuration is valid when
no pair overlaps; Sec. 2.3 / Eq. 2 for the test itself).  No cell list is
involved, so the count pins the periodic stencil of a cell-list count.
"""
from __future__ import annotations

import numpy as np


def oracle_pair_count(ref, pos, ori, chunk=2048):
    """Number of overlapping unordered pairs of (pos, ori) in the oracle
    system `ref` (an oracle.OracleSystem of the same box and shape)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    ori = np.ascontiguousarray(ori, dtype=np.float64)
    N, dim = pos.shape
    L = np.asarray(ref.box, dtype=np.float64)
    halfL = 0.5 * L
    rc2 = ref.geometry()["rc2"]
    total = 0
    for i0 in range(0, N, chunk):
        i1 = min(N, i0 + chunk)
        I, J = [], []
        for i in range(i0, i1):
            d = pos[i + 1:] - pos[i]
            d = np.where(d > halfL, d - L, np.where(d < -halfL, d + L, d))
            q2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]
            if dim == 3:
                q2 = q2 + d[:, 2] * d[:, 2]
            near = np.nonzero(q2 <= rc2)[0]
            if near.size:
                I.append(np.full(near.size, i))
                J.append(i + 1 + near)
        if not I:
            continue
        I = np.concatenate(I)
        J = np.concatenate(J)
        D = pos[J] - pos[I]
        D = np.where(D > halfL, D - L, np.where(D < -halfL, D + L, D))
        total += int(ref.overlap(D, ori[I], ori[J]).sum())
    return total


def plant_wrap_pairs(pos, L, seed=0):
    """A copy of a 2D configuration with pairs placed across the periodic
    boundaries: overlapping pairs straddling the x wrap, the y wrap and the
    corner, plus pairs whose centres sit between the inscribed and the
    circumscribed diameter of a shape of circumradius 0.5 across the x and
    y wraps (their verdict depends on the orientations)."""
    rng = np.random.default_rng(seed)
    p = np.array(pos, dtype=np.float64, copy=True)
    Lx, Ly = float(L[0]), float(L[1])
    p[0] = (Lx - 0.1, 0.37 * Ly)
    p[1] = (0.2, 0.37 * Ly)
    p[2] = (0.61 * Lx, Ly - 0.15)
    p[3] = (0.61 * Lx, 0.1)
    p[4] = (Lx - 0.12, Ly - 0.1)
    p[5] = (0.14, 0.13)
    k = 6
    for j in range(8):
        dist = rng.uniform(0.75, 0.98)
        u = rng.uniform(0.05, dist - 0.05)
        y = (0.45 + 0.05 * j) * Ly
        p[k] = (Lx - u, y)
        p[k + 1] = (dist - u, y)
        x = (0.1 + 0.05 * j) * Lx
        p[k + 2] = (x, Ly - u)
        p[k + 3] = (x, dist - u)
        k += 4
    assert (p >= 0).all() and (p[:, 0] < Lx).all() and (p[:, 1] < Ly).all()
    return p
