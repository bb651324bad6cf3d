"""Pins of the oracle's cell list (Sec. 2.2.1), grid shift (Sec. 2.5.1) and
trial-move arithmetic (Sec. 2.1) against their definitions."""
import numpy as np
import pytest
from scipy import stats

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs


def _pent(L, w_min=0.0):
    return orc.OracleSystem(2, [L, L], inputs.regular_polygon(5, 0.5), w_min=w_min)


def test_cell_geometry_rules():
    g = _pent(34.890576677059904).geometry()
    assert list(g["nc"]) == [34, 34]
    g = _pent(63.70).geometry()            # floor(63.70) = 63 is odd -> 62
    assert list(g["nc"]) == [62, 62]
    assert g["w"][0] >= 1.0
    g = _pent(4076.876, w_min=1.99).geometry()
    assert list(g["nc"]) == [2048, 2048]
    with pytest.raises(ValueError):
        _pent(3.9)                         # fewer than 4 cells per axis
    with pytest.raises(ValueError):        # clockwise polygon
        orc.OracleSystem(2, [20, 20], inputs.regular_polygon(5, 0.5)[::-1])
    with pytest.raises(ValueError):        # non-convex polygon
        orc.OracleSystem(2, [20, 20], np.array([[0, 0], [1, 0], [0.2, 0.2], [0, 1.0]]))


def test_grid_shift_range_and_variation():
    s = _pent(20.0)
    s.set_moves(0.1, 0.1, 4, 42)
    w = s.geometry()["w"]
    sh = np.array([s.grid_shift(k)[:2] for k in range(4000)])
    assert (sh >= 0).all() and (sh < w[None, :]).all()
    for a in range(2):
        assert stats.kstest(sh[:, a] / w[a], "uniform").pvalue > 1e-4


def test_cell_list_definition():
    rng = np.random.default_rng(5)
    L = 23.3
    s = _pent(L)
    s.set_moves(0.1, 0.1, 4, 9)
    g = s.geometry()
    pos = rng.uniform(0, L, (3000, 2))
    pos[:5] = [[0, 0], [L * (1 - 2 ** -52), 0], [g["w"][0], 0], [0, L - 1e-300], [L / 2, L / 2]]
    pos[pos >= L] = 0.0
    for sweep in range(3):
        sh = s.grid_shift(sweep)
        start, idx, cof = s.build_cells(pos, sh)
        nc = g["nc"]
        assert start[0] == 0 and start[-1] == pos.shape[0]
        seen = np.zeros(pos.shape[0], int)
        for c in range(nc[0] * nc[1]):
            members = idx[start[c]:start[c + 1]]
            assert np.all(np.diff(members.astype(np.int64)) > 0)   # ascending tags
            seen[members] += 1
            assert np.all(cof[members] == c)                        # per-particle cell agrees
            ix, iy = c % nc[0], c // nc[0]
            for t in members:
                for a, i in ((0, ix), (1, iy)):
                    y = (pos[t, a] - sh[a]) % L
                    lo, hi = i * g["w"][a], (i + 1) * g["w"][a]
                    assert lo - 1e-9 <= y < hi + 1e-9 or (i == nc[a] - 1 and y >= L - 1e-9)
        assert (seen == 1).all()


def test_translation_rotation_and_pick_distributions():
    s = _pent(30.0)
    d, a = 0.2, 0.3
    s.set_moves(d, a, 8, 1234)
    x0 = np.array([15.0, 15.0])
    z0 = np.array([1.0, 0.0])
    dx, dth, picks = [], [], []
    for cell in range(0, 4000):
        for k in range(2):
            pick, xn, zn = s.propose(7, cell % 4, cell, k, 5, x0, z0)
            dx.append(xn - x0)
            dth.append(np.arctan2(zn[1], zn[0]))
            picks.append(pick)
            assert abs(np.hypot(*zn) - 1.0) < 4e-16
    dx = np.array(dx)
    for ax in range(2):
        assert stats.kstest((dx[:, ax] + d) / (2 * d), "uniform").pvalue > 1e-4
    # rotation: tan(angle/2) uniform on [-tan(a/2), tan(a/2))
    t = np.tan(np.array(dth) / 2) / np.tan(a / 2)
    assert np.abs(np.array(dth)).max() <= a + 1e-12
    assert stats.kstest((t + 1) / 2, "uniform").pvalue > 1e-4
    h = np.bincount(picks, minlength=5)
    assert stats.chisquare(h).pvalue > 1e-4


def test_3d_rotation_distribution_and_norm():
    s = orc.OracleSystem(3, [20, 20, 20], inputs.cube(1.0))
    d, a = 0.1, 0.4
    s.set_moves(d, a, 4, 77)
    x0 = np.array([5.0, 5.0, 5.0])
    q0 = np.array([1.0, 0, 0, 0])
    vs = []
    for cell in range(6000):
        _, xn, qn = s.propose(3, 5, cell, 1, 1, x0, q0)
        assert abs(np.linalg.norm(qn) - 1.0) < 8e-16
        assert np.all(np.abs(xn - x0) <= d)
        vs.append(qn[1:] / qn[0])                 # = v, uniform in the cube
    vs = np.array(vs) / np.tan(a / 2)
    for ax in range(3):
        assert stats.kstest((vs[:, ax] + 1) / 2, "uniform").pvalue > 1e-4


def test_position_wrap_stays_in_box():
    s = _pent(10.0)
    s.set_moves(0.5, 0.1, 4, 3)
    for cell in range(2000):
        for x0 in ([0.0, 0.0], [10.0 - 1e-15, 9.99999], [1e-300, 5.0]):
            _, xn, _ = s.propose(1, 0, cell, 0, 1, np.array(x0), np.array([1.0, 0.0]))
            assert (xn >= 0).all() and (xn < 10.0).all()
