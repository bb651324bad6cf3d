"""NPT volume moves on the GPU: the sequence of accept / reject decisions,
the boxes and the trajectories equal the oracle's bit for bit (disks and
pentagons, including moves that change the cell grid), and hard disks at
the paper's validation pressure settle at its area fraction."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs

pytestmark = pytest.mark.gpu

hpmc = pytest.importorskip("paper_1509_04692_gb300.hpmc")


def _run_both(s, rounds, sweeps, moves, bP, dV, mode):
    o = orc.OracleSystem(s.dim, s.L, s.verts, w_min=s.w_min)
    o.set_moves(s.d, s.a, s.nselect, s.seed)
    p, q = s.pos.copy(), s.orient.copy()
    b = hpmc.from_system(s)
    b.set_precision(mode)
    acc_o, acc_g, sw, m = [], [], 0, 0
    nc_seen = set()
    for _ in range(rounds):
        o.sweep(p, q, sw, sweeps)
        b.sweep(sweeps, graph=True)
        sw += sweeps
        for _ in range(moves):
            acc_o.append(o.box_move(p, q, bP, dV, m))
            acc_g.append(int(b.box_move(bP, dV)))
            m += 1
            nc_seen.add(int(o.geometry()["nc"][0]))
    gp, gq, gsw = b.get_state()
    box = b.box()
    b.close()
    return acc_o, acc_g, (p, q, o.box), (gp, gq, box), nc_seen


@pytest.mark.parametrize("mode", [0, 1])
def test_disks_npt_bit_exact(mode):
    # w_min just below L / 24: the first compression drops the grid to 22 cells
    s = inputs.disk_system(512, 0.60, 21, d=0.12, w_min=1.0782)
    acc_o, acc_g, ref, got, nc_seen = _run_both(s, 30, 2, 4, 30.0, 0.4, mode)
    assert acc_g == acc_o
    assert 0 < sum(acc_o) < len(acc_o)
    assert len(nc_seen) > 1                          # the cell grid changed along the way
    assert np.array_equal(got[2], ref[2])
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_pentagons_npt_bit_exact():
    s = inputs.pentagon_system(400, 0.55, 22, d=0.1, a=0.2)
    acc_o, acc_g, ref, got, _ = _run_both(s, 20, 2, 3, 12.0, 0.3, 1)
    assert acc_g == acc_o and 0 < sum(acc_o)
    assert np.array_equal(got[2], ref[2])
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_disks_at_the_validation_pressure_settle_at_its_density():
    # NVT at area fraction 0.698 has P* = 9.1707 (Sec. 4); NPT at that
    # pressure must give back area fraction 0.698 on average
    s = inputs.disk_system(4096, 0.698, 23, d=0.14, w_min=1.0)
    b = hpmc.from_system(s)
    b.sweep(5000, graph=True)
    area = math.pi * 0.25
    phis = []
    for k in range(12000):
        b.sweep(1, graph=True)
        b.box_move(9.1707, 1.0)
        if k >= 4000 and k % 10 == 0:
            L = b.box()
            phis.append(s.N * area / (L[0] * L[1]))
    phis = np.array(phis)
    assert abs(phis.mean() - 0.698) < 0.004, (phis.mean(), phis.std())
    assert b.check_overlaps() == 0
    b.close()
