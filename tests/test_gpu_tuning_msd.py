"""Move-size tuning in the library and the mean squared displacement (the
paper's efficiency measure).  The tuner takes the same pilots as the host
bisection in tune.py and leaves the trajectory untouched; the MSD equals
the unwrapped displacement of the oracle's own trajectory."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs, tune

pytestmark = pytest.mark.gpu

hpmc = pytest.importorskip("paper_1509_04692_gb300.hpmc")


def test_tuner_matches_host_bisection_and_restores_state():
    s = inputs.pentagon_system(1024, 0.55, 31, d=0.1, a=0.1)
    b = hpmc.from_system(s)
    b.sweep(50)
    p0, q0, sw0 = b.get_state()
    c0 = b.counters()

    def pilot(d, a):
        b.set_state(p0, q0, sw0)
        b.set_moves(d, a, 4)
        b.reset_counters()
        b.sweep(20)
        c = b.counters()
        return c["accept"] / c["moves"]
    ref = tune.tune_scale(pilot, 0.1, 0.1, 0.30, lo=0.25, hi=8.0, iters=8)
    b.close()

    b = hpmc.from_system(s)
    b.sweep(50)
    got = b.tune_moves(0.30, 20, 8, 0.25, 8.0)
    assert got == pytest.approx(ref, rel=0, abs=0)
    assert b.counters() == c0                                # counters restored
    p1, q1, sw1 = b.get_state()
    assert sw1 == sw0 and np.array_equal(p1, p0) and np.array_equal(q1, q0)
    # the run continues exactly as one given the tuned moves directly
    b.sweep(10)
    b2 = hpmc.from_system(s)
    b2.sweep(50)
    b2.set_moves(got[0], got[1], 4)
    b2.sweep(10)
    assert np.array_equal(b.get_state()[0], b2.get_state()[0])
    b.close()
    b2.close()


def _min_image(d, L):
    d = d.copy()
    h = 0.5 * L
    d = np.where(d > h, d - L, d)
    return np.where(d < -h, d + L, d)


@pytest.mark.parametrize("shape", ["pentagons", "disks"])
def test_msd_equals_the_oracle_trajectory(shape):
    s = (inputs.pentagon_system(900, 0.45, 32, d=0.2, a=0.3) if shape == "pentagons"
         else inputs.disk_system(900, 0.45, 33, d=0.25))
    o = orc.OracleSystem(2, s.L, s.verts, w_min=s.w_min)
    o.set_moves(s.d, s.a, s.nselect, s.seed)
    p, q = s.pos.copy(), s.orient.copy()
    acc = np.zeros_like(p)
    last = p.copy()
    b = hpmc.from_system(s)
    b.msd_reset()
    for k in range(30):
        o.sweep(p, q, 2 * k, 2)
        acc += _min_image(p - last, s.L)
        last = p.copy()
        b.sweep(2)
        b.msd_update()
    ref = (acc ** 2).sum(1).mean()
    got = b.msd()
    assert ref > 0.1
    assert abs(got - ref) < 1e-12 * ref
    b.close()
