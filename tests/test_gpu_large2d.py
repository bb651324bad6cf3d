"""Full-size parity of the large 2D system: 2^24 pentagons at area fraction
0.60 on a 2048 x 2048 cell list, FP32-filtered form, graph-replayed sweeps in
the autotuned launch configuration.  The oracle finishes one sweep of this
system in seconds, so whole trajectories are compared, not samples."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs

pytestmark = pytest.mark.gpu

hpmc = pytest.importorskip("paper_1509_04692_gb300.hpmc")


def test_large2d_two_sweeps_bit_exact():
    s = inputs.large2d(42)
    assert s.N == 1 << 24
    g = orc.OracleSystem(2, s.L, s.verts, w_min=s.w_min).geometry()
    assert tuple(g["nc"][:2]) == (2048, 2048)
    b = hpmc.from_system(s)
    b.set_precision(hpmc.HPMC_FP32_FILTERED)
    lanes, warps = b.autotune(2)              # restores state and counters
    b.reset_counters()
    b.sweep(2, graph=True)
    b.sync()
    c = b.counters()
    p, o, sw = b.get_state()
    assert sw == 2
    assert b.check_overlaps() == 0

    ref = orc.OracleSystem(2, s.L, s.verts, w_min=s.w_min)
    ref.set_moves(s.d, s.a, s.nselect, s.seed)
    rp, ro = s.pos.copy(), s.orient.copy()
    rc = ref.sweep(rp, ro, 0, 2)
    assert (c["accept"], c["reject_overlap"], c["reject_boundary"]) == tuple(int(x) for x in rc[:3]), \
        (c, rc, lanes, warps)
    assert c["moves"] == int(rc[0] + rc[1] + rc[2])
    diff = np.nonzero(np.any(p != rp, axis=1) | np.any(o != ro, axis=1))[0]
    assert diff.size == 0, (diff[:10], diff.size)
    b.close()
