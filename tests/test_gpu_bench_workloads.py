"""The benchmark workloads at their full sizes, in the launch configurations
the benchmark times: the 4096-pentagon fluid (graph-replayed melt, the
autotuner's trial runs, then the latency-regime configuration of 32 lanes
per cell in one-warp blocks) against the oracle's whole trajectory, and the
batch of 512 independent replicas (about 2.2 million particles) against
oracle runs of sampled replicas, each replica being its own chain."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs

pytestmark = pytest.mark.gpu

hpmc = pytest.importorskip("paper_1509_04692_gb300.hpmc")
F32 = 1


def _oracle_run(s, n):
    o = orc.OracleSystem(s.dim, s.L, s.verts, w_min=s.w_min)
    o.set_moves(s.d, s.a, s.nselect, s.seed)
    p, q = s.pos.copy(), s.orient.copy()
    rc = o.sweep(p, q, 0, n)
    return p, q, tuple(int(x) for x in rc[:3])


def _same(gp, gq, p, q):
    bad = np.nonzero(np.any(gp != p, axis=1) | np.any(gq != q, axis=1))[0]
    assert bad.size == 0, f"{bad.size} particles differ, first {bad[:5]}"


def test_fluid4096_as_timed():
    s = inputs.fluid4096(42)
    b = hpmc.from_system(s)
    b.set_precision(F32)
    b.sweep(1000, graph=True)                       # the melt
    b.autotune(8)                                   # trial runs; state restored
    assert b.get_state()[2] == 1000
    b.set_group_size(32, 1)
    b.sweep(200, graph=True)                        # one timed step
    c = b.counters()
    gp, gq, sw = b.get_state()
    b.close()
    p, q, rc = _oracle_run(s, 1200)
    assert sw == 1200
    assert (c["accept"], c["reject_overlap"], c["reject_boundary"]) == rc
    _same(gp, gq, p, q)
    assert 0.2 < c["accept"] / c["moves"] < 0.4


def test_replica_batch_512_sampled():
    systems = inputs.replica_systems(512)
    b = hpmc.from_systems(systems)
    b.set_precision(F32)
    b.sweep(20, graph=True)                         # the melt
    b.autotune(8)
    b.sweep(4, graph=True)                          # the autotuner's choice
    b.set_group_size(1, 4)
    b.sweep(2, graph=True)                          # the profiled configuration
    b.sweep(1)                                      # and one direct launch sequence
    Ns = np.array([x.N for x in systems])
    phis = np.array([x.phi for x in systems])
    sample = sorted({0, 1, 255, 511, int(Ns.argmin()), int(Ns.argmax()), int(phis.argmin()),
                     int(phis.argmax())})
    for r in sample:
        s = systems[r]
        p, q, rc = _oracle_run(s, 27)
        c = b.counters(r)
        gp, gq, sw = b.get_state(r)
        assert sw == 27
        assert (c["accept"], c["reject_overlap"], c["reject_boundary"]) == rc, r
        _same(gp, gq, p, q)
    # every replica moved, none overlaps (FP64 contract predicate on the device)
    for r in range(0, 512, 37):
        assert b.counters(r)["accept"] > 0
        assert b.check_overlaps(r) == 0
    b.close()
