"""Bit-exact parity at the states the benchmark times.

The benchmark times its systems after long melts from lattice starts, in the
launch configuration the autotuner picks.  Here the GPU runs exactly that
(graph-replayed melt, autotune, then graph-replayed sweeps in the tuned
configuration), in both precision forms, and the oracle runs the same whole
trajectory from the same seeded start on the host's cores (its threaded set
sweep, byte-identical to the serial one).  Positions, orientations and the
accept / reject counters must agree bit for bit after the compared sweeps.
The oracle never takes a GPU state as input: both sides start from the
seeded lattice.

Systems and lengths (the benchmark's melts):
  * 2^24 pentagons at area fraction 0.60, 2048^2 cells: 200-sweep melt + 2;
  * 32768 cubes and 32000 dodecahedra at volume fraction 0.50: 1000 + 50;
  * 512 replicas (N ~ U{256..8192}, phi ~ U[0.40, 0.70]): 1000 + 20, sampled
    replicas compared;
  * 32 cube replicas (N ~ U{2048..16384}, phi ~ U[0.40, 0.55]): 1000 + 20,
    sampled replicas compared, both forms.
"""
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs

pytestmark = pytest.mark.gpu

hpmc = pytest.importorskip("paper_1509_04692_gb300.hpmc")
F64, F32 = 0, 1
THREADS = max(1, os.cpu_count() or 1)


def _oracle(s, n):
    o = orc.OracleSystem(s.dim, s.L, s.verts, w_min=s.w_min)
    o.set_moves(s.d, s.a, s.nselect, s.seed)
    o.set_threads(THREADS)
    p, q = s.pos.copy(), s.orient.copy()
    c = o.sweep(p, q, 0, n)
    return p, q, tuple(int(x) for x in c[:3])


def _gpu_as_timed(make, mode, melt, n, n_tune):
    """The benchmark's sequence: melt, autotune (state restored), then n
    sweeps in the tuned configuration.  Returns the batch and the tuned
    (lanes per cell, warps per block)."""
    b = make()
    b.set_precision(mode)
    b.sweep(melt, graph=True)
    lanes, warps = b.autotune(n_tune)
    b.sweep(n, graph=True)
    return b, (lanes, warps)


def _counters3(c):
    return (c["accept"], c["reject_overlap"], c["reject_boundary"])


def _same(gp, gq, p, q, what):
    bad = np.nonzero(np.any(gp != p, axis=1) | np.any(gq != q, axis=1))[0]
    assert bad.size == 0, f"{what}: {bad.size} particles differ, first {bad[:5]}"


@pytest.mark.parametrize("name, make, melt, n, n_tune", [
    ("cubes32768", inputs.cubes32768, 1000, 50, 4),
    ("dodecahedra32000", inputs.dodecahedra32000, 1000, 50, 4),
])
def test_3d_melted_state_both_forms(name, make, melt, n, n_tune):
    s = make(42)
    got = {}
    for mode in (F32, F64):
        b, cfg = _gpu_as_timed(lambda: hpmc.from_system(s), mode, melt, n, n_tune)
        c = b.counters()
        p, q, sw = b.get_state()
        assert sw == melt + n
        assert b.check_overlaps() == 0
        got[mode] = (p, q, _counters3(c), cfg, c)
        b.close()
    rp, rq, rc = _oracle(s, melt + n)
    for mode in (F32, F64):
        p, q, c3, cfg, c = got[mode]
        assert c3 == rc, (name, mode, cfg, c3, rc)
        _same(p, q, rp, rq, f"{name} mode {mode} config {cfg}")
    # the compared stretch is a melted fluid, and the filter was exercised
    assert 0.2 < rc[0] / sum(rc) < 0.45
    assert got[F32][4]["fp64_rechecks"] > 0


def test_large2d_melted_state_both_forms():
    s = inputs.large2d(42)
    melt, n = 200, 2
    got = {}
    for mode in (F32, F64):
        b, cfg = _gpu_as_timed(lambda: hpmc.from_system(s), mode, melt, n, 2)
        c = b.counters()
        p, q, sw = b.get_state()
        assert sw == melt + n
        got[mode] = (p, q, _counters3(c), cfg)
        b.close()
    rp, rq, rc = _oracle(s, melt + n)
    for mode in (F32, F64):
        p, q, c3, cfg = got[mode]
        assert c3 == rc, (mode, cfg, c3, rc)
        _same(p, q, rp, rq, f"2^24 pentagons mode {mode} config {cfg}")


def test_replica_batch_melted_state_sampled():
    systems = inputs.replica_systems(512)
    melt, n = 1000, 20
    b, cfg = _gpu_as_timed(lambda: hpmc.from_systems(systems), F32, melt, n, 8)
    Ns = np.array([x.N for x in systems])
    phis = np.array([x.phi for x in systems])
    sample = sorted({0, 511, int(Ns.argmax()), int(phis.argmax())})
    for r in sample:
        s = systems[r]
        p, q, rc = _oracle(s, melt + n)
        gp, gq, sw = b.get_state(r)
        assert sw == melt + n
        assert _counters3(b.counters(r)) == rc, (r, cfg)
        _same(gp, gq, p, q, f"replica {r} config {cfg}")
    b.close()


def test_cube_replica_batch_melted_state_sampled_both_forms():
    systems = inputs.cube_replica_systems()
    melt, n = 1000, 20
    Ns = np.array([x.N for x in systems])
    phis = np.array([x.phi for x in systems])
    sample = sorted({0, 31, int(Ns.argmax()), int(phis.argmax())})
    refs = {r: _oracle(systems[r], melt + n) for r in sample}
    for mode in (F32, F64):
        b, cfg = _gpu_as_timed(lambda: hpmc.from_systems(systems), mode, melt, n, 4)
        for r in sample:
            p, q, rc = refs[r]
            gp, gq, sw = b.get_state(r)
            assert sw == melt + n
            assert _counters3(b.counters(r)) == rc, (r, mode, cfg)
            _same(gp, gq, p, q, f"cube replica {r} mode {mode} config {cfg}")
        b.close()
