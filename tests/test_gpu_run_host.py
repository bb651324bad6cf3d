"""The end-to-end call with host buffers (hpmc_run_host) against the oracle:
replica batches in 2D and 3D, the state uploaded from interleaved host
arrays (replicas concatenated, tag order inside), swept, downloaded; two
calls in a row, the second continuing the sweep counter.  Positions,
orientations and counters bit for bit."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs

pytestmark = pytest.mark.gpu

hpmc = pytest.importorskip("paper_1509_04692_gb300.hpmc")


def _oracle(s, pos, ori, sweep0, n):
    o = orc.OracleSystem(s.dim, s.L, s.verts, w_min=s.w_min)
    o.set_moves(s.d, s.a, s.nselect, s.seed)
    p, q = pos.copy(), ori.copy()
    c = o.sweep(p, q, sweep0, n)
    return p, q, c


@pytest.mark.parametrize("dim", [2, 3])
def test_run_host_two_calls_match_the_oracle(dim):
    if dim == 2:
        systems = [inputs.pentagon_system(N, phi, sd, d=0.15, a=0.2) for N, phi, sd in
                   [(500, 0.55, 3), (1300, 0.45, 4)]]
    else:
        systems = [inputs.cube_system(N, phi, sd, d=0.1, a=0.2) for N, phi, sd in [(343, 0.45, 5), (512, 0.5, 6)]]
    b = hpmc.from_systems(systems)
    qd = 2 if dim == 2 else 4
    pos = np.concatenate([s.pos for s in systems])
    ori = np.concatenate([s.orient for s in systems])
    refs = [(s.pos.copy(), s.orient.copy()) for s in systems]
    sweep0 = 0
    for n in (7, 5):
        po, oo = np.zeros_like(pos), np.zeros_like(ori)
        c = b.run_host(pos, ori, n, po, oo)
        tot = np.zeros(3, dtype=np.int64)
        k = 0
        for r, s in enumerate(systems):
            p, q, cr = _oracle(s, refs[r][0], refs[r][1], sweep0, n)
            refs[r] = (p, q)
            assert np.array_equal(po[k:k + s.N], p) and np.array_equal(oo[k:k + s.N], q), (dim, r, n)
            k += s.N
            tot += np.array([int(x) for x in cr[:3]])
        # counters accumulate over the calls; compare this call's share
        if sweep0 == 0:
            first = np.array([c["accept"], c["reject_overlap"], c["reject_boundary"]])
            assert np.array_equal(first, tot)
        else:
            assert np.array_equal(np.array([c["accept"], c["reject_overlap"], c["reject_boundary"]]) - first, tot)
        assert po.shape == pos.shape and oo.shape[1] == qd
        pos, ori = po, oo
        sweep0 += n
    assert b.get_state(0)[2] == 12
    b.close()
