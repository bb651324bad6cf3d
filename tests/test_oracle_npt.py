"""Oracle pins for the isotropic volume move (NPT).

An ideal gas (point-like disks) at fixed beta P has the volume law
P(V) ~ V^N exp(-beta P V) for uniform proposals in V, a Gamma(N + 1,
beta P) law: mean (N + 1) / (beta P), variance (N + 1) / (beta P)^2.  Hard
particles: a compression that would create an overlap is never accepted."""
import math

import numpy as np

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs


def test_ideal_gas_volume_law():
    N, bP = 4, 0.02
    L0 = math.sqrt((N + 1) / bP)
    o = orc.OracleSystem(2, [L0, L0], radius=1e-4)
    o.set_moves(0.1, 0.0, 1, 99)
    pos = np.random.default_rng(1).uniform(0, L0, (N, 2))
    ori = np.tile([1.0, 0.0], (N, 1))
    V = []
    for m in range(40000):
        o.box_move(pos, ori, bP, 150.0, m)
        if m >= 2000:
            L = o.box
            V.append(L[0] * L[1])
    V = np.array(V)
    # correlated chain: compare with generous but discriminating tolerances
    assert abs(V.mean() - (N + 1) / bP) < 0.05 * (N + 1) / bP
    assert abs(V.var() / ((N + 1) / bP ** 2) - 1.0) < 0.15
    assert np.all(pos >= 0.0) and np.all(pos < o.box)


def test_hard_disk_compression_never_overlaps():
    s = inputs.disk_system(300, 0.60, 4, d=0.1)
    o = orc.OracleSystem(2, s.L, s.verts)
    o.set_moves(0.1, 0.0, 4, 5)
    pos, ori = s.pos.copy(), s.orient.copy()
    acc = 0
    for m in range(60):
        o.sweep(pos, ori, m, 2)
        acc += o.box_move(pos, ori, 8.0, 2.0, m)             # above the fluid pressure: compressions tried
        L = o.box
        D = pos[:, None, :] - pos[None, :, :]
        D -= L * np.round(D / L)
        r2 = (D ** 2).sum(-1) + np.eye(len(pos)) * 10
        assert r2.min() > 1.0
    assert 0 < acc < 60
