"""Oracle pins for the isotropic volume move (NPT).

An ideal gas (point-like disks) at fixed beta P has the volume law
P(V) ~ V^N exp(-beta P V) for uniform proposals in V, a Gamma(N + 1,
beta P) law: mean (N + 1) / (beta P), variance (N + 1) / (beta P)^2.  Hard
particles: a compression that would create an overlap is never accepted."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs


@pytest.mark.parametrize("dim", [2, 3])
def test_ideal_gas_volume_law(dim):
    # the scale factor is the d-th root of the volume ratio; the law is the
    # same in 2D and 3D
    N, bP = 4, 0.02
    L0 = ((N + 1) / bP) ** (1.0 / dim)
    o = orc.OracleSystem(dim, [L0] * dim, radius=1e-4)
    o.set_moves(0.1, 0.0, 1, 99)
    pos = np.random.default_rng(1).uniform(0, L0, (N, dim))
    ori = np.tile([1.0, 0.0] if dim == 2 else [1.0, 0.0, 0.0, 0.0], (N, 1))
    V = []
    for m in range(40000):
        o.box_move(pos, ori, bP, 150.0, m)
        if m >= 2000:
            V.append(float(np.prod(o.box)))
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


@pytest.mark.parametrize("dim", [2, 3])
def test_volume_move_scales_isotropically(dim):
    # an accepted move multiplies every box length by the same factor and
    # keeps every particle's fractional coordinates; a rejected one changes
    # nothing
    N = 6
    L0 = np.array([12.0, 15.0, 18.0][:dim])
    o = orc.OracleSystem(dim, L0, radius=1e-4)
    o.set_moves(0.1, 0.0, 1, 7)
    pos = np.random.default_rng(2).uniform(0, 1, (N, dim)) * L0
    ori = np.tile([1.0, 0.0] if dim == 2 else [1.0, 0.0, 0.0, 0.0], (N, 1))
    seen = [0, 0]
    for m in range(200):
        L, p = o.box.copy(), pos.copy()
        acc = o.box_move(pos, ori, 0.05, 40.0, m)
        seen[int(acc)] += 1
        if acc:
            f = o.box / L
            assert np.allclose(f, f[0], rtol=1e-15, atol=0)
            assert np.allclose(pos / o.box, p / L, rtol=0, atol=1e-14)
            assert np.all((pos >= 0) & (pos < o.box))
        else:
            assert np.array_equal(o.box, L) and np.array_equal(pos, p)
    assert seen[0] > 10 and seen[1] > 10
