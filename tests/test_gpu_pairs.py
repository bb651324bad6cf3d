"""Pair-level parity of the overlap tests on the GPU.

For many random and near-contact pairs: the GPU's FP64 contract equals the
oracle's verdict on every pair (2D separating axes, 3D GJK), and the FP32
filter never contradicts it (it answers the same verdict or "uncertain", in
which case the sweep re-decides in FP64).  For 3D this also checks, on
near-contact pairs, the step of the certificate argument that is tested
rather than proved: FP64 GJK answers "separated" whenever the exact shapes
are certified apart by more than the band."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs
from tests import bruteforce as bf

pytestmark = pytest.mark.gpu

hpmc = pytest.importorskip("paper_1509_04692_gb300.hpmc")


def _quats(rng, n):
    q = rng.normal(size=(n, 4))
    return q / np.linalg.norm(q, axis=1)[:, None]


def _check(dim, v, D, qA, qB, max_uncertain):
    s = orc.OracleSystem(dim, [50.0] * dim, v)
    ref = s.overlap(D, qA, qB)
    o64, o32 = hpmc.pair_test(dim, v, D, qA, qB)
    assert np.array_equal(o64, ref), np.nonzero(o64 != ref)[0][:10]
    cert = o32 < 2
    assert np.array_equal(o32[cert], ref[cert]), np.nonzero(cert & (o32 != ref))[0][:10]
    assert (~cert).mean() <= max_uncertain, ((~cert).mean(), np.bincount(o32))
    return ref, o32


def test_pentagon_pairs_random_and_near_contact():
    rng = np.random.default_rng(1)
    v = inputs.regular_polygon(5, 0.5)
    n = 200000
    ang = rng.uniform(0, 2 * np.pi, n)
    r = 1.02 * np.sqrt(rng.uniform(0, 1, n))
    D = np.stack([r * np.cos(ang), r * np.sin(ang)], 1)
    ta, tb = rng.uniform(0, 2 * np.pi, n), rng.uniform(0, 2 * np.pi, n)
    zA = np.stack([np.cos(ta), np.sin(ta)], 1)
    zB = np.stack([np.cos(tb), np.sin(tb)], 1)
    ref, _ = _check(2, v, D, zA, zB, 1e-3)
    assert 0.2 < ref.mean() < 0.8
    # near contact: bisect to the contact distance, then +- 1e-9 .. 1e-4
    m = 20000
    u = np.stack([np.cos(ang[:m]), np.sin(ang[:m])], 1)
    lo, hi = np.zeros(m), np.full(m, 1.001)
    for _ in range(50):
        mid = 0.5 * (lo + hi)
        ov, _ = bf.classify_2d(v, u * mid[:, None], zA[:m], zB[:m], eps=0.0)
        lo, hi = np.where(ov, mid, lo), np.where(ov, hi, mid)
    off = rng.choice([-1, 1], m) * 10.0 ** rng.uniform(-9, -4, m)
    # offsets deliberately straddle the error bound: only non-contradiction
    # is asserted, plus certainty beyond a few bounds
    _, o32 = _check(2, v, u * (0.5 * (lo + hi) + off)[:, None], zA[:m], zB[:m], 1.0)
    far = np.abs(off) > 1e-5
    assert (o32[far] >= 2).mean() < 0.05


@pytest.mark.parametrize("shape", ["cube", "octahedron", "random12", "dodecahedron"])
def test_polyhedron_pairs_random_and_near_contact(shape):
    # cubes take the box test, octahedra and dodecahedra (origin interior)
    # the portal refinement with the GJK behind it, random12 the GJK
    rng = np.random.default_rng({"cube": 2, "octahedron": 3, "random12": 4, "dodecahedron": 5}[shape])
    if shape == "cube":
        v = inputs.cube(1.0)
    elif shape == "dodecahedron":
        v = inputs.dodecahedron(1.0)
    elif shape == "octahedron":
        v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float) * 0.6
    else:
        p = rng.normal(size=(12, 3))
        v = 0.5 * p / np.linalg.norm(p, axis=1)[:, None]
    R = np.sqrt((v ** 2).sum(1)).max()
    n = 100000
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    D = d * (2 * R * 1.02 * rng.uniform(0, 1, n) ** (1 / 3))[:, None]
    qA, qB = _quats(rng, n), _quats(rng, n)
    ref, _ = _check(3, v, D, qA, qB, 0.01)
    assert 0.1 < ref.mean() < 0.9
    # near contact along random directions (bisection on the oracle verdict)
    m = 20000
    s = orc.OracleSystem(3, [50.0] * 3, v)
    lo, hi = np.zeros(m), np.full(m, 2 * R * 1.001)
    for _ in range(45):
        mid = 0.5 * (lo + hi)
        ov = s.overlap(d[:m] * mid[:, None], qA[:m], qB[:m]).astype(bool)
        lo, hi = np.where(ov, mid, lo), np.where(ov, hi, mid)
    off = rng.choice([-1, 1], m) * 10.0 ** rng.uniform(-8, -3, m)
    _, o32 = _check(3, v, d[:m] * (0.5 * (lo + hi) + off)[:, None], qA[:m], qB[:m], 1.0)
    far = np.abs(off) > 5e-4
    assert (o32[far] >= 2).mean() < 0.05, np.bincount(o32[far])


def test_aligned_cubes_ties():
    # identical orientations: every support query ties; certificates still
    # decide, or the pair is left to FP64, never contradicting it
    rng = np.random.default_rng(5)
    v = inputs.cube(1.0)
    n = 50000
    D = rng.uniform(-1.6, 1.6, size=(n, 3))
    I = np.tile([1.0, 0, 0, 0], (n, 1))
    _check(3, v, D, I, I, 0.5)


def _polyhedron(name, rng):
    if name == "cube":
        return inputs.cube(1.0)
    if name == "octahedron":
        return np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float) * 0.6
    if name == "dodecahedron":
        return inputs.dodecahedron(1.0)
    p = rng.normal(size=(int(name[6:]), 3))                  # "random<n>": points on a sphere
    return 0.5 * p / np.linalg.norm(p, axis=1)[:, None]


@pytest.mark.parametrize("shape", ["cube", "octahedron", "random16", "dodecahedron", "random24", "random32"])
def test_warp_gjk_equals_the_contract(shape):
    # the FP64 GJK the FP32-filtered 3D sweep uses for its re-checks (one warp
    # per pair, lanes sharing the vertices, supports and faces) gives the
    # oracle's verdict after the same number of support evaluations
    rng = np.random.default_rng(sum(map(ord, shape)))
    v = _polyhedron(shape, rng)
    R = np.sqrt((v ** 2).sum(1)).max()
    s = orc.OracleSystem(3, [50.0] * 3, v)
    n = 40000
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    D = d * (2 * R * 1.02 * rng.uniform(0, 1, n) ** (1 / 3))[:, None]
    qA, qB = _quats(rng, n), _quats(rng, n)
    m = 10000                                       # the first m pairs moved to near contact
    lo, hi = np.zeros(m), np.full(m, 2 * R * 1.001)
    for _ in range(45):
        mid = 0.5 * (lo + hi)
        ov = s.overlap(d[:m] * mid[:, None], qA[:m], qB[:m]).astype(bool)
        lo, hi = np.where(ov, mid, lo), np.where(ov, hi, mid)
    off = rng.choice([-1, 1], m) * 10.0 ** rng.uniform(-12, -3, m)
    D[:m] = d[:m] * (0.5 * (lo + hi) + off)[:, None]
    ref, rit = s.overlap(D, qA, qB, iters=True)
    got, git = hpmc.pair_test_warp3d(v, D, qA, qB)
    assert np.array_equal(got, ref), np.nonzero(got != ref)[0][:10]
    assert np.array_equal(git, rit), np.nonzero(git != rit)[0][:10]
    assert 0.1 < ref.mean() < 0.9 and rit.max() >= 3


def test_warp_gjk_ties_and_spheres():
    # identical orientations make every support query tie (the first vertex
    # of the extremum must win, as in the one-lane scan); spheres take the
    # distance branch
    rng = np.random.default_rng(6)
    v = inputs.cube(1.0)
    n = 30000
    D = rng.uniform(-1.6, 1.6, size=(n, 3))
    D[: n // 3] = np.round(D[: n // 3] * 4) / 4                # exact ties of the dot products too
    I = np.tile([1.0, 0, 0, 0], (n, 1))
    s = orc.OracleSystem(3, [50.0] * 3, v)
    ref, rit = s.overlap(D, I, I, iters=True)
    got, git = hpmc.pair_test_warp3d(v, D, I, I)
    assert np.array_equal(got, ref) and np.array_equal(git, rit)
    sph = orc.OracleSystem(3, [50.0] * 3, 0.5)
    qA, qB = _quats(rng, n), _quats(rng, n)
    ref = sph.overlap(D, qA, qB)
    got, git = hpmc.pair_test_warp3d(np.array(0.5), D, qA, qB)
    assert np.array_equal(got, ref) and not git.any()


def _cuboid(hx, hy, hz):
    return np.array([[sx * hx, sy * hy, sz * hz] for sz in (-1, 1) for sy in (-1, 1) for sx in (-1, 1)], float)


@pytest.mark.parametrize("h", [(0.5, 0.5, 0.5), (0.7, 0.35, 0.2)])
def test_box_certificates_never_contradict_the_contract(h):
    # boxes take the FP32 separating-axis certificate in place of the FP32
    # GJK, and their FP32-uncertain pairs the FP64 one before the FP64 GJK:
    # every certified verdict equals the oracle's GJK, and the FP64 band of
    # uncertain pairs is far narrower than the FP32 one
    rng = np.random.default_rng(int(1000 * h[2]))
    v = _cuboid(*h)
    R = float(np.linalg.norm(h))
    s = orc.OracleSystem(3, [50.0] * 3, v)
    n = 60000
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    D = d * (2 * R * 1.02 * rng.uniform(0, 1, n) ** (1 / 3))[:, None]
    qA, qB = _quats(rng, n), _quats(rng, n)
    qB[:500] = qA[:500]                                    # parallel edges: degenerate crosses
    ref, o32 = _check(3, v, D, qA, qB, 0.005)
    assert 0.1 < ref.mean() < 0.9
    b64 = hpmc.pair_test_box64(v, D, qA, qB)
    cert = b64 < 2
    assert np.array_equal(b64[cert], ref[cert]), np.nonzero(cert & (b64 != ref))[0][:10]
    assert (~cert[500:]).mean() < 1e-3
    # near contact along random directions
    m = 20000
    lo, hi = np.zeros(m), np.full(m, 2 * R * 1.001)
    for _ in range(45):
        mid = 0.5 * (lo + hi)
        ov = s.overlap(d[:m] * mid[:, None], qA[:m], qB[:m]).astype(bool)
        lo, hi = np.where(ov, mid, lo), np.where(ov, hi, mid)
    # offsets log-uniform in [1e-10, 1e-2] (both signs) on the first half,
    # uniform in [-1e-3, 1e-3] on the second (the bands' widths compared)
    off = rng.choice([-1, 1], m) * 10.0 ** rng.uniform(-10, -2, m)
    off[m // 2:] = rng.uniform(-1e-3, 1e-3, m - m // 2)
    Dn = d[:m] * (0.5 * (lo + hi) + off)[:, None]
    ref, o32 = _check(3, v, Dn, qA[:m], qB[:m], 1.0)
    b64 = hpmc.pair_test_box64(v, Dn, qA[:m], qB[:m])
    cert = b64 < 2
    assert np.array_equal(b64[cert], ref[cert]), np.nonzero(cert & (b64 != ref))[0][:10]
    far = np.abs(off) > 1e-4
    far[:500] = False
    assert (o32[far] >= 2).mean() < 0.5 and (b64[far] == 2).mean() < 0.05, (
        (o32[far] >= 2).mean(), (b64[far] == 2).mean())
    lin = slice(m // 2, m)
    assert (b64[lin] == 2).sum() < 0.2 * (o32[lin] >= 2).sum(), ((b64[lin] == 2).sum(), (o32[lin] >= 2).sum())


def test_box64_rejects_other_shapes():
    rng = np.random.default_rng(8)
    D = rng.normal(size=(4, 3))
    q = _quats(rng, 4)
    with pytest.raises(hpmc.HPMCError):
        hpmc.pair_test_box64(_polyhedron("octahedron", rng), D, q, q)
