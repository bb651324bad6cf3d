"""Host logic of the 3D shape classification (CPU).

The FP32 filter of the 3D kernels takes the separating-axis test for boxes,
the portal refinement for polyhedra whose local origin is interior, and the
symmetric support query for centrally symmetric polyhedra, whose FP32 vertex
copies it reorders into pairs.  `tests/shape_host.cpp` runs the library's
host code (`build_shapes`, the box margins) on vertex lists given here; this
test checks each classification against what the geometry fixes, that the
reordered FP32 copies are still the vertices' casts, and that the box
margins sit between their floors and a small fraction of the size."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1509_04692_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1509_04692_gb300", "csrc")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "vector_types.h")):
            return os.path.join(d, "include")
    nvcc = shutil.which("nvcc")
    if nvcc:
        d = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
        if os.path.exists(os.path.join(d, "vector_types.h")):
            return d
    return None


@pytest.fixture(scope="module")
def prog(tmp_path_factory):
    inc = _cuda_include()
    cxx = shutil.which("g++")
    if inc is None or cxx is None:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("shape") / "shape_host")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, "-I", inc, os.path.join(HERE, "shape_host.cpp"), "-o",
                    exe], check=True, capture_output=True)
    return exe


def _run(exe, v, dim=3):
    v = np.asarray(v, dtype=np.float64).reshape(-1, dim)
    txt = f"{dim} {len(v)}\n" + "\n".join(" ".join(repr(float(x)) for x in row) for row in v) + "\n"
    out = subprocess.run([exe], input=txt, capture_output=True, text=True, check=True).stdout.split()
    res = {}
    for kv in out:
        k, _, val = kv.partition("=")
        res[k] = val
    return res


def _cuboid(hx, hy, hz):
    return [[sx * hx, sy * hy, sz * hz] for sz in (-1, 1) for sy in (-1, 1) for sx in (-1, 1)]


def _tetra(shift=0.0):
    t = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float) * 0.5
    return t + shift


def test_boxes(prog):
    r = _run(prog, inputs.cube(1.0))
    assert (r["rc"], r["box"], r["sym"], r["mpr"], r["perm"], r["pairs"]) == ("0", "1", "1", "1", "1", "1")
    assert r["bh"] == "0.5,0.5,0.5"
    c = _run(prog, _cuboid(0.7, 0.35, 0.2))
    assert (c["box"], c["sym"]) == ("1", "1")
    assert [float(x) for x in c["bh"].split(",")] == pytest.approx([0.7, 0.35, 0.2], rel=1e-7)
    # vertex order does not matter; the sign patterns do
    v = np.array(_cuboid(0.7, 0.35, 0.2))[[5, 2, 7, 0, 3, 6, 1, 4]]
    assert _run(prog, v)["box"] == "1"


def test_box_margins(prog):
    for v in (inputs.cube(1.0), _cuboid(0.7, 0.35, 0.2)):
        r = _run(prog, v)
        sep32, ov32, sep64, ov64 = (float(r[k]) for k in ("sep32", "ov32", "sep64", "ov64"))
        # FP32: above the separation floor 4e-6 (of 2R) and the overlap band
        # tau = 1e-9, below a small fraction of the size; overlap wider
        assert 4e-6 < sep32 < 2e-4 and 1e-9 < ov32 < 5e-4 and ov32 > sep32
        # FP64: the floors themselves to within the FP64 rounding terms
        assert sep64 == pytest.approx(4e-6, rel=1e-3)
        assert ov64 == pytest.approx(1e-9, rel=0.1)


def test_not_boxes(prog):
    v = np.array(inputs.cube(1.0))
    v[3] *= 1.01                                       # one vertex off the box
    r = _run(prog, v)
    assert (r["rc"], r["box"], r["sym"]) == ("0", "0", "0")
    r = _run(prog, _cuboid(0.5, 0.5, 0.5)[:4] + [[0.6, 0.6, 0.6]] + _cuboid(0.5, 0.5, 0.5)[5:])
    assert r["box"] == "0"


def test_central_symmetry_and_pairs(prog):
    octa = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float) * 0.6
    for v in (inputs.dodecahedron(1.0), octa):
        r = _run(prog, v)
        assert (r["box"], r["sym"], r["mpr"], r["perm"], r["pairs"]) == ("0", "1", "1", "1", "1")
    rng = np.random.default_rng(4)
    p = rng.normal(size=(12, 3))
    r = _run(prog, 0.5 * p / np.linalg.norm(p, axis=1)[:, None])
    assert (r["sym"], r["perm"]) == ("0", "1")
    # a symmetric set given in scrambled order is reordered into pairs
    d = np.asarray(inputs.dodecahedron(1.0))[rng.permutation(20)]
    r = _run(prog, d)
    assert (r["sym"], r["perm"], r["pairs"]) == ("1", "1", "1")


def test_interior_origin(prog):
    assert _run(prog, _tetra())["mpr"] == "1"
    assert _run(prog, _tetra())["sym"] == "0"
    # origin outside the hull (the tetrahedron moved off it): no portal search
    assert _run(prog, _tetra(np.array([2.0, 0.0, 0.0])))["mpr"] == "0"
    # origin on a face (the centroid of vertices 1-3 moved to it): not interior
    t = _tetra()
    assert _run(prog, t - (t[1] + t[2] + t[3]) / 3.0)["mpr"] == "0"


# ---- the FP32 box test's error bound, checked numerically
#
# The separating-axis test of two boxes (box32_sat) evaluates, in FP32 from
# the FP32-cast inputs, s(n) = |l.n| - sum_k h_k |n_k| - extent_B(n) on 15
# axes n; its certificate needs |s(n) - s*(n)| <= E_sep, s* the same value
# for the exact boxes along the same n, and |s*(n) - s*(n*)| <= E_ov - E_sep
# for the exact axis n* the FP32 axis stands for.  Here the FP32 arithmetic
# is emulated in numpy (float32 operations; a fused multiply-add as the
# float64 sum of the exact float32 product, rounded once more to float32,
# which is within the same one-rounding bound), the exact values in float64,
# and the largest errors over many random pairs are compared with E_sep and
# E_ov as the library derives them (printed relative to 2R by shape_host).

F = np.float32


def _fma(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F)


def _box_axes_fp32(h32, d32, qa32, qb32):
    a0, a1, a2, a3 = qa32[:, 0], -qa32[:, 1], -qa32[:, 2], -qa32[:, 3]
    b0, b1, b2, b3 = qb32[:, 0], qb32[:, 1], qb32[:, 2], qb32[:, 3]
    w = ((a0 * b0 - a1 * b1) - a2 * b2) - a3 * b3
    x = ((a0 * b1 + a1 * b0) + a2 * b3) - a3 * b2
    y = ((a0 * b2 - a1 * b3) + a2 * b0) + a3 * b1
    z = ((a0 * b3 + a1 * b2) - a2 * b1) + a3 * b0
    dx, dy, dz = d32[:, 0], d32[:, 1], d32[:, 2]
    two = F(2.0)
    tx = two * _fma(a2, dz, -(a3 * dy))
    ty = two * _fma(a3, dx, -(a1 * dz))
    tz = two * _fma(a1, dy, -(a2 * dx))
    l = [_fma(a0, tx, dx) + _fma(a2, tz, -(a3 * ty)), _fma(a0, ty, dy) + _fma(a3, tx, -(a1 * tz)),
         _fma(a0, tz, dz) + _fma(a1, ty, -(a2 * tx))]
    one = F(1.0)
    M = [[None] * 3 for _ in range(3)]
    M[0][0] = one - two * _fma(y, y, z * z)
    M[1][1] = one - two * _fma(x, x, z * z)
    M[2][2] = one - two * _fma(x, x, y * y)
    M[1][0] = two * _fma(x, y, w * z)
    M[0][1] = two * _fma(x, y, -(w * z))
    M[2][0] = two * _fma(x, z, -(w * y))
    M[0][2] = two * _fma(x, z, w * y)
    M[2][1] = two * _fma(y, z, w * x)
    M[1][2] = two * _fma(y, z, -(w * x))
    A = [[np.abs(M[k][j]) for j in range(3)] for k in range(3)]
    h = [F(v) for v in h32]
    s, axes = [], []
    for k in range(3):
        eb = _fma(np.full_like(dx, h[2]), A[k][2], _fma(np.full_like(dx, h[1]), A[k][1], h[0] * A[k][0]))
        s.append((np.abs(l[k]) - h[k]) - eb)
        n = np.zeros((len(dx), 3))
        n[:, k] = 1.0
        axes.append(("e", k, None, n))
    for j in range(3):
        c = _fma(l[2], M[2][j], _fma(l[1], M[1][j], l[0] * M[0][j]))
        ea = _fma(np.full_like(dx, h[2]), A[2][j], _fma(np.full_like(dx, h[1]), A[1][j], h[0] * A[0][j]))
        s.append((np.abs(c) - ea) - h[j])
        axes.append(("u", None, j, np.stack([M[0][j], M[1][j], M[2][j]], 1).astype(np.float64)))
    for i in range(3):
        i1, i2 = (i + 1) % 3, (i + 2) % 3
        for j in range(3):
            j1, j2 = (j + 1) % 3, (j + 2) % 3
            c = _fma(l[i2], M[i1][j], -(l[i1] * M[i2][j]))
            ea = _fma(np.full_like(dx, h[i1]), A[i2][j], h[i2] * A[i1][j])
            eb = _fma(np.full_like(dx, h[j1]), A[i][j2], h[j2] * A[i][j1])
            s.append((np.abs(c) - ea) - eb)
            n = np.zeros((len(dx), 3))
            n[:, i1] = -M[i2][j]
            n[:, i2] = M[i1][j]
            axes.append(("x", i, j, n))
    return np.stack(s, 1).astype(np.float64), axes


def _rot64(q):
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.empty((len(q), 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 1, 2] = 2 * (y * z - w * x)
    return R


def _s_exact(h, l, U, n):
    # |l.n| - sum_k h_k |n_k| - sum_m h_m |n.u_m| for the exact boxes
    c = np.abs(np.einsum("pi,pi->p", l, n))
    ea = (np.abs(n) * h).sum(1)
    eb = sum(h[m] * np.abs(np.einsum("pi,pi->p", n, U[:, :, m])) for m in range(3))
    return c - ea - eb


@pytest.mark.parametrize("hh", [(0.5, 0.5, 0.5), (0.7, 0.35, 0.2)])
def test_box_test_errors_within_its_margins(prog, hh):
    h = np.array(hh)
    R = float(np.linalg.norm(h))
    r = _run(prog, _cuboid(*hh))
    e_sep = (float(r["sep32"]) - 4e-6 * 1.0001) / 2            # E_sep / 2R
    e_ov = (float(r["ov32"]) - 1e-9 * 1.0001) / 2              # E_ov / 2R
    rng = np.random.default_rng(11)
    n = 200000
    qa = rng.normal(size=(n, 4))
    qa /= np.linalg.norm(qa, axis=1)[:, None]
    qb = rng.normal(size=(n, 4))
    qb /= np.linalg.norm(qb, axis=1)[:, None]
    d = rng.normal(size=(n, 3))
    d *= (2 * R * rng.uniform(0, 1, n) ** (1 / 3) / np.linalg.norm(d, axis=1))[:, None]
    s32, axes = _box_axes_fp32(h.astype(F), d.astype(F), qa.astype(F), qb.astype(F))
    # exact: l* = R(qA)^T D, B's axes u*_m = columns of R(qA)^T R(qB)
    RA, RB = _rot64(qa), _rot64(qb)
    l = np.einsum("pki,pk->pi", RA, d)
    U = np.einsum("pki,pkj->pij", RA, RB)
    err_sep, err_axis = 0.0, 0.0
    for a, (kind, i, j, nv) in enumerate(axes):
        se = _s_exact(h, l, U, nv)
        err_sep = max(err_sep, float(np.max(np.abs(s32[:, a] - se))))
        if kind == "e":
            nstar = nv
        elif kind == "u":
            nstar = U[:, :, j]
        else:
            e = np.zeros(3)
            e[i] = 1.0
            nstar = np.cross(np.broadcast_to(e, U[:, :, j].shape), U[:, :, j])
        err_axis = max(err_axis, float(np.max(np.abs(se - _s_exact(h, l, U, nstar)))))
    assert err_sep / (2 * R) < e_sep, (err_sep / (2 * R), e_sep)
    assert err_axis / (2 * R) < e_ov - e_sep, (err_axis / (2 * R), e_ov - e_sep)
    # the bounds are not vacuous: the worst errors seen are within two
    # orders of magnitude of them
    assert err_sep / (2 * R) > e_sep / 300


# ---- the FP32 separating-axis test of polygons, checked the same way
#
# sat32 evaluates, in FP32 from FP32 casts, each axis' gap max(lo - a_hi,
# a_lo - hi) of the two halves (A's edge normals with B in A's frame, then
# B's with A in B's frame); its certificate needs |gap32 - gap64| <= E / 2,
# gap64 the FP64 contract's value (sat2_margin returns twice the sum of the
# FP32 and FP64 error bounds).


def _sat_gaps(dtype, fma, V, D, cA, sA, cB, sB):
    """Every axis gap of both halves (pairs x 2 nv), with the FP32 filter's
    operations (fma given) or the FP64 contract's (fma None)."""
    nv = len(V)
    vx, vy = V[:, 0].astype(np.float64), V[:, 1].astype(np.float64)
    nx = np.roll(vy, -1) - vy
    ny = vx - np.roll(vx, -1)
    t = nx[:, None] * vx[None, :] + ny[:, None] * vy[None, :]
    alo, ahi = t.min(1), t.max(1)
    c = lambda a: np.asarray(a, dtype=dtype)                       # noqa: E731
    fvx, fvy, fnx, fny, falo, fahi = map(c, (vx, vy, nx, ny, alo, ahi))
    dx, dy = c(D[:, 0]), c(D[:, 1])
    cA, sA, cB, sB = map(c, (cA, sA, cB, sB))
    if fma:
        cr = fma(cA, cB, sA * sB)
        sr = fma(cA, sB, -(sA * cB))
        lx, ly = fma(cA, dx, sA * dy), fma(cA, dy, -(sA * dx))
        mx, my = fma(cB, dx, sB * dy), fma(cB, dy, -(sB * dx))
    else:
        cr, sr = cA * cB + sA * sB, cA * sB - sA * cB
        lx, ly = cA * dx + sA * dy, cA * dy - sA * dx
        mx, my = cB * dx + sB * dy, cB * dy - sB * dx
    gaps = []
    for (r_c, r_s, ox, oy) in ((cr, sr, lx, ly), (cr, -sr, -mx, -my)):
        if fma:
            px = [fma(r_c, np.full_like(dx, fvx[i]), fma(-r_s, np.full_like(dx, fvy[i]), ox)) for i in range(nv)]
            py = [fma(r_s, np.full_like(dx, fvx[i]), fma(r_c, np.full_like(dx, fvy[i]), oy)) for i in range(nv)]
        else:
            px = [(r_c * fvx[i] - r_s * fvy[i]) + ox for i in range(nv)]
            py = [(r_s * fvx[i] + r_c * fvy[i]) + oy for i in range(nv)]
        for k in range(nv):
            if fma:
                tk = [fma(np.full_like(dx, fnx[k]), px[i], fny[k] * py[i]) for i in range(nv)]
            else:
                tk = [fnx[k] * px[i] + fny[k] * py[i] for i in range(nv)]
            lo, hi = np.min(tk, axis=0), np.max(tk, axis=0)
            gaps.append(np.maximum(lo - fahi[k], falo[k] - hi).astype(np.float64))
    return np.stack(gaps, 1)


@pytest.mark.parametrize("nv", [5, 3, 7])
def test_polygon_test_errors_within_its_margin(prog, nv):
    V = inputs.regular_polygon(nv, 0.5)
    r = _run(prog, V, dim=2)
    E = float(r["E"])
    R = float(r["Rc"])
    rng = np.random.default_rng(nv)
    n = 200000
    ang = rng.uniform(0, 2 * np.pi, n)
    D = np.stack([np.cos(ang), np.sin(ang)], 1) * (2 * R * np.sqrt(rng.uniform(0, 1, n)))[:, None]
    tA, tB = rng.uniform(0, 2 * np.pi, n), rng.uniform(0, 2 * np.pi, n)
    cA, sA, cB, sB = np.cos(tA), np.sin(tA), np.cos(tB), np.sin(tB)
    g32 = _sat_gaps(F, _fma, V, D, cA, sA, cB, sB)
    g64 = _sat_gaps(np.float64, None, V, D, cA, sA, cB, sB)
    err = float(np.max(np.abs(g32 - g64)))
    assert err < E / 2, (err, E / 2)
    assert err > E / 2 / 300


def test_polygon_validation(prog):
    # counter-clockwise convex polygons are accepted; clockwise, non-convex
    # and degenerate (collinear) vertex lists are refused
    pent = np.asarray(inputs.regular_polygon(5, 0.5))
    assert _run(prog, pent, dim=2)["rc"] == "0"
    assert _run(prog, pent[::-1], dim=2)["rc"] != "0"                 # clockwise
    dart = np.array([[0.0, -0.5], [0.5, 0.5], [0.0, 0.1], [-0.5, 0.5]])
    assert _run(prog, dart, dim=2)["rc"] != "0"                        # a reflex vertex
    line = np.array([[-0.5, -0.5], [0.0, -0.5], [0.5, -0.5], [0.0, 0.5]])
    assert _run(prog, line, dim=2)["rc"] != "0"                        # three collinear vertices
    assert _run(prog, np.array([[0.0, 0.0], [1.0, 0.0]]), dim=2)["rc"] != "0"    # too few
