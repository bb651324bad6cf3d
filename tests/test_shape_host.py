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


def _run(exe, v):
    v = np.asarray(v, dtype=np.float64).reshape(-1, 3)
    txt = f"{len(v)}\n" + "\n".join(" ".join(repr(float(x)) for x in row) for row in v) + "\n"
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
