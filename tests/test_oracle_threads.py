"""The oracle's threaded set sweep (the active cells of one set shared out
over host threads) gives the serial trajectory byte for byte: the cells of
one checkerboard set are independent (Sec. 2.5.2), so sharing them out
cannot change any decision."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1509_04692_gb300 import inputs
from tests.test_oracle_sweep import load_rsa_start


def _run(dim, L, verts, pos, ori, d, a, seed, n, threads):
    ref = orc.OracleSystem(dim, L, verts)
    ref.set_moves(d, a, 4, seed)
    ref.set_threads(threads)
    p, o = pos.copy(), ori.copy()
    c = ref.sweep(p, o, 0, n)
    return p, o, c


@pytest.mark.parametrize("threads", [2, 3, 8])
def test_threaded_pentagon_sweeps_equal_serial(threads):
    pos, ori, L = load_rsa_start()
    v = inputs.regular_polygon(5, 0.5)
    want = _run(2, L, v, pos, ori, 0.1, 0.1, 42, 60, 1)
    got = _run(2, L, v, pos, ori, 0.1, 0.1, 42, 60, threads)
    assert want[0].tobytes() == got[0].tobytes() and want[1].tobytes() == got[1].tobytes()
    assert np.array_equal(want[2], got[2])


@pytest.mark.parametrize("threads", [2, 5])
def test_threaded_cube_sweeps_equal_serial(threads):
    s = inputs.cube_system(512, 0.45, seed=7, d=0.1)
    want = _run(3, s.L, s.verts, s.pos, s.orient, 0.1, 0.1, 7, 20, 1)
    got = _run(3, s.L, s.verts, s.pos, s.orient, 0.1, 0.1, 7, 20, threads)
    assert want[0].tobytes() == got[0].tobytes() and want[1].tobytes() == got[1].tobytes()
    assert np.array_equal(want[2], got[2])
    assert want[2][0] > 0 and want[2][1] > 0          # moves were accepted and rejected


def test_thread_count_is_checked():
    ref = orc.OracleSystem(2, 20.0, inputs.regular_polygon(5, 0.5))
    with pytest.raises(ValueError):
        ref.set_threads(0)
