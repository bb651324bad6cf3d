"""ctypes wrapper around the plain C oracle (hpmc_oracle.c).

TEST INFRASTRUCTURE ONLY: the CPU tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this module.  The CUDA library never
imports it, links it or calls it, and this module never imports the library.

Every routine here is the slow, obviously-correct FP64 statement of the
checkerboard hard-particle Metropolis sweep (Sec. 2.1, 2.2.1, 2.3 with Eq. 2,
2.5 and 2.5.1-2.5.2 of Anderson, Irrgang & Glotzer).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hpmc_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD_DIR, "liboracle.so")
# -ffp-contract=off: no fused multiply-add anywhere (gcc on aarch64 would
# otherwise contract a*b+c); no fast-math; every FP64 op rounds once.
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, plain C)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm", "-pthread"])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            dp = ctypes.POINTER(ctypes.c_double)
            L.or_system_size.restype = ctypes.c_size_t
            L.or_init.restype = ctypes.c_int
            L.or_init.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, dp, ctypes.c_int, ctypes.c_double]
            L.or_set_moves.restype = ctypes.c_int
            L.or_set_moves.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_uint32, ctypes.c_uint64]
            L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.or_u53.restype = ctypes.c_double
            L.or_u53.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            L.or_grid_shift.argtypes = [ctypes.c_void_p, ctypes.c_uint64, dp]
            L.or_cell_of.restype = ctypes.c_int
            L.or_cell_of.argtypes = [ctypes.c_void_p, dp, dp, ctypes.POINTER(ctypes.c_int)]
            L.or_build_cells.argtypes = [ctypes.c_void_p, ctypes.c_uint32, dp, dp, u32p, u32p,
                                         ctypes.POINTER(ctypes.c_int)]
            L.or_overlap_batch.argtypes = [ctypes.c_void_p, ctypes.c_uint32, dp, dp, dp,
                                           ctypes.POINTER(ctypes.c_int32)]
            L.or_overlap_batch_it.argtypes = [ctypes.c_void_p, ctypes.c_uint32, dp, dp, dp,
                                              ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
            L.or_sweep_repeats.restype = ctypes.c_int
            L.or_sweep_repeats.argtypes = [ctypes.c_void_p, ctypes.c_uint32, dp, dp, ctypes.c_uint64,
                                           ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint8), dp]
            L.or_set_threads.restype = ctypes.c_int
            L.or_set_threads.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.or_sweep.restype = ctypes.c_int
            L.or_sweep.argtypes = [ctypes.c_void_p, ctypes.c_uint32, dp, dp, ctypes.c_uint64,
                                   ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64)]
            L.or_propose_from_stream.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                                 ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                                 dp, dp, u32p, dp, dp]
            L.or_get_geometry.argtypes = [ctypes.c_void_p, dp, dp, ctypes.POINTER(ctypes.c_int), dp, dp]
            L.or_get_tau.restype = ctypes.c_double
            L.or_get_tau.argtypes = [ctypes.c_void_p]
            L.or_get_box.argtypes = [ctypes.c_void_p, dp]
            L.or_box_move.restype = ctypes.c_int
            L.or_box_move.argtypes = [ctypes.c_void_p, ctypes.c_uint32, dp, dp, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_uint64]
            L.or_sdf_histogram.restype = ctypes.c_int
            L.or_sdf_histogram.argtypes = [ctypes.c_void_p, ctypes.c_uint32, dp, dp, ctypes.c_double,
                                           ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64)]
            L.or_rsa_2d.restype = ctypes.c_int
            L.or_rsa_2d.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                    ctypes.c_uint64, dp, dp, ctypes.POINTER(ctypes.c_uint64)]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def philox4x32_10(ctr, key):
    """Philox4x32-10 block (Salmon et al., SC'11) -> 4 uint32 words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_u32p(c), _u32p(k), _u32p(o))
    return o


def u53(a: int, b: int) -> float:
    return lib().or_u53(a, b)


class OracleSystem:
    """One periodic box with one convex shape type (the oracle's view).
    ``radius`` instead of ``verts`` selects disks (2D) or spheres (3D)."""

    def __init__(self, dim, L, verts=None, w_min=0.0, radius=None):
        self.dim = int(dim)
        self._buf = ctypes.create_string_buffer(lib().or_system_size())
        Ls = np.ascontiguousarray(np.broadcast_to(np.asarray(L, dtype=np.float64), (dim,)))
        if radius is None and verts is not None and np.ndim(verts) == 0:
            radius = float(verts)              # a scalar is the radius of disks / spheres
        if radius is not None:
            v = np.array([float(radius)] * dim, dtype=np.float64)
            nv = 0
        else:
            v = np.ascontiguousarray(verts, dtype=np.float64).reshape(-1, dim)
            nv = v.shape[0]
        self.verts = v.copy()
        self.L = Ls.copy()
        rc = lib().or_init(self._buf, self.dim, _dp(Ls), _dp(v), nv, float(w_min))
        if rc != 0:
            raise ValueError(f"oracle or_init failed ({rc})")
        self.seed = 0
        self.nselect = 0

    def box_move(self, pos, orient, beta_P, dV_max, m):
        """One isotropic volume move (attempt number m) in place; returns 1
        when accepted (pos and the box are then scaled)."""
        assert pos.dtype == np.float64 and pos.flags.c_contiguous
        o = np.ascontiguousarray(orient, dtype=np.float64)
        rc = lib().or_box_move(self.ptr, pos.shape[0], _dp(pos), _dp(o), float(beta_P), float(dV_max), int(m))
        if rc < 0:
            raise RuntimeError("or_box_move failed")
        return rc

    @property
    def box(self):
        L = np.zeros(3)
        lib().or_get_box(self.ptr, _dp(L))
        return L[: self.dim].copy()

    def sdf_histogram(self, pos, x_max, nbins, orient=None):
        """Counts of pair compression factors x* in [0, x_max), nbins bins,
        every unordered pair once (disks / spheres: x* = 1 - sigma / r;
        shaped particles: bisection over the bin edges, orientations needed)."""
        p = np.ascontiguousarray(pos, dtype=np.float64)
        qd = 2 if self.dim == 2 else 4
        o = (np.zeros((p.shape[0], qd)) if orient is None
             else np.ascontiguousarray(orient, dtype=np.float64))
        h = np.zeros(int(nbins), dtype=np.uint64)
        rc = lib().or_sdf_histogram(self.ptr, p.shape[0], _dp(p), _dp(o), float(x_max), int(nbins),
                                    h.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
        if rc != 0:
            raise ValueError("or_sdf_histogram failed")
        return h

    @property
    def ptr(self):
        return ctypes.cast(self._buf, ctypes.c_void_p)

    def set_moves(self, d, a, nselect, seed):
        rc = lib().or_set_moves(self.ptr, float(d), float(a), int(nselect), int(seed))
        if rc != 0:
            raise ValueError("bad move parameters")
        self.seed = int(seed)
        self.nselect = int(nselect)

    def set_threads(self, n):
        """Host threads sharing the active cells of each set in sweep()
        (1 = serial, the default); the trajectory does not depend on it."""
        if lib().or_set_threads(self.ptr, int(n)) != 0:
            raise ValueError("thread count must be 1..1024")

    def geometry(self):
        R = ctypes.c_double()
        rc2 = ctypes.c_double()
        nc = (ctypes.c_int * 3)()
        w = np.zeros(3)
        iw = np.zeros(3)
        lib().or_get_geometry(self.ptr, ctypes.byref(R), ctypes.byref(rc2), nc, _dp(w), _dp(iw))
        return dict(R=R.value, rc2=rc2.value, nc=np.array(list(nc)[: self.dim]),
                    w=w[: self.dim].copy(), inv_w=iw[: self.dim].copy())

    @property
    def tau(self):
        return lib().or_get_tau(self.ptr)

    def grid_shift(self, sweep):
        s = np.zeros(3)
        lib().or_grid_shift(self.ptr, int(sweep), _dp(s))
        return s

    def cell_of(self, shift, x):
        sh = np.ascontiguousarray(shift, dtype=np.float64)
        xx = np.ascontiguousarray(x, dtype=np.float64)
        idx = (ctypes.c_int * 3)()
        c = lib().or_cell_of(self.ptr, _dp(sh), _dp(xx), idx)
        return c, np.array(list(idx)[: self.dim])

    def build_cells(self, pos, shift):
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        N = pos.shape[0]
        C = int(np.prod(self.geometry()["nc"]))
        start = np.zeros(C + 1, dtype=np.uint32)
        idx = np.zeros(max(N, 1), dtype=np.uint32)
        cof = np.zeros(max(N, 1), dtype=np.int32)
        sh = np.ascontiguousarray(shift, dtype=np.float64)
        lib().or_build_cells(self.ptr, N, _dp(pos), _dp(sh), _u32p(start), _u32p(idx),
                             cof.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return start, idx[:N], cof[:N]

    def overlap(self, D, qA, qB, iters=False):
        """Vectorised overlap contract D over pairs; returns int32 (1 = overlap),
        and with iters=True (3D) also the GJK's support evaluations after the
        first for each pair."""
        D = np.ascontiguousarray(D, dtype=np.float64).reshape(-1, self.dim)
        qd = 2 if self.dim == 2 else 4
        qA = np.ascontiguousarray(qA, dtype=np.float64).reshape(-1, qd)
        qB = np.ascontiguousarray(qB, dtype=np.float64).reshape(-1, qd)
        n = D.shape[0]
        out = np.zeros(n, dtype=np.int32)
        its = np.zeros(n, dtype=np.int32)
        ip = ctypes.POINTER(ctypes.c_int32)
        lib().or_overlap_batch_it(self.ptr, n, _dp(D), _dp(qA), _dp(qB), out.ctypes.data_as(ip),
                                  its.ctypes.data_as(ip))
        return (out, its) if iters else out

    def sweep(self, pos, orient, sweep0, nsweeps):
        """Run nsweeps sweeps in place on (pos, orient) in tag order.

        Returns the counters [accept, reject_overlap, reject_boundary, gjk_cap].
        """
        assert pos.dtype == np.float64 and pos.flags.c_contiguous
        assert orient.dtype == np.float64 and orient.flags.c_contiguous
        N = pos.shape[0]
        cnt = np.zeros(4, dtype=np.uint64)
        rc = lib().or_sweep(self.ptr, N, _dp(pos), _dp(orient), int(sweep0), int(nsweeps),
                            cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
        if rc != 0:
            raise RuntimeError(f"or_sweep failed ({rc})")
        return cnt

    def sweep_repeats(self, pos, orient, sweep0, n):
        """n independent single sweeps, each from (pos, orient) at sweep index
        sweep0 + k.  Returns (moved[n, N] bool, shifts[n, dim])."""
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        orient = np.ascontiguousarray(orient, dtype=np.float64)
        N = pos.shape[0]
        moved = np.zeros((n, N), dtype=np.uint8)
        shifts = np.zeros((n, 3))
        rc = lib().or_sweep_repeats(self.ptr, N, _dp(pos), _dp(orient), int(sweep0), int(n),
                                    moved.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), _dp(shifts))
        if rc != 0:
            raise RuntimeError(f"or_sweep_repeats failed ({rc})")
        return moved.astype(bool), shifts[:, : self.dim].copy()

    def propose(self, sweep, set_, cell, k, n_c, x, q):
        x = np.ascontiguousarray(x, dtype=np.float64)
        q = np.ascontiguousarray(q, dtype=np.float64)
        xn = np.zeros(3)
        qn = np.zeros(4)
        pick = ctypes.c_uint32()
        lib().or_propose_from_stream(self.ptr, int(sweep), int(set_), int(cell), int(k), int(n_c),
                                     _dp(x), _dp(q), ctypes.byref(pick), _dp(xn), _dp(qn))
        qd = 2 if self.dim == 2 else 4
        return pick.value, xn[: self.dim].copy(), qn[:qd].copy()

    def rsa_2d(self, N, seed, max_attempts):
        """Random sequential addition of N shapes (test-input generation only)."""
        pos = np.zeros((N, 2))
        ori = np.zeros((N, 2))
        used = ctypes.c_uint64()
        rc = lib().or_rsa_2d(self.ptr, N, int(seed), int(max_attempts), _dp(pos), _dp(ori),
                             ctypes.byref(used))
        if rc != 0:
            raise RuntimeError(f"RSA did not place {N} shapes within {max_attempts} attempts")
        return pos, ori, used.value
