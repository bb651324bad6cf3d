"""Thin ctypes binding of libhpmc.so (the C ABI of include/hpmc.h).

Argument marshalling only: every step of a sweep runs in the library's CUDA
kernels.  There is no CPU fallback: importing this module raises if the
library cannot be loaded, and every call raises ``HPMCError`` on a non-zero
return code.  Streams are passed as raw ``cudaStream_t`` handles (an int, e.g.
``torch.cuda.current_stream().cuda_stream``; 0 = the legacy default stream).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

HPMC_FP64 = 0
HPMC_FP32_FILTERED = 1

ERRORS = {
    -1: "HPMC_ERR_INVALID_ARG", -2: "HPMC_ERR_BOX_TOO_SMALL", -3: "HPMC_ERR_OVERLAP",
    -4: "HPMC_ERR_OOM", -5: "HPMC_ERR_CUDA", -6: "HPMC_ERR_TIMEOUT", -7: "HPMC_ERR_CAPACITY",
    -8: "HPMC_ERR_NOT_READY", -9: "HPMC_ERR_SCRATCH_LIMIT",
}

# every symbol include/hpmc.h declares (the CPU tests check the exports)
EXPORTS = [
    "hpmc_batch_create", "hpmc_create", "hpmc_destroy", "hpmc_set_moves", "hpmc_set_precision",
    "hpmc_set_group_size", "hpmc_sweep", "hpmc_sweep_graph", "hpmc_sync", "hpmc_counters",
    "hpmc_reset_counters", "hpmc_check_overlaps", "hpmc_get_state", "hpmc_set_state",
    "hpmc_run_host", "hpmc_autotune", "hpmc_geometry", "hpmc_launches_per_sweep",
    "hpmc_filter_margins", "hpmc_strerror", "hpmc_profile_sweeps", "hpmc_count_overlaps_noalloc",
    "hpmc_trace_read", "hpmc_pair_test", "hpmc_sdf", "hpmc_box_move", "hpmc_get_box",
    "hpmc_tune_moves", "hpmc_msd_reset", "hpmc_msd_update", "hpmc_msd_read", "hpmc_debug_fail_alloc",
    "hpmc_pair_test_warp3d", "hpmc_set_cell_width_min", "hpmc_measure_fma_peak", "hpmc_pressure",
    "hpmc_pair_test_box64",
]


class HPMCError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)} ({_lib.hpmc_strerror(code).decode()})")


class Counters(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "moves", "accept", "reject_overlap", "reject_boundary", "cull_pairs", "overlap_checks",
        "fp64_rechecks", "gjk_cap")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class PressureOut(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "beta_P_over_rho", "beta_P_over_rho_err", "P_star", "P_star_err", "h0", "h0_err")]

    def as_dict(self):
        return {n: float(getattr(self, n)) for n, _ in self._fields_}


class ReplicaDesc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_uint32), ("box", ctypes.c_double * 3),
                ("pos", ctypes.POINTER(ctypes.c_double)), ("orient", ctypes.POINTER(ctypes.c_double)),
                ("seed", ctypes.c_uint64), ("d", ctypes.c_double), ("a", ctypes.c_double),
                ("nselect", ctypes.c_uint32)]


def _load():
    # HPMC_TRACE=1 selects the trace build (per-warp phase stamps)
    trace = os.environ.get("HPMC_TRACE", "") not in ("", "0")
    path = _build.LIB_TRACE if trace else _build.LIB
    if not os.path.exists(path):
        path = _build.build(trace=trace)
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    vp = ctypes.c_void_p
    i32, u32, u64 = ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64
    sig = {
        "hpmc_batch_create": [ctypes.c_int, dp, u32, ctypes.c_double, u32, ctypes.POINTER(ReplicaDesc),
                              ctypes.POINTER(vp)],
        "hpmc_create": [dp, ctypes.c_int, u32, dp, u32, dp, dp, u64, ctypes.c_double, ctypes.POINTER(vp)],
        "hpmc_destroy": [vp],
        "hpmc_set_moves": [vp, i32, ctypes.c_double, ctypes.c_double, u32],
        "hpmc_set_precision": [vp, ctypes.c_int],
        "hpmc_set_group_size": [vp, ctypes.c_int, ctypes.c_int],
        "hpmc_set_cell_width_min": [vp, ctypes.c_double],
        "hpmc_sweep": [vp, u32, vp],
        "hpmc_sweep_graph": [vp, u32, vp],
        "hpmc_sync": [vp],
        "hpmc_counters": [vp, i32, ctypes.POINTER(Counters)],
        "hpmc_reset_counters": [vp],
        "hpmc_check_overlaps": [vp, i32, ctypes.POINTER(u64)],
        "hpmc_get_state": [vp, i32, dp, dp, ctypes.POINTER(u64)],
        "hpmc_set_state": [vp, i32, dp, dp, u64],
        "hpmc_run_host": [vp, dp, dp, u32, dp, dp, ctypes.POINTER(Counters), vp],
        "hpmc_autotune": [vp, u32, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
        "hpmc_geometry": [vp, i32, ctypes.POINTER(i32), dp, dp],
        "hpmc_launches_per_sweep": [vp, ctypes.POINTER(u32)],
        "hpmc_filter_margins": [vp, i32, dp, dp, dp],
        "hpmc_profile_sweeps": [vp, u32, vp, dp, dp],
        "hpmc_trace_read": [vp, ctypes.POINTER(u64), u32, ctypes.POINTER(u32)],
        "hpmc_pair_test": [ctypes.c_int, dp, u32, u32, dp, dp, dp, ctypes.POINTER(ctypes.c_int32),
                           ctypes.POINTER(ctypes.c_int32)],
        "hpmc_pair_test_warp3d": [dp, u32, u32, dp, dp, dp, ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_int32)],
        "hpmc_pair_test_box64": [dp, u32, u32, dp, dp, dp, ctypes.POINTER(ctypes.c_int32)],
        "hpmc_sdf": [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, u32, ctypes.POINTER(ctypes.c_uint64)],
        "hpmc_box_move": [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                          ctypes.POINTER(ctypes.c_int)],
        "hpmc_get_box": [ctypes.c_void_p, ctypes.c_int32, dp],
        "hpmc_tune_moves": [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, u32, u32, ctypes.c_double,
                            ctypes.c_double, dp, dp, dp],
        "hpmc_msd_reset": [ctypes.c_void_p],
        "hpmc_msd_update": [ctypes.c_void_p],
        "hpmc_msd_read": [ctypes.c_void_p, ctypes.c_int32, dp],
        "hpmc_debug_fail_alloc": [ctypes.c_int32],
        "hpmc_measure_fma_peak": [ctypes.c_int, u32, ctypes.c_int, dp, dp],
        "hpmc_pressure": [ctypes.POINTER(u64), u32, u64, ctypes.c_double, u64, ctypes.c_double, ctypes.c_int,
                          ctypes.c_int, ctypes.c_double, ctypes.POINTER(PressureOut)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.hpmc_strerror.argtypes = [ctypes.c_int]
    lib.hpmc_strerror.restype = ctypes.c_char_p
    return lib


_lib = _load()


def lib():
    return _lib


def _ck(rc, where):
    if rc != 0:
        raise HPMCError(rc, where)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _sized(a, n, what):
    """Contiguous float64 copy of `a` holding exactly n values (the library
    reads n values through the pointer)."""
    a = _c64(a)
    if a.size != n:
        raise ValueError(f"{what}: {a.size} values given, {n} expected")
    return a


def _out(a, n, what, dtype=np.float64):
    """An output array the library writes n values into: it must be a
    writable C-contiguous array of `dtype` with exactly n elements."""
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous \
            or not a.flags.writeable or a.size != n:
        raise ValueError(f"{what}: a writable C-contiguous {np.dtype(dtype).name} array of {n} "
                         f"elements is needed")
    return a


class Batch:
    """A batch of R replicas of one convex shape (R = 1: a single system)."""

    def __init__(self, dim, verts, replicas, w_min=0.0):
        """replicas: list of dicts with keys N, box, pos, orient, seed, d, a, nselect."""
        self.dim = int(dim)
        self.qd = 2 if self.dim == 2 else 4
        # a scalar is the radius of disks (2D) / spheres (3D): nv = 0
        round_ = np.ndim(verts) == 0
        v = np.array([float(verts)]) if round_ else _c64(verts).reshape(-1, self.dim)
        nv = 0 if round_ else v.shape[0]
        self._keep = []
        descs = (ReplicaDesc * len(replicas))()
        self.N = []
        for i, r in enumerate(replicas):
            pos = _c64(r["pos"]).reshape(-1, self.dim)
            ori = _sized(r["orient"], pos.shape[0] * self.qd, f"replica {i} orient").reshape(-1, self.qd)
            self._keep += [pos, ori]
            box = list(np.broadcast_to(np.asarray(r["box"], dtype=np.float64), (self.dim,))) + [1.0] * (3 - self.dim)
            descs[i].N = pos.shape[0]
            descs[i].box = (ctypes.c_double * 3)(*box)
            descs[i].pos = _dp(pos)
            descs[i].orient = _dp(ori)
            descs[i].seed = int(r["seed"])
            descs[i].d = float(r.get("d", 0.1))
            descs[i].a = float(r.get("a", 0.1))
            descs[i].nselect = int(r.get("nselect", 4))
            self.N.append(pos.shape[0])
        h = ctypes.c_void_p()
        _ck(_lib.hpmc_batch_create(self.dim, _dp(v), nv, float(w_min), len(replicas), descs,
                                   ctypes.byref(h)), "hpmc_batch_create")
        self.h = h
        self.R = len(replicas)
        self._keep = []

    @classmethod
    def single(cls, dim, verts, box, pos, orient, seed, d=0.1, a=0.1, nselect=4, w_min=0.0):
        return cls(dim, verts, [dict(box=box, pos=pos, orient=orient, seed=seed, d=d, a=a,
                                     nselect=nselect)], w_min=w_min)

    def close(self):
        if getattr(self, "h", None):
            _lib.hpmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---- configuration
    def set_moves(self, d, a, nselect, r=-1):
        _ck(_lib.hpmc_set_moves(self.h, int(r), float(d), float(a), int(nselect)), "hpmc_set_moves")

    def set_cell_width_min(self, w_min):
        """Floor on the cell width of every replica (0 = the circumdiameter)."""
        _ck(_lib.hpmc_set_cell_width_min(self.h, float(w_min)), "hpmc_set_cell_width_min")

    def set_precision(self, mode):
        _ck(_lib.hpmc_set_precision(self.h, int(mode)), "hpmc_set_precision")

    def set_group_size(self, lanes, warps=4):
        _ck(_lib.hpmc_set_group_size(self.h, int(lanes), int(warps)), "hpmc_set_group_size")

    # ---- running
    def sweep(self, n, stream=0, graph=False):
        f = _lib.hpmc_sweep_graph if graph else _lib.hpmc_sweep
        _ck(f(self.h, int(n), ctypes.c_void_p(int(stream) if stream else None)), "hpmc_sweep")

    def sync(self):
        _ck(_lib.hpmc_sync(self.h), "hpmc_sync")

    def counters(self, r=-1):
        c = Counters()
        _ck(_lib.hpmc_counters(self.h, int(r), ctypes.byref(c)), "hpmc_counters")
        return c.as_dict()

    def reset_counters(self):
        _ck(_lib.hpmc_reset_counters(self.h), "hpmc_reset_counters")

    def check_overlaps(self, r=-1):
        n = ctypes.c_uint64()
        _ck(_lib.hpmc_check_overlaps(self.h, int(r), ctypes.byref(n)), "hpmc_check_overlaps")
        return int(n.value)

    def get_state(self, r=0):
        N = self.N[r]
        pos = np.zeros((N, self.dim))
        ori = np.zeros((N, self.qd))
        sw = ctypes.c_uint64()
        _ck(_lib.hpmc_get_state(self.h, int(r), _dp(pos), _dp(ori), ctypes.byref(sw)), "hpmc_get_state")
        return pos, ori, int(sw.value)

    def set_state(self, pos, orient, sweep=0, r=0):
        N = self.N[r]
        pos = _sized(pos, N * self.dim, "set_state pos")
        ori = _sized(orient, N * self.qd, "set_state orient")
        _ck(_lib.hpmc_set_state(self.h, int(r), _dp(pos), _dp(ori), int(sweep)), "hpmc_set_state")

    def run_host(self, pos, orient, n, pos_out, orient_out, stream=0):
        """pos/orient: every replica's configuration, concatenated in replica
        order (tag order inside); the result is written into pos_out /
        orient_out (same sizes).  Returns the summed counters."""
        nt = sum(self.N)
        pos = _sized(pos, nt * self.dim, "run_host pos")
        orient = _sized(orient, nt * self.qd, "run_host orient")
        _out(pos_out, nt * self.dim, "run_host pos_out")
        _out(orient_out, nt * self.qd, "run_host orient_out")
        c = Counters()
        _ck(_lib.hpmc_run_host(self.h, _dp(pos), _dp(orient), int(n), _dp(pos_out), _dp(orient_out),
                               ctypes.byref(c), ctypes.c_void_p(int(stream) if stream else None)),
            "hpmc_run_host")
        return c.as_dict()

    def box_move(self, beta_P, dV_max, r=0):
        """One isotropic volume move of replica r; True when accepted."""
        acc = ctypes.c_int()
        _ck(_lib.hpmc_box_move(self.h, int(r), float(beta_P), float(dV_max), ctypes.byref(acc)),
            "hpmc_box_move")
        return bool(acc.value)

    def tune_moves(self, target=0.30, n_pilot=100, iters=14, lo=0.25, hi=8.0, r=-1):
        """Scale d and a together for a target acceptance (pilots from a
        saved state, restored afterwards).  Returns (d, a, acceptance)."""
        d, a, acc = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _ck(_lib.hpmc_tune_moves(self.h, int(r), float(target), int(n_pilot), int(iters), float(lo),
                                 float(hi), ctypes.byref(d), ctypes.byref(a), ctypes.byref(acc)),
            "hpmc_tune_moves")
        return d.value, a.value, acc.value

    def msd_reset(self):
        _ck(_lib.hpmc_msd_reset(self.h), "hpmc_msd_reset")

    def msd_update(self):
        _ck(_lib.hpmc_msd_update(self.h), "hpmc_msd_update")

    def msd(self, r=-1):
        v = ctypes.c_double()
        _ck(_lib.hpmc_msd_read(self.h, int(r), ctypes.byref(v)), "hpmc_msd_read")
        return v.value

    def box(self, r=0):
        L = np.zeros(3)
        _ck(_lib.hpmc_get_box(self.h, int(r), _dp(L)), "hpmc_get_box")
        return L[: self.dim].copy()

    def sdf(self, x_max, nbins, r=-1, hist=None):
        """Add the current configuration's scale-factor histogram (disks /
        spheres) to ``hist`` (uint64[nbins], created when None); returns it."""
        if hist is None:
            hist = np.zeros(int(nbins), dtype=np.uint64)
        _out(hist, int(nbins), "sdf hist", np.uint64)
        _ck(_lib.hpmc_sdf(self.h, int(r), float(x_max), int(nbins),
                          hist.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))), "hpmc_sdf")
        return hist

    def autotune(self, n_trial=8):
        g = ctypes.c_int()
        w = ctypes.c_int()
        _ck(_lib.hpmc_autotune(self.h, int(n_trial), ctypes.byref(g), ctypes.byref(w)), "hpmc_autotune")
        return g.value, w.value

    def profile_sweeps(self, n, stream=0):
        """Mean ms per sweep of (rebuild, sets), CUDA events on `stream`."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _ck(_lib.hpmc_profile_sweeps(self.h, int(n), ctypes.c_void_p(int(stream) if stream else None),
                                     ctypes.byref(a), ctypes.byref(b)), "hpmc_profile_sweeps")
        return a.value, b.value

    def trace_read(self, max_warps=65536):
        """Per-warp clock64() phase stamps of the last set kernel (trace builds)."""
        buf = np.zeros((max_warps, 32), dtype=np.uint64)
        n = ctypes.c_uint32()
        _ck(_lib.hpmc_trace_read(self.h, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), max_warps,
                                 ctypes.byref(n)), "hpmc_trace_read")
        return buf[:, : n.value]

    def geometry(self, r=0):
        nc = (ctypes.c_int32 * 3)()
        w = np.zeros(3)
        R = ctypes.c_double()
        _ck(_lib.hpmc_geometry(self.h, int(r), nc, _dp(w), ctypes.byref(R)), "hpmc_geometry")
        return dict(nc=np.array(list(nc)[: self.dim]), w=w[: self.dim].copy(), R=R.value)

    def launches_per_sweep(self):
        n = ctypes.c_uint32()
        _ck(_lib.hpmc_launches_per_sweep(self.h, ctypes.byref(n)), "hpmc_launches_per_sweep")
        return int(n.value)

    def filter_margins(self, r=0):
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _ck(_lib.hpmc_filter_margins(self.h, int(r), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
            "hpmc_filter_margins")
        return dict(e_in=a.value, e_cull=b.value, e_overlap=c.value)


def pair_test(dim, verts, D, qA, qB):
    """FP64-contract and FP32-filter verdicts on independent pairs (GPU).

    Returns (out64, out32): 1 overlap, 0 separated, 2 (FP32 only) uncertain."""
    v = _c64(verts).reshape(-1, dim)
    D = _c64(D).reshape(-1, dim)
    qd = 2 if dim == 2 else 4
    n = D.shape[0]
    qA = _sized(qA, n * qd, "pair_test qA").reshape(-1, qd)
    qB = _sized(qB, n * qd, "pair_test qB").reshape(-1, qd)
    o64 = np.zeros(n, dtype=np.int32)
    o32 = np.zeros(n, dtype=np.int32)
    ip = ctypes.POINTER(ctypes.c_int32)
    _ck(_lib.hpmc_pair_test(int(dim), _dp(v), v.shape[0], n, _dp(D), _dp(qA), _dp(qB),
                            o64.ctypes.data_as(ip), o32.ctypes.data_as(ip)), "hpmc_pair_test")
    return o64, o32


def pair_test_warp3d(verts, D, qA, qB):
    """The 3D FP64 contract test as the FP32-filtered sweep evaluates its
    re-checks (one warp per pair).  Returns (out64, iters).  A scalar verts
    is the radius of a sphere."""
    round_ = np.ndim(verts) == 0
    v = np.array([float(verts)]) if round_ else _c64(verts).reshape(-1, 3)
    nv = 0 if round_ else v.shape[0]
    D = _c64(D).reshape(-1, 3)
    n = D.shape[0]
    qA = _sized(qA, n * 4, "pair_test_warp3d qA").reshape(-1, 4)
    qB = _sized(qB, n * 4, "pair_test_warp3d qB").reshape(-1, 4)
    o64 = np.zeros(n, dtype=np.int32)
    its = np.zeros(n, dtype=np.int32)
    ip = ctypes.POINTER(ctypes.c_int32)
    _ck(_lib.hpmc_pair_test_warp3d(_dp(v), nv, n, _dp(D), _dp(qA), _dp(qB), o64.ctypes.data_as(ip),
                                   its.ctypes.data_as(ip)), "hpmc_pair_test_warp3d")
    return o64, its


def pair_test_box64(verts, D, qA, qB):
    """The FP64 separating-axis certificate of box pairs (one warp per pair):
    0 separated, 1 overlap, 2 left to the FP64 GJK."""
    v = _c64(verts).reshape(-1, 3)
    D = _c64(D).reshape(-1, 3)
    n = D.shape[0]
    qA = _sized(qA, n * 4, "pair_test_box64 qA").reshape(-1, 4)
    qB = _sized(qB, n * 4, "pair_test_box64 qB").reshape(-1, 4)
    out = np.zeros(n, dtype=np.int32)
    _ck(_lib.hpmc_pair_test_box64(_dp(v), v.shape[0], n, _dp(D), _dp(qA), _dp(qB),
                                  out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "hpmc_pair_test_box64")
    return out


def from_system(sysm, w_min=None):
    """Batch of one replica from an inputs.System."""
    return Batch.single(sysm.dim, sysm.verts, sysm.L, sysm.pos, sysm.orient, sysm.seed, d=sysm.d,
                        a=sysm.a, nselect=sysm.nselect,
                        w_min=sysm.w_min if w_min is None else w_min)


def from_systems(systems):
    s0 = systems[0]
    reps = [dict(box=s.L, pos=s.pos, orient=s.orient, seed=s.seed, d=s.d, a=s.a, nselect=s.nselect)
            for s in systems]
    return Batch(s0.dim, s0.verts, reps, w_min=s0.w_min)


def pressure(hist, n_samples, x_max, N, volume, dim, sigma=1.0, deg=3):
    """hpmc_pressure on a host histogram (counts of hpmc_sdf): a dict with
    beta_P_over_rho, P_star, h0 and their standard errors."""
    h = np.ascontiguousarray(np.rint(np.asarray(hist, dtype=np.float64)).astype(np.uint64))
    out = PressureOut()
    _ck(_lib.hpmc_pressure(h.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), h.size, int(n_samples),
                           float(x_max), int(N), float(volume), int(dim), int(deg), float(sigma),
                           ctypes.byref(out)), "hpmc_pressure")
    return out.as_dict()


def measure_fma_peak(fp64, iters, reps=3):
    """Measured fused multiply-add rate of the FP64 (fp64=True) or FP32 pipe
    on the current device: (flop/s, ms of the best launch)."""
    f, ms = ctypes.c_double(), ctypes.c_double()
    _ck(_lib.hpmc_measure_fma_peak(1 if fp64 else 0, int(iters), int(reps), ctypes.byref(f), ctypes.byref(ms)),
        "hpmc_measure_fma_peak")
    return f.value, ms.value


def debug_fail_alloc(n):
    """Fault injection for tests: the n-th device allocation from now fails
    as out-of-memory (n < 0 disables)."""
    _ck(_lib.hpmc_debug_fail_alloc(int(n)), "hpmc_debug_fail_alloc")
