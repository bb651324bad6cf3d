"""Benchmark: trial moves/s of the checkerboard hard-particle MC sweep on GB300.

Headline workload (the largest single-GPU configuration): 2^24 regular
pentagons (circumradius 0.5) at area fraction 0.60 on a 2048 x 2048 cell
list (cell width >= 1.99), d = a = 0.165, nselect = 4, Philox seed 42, melted
200 sweeps from the lattice start before timing.  One step = 40 sweeps
(shift + cell-list rebuild + 4 checkerboard sets each), replayed from CUDA
graphs.  The state (2 GB) is larger than L2, and L2 is also flushed between
timed steps.

Headline `value`: FP32-filtered form (decisions identical to FP64), inputs
resident in HBM.  `forms` reports the plain FP64 form of the same system from
the same melted state (its accept / reject counts must equal the filtered
form's, else the run stops), and every other configuration in both forms
with the same check: 1024 pentagons from their random-sequential-addition
start, the 4096-pentagon fluid, 32768 cubes and 32000 dodecahedra at volume
fraction 0.50, the batch of 512 independent pentagon replicas (N ~
U{256..8192}, phi ~ U[0.40, 0.70]) and a batch of 32 cube replicas (N ~
U{2048..16384}, phi ~ U[0.40, 0.55]).  `roofline`: the set kernel's algorithmic flops over
its CUDA-event duration against the FP32 fused multiply-add rate measured in
the same run.  `e2e`: the same metric through hpmc_run_host with host
buffers (H2D + sweeps + D2H inside the timed region).  `cpu_baseline`: the C
oracle on all host cores (and on one).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--quick]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1509_04692_gb300 import inputs  # noqa: E402

METRIC = "trial moves/sec on 1 GB300 (FP32-filtered+batched vs plain FP64), % of roofline"
UNIT = "trial moves/s"
# the headline workload: the largest single-GPU configuration
WORKLOAD = ("2^24 regular pentagons (circumradius 0.5), area fraction 0.60, 2048^2 cells (w_min 1.99), "
            "d=a=0.165, nselect=4, Philox seed 42")
MELT_LARGE = 200              # graph-replayed sweeps from the lattice before timing
SWEEPS_LARGE = 40             # sweeps per timed step
MELT = 1000                   # melt of the smaller systems
RSA1024 = os.path.join(ROOT, "tests", "golden", "rsa_pentagons_N1024_phi050_seed42.txt")
# algorithmic flops per unit of work, per dimension: (trial move arithmetic,
# circumsphere cull candidate, full overlap test: the pentagon separating-axis
# test / the cube GJK estimate)
FLOPS = {2: (30, 5, 330), 3: (80, 8, 1000)}
# FMA-chain sizes of the peak measurement (each launch lasts ~20-40 ms)
PEAK_ITERS = {False: 400000, True: 6000}


def job_totals(torch, ms, moves, device):
    """Whole-job time and work over the ranks of an initialised process
    group: the slowest rank's time, the sum of the ranks' moves (one
    independent replica per rank: weak scaling).  One process: unchanged."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(moves)
    t = torch.tensor([float(ms), float(moves)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples during the timed region: the constructor returns once
    the sampler has written its first line (at most `wait_s` later), and the
    lines written before that point are left out of the record unless no
    other line came."""

    def __init__(self, gpu, period_ms=100, wait_s=5.0):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.skip = 0
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", str(period_ms)],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
            return
        t_end = time.time() + wait_s
        while time.time() < t_end and self.p.poll() is None:
            with open(self.f.name) as g:
                n = g.read().count("\n")
            if n:
                self.skip = n
                break
            time.sleep(0.02)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.f.read().splitlines()
        if len(lines) > self.skip:
            lines = lines[self.skip:]
        for line in lines:
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                mx.append(float(c[2]))
            except ValueError:
                continue
            for n, v in zip(names, c[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def host_cpu():
    """The host the oracle ran on: CPU model (from /proc/cpuinfo where it
    names one) and the number of logical CPUs."""
    import platform
    seen = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                if v.strip():
                    seen.setdefault(k.strip(), v.strip())
    except OSError:
        pass
    model = seen.get("model name") or seen.get("Model") or seen.get("Hardware")
    if not model and "CPU part" in seen:              # Arm: implementer and part number
        model = f"{platform.machine()} (CPU implementer {seen.get('CPU implementer', '?')}, " \
                f"part {seen['CPU part']})"
    return {"model": model or platform.processor() or platform.machine(), "nproc": os.cpu_count()}


def load_rsa1024():
    """The 1024-pentagon random-sequential-addition start (area fraction
    0.50, seed 42; hex floats x y cos sin), an inputs.System with the
    configuration's move sizes d = a = 0.1, nselect 4."""
    rows, L = [], None
    with open(RSA1024) as f:
        for line in f:
            if line.startswith("#"):
                if " L=" in line:
                    L = float.fromhex(line.split("L=")[1].split(",")[0])
                continue
            rows.append([float.fromhex(t) for t in line.split()])
    a = np.array(rows)
    return inputs.System(name="pentagons N=1024 phi=0.50 (RSA start)", dim=2, verts=inputs.regular_polygon(5, 0.5),
                         L=np.array([L, L]), pos=a[:, :2].copy(), orient=a[:, 2:].copy(), seed=42, d=0.1,
                         a=0.1, nselect=4, phi=0.50)


def oracle_rate(s, pos, ori, sweep0, sweeps, threads):
    """The C oracle (threaded set sweep) on `sweeps` sweeps of system s from
    (pos, ori) at sweep index sweep0: (moves/s, moves, seconds)."""
    from oracle import oracle as orc
    ref = orc.OracleSystem(s.dim, s.L, s.verts, w_min=s.w_min)
    ref.set_moves(s.d, s.a, s.nselect, s.seed)
    ref.set_threads(threads)
    p, q = np.ascontiguousarray(pos).copy(), np.ascontiguousarray(ori).copy()
    t0 = time.perf_counter()
    c = ref.sweep(p, q, sweep0, sweeps)
    dt = time.perf_counter() - t0
    moves = int(c[0] + c[1] + c[2])
    return moves / dt, moves, dt


def run_reference(args, system=None, melt=MELT_LARGE):
    """The oracle as it stands, on the host cores (threaded set sweep, every
    logical CPU), on the headline workload: the same melt from the same
    lattice start (untimed), then warm-up and timed steps of one sweep.
    (`system` and `melt` replace the workload in the CPU tests.)"""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as orc
    s = system if system is not None else inputs.large2d(42)
    threads = os.cpu_count() or 1
    ref = orc.OracleSystem(2, s.L, s.verts, w_min=s.w_min)
    ref.set_moves(s.d, s.a, s.nselect, s.seed)
    ref.set_threads(threads)
    pos, ori = s.pos.copy(), s.orient.copy()
    ref.sweep(pos, ori, 0, melt)
    sweep = melt
    per_step = 1
    for _ in range(args.warmup):
        ref.sweep(pos, ori, sweep, per_step)
        sweep += per_step
    moves = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        c = ref.sweep(pos, ori, sweep, per_step)
        sweep += per_step
        moves += int(c[0] + c[1] + c[2])
    dt = time.perf_counter() - t0
    v = moves / dt
    out = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOAD if system is None else s.name, "sweeps_per_step": per_step,
                      "melt_sweeps": melt},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": f"{args.steps} x {per_step} sweep(s) of {s.name} after "
                                      f"the oracle's own {melt}-sweep melt from the lattice (plain C "
                                      f"oracle, cells of each set shared over {threads} threads)",
                            "host": host_cpu()},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "gpu_launches": 0}
    print(json.dumps(out))


def time_steps(b, torch, stream, steps, warmup, flush, sweeps):
    """warmup + steps graph-replayed steps of `sweeps` sweeps; CUDA events on
    the launching stream around each timed step, L2 flushed before each.
    Returns (total ms of the timed steps, counter deltas of the timed steps,
    cumulative (accept, reject_overlap, reject_boundary) after each step
    from the start, warm-up steps included)."""
    c_start = b.counters()
    cum = []

    def mark():
        c = b.counters()
        cum.append(tuple(c[k] - c_start[k] for k in ("accept", "reject_overlap", "reject_boundary")))
    for _ in range(warmup):
        b.sweep(sweeps, stream=stream.cuda_stream, graph=True)
        mark()
    torch.cuda.synchronize()
    c0 = b.counters()
    total_ms = 0.0
    for _ in range(steps):
        flush.zero_()                                  # evict the state from L2 between steps
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.sweep(sweeps, stream=stream.cuda_stream, graph=True)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        mark()
    c1 = b.counters()
    d = {k: c1[k] - c0[k] for k in c1}
    return total_ms, d, cum


def set_kernel_roofline(b, stream, n_prof, peak):
    """Algorithmic flops of the set kernels over `n_prof` directly launched
    sweeps, divided by their mean duration (CUDA events on the stream the
    kernels run on), against `peak`: the measured fused multiply-add rate of
    the pipe the form's arithmetic runs on (FP32 for the filtered form, FP64
    for the plain form).  The state advances by n_prof sweeps."""
    b.reset_counters()
    ms_rebuild, ms_sets = b.profile_sweeps(n_prof, stream=stream.cuda_stream)
    cp = b.counters()
    nsets = 1 << b.dim
    fm, fc, ft = FLOPS[b.dim]
    flop_per_launch = (fm * cp["moves"] + fc * cp["cull_pairs"] + ft * cp["overlap_checks"]) / (n_prof * nsets)
    set_ms = ms_sets / nsets
    achieved = flop_per_launch / (set_ms * 1e-3)
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None,
            "set_kernel_ms": set_ms, "rebuild_ms_per_sweep": ms_rebuild,
            "flop_per_launch": flop_per_launch,
            "moves_per_launch": cp["moves"] / (n_prof * nsets),
            "flops_model": f"{fm} per trial move + {fc} per cull candidate + {ft} per full overlap test"}


def measure_form(b, torch, stream, flush, precision, melt, sweeps, steps, peaks, n_tune=4):
    """Melt (untimed, graph-replayed), autotune (state restored), one warm-up
    step, then `steps` timed steps of `sweeps` sweeps; L2 flushed between
    steps; then the set kernels' roofline over a few more sweeps."""
    from paper_1509_04692_gb300 import hpmc
    b.set_precision(precision)
    if melt:
        b.sweep(melt, stream=stream.cuda_stream, graph=True)
    lanes, warps = b.autotune(n_tune)
    ms, c, cum = time_steps(b, torch, stream, steps, 1, flush, sweeps)
    peak = peaks[1] if precision == hpmc.HPMC_FP64 else peaks[0]
    rf = set_kernel_roofline(b, stream, max(1, min(sweeps, 20)), peak)
    return {"value": c["moves"] / (ms * 1e-3),
            "precision": "FP64" if precision == hpmc.HPMC_FP64 else "FP32_FILTERED",
            "lanes_per_cell": lanes, "warps_per_block": warps, "ms_per_step": ms / steps,
            "sweeps_per_step": sweeps, "steps": steps, "melt_sweeps": melt,
            "acceptance": c["accept"] / max(1, c["moves"]),
            "overlap_checks": c["overlap_checks"], "fp64_rechecks": c["fp64_rechecks"],
            "accept": c["accept"], "reject_overlap": c["reject_overlap"],
            "reject_boundary": c["reject_boundary"], "moves": c["moves"],
            "set_kernel_frac_alu": rf["frac"], "set_kernel_tflops": rf["achieved"],
            "set_kernel_peak": "FP64 FMA rate" if precision == hpmc.HPMC_FP64 else "FP32 FMA rate",
            "set_kernel_ms": rf["set_kernel_ms"]}


def same_decisions(a, b, what):
    """The FP32-filtered and plain FP64 forms of one workload must make the
    same accept / reject decisions; a difference stops the benchmark."""
    ka = (a["accept"], a["reject_overlap"], a["reject_boundary"])
    kb = (b["accept"], b["reject_overlap"], b["reject_boundary"])
    if ka != kb:
        raise SystemExit(f"{what}: FP32-filtered and FP64 decisions differ: {ka} vs {kb}")
    return True


def measure_peaks(hpmc, local):
    """Measured FP32 and FP64 fused multiply-add rates (flop/s) with the SM
    clock sampled during the measurement."""
    sampler = ClockSampler(local)
    p32, ms32 = hpmc.measure_fma_peak(False, PEAK_ITERS[False], reps=5)
    p64, ms64 = hpmc.measure_fma_peak(True, PEAK_ITERS[True], reps=5)
    clk = sampler.stop()
    return p32, p64, {"fp32_tflops": p32 / 1e12, "fp64_tflops": p64 / 1e12, "fp32_launch_ms": ms32,
                      "fp64_launch_ms": ms64, "clocks": clk,
                      "method": "8 independent FMA chains per thread, 2048 threads per SM on every SM, "
                                "best of 5 launches, CUDA events"}


def run_ours(args):
    import torch
    from paper_1509_04692_gb300 import hpmc
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    multi = ws > 1

    p32, p64, peaks = measure_peaks(hpmc, local)

    # ---- headline: the 2^24-pentagon system, FP32-filtered
    s = inputs.large2d(42 + rank)
    b = hpmc.from_system(s)
    b.set_precision(hpmc.HPMC_FP32_FILTERED)
    b.sweep(MELT_LARGE, stream=stream.cuda_stream, graph=True)      # melt (untimed)
    lanes, warps = b.autotune(2)                                      # state restored afterwards
    snap = b.get_state() if not multi else None                      # for the FP64 form and the CPU baseline
    torch.cuda.synchronize()

    if multi:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local) if rank == 0 else None
    ms, cnt, cum32 = time_steps(b, torch, stream, args.steps, args.warmup, flush, SWEEPS_LARGE)
    clocks = sampler.stop() if sampler else None
    moves = cnt["moves"]
    ms_job, moves_job = job_totals(torch, ms, moves, "cuda")
    value = moves_job / (ms_job * 1e-3)

    # ---- end to end through the C ABI with host buffers, on every rank
    # (whole job: the slowest rank's time, the moves and bytes of all ranks)
    N = s.N
    p_in, o_in, _ = b.get_state()
    pin_p = torch.from_numpy(np.ascontiguousarray(p_in)).pin_memory()
    pin_o = torch.from_numpy(np.ascontiguousarray(o_in)).pin_memory()
    out_p = torch.empty_like(pin_p).pin_memory()
    out_o = torch.empty_like(pin_o).pin_memory()
    del p_in, o_in
    torch.cuda.synchronize()
    b.run_host(pin_p.numpy(), pin_o.numpy(), SWEEPS_LARGE, out_p.numpy(), out_o.numpy(),
               stream=stream.cuda_stream)                    # warm-up
    e2e_moves, e2e_dt = 0, 0.0
    e2e_steps = max(3, args.steps // 2)
    if multi:
        dist.barrier()
    for _ in range(e2e_steps):
        b.reset_counters()
        t0 = time.perf_counter()
        c = b.run_host(pin_p.numpy(), pin_o.numpy(), SWEEPS_LARGE, out_p.numpy(), out_o.numpy(),
                       stream=stream.cuda_stream)
        e2e_dt += time.perf_counter() - t0
        e2e_moves += c["moves"]
        pin_p.copy_(out_p)
        pin_o.copy_(out_o)
    e2e_ms_job, e2e_moves_job = job_totals(torch, e2e_dt * 1e3, e2e_moves, "cuda")
    state_bytes = int(ws * N * 4 * 8)
    e2e = {"value": e2e_moves_job / (e2e_ms_job * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": state_bytes, "d2h_bytes_per_step": state_bytes,
           "api": f"hpmc_run_host (pinned host buffers, H2D + {SWEEPS_LARGE} sweeps + D2H + counters)"}
    del pin_p, pin_o, out_p, out_o
    b.reset_counters()
    if rank != 0:
        b.close()
        if multi:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (the set kernel), CUDA events live
    roofline = set_kernel_roofline(b, stream, 8, p32)
    roofline["kernel"] = ("k_set2d_direct<5> (checkerboard set, one lane per active cell)" if lanes == 0 else
                          f"k_set2d<{lanes}, 1, 5> (checkerboard set, {lanes} lanes per cell)") + \
        ", 2^24-pentagon system"
    roofline["peak_source"] = "FP32 fused multiply-add rate measured in this run (hpmc_measure_fma_peak)"
    roofline["traffic_note"] = ("DRAM bytes of this kernel come from a separate ncu capture of a 2^22-particle "
                                "instance (kept with the profiles), not from this run")
    launches = args.steps * SWEEPS_LARGE * b.launches_per_sweep()
    b.close()

    forms = {"large2d_2p24_fp32_filtered": {"value": value, "fp64_rechecks": cnt["fp64_rechecks"],
                                            "overlap_checks": cnt["overlap_checks"],
                                            "acceptance": cnt["accept"] / max(1, moves),
                                            "lanes_per_cell": lanes, "warps_per_block": warps}}
    cpu = None
    if not multi:
        # ---- the plain FP64 form of the headline, from the same melted state:
        # its cumulative decisions must equal the FP32-filtered form's
        b64 = hpmc.from_system(s)
        b64.set_state(*snap)
        b64.set_precision(hpmc.HPMC_FP64)
        l64, w64 = b64.autotune(2)
        k64 = min(args.steps, 5)
        ms64, c64, cum64 = time_steps(b64, torch, stream, k64, args.warmup, flush, SWEEPS_LARGE)
        b64.close()
        n_cmp = args.warmup + k64
        if cum64[n_cmp - 1] != cum32[n_cmp - 1]:
            raise SystemExit(f"2^24 system: FP32-filtered and FP64 decisions differ after {n_cmp} steps: "
                             f"{cum32[n_cmp - 1]} vs {cum64[n_cmp - 1]}")
        forms["large2d_2p24_fp64"] = {"value": c64["moves"] / (ms64 * 1e-3), "steps": k64,
                                      "lanes_per_cell": l64, "warps_per_block": w64,
                                      "decisions_equal_fp32_filtered": True,
                                      "compared_sweeps": n_cmp * SWEEPS_LARGE}

        # ---- the other configurations (one GPU)
        def pair(key, make, melt, sweeps, steps, n_tune, batched=False):
            out = {}
            for prec, tag in ((hpmc.HPMC_FP32_FILTERED, "fp32_filtered"), (hpmc.HPMC_FP64, "fp64")):
                if args.quick and prec == hpmc.HPMC_FP64:
                    continue
                bb = make()
                out[tag] = measure_form(bb, torch, stream, flush, prec, melt, sweeps, steps, (p32, p64), n_tune)
                bb.close()
            if "fp64" in out:
                out["fp32_filtered"]["decisions_equal_fp64"] = same_decisions(out["fp32_filtered"], out["fp64"], key)
            for tag, f in out.items():
                forms[f"{key}_{tag}"] = f

        s1 = load_rsa1024()
        pair("rsa1024", lambda: hpmc.from_system(s1), 0, 1000, 3, 8)
        sf = inputs.fluid4096(42)
        pair("fluid4096", lambda: hpmc.from_system(sf), MELT, 200, 5, 8)
        if not args.no_cubes:
            sc = inputs.cubes32768(42)
            pair("cubes32768", lambda: hpmc.from_system(sc), MELT, 100, 5, 4)
            sd = inputs.dodecahedra32000(42)
            pair("dodecahedra32000", lambda: hpmc.from_system(sd), MELT, 50, 5, 4)
        if not args.no_batched:
            reps = inputs.replica_systems(512)
            pair("batched512", lambda: hpmc.from_systems(reps), MELT, 200, 5, 8)
            forms["batched512_fp32_filtered"].update(replicas=512, particles=int(sum(r.N for r in reps)))
        if not args.no_batched and not args.no_cubes:
            creps = inputs.cube_replica_systems()
            pair("batched_cubes32", lambda: hpmc.from_systems(creps), MELT, 100, 5, 4)
            forms["batched_cubes32_fp32_filtered"].update(replicas=len(creps),
                                                          particles=int(sum(r.N for r in creps)))

        # ---- CPU baseline: the oracle on the host cores, bounded sample of
        # the headline workload (from the GPU's melted state: a timing sample)
        if not args.no_cpu:
            threads = os.cpu_count() or 1
            rate, cmoves, cdt = oracle_rate(s, snap[0], snap[1], snap[2], 2, threads)
            rate1, cmoves1, cdt1 = oracle_rate(s, snap[0], snap[1], snap[2], 1, 1)
            cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle", "host": host_cpu(),
                   "sample": f"2 sweeps ({cmoves} trial moves, {cdt:.1f} s) of the 2^24-pentagon system from "
                             f"the state after the {MELT_LARGE}-sweep melt, plain C oracle with the cells of "
                             f"each set shared over {threads} threads",
                   "single_core": {"value": rate1, "cores": 1,
                                   "sample": f"1 sweep ({cmoves1} trial moves, {cdt1:.1f} s), 1 thread"}}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_job / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (FP32 certified filter, FP64 state)",
           "data": "synthetic",
           "config": {"workload": WORKLOAD, "N": N, "cells": 2048 * 2048, "phi": 0.60, "d": s.d, "a": s.a,
                      "nselect": s.nselect, "sweeps_per_step": SWEEPS_LARGE, "melt_sweeps": MELT_LARGE,
                      "precision": "FP32_FILTERED", "lanes_per_cell": lanes, "warps_per_block": warps,
                      "l2": "inputs larger than L2 (2 GB of state against 129 MB) and a 256 MiB write "
                            "between timed steps",
                      "parallelism": f"replicas only: {ws} independent system(s), one per GPU"},
           "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks, "e2e": e2e,
           "gpu_launches": launches, "peaks": peaks, "forms": forms, "counters": cnt}
    print(json.dumps(out))
    if multi:
        dist.destroy_process_group()


def run_profile(args):
    """Small case for ncu captures: the benchmark fluid, a short melt, then
    `--profile-sweeps` sweeps of the chosen precision form (direct launches)."""
    import torch
    if args.trace:
        os.environ["HPMC_TRACE"] = "1"          # load the -DHPMC_TRACE build
    from paper_1509_04692_gb300 import hpmc
    torch.cuda.set_device(0)
    if args.profile_workload == "batched":
        b = hpmc.from_systems(inputs.replica_systems(512))
    elif args.profile_workload == "cubes":
        b = hpmc.from_system(inputs.cubes32768(42))
    elif args.profile_workload == "batched_cubes":
        b = hpmc.from_systems(inputs.cube_replica_systems())
    elif args.profile_workload == "dodecahedra":
        b = hpmc.from_system(inputs.dodecahedra32000(42))
    elif args.profile_workload == "large2d":
        b = hpmc.from_system(inputs.large2d(42, N=args.profile_n or inputs.LARGE2D_N))
    else:
        b = hpmc.from_system(inputs.fluid4096(42))
    b.set_precision(hpmc.HPMC_FP64 if args.profile_fp64 else hpmc.HPMC_FP32_FILTERED)
    if args.lanes >= 0:
        b.set_group_size(args.lanes, args.warps)
    b.sweep(args.profile_melt, graph=True)
    b.sweep(args.profile_sweeps)
    c = b.counters()
    out = {"profile": args.profile_workload, "sweeps": args.profile_sweeps, "counters": c}
    if args.trace:
        # clock64() stamps of the first item of every warp of the last set
        # kernel: per-phase cycles (median / p90 over warps)
        tr = b.trace_read().astype(np.int64)
        used = tr[:, 0] != 0
        tr = tr[used]
        names = {1: "prologue", 2: "capacity check", 3: "staging", 4: "stencil tables",
                 5: "precompute"}
        phases = {}
        prev = tr[:, 0]
        for p in range(1, 28):
            col = tr[:, p]
            ok = col != 0
            if not ok.any():
                continue
            d = (col - prev)[ok]
            name = names.get(p, f"move{(p - 6) // 3}:" + ["propose", "cull+overlap", "accept"][(p - 6) % 3]
                             if 6 <= p < 30 else "tail")
            phases[name] = {"median": float(np.median(d)), "p90": float(np.percentile(d, 90))}
            prev = np.where(ok, col, prev)
        out["trace_cycles"] = phases
        out["warps_traced"] = int(used.sum())
        # global-timer entry (28) / exit (29) stamps: start spread and span, ns
        ent, ex = tr[:, 28], tr[:, 29]
        okx = (ent != 0) & (ex != 0)
        if okx.any():
            e0 = ent[okx].min()
            out["warp_entry_ns"] = {"p50": float(np.median(ent[okx] - e0)),
                                    "p90": float(np.percentile(ent[okx] - e0, 90)),
                                    "max": float((ent[okx] - e0).max())}
            out["warp_run_ns"] = {"p50": float(np.median(ex[okx] - ent[okx])),
                                  "max": float((ex[okx] - ent[okx]).max())}
            out["kernel_span_ns"] = float(ex[okx].max() - e0)
        out["total_cycles_median"] = float(np.median(tr[:, 30] - tr[:, 0])) if (tr[:, 30] != 0).any() else None
        # 3D kernel: point 31 holds the traced item's FP64 re-check count
        rc = tr[:, 31]
        if rc.any() and okx.any():
            run = (ex - ent).astype(float)
            w0, w1 = okx & (rc == 0), okx & (rc > 0)
            out["rechecks_per_traced_item"] = {
                "mean": float(rc.mean()), "frac_items_with": float((rc > 0).mean()),
                "run_ns_p50_without": float(np.median(run[w0])) if w0.any() else None,
                "run_ns_p50_with": float(np.median(run[w1])) if w1.any() else None,
                "run_ns_max_without": float(run[w0].max()) if w0.any() else None}
    b.close()
    print(json.dumps(out))


VALIDATION = {
    # the paper's NVT validation state points (Sec. 4, Table 2)
    "disks": ("hard disks N=65536 phi=0.698 (paper Sec. 4: P* = beta P sigma^2 = 9.1707(2))",
              lambda: inputs.disk_system(65536, 0.698, 42, d=0.05, w_min=1.06)),
    "spheres": ("hard spheres N=131072 phi=0.60, FCC (paper Sec. 4: P* = beta P v0 = 9.3135(4))",
                lambda: inputs.sphere_system(32, 0.60, 42, d=0.05, w_min=1.06)),
}


def run_validate_pressure(args):
    """A state point of the paper's NVT validation (Sec. 4): hard disks at
    area fraction 0.698 (65536, P* = 9.1707(2)) or hard spheres at volume
    fraction 0.60 on their FCC lattice (131072, P* = 9.3135(4)): equilibrate
    from the lattice, then sample the scale distribution every
    `--sample-every` sweeps and extrapolate the pressure (block averages show
    the drift)."""
    import torch
    from paper_1509_04692_gb300 import hpmc, pressure, tune
    torch.cuda.set_device(0)
    x_max, nbins = 0.05, 25
    label, make = VALIDATION[args.validate_system]
    s = make()
    b = hpmc.from_system(s)
    b.set_precision(hpmc.HPMC_FP32_FILTERED)
    t0 = time.time()
    b.sweep(2000, graph=True)
    p0, q0, sw0 = b.get_state()

    def pilot(d, a):
        b.set_state(p0, q0, sw0)
        b.set_moves(d, 0.0, 4)
        b.reset_counters()
        b.sweep(50, graph=True)
        c = b.counters()
        return c["accept"] / c["moves"]
    d, _, acc = tune.tune_scale(pilot, 0.05, 0.05, 0.30, lo=0.1, hi=10.0, iters=10)
    b.set_state(p0, q0, sw0)
    b.set_moves(d, 0.0, 4)
    b.reset_counters()
    te = time.time()
    b.sweep(args.validate_pressure, graph=True)              # equilibration
    b.sync()
    eq_s = time.time() - te
    blocks = []
    hist_all = np.zeros(nbins, dtype=np.uint64)
    n_all = 0
    per_block = max(1, args.validate_samples // 5)
    ts = time.time()
    for blk in range(5):
        h = np.zeros(nbins, dtype=np.uint64)
        for _ in range(per_block):
            b.sweep(args.sample_every, graph=True)
            b.sdf(x_max, nbins, hist=h)
        hist_all += h
        n_all += per_block
        blocks.append(pressure.pressure(h, per_block, x_max, s.N, float(np.prod(s.L)), s.dim)["P_star"])
    samp_s = time.time() - ts
    vol = float(np.prod(s.L))
    out = pressure.pressure(hist_all, n_all, x_max, s.N, vol, s.dim)
    c = b.counters()
    bm = np.array(blocks)
    # sensitivity of the extrapolation: polynomial degree and fitted range
    variants = {}
    for deg, nb in ((1, 10), (2, 25), (3, 25), (2, 12)):
        v = pressure.pressure(hist_all[:nb], n_all, x_max * nb / nbins, s.N, vol, s.dim, deg=deg)
        variants[f"deg{deg}_x{x_max * nb / nbins:.3f}"] = v["P_star"]
    print(json.dumps({
        "P_star_fit_variants": variants,
        "validate": label,
        "P_star": out["P_star"], "P_star_fit_err": out["P_star_err"],
        "P_star_blocks": blocks, "P_star_block_sem": float(bm.std(ddof=1) / np.sqrt(len(bm))),
        "d": d, "acceptance": c["accept"] / max(1, c["moves"]),
        "equilibration_sweeps": args.validate_pressure, "samples": n_all, "sample_every": args.sample_every,
        "moves_per_s": c["moves"] / (eq_s + samp_s), "seconds": time.time() - t0,
        "fp64_rechecks": c["fp64_rechecks"], "overlaps_after": b.check_overlaps()}))
    b.close()


def run_efficiency(args):
    """Sampling efficiency against move size (Sec. 2.1: the diffusion rate in
    wall-clock time peaks near the acceptance the paper tunes to): the
    4096-pentagon fluid at area fraction 0.60, d = a scaled together; for each
    scale, the mean squared displacement after `--efficiency` sweeps divided
    by the GPU time of those sweeps (CUDA events around the sweeps only)."""
    import torch
    from paper_1509_04692_gb300 import hpmc
    torch.cuda.set_device(0)
    s = inputs.fluid4096(42)
    b = hpmc.from_system(s)
    b.set_precision(hpmc.HPMC_FP32_FILTERED)
    b.sweep(MELT, graph=True)
    b.autotune(4)
    p0, q0, sw0 = b.get_state()
    rows = []
    chunk = 20
    for f in (0.15, 0.25, 0.4, 0.6, 0.8, 1.0, 1.3, 1.7, 2.3, 3.0):
        b.set_state(p0, q0, sw0)
        b.set_moves(s.d * f, s.a * f, s.nselect)
        b.sweep(100, graph=True)                             # settle at this move size
        b.reset_counters()
        b.msd_reset()
        ms = 0.0
        for _ in range(max(1, args.efficiency // chunk)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            b.sweep(chunk, graph=True)
            e1.record()
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            b.msd_update()
        c = b.counters()
        msd = b.msd()
        rows.append({"scale": f, "d": s.d * f, "a": s.a * f, "acceptance": c["accept"] / c["moves"],
                     "msd": msd, "gpu_s": ms * 1e-3, "msd_per_gpu_s": msd / (ms * 1e-3),
                     "moves_per_s": c["moves"] / (ms * 1e-3)})
    best = max(rows, key=lambda r: r["msd_per_gpu_s"])
    print(json.dumps({"efficiency": "4096 pentagons, area fraction 0.60, d = a scaled together",
                      "sweeps_per_point": args.efficiency, "rows": rows,
                      "best_acceptance": best["acceptance"], "best_scale": best["scale"]}))
    b.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--profile-sweeps", type=int, default=0,
                    help="run the small ncu case instead of the benchmark")
    ap.add_argument("--profile-workload", default="fluid4096",
                    choices=["fluid4096", "batched", "cubes", "batched_cubes", "dodecahedra", "large2d"])
    ap.add_argument("--profile-fp64", action="store_true")
    ap.add_argument("--profile-n", type=int, default=0, help="N of the large2d profile case")
    ap.add_argument("--profile-melt", type=int, default=20, help="graph-replayed sweeps before profiling")
    ap.add_argument("--lanes", type=int, default=-1,
                    help="lanes per cell of the profiled set kernel (0: the 2D direct kernel; default: as created)")
    ap.add_argument("--warps", type=int, default=4)
    ap.add_argument("--trace", action="store_true", help="with --profile-sweeps: per-warp phase stamps")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-cubes", action="store_true")
    ap.add_argument("--validate-pressure", type=int, default=0,
                    help="hard-disk pressure validation: equilibration sweeps (then sampling)")
    ap.add_argument("--validate-samples", type=int, default=2000)
    ap.add_argument("--validate-system", default="disks", choices=sorted(VALIDATION))
    ap.add_argument("--efficiency", type=int, default=0,
                    help="diffusion per GPU second against move size (sweeps per point)")
    ap.add_argument("--sample-every", type=int, default=50)
    ap.add_argument("--quick", action="store_true", help="skip the plain FP64 forms of the smaller systems")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.validate_pressure:
        run_validate_pressure(args)
    elif args.efficiency:
        run_efficiency(args)
    elif args.profile_sweeps:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
