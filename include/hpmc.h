/*
 * hpmc.h -- C ABI of the GB300 (sm_103a) checkerboard hard-particle Monte
 * Carlo library libhpmc.so.
 *
 * The library implements the data-parallel hot path of hard-particle
 * Metropolis Monte Carlo (Anderson, Irrgang & Glotzer, "Scalable Metropolis
 * Monte Carlo for simulation of hard shapes"): per sweep a random shift of
 * the cell grid, a cell-list rebuild, and 2^d checkerboard sets in which
 * every active cell makes `nselect` sequential trial moves (translation and
 * rotation), each rejected when it leaves its cell or overlaps a neighbour.
 *
 * Conventions for every function below:
 *   - Return value: 0 on success or a negative HPMC_ERR_* code.  The library
 *     never exits, aborts or traps; errors raised by device code (capacity
 *     overflow, bounded waits) are recorded in the handle and returned by the
 *     next call that synchronises (hpmc_counters, hpmc_get_state,
 *     hpmc_check_overlaps, hpmc_sync).  hpmc_strerror() names a code.
 *   - Host pointers are owned by the caller and only read/written during the
 *     call.  The library owns all device memory; it allocates in *_create and
 *     frees in *_destroy.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Functions that take a stream only enqueue work on it.
 *   - dim is 2 (convex polygons, orientation (cos, sin)) or 3 (convex
 *     polyhedra, unit quaternion (w, x, y, z)).  Positions lie in [0, L).
 *   - A "batch" holds R independent replicas of one shape type; a single
 *     system is a batch with R = 1.  Replica index r selects one replica.
 */
#ifndef HPMC_H
#define HPMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HPMC_OK                0
#define HPMC_ERR_INVALID_ARG  -1   /* NaN, N = 0, dim not 2/3, bad vertices, sizes */
#define HPMC_ERR_BOX_TOO_SMALL -2  /* fewer than 4 cells on an axis */
#define HPMC_ERR_OVERLAP      -3   /* (reserved) overlapping input where forbidden */
#define HPMC_ERR_OOM          -4   /* device allocation failed */
#define HPMC_ERR_CUDA         -5   /* a CUDA runtime call failed */
#define HPMC_ERR_TIMEOUT      -6   /* (reserved) a bounded device wait gave up: no kernel here waits */
#define HPMC_ERR_CAPACITY     -7   /* a cell or stencil exceeded the staging capacity */
#define HPMC_ERR_NOT_READY    -8   /* call order violated (e.g. no moves set) */

#define HPMC_FP64          0       /* plain form: every decision in FP64 */
#define HPMC_FP32_FILTERED 1       /* FP32 with certified bounds, FP64 re-check */

/* Counters accumulated since the last reset, summed over replicas. */
typedef struct {
    uint64_t moves;            /* trial moves proposed = accept + both rejects */
    uint64_t accept;
    uint64_t reject_overlap;
    uint64_t reject_boundary;  /* trial left its active cell (checkerboard rule) */
    uint64_t cull_pairs;       /* stencil neighbours tested by circumsphere */
    uint64_t overlap_checks;   /* full SAT / GJK evaluations */
    uint64_t fp64_rechecks;    /* FP32 verdicts that were not certified */
    uint64_t gjk_cap;          /* 3D: GJK iteration cap reached (counted as overlap) */
} hpmc_counters_t;

typedef struct hpmc_batch* hpmc_t;

/* One replica of a batch.  pos[N*dim] and orient[N*(2|4)] are its starting
 * configuration in tag order (caller-owned host arrays, read during create). */
typedef struct {
    uint32_t N;
    double box[3];             /* L per axis (box[2] ignored in 2D) */
    const double* pos;
    const double* orient;
    uint64_t seed;             /* Philox key of this replica */
    double d;                  /* translation half-width */
    double a;                  /* rotation half-angle parameter (radians) */
    uint32_t nselect;          /* sequential trial moves per active cell */
} hpmc_replica_desc_t;

/*
 * hpmc_batch_create -- allocate a batch of R replicas of one convex shape.
 *   dim       2 or 3.
 *   verts     nv*dim doubles, the shape in its local frame (2D: convex and
 *             counter-clockwise; 3D: the vertices of a convex polyhedron).
 *   nv        3..16 (2D) or 4..32 (3D); or 0: hard disks (2D) / spheres
 *             (3D) of radius verts[0] (the paper's validation systems,
 *             Sec. 4), which overlap when their centres are at most one
 *             diameter apart.
 *   w_min     floor on the cell width (0 = the circumdiameter, the paper's
 *             minimum, Sec. 2.2.1).
 *   reps      R replica descriptors (see above).
 *   out       receives the handle.
 * Cell geometry per axis: nc = floor(L / max(2R, w_min)), made even, >= 4
 * (BOX_TOO_SMALL otherwise).  Limits (INVALID_ARG beyond them): nc <= 65536
 * per axis, and at most 2^31 - 1 cells in a replica, cells in the batch and
 * particles in the batch (cell and particle indices are 32-bit).
 * Errors: INVALID_ARG, BOX_TOO_SMALL, OOM, CUDA.  Synchronous.
 */
int hpmc_batch_create(int dim, const double* verts, uint32_t nv, double w_min,
                      uint32_t R, const hpmc_replica_desc_t* reps, hpmc_t* out);

/*
 * hpmc_create -- single-system form of hpmc_batch_create (R = 1) taking the
 * box, shape, configuration and Philox seed; moves default to d = a = 0.1,
 * nselect = 4 until hpmc_set_moves is called.  The system is the one Sec. 2.1
 * simulates: N hard convex shapes of one type in a periodic box, each with a
 * position and an orientation, no two overlapping; the seed keys the
 * per-move random streams of Sec. 2.5 (hash-style counters instead of a
 * stored generator state).  Same arguments and errors as
 * hpmc_batch_create (pos[N*dim], orient[N*(2|4)] host arrays in tag order).
 */
int hpmc_create(const double* box, int dim, uint32_t N, const double* verts, uint32_t nv,
                const double* pos, const double* orient, uint64_t seed, double w_min,
                hpmc_t* out);

/* Release every device and host resource of the handle (synchronises it).
 * Resource management: no counterpart in the paper. */
int hpmc_destroy(hpmc_t h);

/*
 * hpmc_set_moves -- trial-move sizes of replica r (r = -1: all replicas).
 *   d >= 0 translation half-width; a in [0, pi) rotation parameter; nselect
 *   1..65535.  Sec. 2.1: r' = r + dr, q' = q * dq.
 */
int hpmc_set_moves(hpmc_t h, int32_t r, double d, double a, uint32_t nselect);

/*
 * hpmc_set_cell_width_min -- new floor w_min >= 0 on the cell width of every
 * replica (the w_min of creation; 0 = the circumdiameter, the paper's
 * minimum, Sec. 2.2.1).  The cell grid follows the creation rule; the next
 * sweep rebuilds the cell list.  Moves per sweep depend on the grid (one
 * select stream per cell), so trajectories with different floors differ.
 * BOX_TOO_SMALL (grid unchanged) when a replica would get fewer than 4 cells
 * on an axis; INVALID_ARG for a negative or non-finite w_min.  Synchronous.
 */
int hpmc_set_cell_width_min(hpmc_t h, double w_min);

/*
 * hpmc_set_precision -- HPMC_FP64 or HPMC_FP32_FILTERED (default).  Sec. 2.3
 * runs the overlap tests in single precision on double-precision separations
 * in the frame of one particle (Eq. 2); here the single-precision verdict is
 * used only when a forward error bound certifies that it equals the FP64
 * test's, and the test is re-run in FP64 otherwise, so both modes give
 * identical trajectories; the filtered form is faster.  INVALID_ARG for any
 * other mode.  Takes effect at the next sweep.
 */
int hpmc_set_precision(hpmc_t h, int mode);

/*
 * hpmc_set_group_size -- lanes per active cell in the set kernel (1, 2, 4, 8,
 * 16 or 32; or 0: the 2D direct kernel, one lane per cell reading its
 * neighbours without shared-memory staging; the FP32-filtered form also
 * skips the stencil layers a trial cannot reach -- INVALID_ARG in 3D) and
 * warps per block (1..16,
 * at most the kernel's launch bound: 8 warps for 8+ lanes per cell in 2D and
 * for the direct kernel, 6 for fewer, 8 in 3D; INVALID_ARG beyond it).  The
 * checkerboard schedule of Sec. 2.5.2 is the same for every choice, so the
 * trajectory does not change.  hpmc_autotune picks them by timing.
 */
int hpmc_set_group_size(hpmc_t h, int lanes_per_cell, int warps_per_block);

/*
 * hpmc_sweep -- enqueue n sweeps on `stream`: per sweep the grid shift,
 * the cell-list rebuild and the 2^d checkerboard sets (Sec. 2.5.2), for
 * every replica.  Asynchronous; the sweep counter advances on the device.
 * hpmc_sweep launches the kernels directly; hpmc_sweep_graph captures the
 * launch sequence of 16 sweeps (for runs of 16 or more) and of two sweeps
 * once into CUDA graphs (per buffer parity) and replays them.  Both give the
 * same trajectory.  With 8 or more lanes per
 * cell each sweep also runs one kernel on an internal second stream (the
 * state-independent part of every select, computed beside the rebuild and
 * joined before the first set); the first sweep after a change of group
 * size, precision, nselect or cell grid allocates its table, so a caller
 * that captures hpmc_sweep into a graph of its own runs one sweep first.
 */
int hpmc_sweep(hpmc_t h, uint32_t n, void* stream);
int hpmc_sweep_graph(hpmc_t h, uint32_t n, void* stream);

/* Wait for the handle's last stream; returns a recorded device error.
 * Host synchronisation: no counterpart in the paper. */
int hpmc_sync(hpmc_t h);

/*
 * hpmc_counters -- synchronise, then copy the counters of replica r (r = -1:
 * the sum over replicas) into *out.  hpmc_reset_counters zeroes them.  The
 * accept / reject counts are the outcomes of the Metropolis steps of Sec.
 * 2.1 (accepted when the trial overlaps nothing) and of the checkerboard
 * rule of Sec. 2.5.2 (rejected when the trial leaves its active cell); their
 * ratio is the acceptance the paper tunes move sizes to.  INVALID_ARG for a
 * null handle or output or r out of range; a recorded device error is
 * returned.
 */
int hpmc_counters(hpmc_t h, int32_t r, hpmc_counters_t* out);
int hpmc_reset_counters(hpmc_t h);

/*
 * hpmc_check_overlaps -- synchronise, rebuild the cell list and count the
 * overlapping pairs of replica r (r = -1: all) with the FP64 contract
 * predicate (circumsphere cull, then SAT / GJK; Sec. 2.1 defines a valid
 * configuration as one in which no pair overlaps, and the system tests of
 * Sec. 4 check runs for overlaps).  *n_pairs receives the count.  The grid
 * shift of the running sweep is kept, so the trajectory is unaffected.
 * INVALID_ARG for a null handle or output or r out of range.
 */
int hpmc_check_overlaps(hpmc_t h, int32_t r, uint64_t* n_pairs);

/*
 * hpmc_get_state / hpmc_set_state -- copy replica r's configuration in tag
 * order to / from caller-owned host arrays pos[N*dim], orient[N*(2|4)], and
 * its sweep counter.  The state of Sec. 2.1 is exactly this: every
 * particle's position and orientation; with the sweep counter (the step
 * index that keys the random streams of Sec. 2.5) it fixes the rest of the
 * trajectory, so a state read and written back continues bit for bit
 * (checkpoint and restart).  Both synchronise.  set_state checks that
 * positions are finite and inside [0, L) and orientations finite
 * (INVALID_ARG otherwise); it does not check overlaps (see
 * hpmc_check_overlaps).
 */
int hpmc_get_state(hpmc_t h, int32_t r, double* pos, double* orient, uint64_t* sweep);
int hpmc_set_state(hpmc_t h, int32_t r, const double* pos, const double* orient, uint64_t sweep);

/*
 * hpmc_run_host -- end-to-end call for callers holding host buffers: upload
 * every replica's configuration from pos/orient (all replicas concatenated in
 * replica order, tag order inside: pos[Ntot*dim], orient[Ntot*(2|4)], Ntot
 * the batch's particle count), run n sweeps, download the result into
 * pos_out/orient_out (same sizes, caller-owned) and the summed counters into
 * *out (may be NULL).  The state is what Sec. 2.1 evolves (positions and
 * orientations); the sweeps are those of hpmc_sweep_graph.  Each array moves
 * in one copy on `stream` (direct DMA when the caller's buffers are pinned)
 * through a device staging area of Ntot*(dim + (2|4)) doubles that the first
 * call allocates and the handle keeps; the layout change runs on the device.
 * The sweep counter continues from the handle's.  Synchronous.  Errors:
 * INVALID_ARG (null pointers), OOM (staging area), CUDA, and device errors
 * of the sweeps.
 */
int hpmc_run_host(hpmc_t h, const double* pos, const double* orient, uint32_t n,
                  double* pos_out, double* orient_out, hpmc_counters_t* out, void* stream);

/*
 * hpmc_autotune -- the launch-parameter autotuner of Sec. 2.5.3 (the fastest
 * group size and block size by timing).  Times each (lanes per cell, warps
 * per block) choice on n_trial sweeps from a saved copy of the state, restore the state and
 * sweep counters, and keep the fastest choice.  The trajectory does not
 * depend on the choice.  *best_lanes / *best_warps receive it.  A choice
 * whose sweeps cannot be launched is skipped; a failing CUDA call restores
 * the previous choice and the state before returning its error.  Synchronous.
 */
int hpmc_autotune(hpmc_t h, uint32_t n_trial, int* best_lanes, int* best_warps);

/*
 * hpmc_profile_sweeps -- the time per sweep that Sec. 3's benchmarks report,
 * split by phase: run n sweeps on `stream` with CUDA events recorded
 * around the rebuild (shift + cell list) and around the 2^d set kernels of
 * every sweep; synchronise and return the mean milliseconds per sweep of
 * each phase.  The set kernels' mean duration is *ms_sets / 2^d.
 */
int hpmc_profile_sweeps(hpmc_t h, uint32_t n, void* stream, double* ms_rebuild, double* ms_sets);

/*
 * hpmc_trace_read -- libraries built with -DHPMC_TRACE record, for the first
 * work item of every warp of the last set kernel, clock64() stamps at its
 * phase boundaries (*n_points per warp; see HPMC_STAMP in the kernel source).
 * Copies up to max_warps warps' stamps into out[max_warps * *n_points].
 * Returns HPMC_ERR_NOT_READY in ordinary builds.  Synchronous.  A profiling
 * aid: no counterpart in the paper.
 */
int hpmc_trace_read(hpmc_t h, uint64_t* out, uint32_t max_warps, uint32_t* n_points);

/*
 * hpmc_box_move -- one isotropic volume move of replica r (the NPT ensemble
 * that Sec. 1 lists among the paper's HPMC capabilities and whose
 * acceptance rule it takes from its NPT references): V' = V + dV_max (2u - 1)
 * with u from the replica's volume-move stream (Philox key = the replica's
 * seed, counter (lo32(m), hi32(m), 0, 4 << 24) for its m-th attempt; u from
 * words 0-1, u' from words 2-3); every box length and position scaled by
 * f = (V'/V)^(1/dim) (a position that rounds onto L' wraps to 0); the cell
 * grid follows the creation rule for the new box (a trial with fewer than 4
 * cells on an axis is rejected).  Any overlapping pair rejects; otherwise
 * the move is accepted when u' < exp(-beta_P (V' - V) + N log(V'/V)) (host
 * libm).  *accepted receives 1 or 0.  dV_max >= 0.  Synchronous.
 */
int hpmc_box_move(hpmc_t h, int32_t r, double beta_P, double dV_max, int* accepted);

/*
 * hpmc_debug_fail_alloc -- fault injection for tests: the n-th device
 * allocation the library makes from now on (n = 0: the next one) fails as
 * if the device were out of memory; the call that made it returns
 * HPMC_ERR_OOM and releases what it had allocated.  n < 0 disables it.
 * Host-side only: nothing runs on or faults the device.  A test hook with
 * no counterpart in the paper.
 */
int hpmc_debug_fail_alloc(int32_t n);

/* hpmc_get_box -- the current box lengths of replica r (box[3]; 0 beyond
 * dim), which hpmc_box_move changes (the NPT ensemble of Sec. 1). */
int hpmc_get_box(hpmc_t h, int32_t r, double* box);

/*
 * hpmc_tune_moves -- move sizes for a target acceptance ratio (Sec. 2.1: the
 * paper tunes to a fixed acceptance, then fixes the sizes).  A geometric
 * bisection over a common factor f in [lo, hi] of replica r's current d and a
 * (r = -1: every replica, acceptance pooled): each of `iters` pilots runs
 * n_pilot sweeps from the same saved state; the pilot whose acceptance is
 * closest to `target` sets the moves.  The configuration, sweep counters
 * and event counters are restored afterwards, so the trajectory continues
 * as if no pilot had run.  *d_out, *a_out (replica r, or replica 0 when
 * r = -1) and *acc_out (may be NULL) receive the result.  A failing pilot
 * restores the state and the previous moves before its error is returned.
 * Synchronous.
 */
int hpmc_tune_moves(hpmc_t h, int32_t r, double target, uint32_t n_pilot, uint32_t iters, double lo,
                    double hi, double* d_out, double* a_out, double* acc_out);

/*
 * Mean squared displacement (the paper's efficiency measure for fluids is
 * the diffusion rate per wall-clock time, Sec. 2.1).  hpmc_msd_reset makes
 * the current positions the reference; hpmc_msd_update adds every
 * particle's minimum-image step since the previous call to its unwrapped
 * displacement (call it often enough that no particle moves half a box in
 * between; NVT only: a volume move would count as displacement);
 * hpmc_msd_read returns the mean over replica r's particles (r = -1: all)
 * of |displacement|^2 (NOT_READY before a reset).  Synchronous.
 */
int hpmc_msd_reset(hpmc_t h);
int hpmc_msd_update(hpmc_t h);
int hpmc_msd_read(hpmc_t h, int32_t r, double* msd);

/*
 * hpmc_sdf -- pressure sampling by the scale distribution (Sec. 4): for
 * every pair of replica r (r = -1: all replicas) whose compression factor x*
 * (the uniform compression of positions by 1 - x, shapes unchanged, that
 * makes the pair touch) lies in [0, x_max), adds one to the bin of x*.
 * Disks / spheres (nv = 0): x* = 1 - 2R/|D|, bin (int)(x* * nbins / x_max).
 * Shaped particles: the bin by bisection over the bin edges e_k = k h,
 * h = x_max / nbins, with the overlap test along D (1 - e_k): the smallest
 * overlapping edge k gives bin k - 1.  hist is a caller-owned host array of
 * nbins uint64 that is accumulated, not cleared, so successive samples add
 * up.  beta P / rho = 1 + h(0) / (dim N), h(x) the pair count per unit x
 * per configuration extrapolated to x = 0.  Requires 0 < x_max < 1,
 * 1 <= nbins <= 2^20 and 2R / (1 - x_max) <= the cell width on every axis
 * (w_min at creation sets it); INVALID_ARG otherwise.  Rebuilds the cell
 * list (the trajectory is unaffected).
 * Synchronous.
 */
int hpmc_sdf(hpmc_t h, int32_t r, double x_max, uint32_t nbins, uint64_t* hist);

/* Result of hpmc_pressure. */
typedef struct {
    double beta_P_over_rho;       /* 1 + h(0) / (dim N) */
    double beta_P_over_rho_err;   /* standard error from the fit */
    double P_star;                /* beta P sigma^2 (2D) or beta P v0, v0 = pi sigma^3 / 6 (3D) */
    double P_star_err;
    double h0;                    /* extrapolated pairs per unit x per configuration at x = 0 */
    double h0_err;
} hpmc_pressure_t;

/*
 * hpmc_pressure -- pressure from a scale-distribution histogram (Sec. 4: the
 * volume-perturbation estimator).  hist[nbins] holds the counts hpmc_sdf
 * accumulated over n_samples configurations of N particles in a box of
 * volume `volume` (area in 2D), bins of width x_max / nbins from x = 0.
 * h(x) = count / (n_samples * bin width) is extrapolated to x = 0 by a
 * weighted least-squares fit of log h on the bin centres with a polynomial
 * of degree `deg` (0..8; weights sqrt(count), the inverse standard error of
 * a Poisson log count; empty bins left out), and beta P / rho = 1 + h(0) /
 * (dim N).  P* uses `sigma`, the diameter of the disks / spheres the paper
 * reports (any length scale for shaped particles).  Host computation only
 * (no device work, no allocation on the device).  Errors: INVALID_ARG (null
 * pointers, nbins = 0, n_samples = 0, N = 0, dim not 2/3, deg outside 0..8,
 * non-positive or non-finite x_max, volume or sigma, at most deg + 1
 * populated bins).
 */
int hpmc_pressure(const uint64_t* hist, uint32_t nbins, uint64_t n_samples, double x_max, uint64_t N,
                  double volume, int dim, int deg, double sigma, hpmc_pressure_t* out);

/*
 * hpmc_pair_test -- evaluate the overlap test of Sec. 2.3 (the separating
 * axis test in 2D, GJK in 3D, and the single-precision check of its mixed
 * precision mode) on n independent pairs on the GPU, for validation.  A sits at the origin with orientation qA, B at Delta
 * (minimum image already applied) with orientation qB; host arrays
 * D[n*dim], qA[n*(2|4)], qB[n*(2|4)] in FP64.  out64[n] receives the FP64
 * contract's verdict (1 overlap, 0 separated); out32[n] the FP32 filter's
 * verdict from the FP32-cast inputs (1 overlap, 0 separated, >= 2
 * uncertain: the sweep would re-decide in FP64; in 3D the value says why:
 * 2 converged apart within the error bound, 3 enclosed but the origin within
 * the bound of a face, 4 degenerate simplex, 5 iteration cap).  3D boxes take
 * the separating-axis certificate (2 = uncertain), polyhedra with an
 * interior origin the portal refinement before the GJK.  Shape and dim as in
 * hpmc_batch_create.  Synchronous; allocates and frees its own device
 * buffers.
 */
int hpmc_pair_test(int dim, const double* verts, uint32_t nv, uint32_t n, const double* D,
                   const double* qA, const double* qB, int32_t* out64, int32_t* out32);

/*
 * hpmc_pair_test_warp3d -- the 3D FP64 contract test (GJK, Sec. 2.3 / Eq. 2)
 * as the FP32-filtered 3D sweep evaluates its re-checks: one warp per pair,
 * the independent parts of the computation spread over its lanes.  Inputs
 * as hpmc_pair_test with dim = 3; out64[n] the verdict (1 overlap, 0
 * separated), iters[n] the support evaluations after the first (33 when the
 * iteration cap is reached).  For validation; synchronous; allocates and
 * frees its own device buffers.
 */
int hpmc_pair_test_warp3d(const double* verts, uint32_t nv, uint32_t n, const double* D, const double* qA,
                          const double* qB, int32_t* out64, int32_t* iters);

/*
 * hpmc_pair_test_box64 -- the FP64 separating-axis certificate the
 * FP32-filtered 3D sweep applies to box pairs (vertices (+-h0, +-h1, +-h2))
 * before re-deciding them with the FP64 GJK of the contract (Sec. 2.3 /
 * Eq. 2): one warp per pair.  Inputs as hpmc_pair_test with dim = 3; out[n]
 * receives 0 (certified separated: the boxes are more than 4e-6 of the
 * circumdiameter apart), 1 (certified overlap: deeper than 1e-9 of it) or 2
 * (left to the GJK).  INVALID_ARG when the shape is not such a box.  For
 * validation; synchronous; allocates and frees its own device buffers.
 */
int hpmc_pair_test_box64(const double* verts, uint32_t nv, uint32_t n, const double* D, const double* qA,
                         const double* qB, int32_t* out);

/* Geometry of replica r: cells per axis, cell width, circumradius (the cell
 * list of Sec. 2.2.1: cells at least the circumdiameter wide). */
int hpmc_geometry(hpmc_t h, int32_t r, int32_t* nc, double* w, double* R);

/* Number of kernel launches one sweep enqueues, the select-table kernel of
 * the latency regime included (for launch accounting; no counterpart in the
 * paper). */
int hpmc_launches_per_sweep(hpmc_t h, uint32_t* n);

/* FP32 filter margins of replica r (in-cell, cull, overlap), for reporting:
 * the certified bounds of the single-precision checks of the mixed
 * precision mode (Sec. 2.3). */
int hpmc_filter_margins(hpmc_t h, int32_t r, double* e_in, double* e_cull, double* e_overlap);

/* Name of an error code (a static string; unknown codes get a generic name).
 * Error reporting: no counterpart in the paper. */
const char* hpmc_strerror(int code);

/*
 * hpmc_measure_fma_peak -- measured peak of the pipe the set kernels' ALU
 * work runs on (the roofline denominator of their arithmetic; the paper
 * states no machine peak: no counterpart in the paper).  Times `iters` iterations of 8 independent fused
 * multiply-adds per thread in 2048 resident threads on every SM, FP64 when
 * fp64 != 0 else FP32, with CUDA events on a private stream, `reps` times
 * after one short warm-up launch; *flops_per_s receives the best rate (2
 * flops per multiply-add) and *ms (may be NULL) that launch's duration.  The
 * rate is at the clock the GPU ran, which the caller samples alongside.
 * Synchronous; allocates and frees its own device buffer.  Errors:
 * INVALID_ARG (null output, iters = 0, reps outside 1..1000), OOM, CUDA.
 */
int hpmc_measure_fma_peak(int fp64, uint32_t iters, int reps, double* flops_per_s, double* ms);

/*
 * hpmc_count_overlaps_noalloc -- count the overlapping pairs of one 2D
 * configuration without allocating any memory.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate
 * device memory where they need the check (code running inside a custom
 * memory pool or a callback that must not touch the allocator, tools that
 * forbid allocation while recording work, embedders that own all device
 * memory up front).
 *   box        host, 2 doubles: L_x, L_y (periodic, positions in [0, L)).
 *   verts      host, nv*2 doubles: convex counter-clockwise polygon, 3..16
 *              vertices, local frame.
 *   N          particles, 1..HPMC_NOALLOC_MAX_N.
 *   pos_dev    device, N*2 doubles (x, y) per particle, caller-owned.
 *   orient_dev device, N*2 doubles (cos, sin) per particle, caller-owned.
 *   count_dev  device, one unsigned 64-bit counter, caller-owned; receives
 *              the number of overlapping unordered pairs.
 *   stream     cudaStream_t as void* (NULL = legacy default stream); the
 *              call only enqueues work on it.
 * The pair rule is the FP64 one of hpmc_check_overlaps (minimum image,
 * circumsphere cull, separating axes) on the same cell grid (width rule of
 * hpmc_batch_create, no shift).  The cell list lives in one fixed
 * file-scope device array of the library (about 1.3 MB) that every device
 * loading the library keeps until the process exits; the call performs no
 * cudaMalloc, cudaFree or other allocation.  The first call on a device looks
 * up that array's device address; make it before any stream capture.  All
 * calls share the array and it keeps the last call's contents (the call
 * clears what must start at zero), so calls whose work overlaps on the GPU
 * (other streams, other threads) race and must be serialised by the caller.
 * Errors: INVALID_ARG (null pointers, bad vertices, non-finite box),
 * BOX_TOO_SMALL, SCRATCH_LIMIT (N > HPMC_NOALLOC_MAX_N or more than
 * HPMC_NOALLOC_MAX_CELLS cells), CUDA.
 */
#define HPMC_ERR_SCRATCH_LIMIT  -9   /* size beyond the fixed no-allocation scratch */
#define HPMC_NOALLOC_MAX_N      65536
#define HPMC_NOALLOC_MAX_CELLS  65536
int hpmc_count_overlaps_noalloc(const double* box, const double* verts, uint32_t nv, uint32_t N,
                                const double* pos_dev, const double* orient_dev,
                                unsigned long long* count_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HPMC_H */
