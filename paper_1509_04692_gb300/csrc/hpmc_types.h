// hpmc_types.h -- device data layout of a batch of replicas (host + device).
//
// All particle arrays are global over the batch: replica r owns the index
// range [pbase, pbase + n) and the cell range [cbase, cbase + ncell).  Inside
// a replica the particles are kept in cell-sorted order (rebuilt every sweep);
// `tag` maps a sorted slot back to the particle's tag (0..n-1 per replica).
#pragma once
#include <cstdint>

namespace hpmc {

constexpr int kMaxV2 = 16;      // polygon vertices
constexpr int kMaxV3 = 32;      // polyhedron vertices
constexpr int kNumCounters = 8; // see hpmc_counters_t
constexpr int kGjkMaxIt = 32;
constexpr int kTracePoints = 32;

// Warp phase stamps (Sec. 2.5.3 used clock64() traces of one warp to compare
// queue designs).  Compiled in only with -DHPMC_TRACE.
#ifdef HPMC_TRACE
#define HPMC_STAMP(dv, warp_id, first, lane, point)                                      \
    do {                                                                                 \
        if ((first) && (lane) == 0 && (dv).trace && (warp_id) < (dv).trace_warps &&      \
            (point) < kTracePoints)                                                      \
            (dv).trace[(size_t)(warp_id) * kTracePoints + (point)] = clock64();          \
    } while (0)
// global nanosecond timer (comparable across SMs) for entry / exit stamps
#define HPMC_STAMP_NS(dv, warp_id, lane, point)                                          \
    do {                                                                                 \
        if ((lane) == 0 && (dv).trace && (warp_id) < (dv).trace_warps) {                 \
            unsigned long long t_;                                                       \
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_));                       \
            (dv).trace[(size_t)(warp_id) * kTracePoints + (point)] = t_;                 \
        }                                                                                \
    } while (0)
#else
#define HPMC_STAMP(dv, warp_id, first, lane, point) do { } while (0)
#define HPMC_STAMP_NS(dv, warp_id, lane, point) do { } while (0)
#endif

enum : int { CNT_MOVES = 0, CNT_ACCEPT, CNT_REJ_OVERLAP, CNT_REJ_BOUNDARY, CNT_CULL,
             CNT_CHECKS, CNT_RECHECK, CNT_GJKCAP };

enum : int { ERR_NONE = 0, ERR_CAPACITY = 1, ERR_TIMEOUT = 2 };

// Per-replica constants (device array, one entry per replica).
struct Rep {
    double L[3], halfL[3], w[3], inv_w[3];
    float w32[3];
    int nc[3];
    uint32_t n, pbase, cbase, ncell;
    uint64_t seed;
    double d, tau;           // move sizes (FP64 contract)
    double d_s, tau_s;       // d * 2^-53 and tau * 2^-53 (exact; see pm53)
    float d32, tau32;        // FP32 copies for the filter
    uint32_t nselect;
    // FP32 filter thresholds (certified; see hpmc_bounds.h), rounded outward:
    float in_lo;             // rel' >  in_lo  and < in_hi[a]  -> inside  (all axes)
    float in_hi[3];
    float out_lo;            // rel' < out_lo or > out_hi[a]   -> outside (any axis)
    float out_hi[3];
    float cull_keep;         // |D32|^2 < cull_keep -> FP64 keeps the pair
    float cull_skip;         // |D32|^2 > cull_skip -> FP64 culls the pair
    float sat_e;             // separating-axis / support gap margin
    float e_dlt32;           // |Delta32 - Delta64| per component (3D GJK input bound)
    float e_ori32;           // |q'32 - q'64| per component of the FP32 trial orientation
    float e_pb32;            // 3D: |pb32 - pb| per component of B's vertices in A's frame
    float e_va32;            // 3D: |fl32(v) - v| per component of A's local vertices
    float tau3;              // 3D: certificate band (depth / extra gap a certificate needs)
    float ins32;             // |D32|^2 < ins32 -> certain overlap (inscribed balls meet)
    float reach_lo[3];       // trial rel' > reach_lo[a]: the lower neighbour layer on axis a is beyond the cull
    float reach_hi[3];       // trial rel' < reach_hi[a]: the upper neighbour layer is beyond the cull
    // FP32 cell rule of the rebuild (certified; see cell_axis_f32)
    float L32[3], inv_w32[3];
    double reach64_lo[3], reach64_hi[3];  // the same reach for the FP64 trial coordinate (FP64 direct kernel)
    float cell_ey[3];        // bound on |y32 - (x - s)| (the sign test)
    float cell_et[3];        // bound on |t32 - t64| in cells (the boundary test)
    float box_esep;          // 3D boxes: a separating-axis gap above this certifies separation
    float box_eov;           // 3D boxes: overlaps above this on all 15 axes certify overlap
    double box_sep64, box_ov64;  // the same two margins of the FP64 separating-axis test
    double ins64;            // the same test on the FP64 |D|^2
    double e_in, e_cull, e_sat;  // the same margins in FP64 (reporting)
};

// Polygon constants (kernel parameter, passed by value).
struct Shape2 {
    int nv;
    int round;               // 1: hard disk (nv = 0), overlap iff |D|^2 <= rc2
    double vx[kMaxV2], vy[kMaxV2];
    double nx[kMaxV2], ny[kMaxV2];
    double alo[kMaxV2], ahi[kMaxV2];
    float fvx[kMaxV2], fvy[kMaxV2], fnx[kMaxV2], fny[kMaxV2], falo[kMaxV2], fahi[kMaxV2];
    double rc2;
    float frc2;
};

// Polyhedron constants (kernel parameter, passed by value).
struct Shape3 {
    int nv;
    int round;               // 1: hard sphere (nv = 0), overlap iff |D|^2 <= rc2
    int box;                 // 1: the 8 vertices are (+-h0, +-h1, +-h2), a box centred on the origin
    int mpr;                 // 1: the local origin is interior (the FP32 filter searches by portal refinement)
    int sym;                 // 1: centrally symmetric; fv is then ordered so that fv[k + nv / 2] = -fv[k]
    float bh[3];             // its half extents (FP32)
    double v[kMaxV3][3];     // the contract's vertices, in the given order
    float fv[kMaxV3][3];     // FP32 copies for the filter (same order unless sym)
    double rc2;
    float frc2;
};

// One copy of the particle state (the rebuild alternates between two).
struct Bufs {
    double* px; double* py; double* pz;
    double* q0; double* q1; double* q2; double* q3;   // 2D uses q0 = cos, q1 = sin
    float4* f4a;             // FP32 (rel.x, rel.y, c, s) 2D or (rel.x, rel.y, rel.z, qw) 3D
    float4* f4b;             // 3D: (qx, qy, qz, 0)
    uint32_t* tag;
};

// Device pointers of one batch (kernel parameter, passed by value).
struct Dev {
    int dim;
    uint32_t R;              // replicas
    uint32_t ntot;           // particles over all replicas
    uint32_t ctot;           // cells over all replicas
    const Rep* reps;
    const uint32_t* rep_of;  // replica of each global particle slot
    Bufs buf[2];             // the rebuild reads buf[cur] and writes buf[cur ^ 1]
    // cell list
    uint32_t* count;         // [ctot]
    uint32_t* start;         // [ctot + 1]
    uint32_t* tile_sums;     // scan scratch
    uint32_t* cellid;        // [ntot] scratch: global cell of each particle
    uint32_t* slot;          // [ntot] scratch: arrival slot in the cell
    uint32_t* tmp_tag;       // [ntot] scratch: tags in arrival order
    double* shift;           // [R * 3] grid shift of the current sweep
    uint64_t* sweep;         // [R] sweep counter per replica
    unsigned long long* counters;   // [R * kNumCounters]
    int* error;              // device error word (ERR_*)
    // state-independent part of the first selects of every cell in the
    // running sweep (latency-regime kernels only): record of select k of
    // global cell c at c * msel_stride + k; msel_n records allocated
    void* msel;
    uint32_t msel_stride;    // min(largest nselect over the replicas, G)
    uint64_t msel_n;
    // warp phase timestamps (trace builds only, -DHPMC_TRACE): kTracePoints
    // clock64() stamps of the first work item of each warp of a set kernel
    unsigned long long* trace;
    uint32_t trace_warps;
};

}  // namespace hpmc
