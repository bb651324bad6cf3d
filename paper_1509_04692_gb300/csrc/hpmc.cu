// hpmc.cu -- C ABI of libhpmc.so: batch state, launch sequence of a sweep,
// CUDA-graph replay, counters, overlap check, state I/O and the autotuner.
//
// Sec. 2.5.2 (GPU checkerboard kernel): the host only enqueues; every step of
// a sweep (shift, cell-list rebuild, 2^d sets) runs in the kernels of this
// library on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/hpmc.h"
#include "hpmc_bounds.h"
#include "hpmc_launch.h"
#include "hpmc_rebuild.cuh"
#include "hpmc_shape.h"

using namespace hpmc;

int hpmc_check3d_launch(const hpmc::Dev& dv, const hpmc::Shape3& sh, int b, int32_t r,
                        unsigned long long* out, uint32_t ntot);

namespace {

// lanes per cell of the set kernels; 0 is the 2D direct kernel (one lane per
// cell, neighbours read through L1 without staging)
constexpr int kNumGroups = 7;
constexpr int kGroupSizes[kNumGroups] = { 1, 2, 4, 8, 16, 32, 0 };

int gidx_of(int G)
{
    for (int i = 0; i < kNumGroups; ++i)
        if (kGroupSizes[i] == G) return i;
    return -1;
}

// cells of a strip of one work item
int cells_per_item(int G)
{
    return G ? 32 / G : 32;
}

struct HostRep {
    uint32_t N;
    double L[3];
    uint64_t seed;
    double d, a;
    uint32_t nselect;
    uint64_t box_moves = 0;   // volume-move attempts (counter of their Philox stream)
};

// Philox4x32-10 on the host (the volume move draws its two numbers here; the
// device version is in hpmc_device.cuh): same rounds and Weyl key bumps.
void philox_host(uint32_t c[4], uint32_t k0, uint32_t k1)
{
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0], p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

double u53_host(uint32_t a, uint32_t b)
{
    return (double)((((uint64_t)a << 32) | b) >> 11) * 0x1.0p-53;
}

}  // namespace

struct hpmc_batch {
    int dim = 2;
    int nv = 0;
    double verts[kMaxV3 * 3] = {};
    double w_min = 0.0;
    double Rc = 0.0, rc2 = 0.0;
    double rin = 0.0;                    // inradius about the local origin
    uint32_t ctot_cap = 0;               // cells the count / start arrays hold
    double* bak[3] = { nullptr, nullptr, nullptr };   // positions saved by a volume move
    double* msd_last = nullptr;          // [ntot * 3] position at the last update, by tag
    double* msd_acc = nullptr;           // [ntot * 3] unwrapped displacement since the reset
    unsigned long long* sdf_hist = nullptr;   // device histogram of hpmc_sdf
    uint32_t sdf_cap = 0;
    uint32_t R = 0, ntot = 0, ctot = 0, ntiles = 0;
    std::vector<HostRep> hr;
    std::vector<Rep> reps;
    Shape2 sh2{};
    Shape3 sh3{};
    Dev dv{};
    int cur = 0;
    int precision = HPMC_FP32_FILTERED;
    int G = 4, wpb = 4;
    int num_sms = 0;
    uint32_t* item_base_dev = nullptr;   // [kNumGroups][R + 1]
    std::vector<uint32_t> items_per_set; // [kNumGroups] totals
    std::vector<void*> allocs;
    cudaStream_t last_stream = nullptr;
    int pending_error = 0;
    // graphs of two and of kLongGraph sweeps per starting buffer parity (an
    // even number of sweeps returns to it); the long one for long runs, so
    // that graph-launch boundaries are rare
    cudaGraphExec_t graph[2] = { nullptr, nullptr };
    cudaGraphExec_t graph_long[2] = { nullptr, nullptr };
    cudaStream_t graph_stream = nullptr;
    // set-kernel launch configuration (recomputed when G, wpb or precision change)
    bool cfg_valid = false;
    const void* cfg_fn = nullptr;
    size_t cfg_smem = 0;
    uint32_t cfg_grid = 0;
    unsigned long long* check_out = nullptr;
    // select table of the latency-regime kernels (G >= 8), filled by k_selects
    // on a second stream while the cell list is rebuilt
    bool use_selects = false;
    void* msel = nullptr;
    uint64_t msel_cap = 0;               // records allocated
    uint32_t sel_grid = 0;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // device copy of a host configuration for hpmc_run_host (positions then
    // orientations, interleaved per particle as the caller holds them),
    // allocated on the first call
    double* stage = nullptr;
};

namespace {

int cuda_fail(cudaError_t e)
{
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? HPMC_ERR_OOM : HPMC_ERR_CUDA;
}

#define CK(x)                                  \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

// Fault injection for tests (hpmc_debug_fail_alloc): when non-negative, the
// allocation with this index (counting from the call) fails as if the device
// were out of memory.  Host-side only; the device is never faulted.
int g_fail_alloc = -1;

template <typename T>
int dalloc(hpmc_batch* h, T** p, size_t n)
{
    void* q = nullptr;
    if (g_fail_alloc >= 0 && g_fail_alloc-- == 0) return HPMC_ERR_OOM;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e);
    h->allocs.push_back(q);
    *p = (T*)q;
    return 0;
}

float f32_down(double x)
{
    float f = (float)x;
    if ((double)f > x) f = std::nextafter(f, -INFINITY);
    return f;
}

float f32_up(double x)
{
    float f = (float)x;
    if ((double)f < x) f = std::nextafter(f, INFINITY);
    return f;
}

bool is_finite(double x) { return std::isfinite(x); }

// geometry shared by every replica: circumradius and the overlap constants
int shape_setup(hpmc_batch* h, int dim, const double* verts, uint32_t nv)
{
    const int rc = build_shapes(dim, verts, nv, h->sh2, h->sh3, h->Rc, h->rc2);
    if (rc) return rc;
    h->dim = dim;
    h->nv = (int)nv;
    std::memcpy(h->verts, verts, sizeof(double) * nv * dim);
    h->rin = shape_inradius(dim, verts, nv);
    return 0;
}

int rep_geometry(const hpmc_batch* h, const HostRep& hr, Rep& rp)
{
    const double dcut = h->Rc + h->Rc;
    const double wmin = dcut > h->w_min ? dcut : h->w_min;
    for (int a = 0; a < 3; ++a) {
        if (a < h->dim) {
            const double L = hr.L[a];
            if (!(L > 0.0) || !is_finite(L)) return HPMC_ERR_INVALID_ARG;
            int n = (int)std::floor(L / wmin);
            if (n % 2) n -= 1;
            if (n < 4) return HPMC_ERR_BOX_TOO_SMALL;
            if (n > 65536) return HPMC_ERR_INVALID_ARG;
            rp.L[a] = L;
            rp.halfL[a] = 0.5 * L;
            rp.nc[a] = n;
            rp.w[a] = L / (double)n;
            rp.inv_w[a] = (double)n / L;
            rp.w32[a] = (float)rp.w[a];
        } else {
            rp.L[a] = 1.0; rp.halfL[a] = 0.5; rp.nc[a] = 1; rp.w[a] = 1.0; rp.inv_w[a] = 1.0;
            rp.w32[a] = 1.0f;
        }
    }
    rp.n = hr.N;
    rp.seed = hr.seed;
    rp.d = hr.d;
    rp.tau = std::tan(0.5 * hr.a);
    rp.d_s = rp.d * 0x1.0p-53;        // exact: power-of-two scaling
    rp.tau_s = rp.tau * 0x1.0p-53;
    rp.d32 = (float)rp.d;
    rp.tau32 = (float)rp.tau;
    rp.nselect = hr.nselect;
    // the cell count in 64 bits: a dilute box can exceed 32 bits (cell
    // indices are 32-bit, so at most 2^31 - 1 cells)
    const uint64_t ncell = (uint64_t)rp.nc[0] * (uint64_t)rp.nc[1] * (uint64_t)(h->dim == 3 ? rp.nc[2] : 1);
    if (ncell > 0x7fffffffull) return HPMC_ERR_INVALID_ARG;
    rp.ncell = (uint32_t)ncell;
    // certified FP32 thresholds
    double wmax = 0.0, Lmax = 0.0;
    for (int a = 0; a < h->dim; ++a) { wmax = std::max(wmax, rp.w[a]); Lmax = std::max(Lmax, rp.L[a]); }
    Margins g = base_margins(h->dim, wmax, Lmax, rp.d, rp.tau, h->rc2);
    double vm = 0.0, nm = 0.0, am = 0.0;
    if (h->dim == 2) {
        for (int k = 0; k < h->sh2.nv; ++k) {
            vm = std::max({ vm, std::fabs(h->sh2.vx[k]), std::fabs(h->sh2.vy[k]) });
            nm = std::max({ nm, std::fabs(h->sh2.nx[k]), std::fabs(h->sh2.ny[k]) });
            am = std::max({ am, std::fabs(h->sh2.alo[k]), std::fabs(h->sh2.ahi[k]) });
        }
        g.e_sat = sat2_margin(g, h->Rc, vm, nm, am);
    } else {
        for (int k = 0; k < h->sh3.nv; ++k)
            for (int a = 0; a < 3; ++a) vm = std::max(vm, std::fabs(h->sh3.v[k][a]));
        // the 3D kernel takes its FP32 trial orientation as a cast of the FP64
        // contract's trial quaternion (|q'| = 1 within 1e-15)
        g.e_ori = kU32 * 1.000001 + 2e-15;
        g.e_sat = gjk3_vertex_margin(g, h->Rc, vm);
    }
    rp.e_pb32 = f32_up(h->dim == 3 ? g.e_sat : 0.0);
    rp.e_va32 = f32_up(2.0 * kU32 * vm);
    // certificate band: an overlap certificate needs the origin this deep
    // inside the Minkowski difference, far above the FP64 rounding of a
    // support query (~1e-13 of the shape size), so that no FP64 support can
    // show a separating plane.  A separation certificate needs, besides
    // tau |n|_1, a gap of |n|_1 times the FP32 vertex error bound (~6e-5 of
    // the size for cubes), outside the zone near contact (below ~3e-7 of
    // the size) where the FP64 GJK may conservatively answer overlap.
    rp.tau3 = f32_up(1e-9 * 2.0 * h->Rc);
    rp.box_esep = rp.box_eov = 0.0f;
    rp.box_sep64 = rp.box_ov64 = 0.0;
    if (h->dim == 3 && h->sh3.box) {
        const double bh[3] = { std::fabs(h->sh3.v[0][0]), std::fabs(h->sh3.v[0][1]), std::fabs(h->sh3.v[0][2]) };
        const BoxMargins bm = box_sat_margins(g, h->Rc, bh, (double)rp.tau3);
        rp.box_esep = f32_up(bm.sep);
        rp.box_eov = f32_up(bm.ov);
        const BoxMargins b64 = box_sat_margins64(h->Rc, bh, (double)rp.tau3);
        rp.box_sep64 = b64.sep;
        rp.box_ov64 = b64.ov;
    }
    rp.in_lo = f32_up(g.e_in);
    rp.out_lo = f32_down(-g.e_in);
    for (int a = 0; a < 3; ++a) {
        rp.in_hi[a] = f32_down(rp.w[a] - g.e_in);
        rp.out_hi[a] = f32_up(rp.w[a] + g.e_in);
    }
    rp.cull_keep = f32_down(h->rc2 - g.e_cull);
    // centres closer than twice the inradius: the inscribed balls meet, so the
    // shapes overlap at depth 2 rin - |Delta|; with the band of the certified
    // GJK (and far above any FP64 rounding) every FP64 test answers overlap
    {
        const double band = 2e-9 * 2.0 * h->Rc;
        const double r2 = 2.0 * h->rin * (1.0 - 1e-12) - band;
        rp.ins64 = r2 > 0.0 ? r2 * r2 * (1.0 - 1e-12) : -1.0;
        rp.ins32 = r2 > 0.0 ? f32_down(r2 * r2 - g.e_cull) : -1.0f;
    }
    rp.cull_skip = f32_up(h->rc2 + g.e_cull);
    // Reach of a trial across the walls of its cell.  A particle of the
    // lower neighbour layer on axis a lies below the cell's lower wall (up to
    // a few FP64 ulps of L from the cell rule), so the contract's |Delta_a|
    // exceeds rel'_exact minus those ulps and its own rounding; rel'_exact is
    // within e_in / 2 of the FP32 trial coordinate.  When the FP32 trial
    // coordinate exceeds 2R (1 + 4 u64) + e_in, every pair with that layer has
    // |Delta_a| >= 2R (1 + 2 u64), so |Delta|^2 rounds above (2R)^2 and the
    // contract culls it.  Likewise for the upper layer below w - reach.
    for (int a = 0; a < 3; ++a) {
        const double reach = h->Rc * 2.0 * (1.0 + 4.0 * kU64) + g.e_in;
        rp.reach_lo[a] = f32_up(reach);
        rp.reach_hi[a] = f32_down(rp.w[a] - reach);
        // the FP64 trial coordinate (x' - s, + L, - i w: a few roundings of
        // magnitude L) in place of the FP32 one: the cell rule's and these
        // roundings together stay far below 32 u64 L + 4 u64 w
        const double reach64 = h->Rc * 2.0 * (1.0 + 4.0 * kU64) + 32.0 * kU64 * rp.L[a] + 4.0 * kU64 * rp.w[a];
        rp.reach64_lo[a] = reach64;
        rp.reach64_hi[a] = rp.w[a] - reach64;
    }
    // FP32 cell rule of the rebuild: x and s truncated to FP32 (relative
    // error below 2^-23), y32 = x32 - s32 (+ L32), t32 = y32 * inv_w32 (each
    // rounding 2^-24 of its magnitude; L32 and inv_w32 within 2^-24).  Then
    // |y32 - (x - s)| < (2^-23 + 2^-24) L + 2^-23 w before the wrap, and
    // |t32 - t64| < 7 2^-24 nc + 2^-23 in cells, t64 the contract's product
    // (within 3 u64 nc of the exact one).  Both bounds are doubled.
    for (int a = 0; a < 3; ++a) {
        rp.L32[a] = (float)rp.L[a];
        rp.inv_w32[a] = (float)rp.inv_w[a];
        const double ey = (0x1.0p-23 + 0x1.0p-24) * rp.L[a] + 0x1.0p-23 * rp.w[a] + 0x1.0p-126;
        const double et = 7.0 * 0x1.0p-24 * (double)rp.nc[a] + 0x1.0p-23 + 3.0 * kU64 * (double)rp.nc[a];
        rp.cell_ey[a] = f32_up(2.0 * ey);
        rp.cell_et[a] = f32_up(2.0 * et);
    }
    rp.sat_e = f32_up(g.e_sat);
    rp.e_dlt32 = f32_up(g.e_dlt);
    rp.e_ori32 = f32_up(g.e_ori);
    rp.e_in = g.e_in;
    rp.e_cull = g.e_cull;
    rp.e_sat = g.e_sat;
    return 0;
}

int check_moves(double d, double a, uint32_t nselect)
{
    // (nonzero sizes below 1e-250 would make d * 2^-53 subnormal)
    if (!is_finite(d) || d < 0.0 || (d > 0.0 && d < 1e-250)) return HPMC_ERR_INVALID_ARG;
    if (!is_finite(a) || a < 0.0 || a >= 3.14159 || (a > 0.0 && a < 1e-250)) return HPMC_ERR_INVALID_ARG;
    if (nselect == 0 || nselect > 65535) return HPMC_ERR_INVALID_ARG;
    return 0;
}

int check_config(int dim, const HostRep& hr, const double* pos, const double* orient)
{
    if (!pos || !orient) return HPMC_ERR_INVALID_ARG;
    const int qd = dim == 2 ? 2 : 4;
    for (uint32_t i = 0; i < hr.N; ++i) {
        for (int a = 0; a < dim; ++a) {
            const double x = pos[(size_t)i * dim + a];
            if (!is_finite(x) || x < 0.0 || x >= hr.L[a]) return HPMC_ERR_INVALID_ARG;
        }
        double n2 = 0.0;
        for (int a = 0; a < qd; ++a) {
            const double q = orient[(size_t)i * qd + a];
            if (!is_finite(q)) return HPMC_ERR_INVALID_ARG;
            n2 += q * q;
        }
        if (std::fabs(n2 - 1.0) > 1e-6) return HPMC_ERR_INVALID_ARG;
    }
    return 0;
}

// the half-width of the rotation and the translation need the filter margins
// recomputed; items per set depend only on the cell grid
void build_item_tables(hpmc_batch* h, std::vector<uint32_t>& tab)
{
    tab.assign(kNumGroups * (h->R + 1), 0);
    h->items_per_set.assign(kNumGroups, 0);
    for (int gi = 0; gi < kNumGroups; ++gi) {
        const int S = cells_per_item(kGroupSizes[gi]);
        uint32_t acc = 0;
        for (uint32_t r = 0; r < h->R; ++r) {
            tab[gi * (h->R + 1) + r] = acc;
            const Rep& rp = h->reps[r];
            const uint32_t nax = (uint32_t)rp.nc[0] / 2;
            const uint32_t spr = (nax + S - 1) / S;
            uint32_t rows = (uint32_t)rp.nc[1] / 2;
            if (h->dim == 3) rows *= (uint32_t)rp.nc[2] / 2;
            acc += rows * spr;
        }
        tab[gi * (h->R + 1) + h->R] = acc;
        h->items_per_set[gi] = acc;
    }
}

void invalidate_graph(hpmc_batch* h)
{
    h->cfg_valid = false;
    for (int p = 0; p < 2; ++p) {
        if (h->graph[p]) {
            cudaGraphExecDestroy(h->graph[p]);
            h->graph[p] = nullptr;
        }
        if (h->graph_long[p]) {
            cudaGraphExecDestroy(h->graph_long[p]);
            h->graph_long[p] = nullptr;
        }
    }
}

int upload_reps(hpmc_batch* h, cudaStream_t st)
{
    CK(cudaMemcpyAsync((void*)h->dv.reps, h->reps.data(), sizeof(Rep) * h->R, cudaMemcpyHostToDevice, st));
    return 0;
}

SetKernel pick_kernel(const hpmc_batch* h)
{
    const bool f32 = h->precision == HPMC_FP32_FILTERED;
    if (h->dim == 2) {
        const bool fixed = h->nv == 5;
        if (h->G == 0) return set2d_direct_kernel(fixed, f32);
        return f32 ? set2d_f32_kernel(h->G, fixed) : set2d_f64_kernel(h->G, fixed);
    }
    if (h->G == 0) return SetKernel{ nullptr, 0 };
    return f32 ? set3d_f32_kernel(h->G, h->nv) : set3d_f64_kernel(h->G, h->nv);
}

// enqueue the rebuild of the cell list from buffer `cur` into cur ^ 1
// Launch configuration with programmatic stream serialisation: the kernel
// may be scheduled while its predecessor in the stream still runs; it waits
// for it in pdl_enter() before touching memory.
struct PdlLaunch {
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[1];
    PdlLaunch(dim3 grid, dim3 block, size_t smem, cudaStream_t st)
    {
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
    }
    PdlLaunch(const PdlLaunch&) = delete;
    PdlLaunch& operator=(const PdlLaunch&) = delete;
};

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*fn)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args)
{
    PdlLaunch L(grid, block, 0, st);
    return cudaLaunchKernelEx(&L.cfg, fn, args...);
}

int enqueue_rebuild(hpmc_batch* h, cudaStream_t st, bool with_shift)
{
    const uint32_t T = 256;
    const dim3 gp((h->ntot + T - 1) / T), gc((h->ctot + T - 1) / T);
    const int cur = h->cur;
    if (with_shift) {
        CK(launch_pdl(k_shift, dim3((h->R + 127) / 128), dim3(128), st, h->dv));
        if (h->use_selects) {
            // fork: the select table of this sweep (it needs the advanced
            // sweep counter only) alongside the rebuild; joined in enqueue_sets
            CK(cudaEventRecord(h->ev_fork, st));
            CK(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
            CK(launch_selects(h->dv, h->dim, h->sel_grid, h->side));
            CK(cudaEventRecord(h->ev_join, h->side));
        }
    }
    CK(launch_pdl(k_count, gp, dim3(T), st, h->dv, cur));
    CK(launch_pdl(k_scan_tiles, dim3(h->ntiles), dim3(kScanThreads), st, h->dv));
    if (h->ntiles > 1) {
        CK(launch_pdl(k_scan_sums, dim3(1), dim3(kScanThreads), st, h->dv, h->ntiles));
        CK(launch_pdl(k_scan_add, gc, dim3(T), st, h->dv));
    }
    CK(launch_pdl(k_scatter_tags, gp, dim3(T), st, h->dv, cur));
    CK(launch_pdl(k_place, gp, dim3(T), st, h->dv, cur));
    return 0;
}

// the set kernels that read their first selects from the sweep's table (the
// latency regime; the direct kernel draws its selects itself)
bool uses_select_table(int G)
{
    return G >= 8;
}

// Select table for the latency-regime kernels: one record for each of the
// first min(nselect, G) selects of every cell of every replica (the chunk in
// which idle lanes would otherwise carry the FP64 steps), grown (never
// shrunk) with the cell count or the stride.  Runs when the launch
// configuration is rebuilt, outside any stream capture of this library.
int prepare_selects(hpmc_batch* h)
{
    h->use_selects = uses_select_table(h->G);
    if (!h->use_selects) return 0;
    uint32_t stride = 1;
    for (const HostRep& r : h->hr) stride = std::max(stride, r.nselect);
    stride = std::min<uint32_t>(stride, (uint32_t)h->G);
    const uint64_t need = (uint64_t)h->ctot * stride;
    const size_t rec = select_record_bytes(h->dim);
    if (need > h->msel_cap) {
        if (h->msel) {
            CK(cudaDeviceSynchronize());
            h->allocs.erase(std::find(h->allocs.begin(), h->allocs.end(), h->msel));
            cudaFree(h->msel);
            h->msel = nullptr;
            h->msel_cap = 0;
            h->dv.msel = nullptr;
            h->dv.msel_n = 0;
        }
        uint4* p = nullptr;
        const int rc = dalloc(h, &p, need * rec / sizeof(uint4));
        if (rc) return rc;
        h->msel = p;
        h->msel_cap = need;
    }
    if (!h->side) CK(cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
    if (!h->ev_fork) CK(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
    if (!h->ev_join) CK(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    h->dv.msel = h->msel;
    h->dv.msel_stride = stride;
    h->dv.msel_n = h->msel_cap;
    const uint64_t blocks = (need + 255) / 256;
    h->sel_grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(blocks, (uint64_t)h->num_sms * 8));
    return 0;
}

int prepare_set(hpmc_batch* h)
{
    if (h->cfg_valid) return 0;
    const SetKernel K = pick_kernel(h);
    if (!K.fn) return HPMC_ERR_INVALID_ARG;
    const int gi = gidx_of(h->G);
    const uint32_t items = h->items_per_set[gi];
    const size_t smem = K.smem_per_warp * (size_t)h->wpb;
    const uint32_t blocks_needed = (items + h->wpb - 1) / h->wpb;
    int per_sm = 0;
    CK(cudaFuncSetAttribute(K.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, K.fn, 32 * h->wpb, smem));
    if (per_sm < 1) return HPMC_ERR_INVALID_ARG;
    h->cfg_fn = K.fn;
    h->cfg_smem = smem;
    h->cfg_grid = std::max<uint32_t>(1, std::min<uint32_t>(blocks_needed, (uint32_t)(per_sm * h->num_sms)));
    int rc = prepare_selects(h);
    if (rc) return rc;
    h->cfg_valid = true;
    return 0;
}

// the set kernels of one sweep (after its rebuild) into buffer cur ^ 1
int enqueue_sets(hpmc_batch* h, cudaStream_t st)
{
    if (h->use_selects) CK(cudaStreamWaitEvent(st, h->ev_join, 0));   // join the select table
    const int nxt = h->cur ^ 1;
    const int gi = gidx_of(h->G);
    const uint32_t* ib = h->item_base_dev + (size_t)gi * (h->R + 1);
    const int nsets = 1 << h->dim;
    for (int sigma = 0; sigma < nsets; ++sigma) {
        void* args[5];
        int nx = nxt, sg = sigma;
        args[0] = &h->dv;
        args[1] = h->dim == 2 ? (void*)&h->sh2 : (void*)&h->sh3;
        args[2] = &nx;
        args[3] = &sg;
        args[4] = (void*)&ib;
        // Sets 1.. are launched with programmatic stream serialisation and
        // only wait (pdl_wait): the next set's launch is prepared while the
        // previous one drains (4096-pentagon fluid +2.5%).  Set 0 keeps the
        // full dependency on the rebuild, whose kernels let their successor
        // be scheduled early: its blocks would wait beside k_place.
        PdlLaunch L(dim3(h->cfg_grid), dim3(32 * h->wpb), h->cfg_smem, st);
        if (sigma == 0) L.cfg.numAttrs = 0;
        CK(cudaLaunchKernelExC(&L.cfg, h->cfg_fn, args));
    }
    h->cur = nxt;
    return 0;
}

int enqueue_sweep(hpmc_batch* h, cudaStream_t st)
{
    int rc = prepare_set(h);
    if (rc) return rc;
    rc = enqueue_rebuild(h, st, true);
    if (rc) return rc;
    return enqueue_sets(h, st);
}

// unsorted copy of the state (tag order) into buffer cur ^ 1
__global__ void k_unsort(Dev dv, int cur)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dv.ntot) return;
    const Bufs& S = dv.buf[cur];
    const Bufs& D = dv.buf[cur ^ 1];
    const uint32_t r = dv.rep_of[i];
    const uint32_t o = dv.reps[r].pbase + S.tag[i];
    D.px[o] = S.px[i];
    D.py[o] = S.py[i];
    D.q0[o] = S.q0[i];
    D.q1[o] = S.q1[i];
    D.tag[o] = S.tag[i];
    if (dv.dim == 3) {
        D.pz[o] = S.pz[i];
        D.q2[o] = S.q2[i];
        D.q3[o] = S.q3[i];
    }
}

// interleaved tag-order state (stage: pos[ntot * dim], then orient[ntot * qd])
// into buffer cur, with identity tags
__global__ void k_from_interleaved(Dev dv, int cur, const double* __restrict__ stage)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dv.ntot) return;
    const Bufs& B = dv.buf[cur];
    const size_t n = dv.ntot;
    if (dv.dim == 2) {
        const double2 p = reinterpret_cast<const double2*>(stage)[i];
        const double2 q = reinterpret_cast<const double2*>(stage + 2 * n)[i];
        B.px[i] = p.x; B.py[i] = p.y;
        B.q0[i] = q.x; B.q1[i] = q.y;
    } else {
        B.px[i] = stage[3 * (size_t)i]; B.py[i] = stage[3 * (size_t)i + 1]; B.pz[i] = stage[3 * (size_t)i + 2];
        const double* q = stage + 3 * n + 4 * (size_t)i;
        B.q0[i] = q[0]; B.q1[i] = q[1]; B.q2[i] = q[2]; B.q3[i] = q[3];
    }
    B.tag[i] = i - dv.reps[dv.rep_of[i]].pbase;
}

// buffer cur (cell-sorted, with tags) into the interleaved tag-order layout
__global__ void k_to_interleaved(Dev dv, int cur, double* __restrict__ stage)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dv.ntot) return;
    const Bufs& B = dv.buf[cur];
    const size_t n = dv.ntot;
    const size_t o = dv.reps[dv.rep_of[i]].pbase + B.tag[i];
    if (dv.dim == 2) {
        reinterpret_cast<double2*>(stage)[o] = make_double2(B.px[i], B.py[i]);
        reinterpret_cast<double2*>(stage + 2 * n)[o] = make_double2(B.q0[i], B.q1[i]);
    } else {
        stage[3 * o] = B.px[i]; stage[3 * o + 1] = B.py[i]; stage[3 * o + 2] = B.pz[i];
        double* q = stage + 3 * n + 4 * o;
        q[0] = B.q0[i]; q[1] = B.q1[i]; q[2] = B.q2[i]; q[3] = B.q3[i];
    }
}

__global__ void k_identity_tags(Dev dv, int cur)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dv.ntot) return;
    dv.buf[cur].tag[i] = i - dv.reps[dv.rep_of[i]].pbase;
}

int read_error(hpmc_batch* h)
{
    int e = 0;
    CK(cudaMemcpy(&e, h->dv.error, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        CK(cudaMemset(h->dv.error, 0, sizeof(int)));
        if (e & ERR_TIMEOUT) return HPMC_ERR_TIMEOUT;
        return HPMC_ERR_CAPACITY;
    }
    int p = h->pending_error;
    h->pending_error = 0;
    return p;
}

// copy a state in tag order into buffer cur (all replicas, concatenated)
int upload_all(hpmc_batch* h, const double* pos, const double* orient, cudaStream_t st)
{
    const int dim = h->dim, qd = dim == 2 ? 2 : 4;
    const size_t n = h->ntot;
    std::vector<double> col(n);
    Bufs& B = h->dv.buf[h->cur];
    double* dst_p[3] = { B.px, B.py, B.pz };
    double* dst_q[4] = { B.q0, B.q1, B.q2, B.q3 };
    for (int a = 0; a < dim; ++a) {
        for (size_t i = 0; i < n; ++i) col[i] = pos[i * dim + a];
        CK(cudaMemcpyAsync(dst_p[a], col.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
    }
    for (int a = 0; a < qd; ++a) {
        for (size_t i = 0; i < n; ++i) col[i] = orient[i * qd + a];
        CK(cudaMemcpyAsync(dst_q[a], col.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
    }
    k_identity_tags<<<(h->ntot + 255) / 256, 256, 0, st>>>(h->dv, h->cur);
    CK(cudaGetLastError());
    return 0;
}

}  // namespace

// ======================================================================= ABI
extern "C" {

const char* hpmc_strerror(int code)
{
    switch (code) {
    case HPMC_OK: return "ok";
    case HPMC_ERR_INVALID_ARG: return "invalid argument";
    case HPMC_ERR_BOX_TOO_SMALL: return "box too small: fewer than 4 cells on an axis";
    case HPMC_ERR_OVERLAP: return "overlapping configuration";
    case HPMC_ERR_OOM: return "device allocation failed";
    case HPMC_ERR_CUDA: return "CUDA runtime error";
    case HPMC_ERR_TIMEOUT: return "bounded device wait gave up";
    case HPMC_ERR_CAPACITY: return "a cell stencil exceeded the staging capacity";
    case HPMC_ERR_NOT_READY: return "call order violated";
    case HPMC_ERR_SCRATCH_LIMIT: return "size exceeds the fixed scratch of the no-allocation entry point";
    default: return "unknown error";
    }
}

int hpmc_batch_create(int dim, const double* verts, uint32_t nv, double w_min, uint32_t R,
                      const hpmc_replica_desc_t* reps, hpmc_t* out)
{
    if (!out || !reps || R == 0) return HPMC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!is_finite(w_min) || w_min < 0.0) return HPMC_ERR_INVALID_ARG;
    hpmc_batch* h = new (std::nothrow) hpmc_batch();
    if (!h) return HPMC_ERR_OOM;
    int rc = shape_setup(h, dim, verts, nv);
    if (rc) { delete h; return rc; }
    h->w_min = w_min;
    h->R = R;
    h->hr.resize(R);
    h->reps.resize(R);
    uint64_t ntot = 0, ctot = 0;
    for (uint32_t r = 0; r < R; ++r) {
        const hpmc_replica_desc_t& d = reps[r];
        HostRep& hr = h->hr[r];
        if (d.N == 0) { delete h; return HPMC_ERR_INVALID_ARG; }
        hr.N = d.N;
        for (int a = 0; a < 3; ++a) hr.L[a] = d.box[a];
        hr.seed = d.seed;
        hr.d = d.d;
        hr.a = d.a;
        hr.nselect = d.nselect;
        rc = check_moves(d.d, d.a, d.nselect);
        if (!rc) rc = rep_geometry(h, hr, h->reps[r]);
        if (!rc) rc = check_config(dim, hr, d.pos, d.orient);
        if (rc) { delete h; return rc; }
        h->reps[r].pbase = (uint32_t)ntot;
        h->reps[r].cbase = (uint32_t)ctot;
        ntot += d.N;
        ctot += h->reps[r].ncell;
        if (ntot > 0x7fffffffull || ctot > 0x7fffffffull) { delete h; return HPMC_ERR_INVALID_ARG; }
    }
    h->ntot = (uint32_t)ntot;
    h->ctot = (uint32_t)ctot;
    h->ntiles = (h->ctot + kScanTile - 1) / kScanTile;
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) { delete h; return cuda_fail(ce); }

    Dev& dv = h->dv;
    dv.dim = dim;
    dv.R = R;
    dv.ntot = h->ntot;
    dv.ctot = h->ctot;
    auto fail = [&](int code) { hpmc_destroy(h); return code; };
    Rep* reps_dev = nullptr;
    uint32_t* rep_of = nullptr;
    if ((rc = dalloc(h, &reps_dev, R))) return fail(rc);
    dv.reps = reps_dev;
    if ((rc = dalloc(h, &rep_of, h->ntot))) return fail(rc);
    dv.rep_of = rep_of;
    for (int b = 0; b < 2; ++b) {
        Bufs& B = dv.buf[b];
        if ((rc = dalloc(h, &B.px, h->ntot)) || (rc = dalloc(h, &B.py, h->ntot)) ||
            (rc = dalloc(h, &B.q0, h->ntot)) || (rc = dalloc(h, &B.q1, h->ntot)) ||
            (rc = dalloc(h, &B.f4a, h->ntot)) || (rc = dalloc(h, &B.tag, h->ntot)))
            return fail(rc);
        if (dim == 3) {
            if ((rc = dalloc(h, &B.pz, h->ntot)) || (rc = dalloc(h, &B.q2, h->ntot)) ||
                (rc = dalloc(h, &B.q3, h->ntot)) || (rc = dalloc(h, &B.f4b, h->ntot)))
                return fail(rc);
        }
    }
    h->ctot_cap = h->ctot;
    if ((rc = dalloc(h, &dv.count, h->ctot)) || (rc = dalloc(h, &dv.start, (size_t)h->ctot + 1)) ||
        (rc = dalloc(h, &dv.tile_sums, h->ntiles)) || (rc = dalloc(h, &dv.cellid, h->ntot)) ||
        (rc = dalloc(h, &dv.slot, h->ntot)) || (rc = dalloc(h, &dv.tmp_tag, h->ntot)) ||
        (rc = dalloc(h, &dv.shift, 3 * (size_t)R)) || (rc = dalloc(h, &dv.sweep, R)) ||
        (rc = dalloc(h, &dv.counters, (size_t)R * kNumCounters)) || (rc = dalloc(h, &dv.error, 1)) ||
        (rc = dalloc(h, &h->item_base_dev, kNumGroups * ((size_t)R + 1))) || (rc = dalloc(h, &h->check_out, 1)))
        return fail(rc);
#ifdef HPMC_TRACE
    dv.trace_warps = 65536;
    if ((rc = dalloc(h, &dv.trace, (size_t)dv.trace_warps * kTracePoints))) return fail(rc);
    if (cudaMemset(dv.trace, 0, sizeof(unsigned long long) * dv.trace_warps * kTracePoints) != cudaSuccess)
        return fail(HPMC_ERR_CUDA);
#else
    dv.trace = nullptr;
    dv.trace_warps = 0;
#endif

    std::vector<uint32_t> tab;
    build_item_tables(h, tab);
    std::vector<uint32_t> ro(h->ntot);
    for (uint32_t r = 0; r < R; ++r)
        for (uint32_t i = 0; i < h->hr[r].N; ++i) ro[h->reps[r].pbase + i] = r;
    const uint32_t nt = h->ntot;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpy(rep_of, ro.data(), sizeof(uint32_t) * nt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->item_base_dev, tab.data(), sizeof(uint32_t) * tab.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(reps_dev, h->reps.data(), sizeof(Rep) * R, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dv.count, 0, sizeof(uint32_t) * h->ctot);
    if (e == cudaSuccess) e = cudaMemcpy(dv.start + h->ctot, &nt, sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(dv.sweep, 0, sizeof(uint64_t) * R);
    if (e == cudaSuccess) e = cudaMemset(dv.counters, 0, sizeof(unsigned long long) * R * kNumCounters);
    if (e == cudaSuccess) e = cudaMemset(dv.error, 0, sizeof(int));
    if (e != cudaSuccess) return fail(cuda_fail(e));
    // initial configuration (tag order) into buffer 0
    std::vector<double> P((size_t)h->ntot * dim), Q((size_t)h->ntot * (dim == 2 ? 2 : 4));
    const int qd = dim == 2 ? 2 : 4;
    for (uint32_t r = 0; r < R; ++r) {
        std::memcpy(P.data() + (size_t)h->reps[r].pbase * dim, reps[r].pos, sizeof(double) * reps[r].N * dim);
        std::memcpy(Q.data() + (size_t)h->reps[r].pbase * qd, reps[r].orient, sizeof(double) * reps[r].N * qd);
    }
    h->cur = 0;
    if ((rc = upload_all(h, P.data(), Q.data(), 0))) return fail(rc);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(cuda_fail(e));
    *out = h;
    return 0;
}

int hpmc_create(const double* box, int dim, uint32_t N, const double* verts, uint32_t nv,
                const double* pos, const double* orient, uint64_t seed, double w_min, hpmc_t* out)
{
    if (!box) return HPMC_ERR_INVALID_ARG;
    hpmc_replica_desc_t d{};
    d.N = N;
    for (int a = 0; a < 3; ++a) d.box[a] = (a < dim) ? box[a] : 1.0;
    d.pos = pos;
    d.orient = orient;
    d.seed = seed;
    d.d = 0.1;
    d.a = 0.1;
    d.nselect = 4;
    return hpmc_batch_create(dim, verts, nv, w_min, 1, &d, out);
}

int hpmc_destroy(hpmc_t h)
{
    if (!h) return HPMC_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    invalidate_graph(h);
    if (h->graph_stream) cudaStreamDestroy(h->graph_stream);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    for (void* p : h->allocs) cudaFree(p);
    if (h->sdf_hist) cudaFree(h->sdf_hist);
    delete h;
    return 0;
}

int hpmc_set_moves(hpmc_t h, int32_t r, double d, double a, uint32_t nselect)
{
    if (!h) return HPMC_ERR_INVALID_ARG;
    int rc = check_moves(d, a, nselect);
    if (rc) return rc;
    if (r >= (int32_t)h->R || r < -1) return HPMC_ERR_INVALID_ARG;
    CK(cudaDeviceSynchronize());
    for (uint32_t i = 0; i < h->R; ++i) {
        if (r >= 0 && (uint32_t)r != i) continue;
        h->hr[i].d = d;
        h->hr[i].a = a;
        h->hr[i].nselect = nselect;
        const uint32_t pb = h->reps[i].pbase, cb = h->reps[i].cbase;
        rc = rep_geometry(h, h->hr[i], h->reps[i]);
        h->reps[i].pbase = pb;
        h->reps[i].cbase = cb;
        if (rc) return rc;
    }
    invalidate_graph(h);
    rc = upload_reps(h, 0);
    if (rc) return rc;
    CK(cudaDeviceSynchronize());
    return 0;
}

int relayout(hpmc_batch* h);

int hpmc_set_cell_width_min(hpmc_t h, double w_min)
{
    if (!h || !is_finite(w_min) || w_min < 0.0) return HPMC_ERR_INVALID_ARG;
    CK(cudaDeviceSynchronize());
    const double w_old = h->w_min;
    h->w_min = w_min;
    std::vector<Rep> fresh(h->reps);
    for (uint32_t r = 0; r < h->R; ++r) {
        const int rc = rep_geometry(h, h->hr[r], fresh[r]);
        if (rc) {
            h->w_min = w_old;                           // the grid is unchanged
            return rc;
        }
        fresh[r].pbase = h->reps[r].pbase;
    }
    const std::vector<Rep> old = h->reps;
    h->reps = fresh;                                    // cbase: relayout
    const int rc = relayout(h);
    if (rc) {
        // allocation failed: back to the old grid (it fits the arrays we have)
        h->w_min = w_old;
        h->reps = old;
        const int rc2 = relayout(h);
        return rc2 ? rc2 : rc;
    }
    CK(cudaDeviceSynchronize());                        // the next sweep rebuilds cells and mirrors
    return 0;
}

int hpmc_set_precision(hpmc_t h, int mode)
{
    if (!h || (mode != HPMC_FP64 && mode != HPMC_FP32_FILTERED)) return HPMC_ERR_INVALID_ARG;
    h->precision = mode;
    invalidate_graph(h);
    return 0;
}

int hpmc_set_group_size(hpmc_t h, int lanes_per_cell, int warps_per_block)
{
    if (!h || gidx_of(lanes_per_cell) < 0 || warps_per_block < 1 || warps_per_block > 16)
        return HPMC_ERR_INVALID_ARG;
    const SetKernel K = [&] {
        const int G0 = h->G;
        h->G = lanes_per_cell;
        SetKernel k = pick_kernel(h);
        h->G = G0;
        return k;
    }();
    if (!K.fn || K.smem_per_warp * (size_t)warps_per_block > 227 * 1024) return HPMC_ERR_INVALID_ARG;
    cudaFuncAttributes fa{};
    CK(cudaFuncGetAttributes(&fa, K.fn));
    if (32 * warps_per_block > fa.maxThreadsPerBlock) return HPMC_ERR_INVALID_ARG;   // launch bounds
    h->G = lanes_per_cell;
    h->wpb = warps_per_block;
    invalidate_graph(h);
    return 0;
}

int hpmc_sweep(hpmc_t h, uint32_t n, void* stream)
{
    if (!h) return HPMC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    h->last_stream = st;
    for (uint32_t s = 0; s < n; ++s) {
        int rc = enqueue_sweep(h, st);
        if (rc) return rc;
    }
    return 0;
}

static constexpr uint32_t kLongGraph = 16;

// capture `sweeps` sweeps (even) from the current parity into *out
static int capture_sweeps(hpmc_batch* h, cudaStream_t st, uint32_t sweeps, cudaGraphExec_t* out)
{
    int prc = prepare_set(h);
    if (prc) return prc;
    if (!h->graph_stream) CK(cudaStreamCreateWithFlags(&h->graph_stream, cudaStreamNonBlocking));
    CK(cudaStreamSynchronize(st));
    const int cur0 = h->cur;
    CK(cudaStreamBeginCapture(h->graph_stream, cudaStreamCaptureModeThreadLocal));
    int rc = 0;
    for (uint32_t k = 0; k < sweeps && !rc; ++k) rc = enqueue_sweep(h, h->graph_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->graph_stream, &g);
    h->cur = cur0;
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { *out = nullptr; return cuda_fail(e); }
    return 0;
}

int hpmc_sweep_graph(hpmc_t h, uint32_t n, void* stream)
{
    if (!h) return HPMC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    h->last_stream = st;
    uint32_t s = 0;
    if (n >= kLongGraph) {
        if (!h->graph_long[h->cur]) {
            const int rc = capture_sweeps(h, st, kLongGraph, &h->graph_long[h->cur]);
            if (rc) return rc;
        }
        for (; s + kLongGraph <= n; s += kLongGraph) CK(cudaGraphLaunch(h->graph_long[h->cur], st));
    }
    if (n - s >= 2 && !h->graph[h->cur]) {
        const int rc = capture_sweeps(h, st, 2, &h->graph[h->cur]);
        if (rc) return rc;
    }
    for (; s + 2 <= n; s += 2) CK(cudaGraphLaunch(h->graph[h->cur], st));
    if (s < n) {
        int rc = enqueue_sweep(h, st);
        if (rc) return rc;
    }
    return 0;
}

int hpmc_sync(hpmc_t h)
{
    if (!h) return HPMC_ERR_INVALID_ARG;
    CK(cudaDeviceSynchronize());
    return read_error(h);
}

int hpmc_counters(hpmc_t h, int32_t r, hpmc_counters_t* out)
{
    if (!h || !out || r < -1 || r >= (int32_t)h->R) return HPMC_ERR_INVALID_ARG;
    CK(cudaDeviceSynchronize());
    std::vector<unsigned long long> c((size_t)h->R * kNumCounters);
    CK(cudaMemcpy(c.data(), h->dv.counters, sizeof(unsigned long long) * c.size(), cudaMemcpyDeviceToHost));
    unsigned long long s[kNumCounters] = {};
    for (uint32_t i = 0; i < h->R; ++i) {
        if (r >= 0 && (uint32_t)r != i) continue;
        for (int k = 0; k < kNumCounters; ++k) s[k] += c[(size_t)i * kNumCounters + k];
    }
    out->moves = s[CNT_MOVES];
    out->accept = s[CNT_ACCEPT];
    out->reject_overlap = s[CNT_REJ_OVERLAP];
    out->reject_boundary = s[CNT_REJ_BOUNDARY];
    out->cull_pairs = s[CNT_CULL];
    out->overlap_checks = s[CNT_CHECKS];
    out->fp64_rechecks = s[CNT_RECHECK];
    out->gjk_cap = s[CNT_GJKCAP];
    return read_error(h);
}

int hpmc_reset_counters(hpmc_t h)
{
    if (!h) return HPMC_ERR_INVALID_ARG;
    CK(cudaDeviceSynchronize());
    CK(cudaMemset(h->dv.counters, 0, sizeof(unsigned long long) * h->R * kNumCounters));
    return 0;
}

int hpmc_check_overlaps(hpmc_t h, int32_t r, uint64_t* n_pairs)
{
    if (!h || !n_pairs || r < -1 || r >= (int32_t)h->R) return HPMC_ERR_INVALID_ARG;
    CK(cudaDeviceSynchronize());
    // a cell list with a zero shift, then every pair of stencil neighbours
    CK(cudaMemset(h->dv.shift, 0, sizeof(double) * 3 * h->R));
    int rc = enqueue_rebuild(h, 0, false);
    if (rc) return rc;
    h->cur ^= 1;
    CK(cudaMemset(h->check_out, 0, sizeof(unsigned long long)));
    const int T = 128;
    if (h->dim == 2) {
        if (h->nv == 5) k_check2d<5><<<(h->ntot + T - 1) / T, T>>>(h->dv, h->sh2, h->cur, r, h->check_out);
        else k_check2d<0><<<(h->ntot + T - 1) / T, T>>>(h->dv, h->sh2, h->cur, r, h->check_out);
    } else {
        rc = hpmc_check3d_launch(h->dv, h->sh3, h->cur, r, h->check_out, h->ntot);
        if (rc) return rc;
    }
    CK(cudaGetLastError());
    unsigned long long n = 0;
    CK(cudaMemcpy(&n, h->check_out, sizeof(n), cudaMemcpyDeviceToHost));
    *n_pairs = n;
    return read_error(h);
}

int hpmc_sdf(hpmc_t h, int32_t r, double x_max, uint32_t nbins, uint64_t* hist)
{
    if (!h || !hist || r < -1 || r >= (int32_t)h->R) return HPMC_ERR_INVALID_ARG;
    if (!(x_max > 0.0) || !(x_max < 1.0) || nbins == 0 || nbins > (1u << 20)) return HPMC_ERR_INVALID_ARG;
    const double sigma = h->Rc + h->Rc;
    const double rmax = sigma / (1.0 - x_max);
    for (uint32_t q = 0; q < h->R; ++q) {
        if (r >= 0 && (uint32_t)r != q) continue;
        for (int a = 0; a < h->dim; ++a)
            if (rmax > h->reps[q].w[a]) return HPMC_ERR_INVALID_ARG;
    }
    CK(cudaDeviceSynchronize());
    if (h->sdf_cap < nbins) {
        if (h->sdf_hist) cudaFree(h->sdf_hist);
        h->sdf_hist = nullptr;
        h->sdf_cap = 0;
        CK(cudaMalloc(&h->sdf_hist, sizeof(unsigned long long) * nbins));
        h->sdf_cap = nbins;
    }
    // a cell list with a zero shift, then every pair of stencil neighbours
    CK(cudaMemset(h->dv.shift, 0, sizeof(double) * 3 * h->R));
    int rc = enqueue_rebuild(h, 0, false);
    if (rc) return rc;
    h->cur ^= 1;
    CK(cudaMemset(h->sdf_hist, 0, sizeof(unsigned long long) * nbins));
    const int T = 128;
    if (h->nv == 0)
        k_sdf<<<(h->ntot + T - 1) / T, T>>>(h->dv, h->cur, sigma, x_max, (double)nbins / x_max, nbins, r,
                                            h->sdf_hist);
    else
        k_sdf_shaped<<<(h->ntot + T - 1) / T, T>>>(h->dv, h->cur, h->sh2, h->sh3, x_max / (double)nbins, nbins, r,
                                                   h->sdf_hist);
    CK(cudaGetLastError());
    std::vector<unsigned long long> got(nbins);
    CK(cudaMemcpy(got.data(), h->sdf_hist, sizeof(unsigned long long) * nbins, cudaMemcpyDeviceToHost));
    for (uint32_t b = 0; b < nbins; ++b) hist[b] += got[b];
    return read_error(h);
}

// Cell offsets, scan tiles and work-item tables after a replica's cell grid
// changed (volume moves); the count / start arrays grow by doubling.
int relayout(hpmc_batch* h)
{
    uint64_t ctot = 0;
    for (uint32_t r = 0; r < h->R; ++r) {
        h->reps[r].cbase = (uint32_t)ctot;
        ctot += h->reps[r].ncell;
    }
    if (ctot > 0x7fffffffull) return HPMC_ERR_INVALID_ARG;
    Dev& dv = h->dv;
    if (ctot > h->ctot_cap) {
        // all three arrays first, switched only together: a failed allocation
        // leaves the device layout as it was (the caller restores the host's)
        const uint32_t cap = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(ctot, 2ull * h->ctot_cap), 0x7fffffffull);
        const uint32_t nt = (cap + kScanTile - 1) / kScanTile;
        uint32_t *cnt = nullptr, *sta = nullptr, *tsu = nullptr;
        int rc;
        if ((rc = dalloc(h, &cnt, cap)) || (rc = dalloc(h, &sta, (size_t)cap + 1)) || (rc = dalloc(h, &tsu, nt)))
            return rc;
        dv.count = cnt;
        dv.start = sta;
        dv.tile_sums = tsu;
        h->ctot_cap = cap;
    }
    h->ctot = (uint32_t)ctot;
    h->ntiles = (h->ctot + kScanTile - 1) / kScanTile;
    dv.ctot = h->ctot;
    std::vector<uint32_t> tab;
    build_item_tables(h, tab);
    const uint32_t nt = h->ntot;
    CK(cudaMemcpy(h->item_base_dev, tab.data(), sizeof(uint32_t) * tab.size(), cudaMemcpyHostToDevice));
    CK(cudaMemset(dv.count, 0, sizeof(uint32_t) * h->ctot));
    CK(cudaMemcpy(dv.start + h->ctot, &nt, sizeof(uint32_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy((void*)dv.reps, h->reps.data(), sizeof(Rep) * h->R, cudaMemcpyHostToDevice));
    invalidate_graph(h);
    return 0;
}

// Positions of replica r (slots [pbase, pbase + n) of buffer b) scaled by f,
// wrapped onto [0, L') when the product rounds onto L'.
__global__ void k_scale(Dev dv, int b, uint32_t pbase, uint32_t n, double f, double L0, double L1, double L2)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Bufs& B = dv.buf[b];
    const uint32_t k = pbase + i;
    double x = B.px[k] * f;
    if (x >= L0) x = x - L0;
    B.px[k] = x;
    double y = B.py[k] * f;
    if (y >= L1) y = y - L1;
    B.py[k] = y;
    if (dv.dim == 3) {
        double z = B.pz[k] * f;
        if (z >= L2) z = z - L2;
        B.pz[k] = z;
    }
}

int hpmc_box_move(hpmc_t h, int32_t r, double beta_P, double dV_max, int* accepted)
{
    if (!h || !accepted || r < 0 || r >= (int32_t)h->R) return HPMC_ERR_INVALID_ARG;
    if (!is_finite(beta_P) || !is_finite(dV_max) || dV_max < 0.0) return HPMC_ERR_INVALID_ARG;
    *accepted = 0;
    CK(cudaDeviceSynchronize());
    HostRep& hr = h->hr[r];
    const int dim = h->dim;
    // the two numbers of attempt m: key = seed, ctr = (lo32(m), hi32(m), 0, 4 << 24)
    const uint64_t m = hr.box_moves++;
    uint32_t c[4] = { (uint32_t)m, (uint32_t)(m >> 32), 0u, 4u << 24 };
    philox_host(c, (uint32_t)hr.seed, (uint32_t)(hr.seed >> 32));
    const double u1 = u53_host(c[0], c[1]), u2 = u53_host(c[2], c[3]);
    double V = hr.L[0] * hr.L[1];
    if (dim == 3) V = V * hr.L[2];
    const double dV = dV_max * (2.0 * u1 - 1.0);
    const double Vn = V + dV;
    if (!(Vn > 0.0)) return 0;
    const double ratio = Vn / V;
    const double f = dim == 2 ? std::sqrt(ratio) : std::cbrt(ratio);
    HostRep trial = hr;
    for (int a = 0; a < dim; ++a) trial.L[a] = hr.L[a] * f;
    Rep rp_old = h->reps[r], rp_new = rp_old;
    if (rep_geometry(h, trial, rp_new)) return 0;      // fewer than 4 cells: rejected
    rp_new.pbase = rp_old.pbase;
    const bool grid_changed = rp_new.ncell != rp_old.ncell || rp_new.nc[0] != rp_old.nc[0] ||
                              rp_new.nc[1] != rp_old.nc[1] || rp_new.nc[2] != rp_old.nc[2];
    // save the replica's positions, scale them, switch to the trial geometry
    const uint32_t pb = rp_old.pbase, n = hr.N;
    const int cur0 = h->cur;
    Bufs& B = h->dv.buf[cur0];
    double* src[3] = { B.px, B.py, B.pz };
    for (int a = 0; a < dim; ++a) {
        if (!h->bak[a]) {
            int rc = dalloc(h, &h->bak[a], h->ntot);
            if (rc) return rc;
        }
        CK(cudaMemcpy(h->bak[a] + pb, src[a] + pb, sizeof(double) * n, cudaMemcpyDeviceToDevice));
    }
    k_scale<<<(n + 255) / 256, 256>>>(h->dv, cur0, pb, n, f, rp_new.L[0], rp_new.L[1], rp_new.L[2]);
    CK(cudaGetLastError());
    h->reps[r] = rp_new;
    int rc = grid_changed ? relayout(h) : upload_reps(h, 0);
    if (rc) {
        // the trial grid could not be laid out: positions and grid as before
        for (int a = 0; a < dim; ++a)
            CK(cudaMemcpy(src[a] + pb, h->bak[a] + pb, sizeof(double) * n, cudaMemcpyDeviceToDevice));
        h->reps[r] = rp_old;
        const int rc2 = grid_changed ? relayout(h) : upload_reps(h, 0);
        return rc2 ? rc2 : rc;
    }
    // any overlapping pair of the replica rejects (FP64 contract, cell list of the trial box)
    uint64_t n_ov = 0;
    rc = hpmc_check_overlaps(h, r, &n_ov);
    if (rc) return rc;
    bool acc = false;
    if (n_ov == 0) {
        const double arg = -beta_P * dV + (double)n * std::log(ratio);
        acc = u2 < std::exp(arg);
    }
    if (acc) {
        hr.L[0] = trial.L[0]; hr.L[1] = trial.L[1]; hr.L[2] = trial.L[2];
        *accepted = 1;
        return 0;
    }
    // rejected: the old buffer (untouched but for the scaled positions) and geometry
    h->cur = cur0;
    for (int a = 0; a < dim; ++a)
        CK(cudaMemcpy(src[a] + pb, h->bak[a] + pb, sizeof(double) * n, cudaMemcpyDeviceToDevice));
    h->reps[r] = rp_old;
    rc = grid_changed ? relayout(h) : upload_reps(h, 0);
    if (rc) return rc;
    CK(cudaDeviceSynchronize());      // (the next sweep rebuilds the cell list and mirrors)
    return read_error(h);
}

// Mean squared displacement, by particle tag: mode 0 resets (the current
// positions become the reference), mode 1 adds the minimum-image step since
// the last call to the unwrapped displacement.
__global__ void k_msd(Dev dv, int b, int mode, double* last, double* acc)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dv.ntot) return;
    const Rep& rp = dv.reps[dv.rep_of[i]];
    const Bufs& B = dv.buf[b];
    const size_t g = 3 * (size_t)(rp.pbase + B.tag[i]);
    const double x[3] = { B.px[i], B.py[i], dv.dim == 3 ? B.pz[i] : 0.0 };
    for (int a = 0; a < dv.dim; ++a) {
        if (mode == 0) {
            acc[g + a] = 0.0;
        } else {
            acc[g + a] += min_image(x[a] - last[g + a], rp.L[a], rp.halfL[a]);
        }
        last[g + a] = x[a];
    }
}

int msd_launch(hpmc_batch* h, int mode)
{
    CK(cudaDeviceSynchronize());
    if (!h->msd_last) {
        int rc;
        if ((rc = dalloc(h, &h->msd_last, 3 * (size_t)h->ntot)) || (rc = dalloc(h, &h->msd_acc, 3 * (size_t)h->ntot)))
            return rc;
        mode = 0;
    }
    k_msd<<<(h->ntot + 255) / 256, 256>>>(h->dv, h->cur, mode, h->msd_last, h->msd_acc);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    return read_error(h);
}

int hpmc_msd_reset(hpmc_t h)
{
    if (!h) return HPMC_ERR_INVALID_ARG;
    return msd_launch(h, 0);
}

int hpmc_msd_update(hpmc_t h)
{
    if (!h) return HPMC_ERR_INVALID_ARG;
    return msd_launch(h, 1);
}

int hpmc_msd_read(hpmc_t h, int32_t r, double* msd)
{
    if (!h || !msd || r < -1 || r >= (int32_t)h->R) return HPMC_ERR_INVALID_ARG;
    if (!h->msd_acc) return HPMC_ERR_NOT_READY;
    CK(cudaDeviceSynchronize());
    std::vector<double> acc(3 * (size_t)h->ntot);
    CK(cudaMemcpy(acc.data(), h->msd_acc, sizeof(double) * acc.size(), cudaMemcpyDeviceToHost));
    double sum = 0.0;
    uint64_t n = 0;
    for (uint32_t q = 0; q < h->R; ++q) {
        if (r >= 0 && (uint32_t)r != q) continue;
        const uint32_t pb = h->reps[q].pbase;
        for (uint32_t t = 0; t < h->hr[q].N; ++t) {
            const double* d = acc.data() + 3 * (size_t)(pb + t);
            sum += d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        }
        n += h->hr[q].N;
    }
    *msd = n ? sum / (double)n : 0.0;
    return 0;
}

int hpmc_debug_fail_alloc(int32_t n)
{
    g_fail_alloc = n < 0 ? -1 : n;
    return 0;
}

int hpmc_get_box(hpmc_t h, int32_t r, double* box)
{
    if (!h || !box || r < 0 || r >= (int32_t)h->R) return HPMC_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a) box[a] = a < h->dim ? h->hr[r].L[a] : 0.0;
    return 0;
}

int hpmc_get_state(hpmc_t h, int32_t r, double* pos, double* orient, uint64_t* sweep)
{
    if (!h || r < 0 || r >= (int32_t)h->R) return HPMC_ERR_INVALID_ARG;
    CK(cudaDeviceSynchronize());
    k_unsort<<<(h->ntot + 255) / 256, 256>>>(h->dv, h->cur);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    const Bufs& D = h->dv.buf[h->cur ^ 1];
    const uint32_t N = h->hr[r].N, pb = h->reps[r].pbase;
    const int dim = h->dim, qd = dim == 2 ? 2 : 4;
    std::vector<double> col(N);
    const double* src_p[3] = { D.px, D.py, D.pz };
    const double* src_q[4] = { D.q0, D.q1, D.q2, D.q3 };
    if (pos) {
        for (int a = 0; a < dim; ++a) {
            CK(cudaMemcpy(col.data(), src_p[a] + pb, sizeof(double) * N, cudaMemcpyDeviceToHost));
            for (uint32_t i = 0; i < N; ++i) pos[(size_t)i * dim + a] = col[i];
        }
    }
    if (orient) {
        for (int a = 0; a < qd; ++a) {
            CK(cudaMemcpy(col.data(), src_q[a] + pb, sizeof(double) * N, cudaMemcpyDeviceToHost));
            for (uint32_t i = 0; i < N; ++i) orient[(size_t)i * qd + a] = col[i];
        }
    }
    if (sweep) CK(cudaMemcpy(sweep, h->dv.sweep + r, sizeof(uint64_t), cudaMemcpyDeviceToHost));
    return read_error(h);
}

int hpmc_set_state(hpmc_t h, int32_t r, const double* pos, const double* orient, uint64_t sweep)
{
    if (!h || r < 0 || r >= (int32_t)h->R) return HPMC_ERR_INVALID_ARG;
    int rc = check_config(h->dim, h->hr[r], pos, orient);
    if (rc) return rc;
    CK(cudaDeviceSynchronize());
    // bring every replica to tag order in buffer cur ^ 1, overwrite replica r,
    // then make that buffer current
    k_unsort<<<(h->ntot + 255) / 256, 256>>>(h->dv, h->cur);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    h->cur ^= 1;
    const Bufs& D = h->dv.buf[h->cur];
    const uint32_t N = h->hr[r].N, pb = h->reps[r].pbase;
    const int dim = h->dim, qd = dim == 2 ? 2 : 4;
    std::vector<double> col(N);
    double* dst_p[3] = { D.px, D.py, D.pz };
    double* dst_q[4] = { D.q0, D.q1, D.q2, D.q3 };
    for (int a = 0; a < dim; ++a) {
        for (uint32_t i = 0; i < N; ++i) col[i] = pos[(size_t)i * dim + a];
        CK(cudaMemcpy(dst_p[a] + pb, col.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
    }
    for (int a = 0; a < qd; ++a) {
        for (uint32_t i = 0; i < N; ++i) col[i] = orient[(size_t)i * qd + a];
        CK(cudaMemcpy(dst_q[a] + pb, col.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(h->dv.sweep + r, &sweep, sizeof(uint64_t), cudaMemcpyHostToDevice));
    invalidate_graph(h);
    return 0;
}

int hpmc_run_host(hpmc_t h, const double* pos, const double* orient, uint32_t n, double* pos_out,
                  double* orient_out, hpmc_counters_t* out, void* stream)
{
    if (!h || !pos || !orient || !pos_out || !orient_out) return HPMC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int dim = h->dim, qd = dim == 2 ? 2 : 4;
    const size_t N = h->ntot;
    int rc = 0;
    if (!h->stage && (rc = dalloc(h, &h->stage, N * (size_t)(dim + qd)))) return rc;
    // one copy per array as the caller holds it (a direct DMA when the host
    // buffers are pinned), then the layout change on the device
    CK(cudaMemcpyAsync(h->stage, pos, N * dim * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(h->stage + N * dim, orient, N * qd * sizeof(double), cudaMemcpyHostToDevice, st));
    k_from_interleaved<<<(h->ntot + 255) / 256, 256, 0, st>>>(h->dv, h->cur, h->stage);
    CK(cudaGetLastError());
    rc = hpmc_sweep_graph(h, n, stream);
    if (rc) return rc;
    k_to_interleaved<<<(h->ntot + 255) / 256, 256, 0, st>>>(h->dv, h->cur, h->stage);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(pos_out, h->stage, N * dim * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(orient_out, h->stage + N * dim, N * qd * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (out) return hpmc_counters(h, -1, out);
    return read_error(h);
}

// CUDA events owned by a host scope (destroyed on every return path)
struct Events {
    std::vector<cudaEvent_t> e;
    explicit Events(size_t n) : e(n, nullptr) {}
    ~Events()
    {
        for (cudaEvent_t x : e)
            if (x) cudaEventDestroy(x);
    }
    cudaError_t create()
    {
        for (cudaEvent_t& x : e) {
            const cudaError_t r = cudaEventCreate(&x);
            if (r != cudaSuccess) return r;
        }
        return cudaSuccess;
    }
    Events(const Events&) = delete;
    Events& operator=(const Events&) = delete;
};

// The state in tag order, the sweep counters and the event counters, kept on
// the host while trial runs (tuning) use the device state.
struct Snapshot {
    std::vector<double> P, Q;
    std::vector<uint64_t> sw;
    std::vector<unsigned long long> cnt;
};

int snapshot_take(hpmc_batch* h, Snapshot& s)
{
    CK(cudaDeviceSynchronize());
    const int qd = h->dim == 2 ? 2 : 4;
    const size_t N = h->ntot;
    s.P.resize(N * h->dim);
    s.Q.resize(N * qd);
    s.sw.resize(h->R);
    s.cnt.resize((size_t)h->R * kNumCounters);
    k_unsort<<<(h->ntot + 255) / 256, 256>>>(h->dv, h->cur);
    CK(cudaDeviceSynchronize());
    const Bufs& D = h->dv.buf[h->cur ^ 1];
    const double* sp[3] = { D.px, D.py, D.pz };
    const double* sq[4] = { D.q0, D.q1, D.q2, D.q3 };
    std::vector<double> col(N);
    for (int a = 0; a < h->dim; ++a) {
        CK(cudaMemcpy(col.data(), sp[a], N * sizeof(double), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < N; ++i) s.P[i * h->dim + a] = col[i];
    }
    for (int a = 0; a < qd; ++a) {
        CK(cudaMemcpy(col.data(), sq[a], N * sizeof(double), cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < N; ++i) s.Q[i * qd + a] = col[i];
    }
    CK(cudaMemcpy(s.sw.data(), h->dv.sweep, sizeof(uint64_t) * h->R, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(s.cnt.data(), h->dv.counters, sizeof(unsigned long long) * s.cnt.size(), cudaMemcpyDeviceToHost));
    return 0;
}

int snapshot_restore(hpmc_batch* h, const Snapshot& s)
{
    CK(cudaDeviceSynchronize());
    int rc = upload_all(h, s.P.data(), s.Q.data(), 0);
    if (rc) return rc;
    CK(cudaMemcpy(h->dv.sweep, s.sw.data(), sizeof(uint64_t) * h->R, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(h->dv.counters, s.cnt.data(), sizeof(unsigned long long) * s.cnt.size(), cudaMemcpyHostToDevice));
    CK(cudaDeviceSynchronize());
    return 0;
}

int hpmc_tune_moves(hpmc_t h, int32_t r, double target, uint32_t n_pilot, uint32_t iters, double lo,
                    double hi, double* d_out, double* a_out, double* acc_out)
{
    if (!h || r < -1 || r >= (int32_t)h->R || n_pilot == 0 || iters == 0) return HPMC_ERR_INVALID_ARG;
    if (!(target > 0.0 && target < 1.0) || !(lo > 0.0) || !(hi > lo) || !is_finite(hi)) return HPMC_ERR_INVALID_ARG;
    Snapshot snap;
    int rc = snapshot_take(h, snap);
    if (rc) return rc;
    const std::vector<HostRep> base = h->hr;
    auto set_scale = [&](double f) {
        for (uint32_t q = 0; q < h->R; ++q) {
            if (r >= 0 && (uint32_t)r != q) continue;
            int e = hpmc_set_moves(h, (int32_t)q, base[q].d * f, base[q].a * f, base[q].nselect);
            if (e) return e;
        }
        return 0;
    };
    // a failed pilot leaves the state and the moves as they were
    auto fail = [&](int code) {
        snapshot_restore(h, snap);
        set_scale(1.0);
        return code;
    };
    // geometric bisection on a common scale of (d, a): acceptance falls as the
    // moves grow; the best pilot (closest to the target) wins
    double best_f = 1.0, best_acc = -1.0;
    for (uint32_t it = 0; it < iters; ++it) {
        const double mid = std::sqrt(lo * hi);
        if ((rc = snapshot_restore(h, snap)) || (rc = set_scale(mid))) return fail(rc);
        const cudaError_t ce = cudaMemset(h->dv.counters, 0, sizeof(unsigned long long) * h->R * kNumCounters);
        if (ce != cudaSuccess) return fail(cuda_fail(ce));
        if ((rc = hpmc_sweep(h, n_pilot, nullptr))) return fail(rc);
        hpmc_counters_t c{};
        if ((rc = hpmc_counters(h, r, &c))) return fail(rc);
        const double acc = c.moves ? (double)c.accept / (double)c.moves : 0.0;
        if (best_acc < 0.0 || std::fabs(acc - target) < std::fabs(best_acc - target)) {
            best_acc = acc;
            best_f = mid;
        }
        if (acc > target) lo = mid;        // moves too small: acceptance too high
        else hi = mid;
    }
    if ((rc = snapshot_restore(h, snap)) || (rc = set_scale(best_f))) return rc;
    if (r >= 0) {
        if (d_out) *d_out = h->hr[r].d;
        if (a_out) *a_out = h->hr[r].a;
    } else {
        if (d_out) *d_out = h->hr[0].d;
        if (a_out) *a_out = h->hr[0].a;
    }
    if (acc_out) *acc_out = best_acc;
    return read_error(h);
}

int hpmc_autotune(hpmc_t h, uint32_t n_trial, int* best_lanes, int* best_warps)
{
    if (!h || n_trial == 0) return HPMC_ERR_INVALID_ARG;
    Snapshot snap;
    int rc0 = snapshot_take(h, snap);
    if (rc0) return rc0;
    const int G0 = h->G, W0 = h->wpb;
    float best_ms = 1e30f;
    int bg = G0, bw = W0;
    // a CUDA failure leaves the configuration and the state as they were
    auto fail = [&](cudaError_t e) {
        const int code = cuda_fail(e);
        h->G = G0;
        h->wpb = W0;
        invalidate_graph(h);
        snapshot_restore(h, snap);
        return code;
    };
    Events ev(2);
    cudaError_t ce = ev.create();
    if (ce != cudaSuccess) return fail(ce);
    const int wpbs[4] = { 1, 2, 4, 8 };
    for (int gi = 0; gi < kNumGroups; ++gi) {
        for (int wi = 0; wi < 4; ++wi) {
            if (hpmc_set_group_size(h, kGroupSizes[gi], wpbs[wi]) != 0) continue;
            int rc = hpmc_sweep(h, 1, nullptr);      // warm-up
            if (rc) continue;
            if ((ce = cudaEventRecord(ev.e[0])) != cudaSuccess) return fail(ce);
            rc = hpmc_sweep(h, n_trial, nullptr);
            if ((ce = cudaEventRecord(ev.e[1])) != cudaSuccess) return fail(ce);
            if ((ce = cudaEventSynchronize(ev.e[1])) != cudaSuccess) return fail(ce);
            if (rc) continue;
            float ms = 0.f;
            if ((ce = cudaEventElapsedTime(&ms, ev.e[0], ev.e[1])) != cudaSuccess) return fail(ce);
            if (ms < best_ms) { best_ms = ms; bg = kGroupSizes[gi]; bw = wpbs[wi]; }
        }
    }
    h->G = bg;
    h->wpb = bw;
    invalidate_graph(h);
    int rc = snapshot_restore(h, snap);
    if (rc) return rc;
    if (best_lanes) *best_lanes = bg;
    if (best_warps) *best_warps = bw;
    return read_error(h);
}

int hpmc_profile_sweeps(hpmc_t h, uint32_t n, void* stream, double* ms_rebuild, double* ms_sets)
{
    if (!h || n == 0) return HPMC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    h->last_stream = st;
    int rc = prepare_set(h);
    if (rc) return rc;
    Events evs(3 * (size_t)n);
    CK(evs.create());
    std::vector<cudaEvent_t>& ev = evs.e;
    for (uint32_t s = 0; s < n; ++s) {
        CK(cudaEventRecord(ev[3 * s], st));
        rc = enqueue_rebuild(h, st, true);
        if (rc) break;
        // the rebuild's time includes the select table made alongside it
        if (h->use_selects) CK(cudaStreamWaitEvent(st, h->ev_join, 0));
        CK(cudaEventRecord(ev[3 * s + 1], st));
        rc = enqueue_sets(h, st);
        if (rc) break;
        CK(cudaEventRecord(ev[3 * s + 2], st));
    }
    CK(cudaStreamSynchronize(st));
    double a = 0.0, b = 0.0;
    for (uint32_t s = 0; s < n && !rc; ++s) {
        float x = 0.f, y = 0.f;
        CK(cudaEventElapsedTime(&x, ev[3 * s], ev[3 * s + 1]));
        CK(cudaEventElapsedTime(&y, ev[3 * s + 1], ev[3 * s + 2]));
        a += x;
        b += y;
    }
    if (rc) return rc;
    if (ms_rebuild) *ms_rebuild = a / n;
    if (ms_sets) *ms_sets = b / n;
    return read_error(h);
}

int hpmc_geometry(hpmc_t h, int32_t r, int32_t* nc, double* w, double* R)
{
    if (!h || r < 0 || r >= (int32_t)h->R) return HPMC_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a) {
        if (nc) nc[a] = h->reps[r].nc[a];
        if (w) w[a] = h->reps[r].w[a];
    }
    if (R) *R = h->Rc;
    return 0;
}

int hpmc_launches_per_sweep(hpmc_t h, uint32_t* n)
{
    if (!h || !n) return HPMC_ERR_INVALID_ARG;
    *n = 5 + (h->ntiles > 1 ? 2 : 0) + (1u << h->dim) + (uses_select_table(h->G) ? 1 : 0);
    return 0;
}

int hpmc_trace_read(hpmc_t h, uint64_t* out, uint32_t max_warps, uint32_t* n_points)
{
    if (!h || !out || !n_points) return HPMC_ERR_INVALID_ARG;
    *n_points = kTracePoints;
    if (!h->dv.trace) return HPMC_ERR_NOT_READY;
    CK(cudaDeviceSynchronize());
    const uint32_t n = std::min(max_warps, h->dv.trace_warps);
    CK(cudaMemcpy(out, h->dv.trace, sizeof(uint64_t) * n * kTracePoints, cudaMemcpyDeviceToHost));
    return 0;
}

int hpmc_filter_margins(hpmc_t h, int32_t r, double* e_in, double* e_cull, double* e_overlap)
{
    if (!h || r < 0 || r >= (int32_t)h->R) return HPMC_ERR_INVALID_ARG;
    if (e_in) *e_in = h->reps[r].e_in;
    if (e_cull) *e_cull = h->reps[r].e_cull;
    if (e_overlap) *e_overlap = h->reps[r].e_sat;
    return 0;
}

}  // extern "C"
