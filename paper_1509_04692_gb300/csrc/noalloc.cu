// noalloc.cu -- overlap-pair count that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need an
// overlap check: code running inside a custom memory pool or a host callback
// that may not touch the allocator, graph-building tools that forbid
// allocation while they record work, or embedders whose process owns all
// device memory up front.  hpmc_count_overlaps_noalloc serves them: the caller
// passes its own device arrays for the configuration and the result, and the
// cell list the count needs lives in one fixed array of this file
// (g_noalloc_scratch), reserved when the library is loaded and kept by every
// device that loads it until the process exits.
//
// The pair test is the same FP64 rule hpmc_check_overlaps uses (minimum
// image, circumsphere cull, separating-axis test), on a cell grid built with
// the same width rule and no shift.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>

#include "../../include/hpmc.h"
#include "hpmc_device.cuh"

namespace {

constexpr uint32_t kMaxN = HPMC_NOALLOC_MAX_N;
constexpr uint32_t kMaxCells = HPMC_NOALLOC_MAX_CELLS;
constexpr int kMaxDevices = 64;

// layout: count[kMaxCells] | start[kMaxCells + 1] | cell[kMaxN] | slot[kMaxN] | idx[kMaxN]
constexpr size_t kScratchWords = (size_t)kMaxCells + (kMaxCells + 1) + 3 * (size_t)kMaxN;

static __device__ __align__(256) uint32_t g_noalloc_scratch[kScratchWords];

// device address of g_noalloc_scratch per device, looked up on a device's
// first call; atomic so that host threads making their first calls at the
// same time do not race (each would store the same address)
std::atomic<uint32_t*> g_scratch_ptr[kMaxDevices] = {};

struct Grid2 {
    double L[2], halfL[2], inv_w[2];
    int nc[2];
};

__global__ void k_na_zero(uint32_t* count, uint32_t ncell)
{
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x)
        count[c] = 0u;
}

__global__ void k_na_count(Grid2 g, uint32_t N, const double* __restrict__ pos, uint32_t* count,
                           uint32_t* cell, uint32_t* slot)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    // positions outside [0, L) (or NaN) are the caller's error; clamp the
    // index so that they can never address outside the scratch
    const int ix = max(0, hpmc::cell_axis(pos[2 * i], 0.0, g.L[0], g.inv_w[0], g.nc[0]));
    const int iy = max(0, hpmc::cell_axis(pos[2 * i + 1], 0.0, g.L[1], g.inv_w[1], g.nc[1]));
    const uint32_t c = (uint32_t)ix + (uint32_t)g.nc[0] * (uint32_t)iy;
    cell[i] = c;
    slot[i] = atomicAdd(count + c, 1u);
}

// exclusive scan of count[0..ncell) into start[], one block
__global__ void __launch_bounds__(1024) k_na_scan(const uint32_t* count, uint32_t* start, uint32_t ncell)
{
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t b = 0; b < ncell; b += 1024) {
        const uint32_t i = b + threadIdx.x;
        const uint32_t x = i < ncell ? count[i] : 0u;
        uint32_t incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint32_t w = wsum[lane];
            uint32_t wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            wsum[lane] = wi - w;
        }
        __syncthreads();
        const uint32_t ex = carry + wsum[warp] + incl - x;
        __syncthreads();
        if (i < ncell) start[i] = ex;
        if (threadIdx.x == 1023) carry = ex + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[ncell] = carry;
}

__global__ void k_na_scatter(uint32_t N, const uint32_t* start, const uint32_t* cell, const uint32_t* slot,
                             uint32_t* idx)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    idx[start[cell[i]] + slot[i]] = i;
}

// every unordered pair once (the lower index counts it)
__global__ void k_na_pairs(Grid2 g, hpmc::Shape2 sh, uint32_t N, const double* __restrict__ pos,
                           const double* __restrict__ ori, const uint32_t* start, const uint32_t* cell,
                           const uint32_t* idx, unsigned long long* out)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint32_t c = cell[i];
    const int ix = (int)(c % (uint32_t)g.nc[0]), iy = (int)(c / (uint32_t)g.nc[0]);
    const double xi = pos[2 * i], yi = pos[2 * i + 1], ci = ori[2 * i], si = ori[2 * i + 1];
    unsigned long long n = 0;
    for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
            const int jx = (ix + ox + g.nc[0]) % g.nc[0];
            const int jy = (iy + oy + g.nc[1]) % g.nc[1];
            const uint32_t cc = (uint32_t)jx + (uint32_t)g.nc[0] * (uint32_t)jy;
            for (uint32_t e = start[cc]; e < start[cc + 1]; ++e) {
                const uint32_t j = idx[e];
                if (j <= i) continue;
                const double Dx = hpmc::min_image(pos[2 * j] - xi, g.L[0], g.halfL[0]);
                const double Dy = hpmc::min_image(pos[2 * j + 1] - yi, g.L[1], g.halfL[1]);
                if (Dx * Dx + Dy * Dy > sh.rc2) continue;
                if (hpmc::overlap2d64<0>(sh, Dx, Dy, ci, si, ori[2 * j], ori[2 * j + 1])) n += 1;
            }
        }
    if (n) atomicAdd(out, n);
}

// Look up the device address of the scratch array once per device.  Host
// code may not pass g_noalloc_scratch itself to a kernel: on the host that
// name is only a stand-in for the device symbol.
int scratch_for_current_device(uint32_t** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { (void)cudaGetLastError(); return HPMC_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) return HPMC_ERR_CUDA;
    uint32_t* known = g_scratch_ptr[dev].load(std::memory_order_acquire);
    if (!known) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) { (void)cudaGetLastError(); return HPMC_ERR_CUDA; }
        known = (uint32_t*)p;
        g_scratch_ptr[dev].store(known, std::memory_order_release);
    }
    *out = known;
    return 0;
}

}  // namespace

extern "C" int hpmc_count_overlaps_noalloc(const double* box, const double* verts, uint32_t nv, uint32_t N,
                                           const double* pos_dev, const double* orient_dev,
                                           unsigned long long* count_dev, void* stream)
{
    if (!box || !verts || !pos_dev || !orient_dev || !count_dev) return HPMC_ERR_INVALID_ARG;
    if (nv < 3 || nv > (uint32_t)hpmc::kMaxV2 || N == 0) return HPMC_ERR_INVALID_ARG;
    if (N > kMaxN) return HPMC_ERR_SCRATCH_LIMIT;
    for (uint32_t k = 0; k < 2 * nv; ++k)
        if (!std::isfinite(verts[k])) return HPMC_ERR_INVALID_ARG;
    // shape constants, as the FP64 rule defines them
    hpmc::Shape2 sh{};
    sh.nv = (int)nv;
    double r2 = 0.0;
    for (uint32_t k = 0; k < nv; ++k) {
        sh.vx[k] = verts[2 * k];
        sh.vy[k] = verts[2 * k + 1];
        const double q = sh.vx[k] * sh.vx[k] + sh.vy[k] * sh.vy[k];
        if (q > r2) r2 = q;
    }
    for (uint32_t k = 0; k < nv; ++k) {
        const uint32_t k1 = (k + 1) % nv;
        const double cr = (sh.vx[k1] - sh.vx[k]) * (sh.vy[(k + 2) % nv] - sh.vy[k1]) -
                          (sh.vy[k1] - sh.vy[k]) * (sh.vx[(k + 2) % nv] - sh.vx[k1]);
        if (!(cr > 0.0)) return HPMC_ERR_INVALID_ARG;        // convex, counter-clockwise
        sh.nx[k] = sh.vy[k1] - sh.vy[k];
        sh.ny[k] = sh.vx[k] - sh.vx[k1];
        double lo = 0.0, hi = 0.0;
        for (uint32_t i = 0; i < nv; ++i) {
            const double t = sh.nx[k] * sh.vx[i] + sh.ny[k] * sh.vy[i];
            if (i == 0 || t < lo) lo = t;
            if (i == 0 || t > hi) hi = t;
        }
        sh.alo[k] = lo;
        sh.ahi[k] = hi;
    }
    const double R = std::sqrt(r2);
    if (!(R > 0.0)) return HPMC_ERR_INVALID_ARG;
    const double dcut = R + R;
    sh.rc2 = dcut * dcut;
    Grid2 g{};
    uint64_t ncell = 1;
    for (int a = 0; a < 2; ++a) {
        const double L = box[a];
        if (!(L > 0.0) || !std::isfinite(L)) return HPMC_ERR_INVALID_ARG;
        // range check in double before the cast: a large finite box must
        // read as beyond the scratch, not overflow the integer conversion
        const double fl = std::floor(L / dcut);
        if (!(fl <= (double)kMaxCells + 1.0)) return HPMC_ERR_SCRATCH_LIMIT;
        int n = (int)fl;
        if (n % 2) n -= 1;
        if (n < 4) return HPMC_ERR_BOX_TOO_SMALL;
        if (n > (int)kMaxCells) return HPMC_ERR_SCRATCH_LIMIT;
        g.L[a] = L;
        g.halfL[a] = 0.5 * L;
        g.inv_w[a] = (double)n / L;
        g.nc[a] = n;
        ncell *= (uint64_t)n;
    }
    if (ncell > kMaxCells) return HPMC_ERR_SCRATCH_LIMIT;

    uint32_t* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    uint32_t* count = scratch;
    uint32_t* start = count + kMaxCells;
    uint32_t* cell = start + (kMaxCells + 1);
    uint32_t* slot = cell + kMaxN;
    uint32_t* idx = slot + kMaxN;
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t nc = (uint32_t)ncell;
    // the scratch keeps the previous call's contents: counts must restart at 0
    k_na_zero<<<(nc + 255) / 256, 256, 0, st>>>(count, nc);
    if (cudaMemsetAsync(count_dev, 0, sizeof(unsigned long long), st) != cudaSuccess) {
        (void)cudaGetLastError();
        return HPMC_ERR_CUDA;
    }
    k_na_count<<<(N + 255) / 256, 256, 0, st>>>(g, N, pos_dev, count, cell, slot);
    k_na_scan<<<1, 1024, 0, st>>>(count, start, nc);
    k_na_scatter<<<(N + 255) / 256, 256, 0, st>>>(N, start, cell, slot, idx);
    k_na_pairs<<<(N + 127) / 128, 128, 0, st>>>(g, sh, N, pos_dev, orient_dev, start, cell, idx, count_dev);
    if (cudaGetLastError() != cudaSuccess) return HPMC_ERR_CUDA;
    return 0;
}
