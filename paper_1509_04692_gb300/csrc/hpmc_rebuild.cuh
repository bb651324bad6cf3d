// hpmc_rebuild.cuh -- per-sweep grid shift and cell-list rebuild (Sec. 2.2.1,
// Sec. 2.5.1): count with atomic arrival slots, exclusive scan, scatter of
// tags, then a canonical placement (rank of the tag among the cell's tags)
// that gathers the state into the other buffer in cell-sorted order and
// refreshes the FP32 cell-relative mirror.
#pragma once
#include "hpmc_device.cuh"

namespace hpmc {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// Grid shift of the sweep about to run for replica r, and the sweep counter
// advance (the running sweep is sweep[r] - 1 afterwards).
__device__ __forceinline__ void shift_replica(const Dev& dv, uint32_t r, double out[3])
{
    const Rep& rp = dv.reps[r];
    const uint64_t sweep = dv.sweep[r];
    const uint4 b0 = shift_block(rp.seed, sweep, 0);
    out[0] = rp.w[0] * u53(b0.x, b0.y);
    out[1] = rp.w[1] * u53(b0.z, b0.w);
    if (dv.dim == 3) {
        const uint4 b1 = shift_block(rp.seed, sweep, 1);
        out[2] = rp.w[2] * u53(b1.x, b1.y);
    } else {
        out[2] = 0.0;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) dv.shift[3 * r + a] = out[a];
    dv.sweep[r] = sweep + 1;
}

// One thread per replica.
__global__ void k_shift(Dev dv)
{
    pdl_enter();
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= dv.R) return;
    double s[3];
    shift_replica(dv, r, s);
}

// Local cell (replica-relative linear index) of particle i of buffer cur.
__device__ __forceinline__ uint32_t local_cell(const Dev& dv, const Rep& rp, const Bufs& B, uint32_t i,
                                               const double* sh)
{
    const int ix = cell_axis(B.px[i], sh[0], rp.L[0], rp.inv_w[0], rp.nc[0]);
    const int iy = cell_axis(B.py[i], sh[1], rp.L[1], rp.inv_w[1], rp.nc[1]);
    int iz = 0;
    if (dv.dim == 3) iz = cell_axis(B.pz[i], sh[2], rp.L[2], rp.inv_w[2], rp.nc[2]);
    return (uint32_t)ix + (uint32_t)rp.nc[0] * ((uint32_t)iy + (uint32_t)rp.nc[1] * (uint32_t)iz);
}

// A non-negative double truncated to FP32 from its bit pattern (integer
// operations only: on this GPU every FP64 instruction, conversions included,
// takes the slow FP64 pipe).  Relative error below 2^-23; values below 2^-126
// give 0.  A negative zero reads as zero.
__device__ __forceinline__ float f32_trunc_nonneg(double x)
{
    const uint32_t hi = (uint32_t)__double2hiint(x) & 0x7fffffffu, lo = (uint32_t)__double2loint(x);
    const int e = (int)(hi >> 20) - 1023 + 127;
    if (e <= 0) return 0.0f;
    return __uint_as_float(((uint32_t)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

// The contract's cell index on axis a (cell_axis: y = x - s, + L when
// negative, truncation of y * inv_w, clamp to nc - 1) evaluated in FP32:
// the result is certified when the FP32 y is farther than cell_ey from 0 and
// the FP32 product farther than cell_et from the nearest integer (the
// bounds of the FP32 error, see the host's derivation); otherwise -1, and
// the caller takes the FP64 rule.
__device__ __forceinline__ int cell_axis_f32(const Rep& rp, int a, double x, float s32)
{
    float y = __fsub_rn(f32_trunc_nonneg(x), s32);
    if (!(fabsf(y) > rp.cell_ey[a])) return -1;
    if (y < 0.0f) y = __fadd_rn(y, rp.L32[a]);
    const float t = __fmul_rn(y, rp.inv_w32[a]);
    const float fi = floorf(t);
    const float fr = t - fi;                       // exact
    const float et = rp.cell_et[a];
    if (!(fr > et && fr < 1.0f - et)) return -1;
    return min((int)fi, rp.nc[a] - 1);
}

// Cell of every particle of buffer `cur` and its arrival slot in the cell.
__global__ void k_count(Dev dv, int cur)
{
    pdl_enter();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dv.ntot) return;
    const uint32_t r = dv.rep_of[i];
    const Rep& rp = dv.reps[r];
    const Bufs& S = dv.buf[cur];
    const double* sh = dv.shift + 3 * r;
    uint32_t lc;
    // the FP32 rule first (2D); the FP64 rule where it is not certified
    const int ix = dv.dim == 2 ? cell_axis_f32(rp, 0, S.px[i], f32_trunc_nonneg(sh[0])) : -1;
    const int iy = ix >= 0 ? cell_axis_f32(rp, 1, S.py[i], f32_trunc_nonneg(sh[1])) : -1;
    if (iy >= 0) lc = (uint32_t)ix + (uint32_t)rp.nc[0] * (uint32_t)iy;
    else lc = local_cell(dv, rp, S, i, sh);
    const uint32_t c = rp.cbase + lc;
    dv.cellid[i] = c;
    dv.slot[i] = atomicAdd(dv.count + c, 1u);
}

// Block-wide exclusive scan of one tile of `count` into `start`; the tile
// total goes to tile_sums[tile].  The counts are zeroed for the next sweep.
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(Dev dv)
{
    pdl_enter();
    __shared__ uint32_t wsum[kScanThreads / 32];
    const uint32_t base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t tsum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const uint32_t i = base + k;
        v[k] = (i < dv.ctot) ? dv.count[i] : 0u;
        tsum += v[k];
    }
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const uint32_t i = base + k;
        if (i < dv.ctot) dv.count[i] = 0u;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = wsum[lane];
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        wsum[lane] = wi - w;
        if (lane == 31) dv.tile_sums[blockIdx.x] = wi;
    }
    __syncthreads();
    uint32_t run = wsum[warp] + incl - tsum;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const uint32_t i = base + k;
        if (i < dv.ctot) dv.start[i] = run;
        run += v[k];
    }
}

// Exclusive scan of the tile totals in place (single block, loops if needed).
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(Dev dv, uint32_t ntiles)
{
    pdl_enter();
    __shared__ uint32_t wsum[kScanThreads / 32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t b = 0; b < ntiles; b += kScanThreads) {
        const uint32_t i = b + threadIdx.x;
        const uint32_t x = i < ntiles ? dv.tile_sums[i] : 0u;
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = wsum[lane];
            uint32_t wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            wsum[lane] = wi - w;
        }
        __syncthreads();
        const uint32_t ex = carry + wsum[warp] + incl - x;
        __syncthreads();
        if (i < ntiles) dv.tile_sums[i] = ex;
        if (threadIdx.x == kScanThreads - 1) carry = ex + x;
        __syncthreads();
    }
}

__global__ void k_scan_add(Dev dv)
{
    pdl_enter();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dv.ctot || i < (uint32_t)kScanTile) return;
    dv.start[i] += dv.tile_sums[i / kScanTile];
}

// tags in arrival order
__global__ void k_scatter_tags(Dev dv, int cur)
{
    pdl_enter();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dv.ntot) return;
    dv.tmp_tag[dv.start[dv.cellid[i]] + dv.slot[i]] = dv.buf[cur].tag[i];
}

// A finite double rounded to FP32, to nearest with ties to even, from its bit
// pattern (integer operations only, the FP64 pipe being slow on this GPU):
// the same value as the hardware conversion for results in the normal FP32
// range; magnitudes below 2^-126 give a zero of the same sign.
__device__ __forceinline__ float f32_rn_bits(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const int e = (int)((b >> 52) & 0x7ffu) - 1023 + 127;
    if (e <= 0) return __uint_as_float(sign);
    const uint32_t mant = (uint32_t)((b >> 29) & 0x7fffffu);
    const uint32_t rest = (uint32_t)(b & 0x1fffffffu);
    uint32_t r = ((uint32_t)e << 23) | mant;
    if (rest > 0x10000000u || (rest == 0x10000000u && (mant & 1u))) r += 1u;   // a carry raises the exponent
    return __uint_as_float(sign | r);
}

// FP32 mirror coordinate of x in cell i of an axis: rel = (x - s, + L when
// negative) - i w with the product and difference in one fused multiply-add,
// then rounded to FP32 (within the certified bound of the mirror: a few FP64
// roundings of magnitude L, then the cast).
__device__ __forceinline__ float mirror_rel(double x, double s, double L, double w, int i)
{
    return f32_rn_bits(__fma_rn(-(double)i, w, cell_coord_bits(x, s, L)));
}

// Gather of particle i (tag t) of replica r, cell c, into slot o of buffer
// cur ^ 1, with the FP32 mirror (cell-relative coordinate, orientation).
__device__ __forceinline__ void place_at(const Dev& dv, int cur, uint32_t i, uint32_t t, uint32_t r, uint32_t c,
                                         uint32_t o)
{
    const Bufs& S = dv.buf[cur];
    const Bufs& D = dv.buf[cur ^ 1];
    const Rep& rp = dv.reps[r];
    const uint32_t lc = c - rp.cbase;
    const int ix = (int)(lc % (uint32_t)rp.nc[0]);
    const int iy = (int)((lc / (uint32_t)rp.nc[0]) % (uint32_t)rp.nc[1]);
    const double x = S.px[i], y = S.py[i];
    D.px[o] = x;
    D.py[o] = y;
    D.tag[o] = t;
    const float rx = mirror_rel(x, dv.shift[3 * r], rp.L[0], rp.w[0], ix);
    const float ry = mirror_rel(y, dv.shift[3 * r + 1], rp.L[1], rp.w[1], iy);
    if (dv.dim == 2) {
        const double c0 = S.q0[i], s0 = S.q1[i];
        D.q0[o] = c0;
        D.q1[o] = s0;
        D.f4a[o] = make_float4(rx, ry, f32_rn_bits(c0), f32_rn_bits(s0));
    } else {
        const int iz = (int)(lc / ((uint32_t)rp.nc[0] * (uint32_t)rp.nc[1]));
        const double z = S.pz[i];
        D.pz[o] = z;
        const float rz = mirror_rel(z, dv.shift[3 * r + 2], rp.L[2], rp.w[2], iz);
        const double w0 = S.q0[i], w1 = S.q1[i], w2 = S.q2[i], w3 = S.q3[i];
        D.q0[o] = w0; D.q1[o] = w1; D.q2[o] = w2; D.q3[o] = w3;
        D.f4a[o] = make_float4(rx, ry, rz, f32_rn_bits(w0));
        D.f4b[o] = make_float4(f32_rn_bits(w1), f32_rn_bits(w2), f32_rn_bits(w3), 0.0f);
    }
}

// Canonical placement: a particle's sorted slot is its cell's start b plus
// the number of tags among the cell's n tags (tmp_tag[b..b+n)) below its own
// (ascending-tag order).
__global__ void k_place(Dev dv, int cur)
{
    pdl_enter();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dv.ntot) return;
    const uint32_t c = dv.cellid[i];
    const uint32_t b = dv.start[c];
    const uint32_t n = dv.start[c + 1] - b;
    const uint32_t t = dv.buf[cur].tag[i];
    uint32_t rank = 0;
    for (uint32_t j = 0; j < n; ++j) rank += (dv.tmp_tag[b + j] < t) ? 1u : 0u;
    place_at(dv, cur, i, t, dv.rep_of[i], c, b + rank);
}

// ------------------------------------------------ pressure (disks, spheres)
// Scale-distribution histogram (Sec. 4): every unordered pair of stencil
// neighbours (the higher tag counts it) with 0 <= x* = 1 - sigma / r < x_max
// adds one to bin (int)(x* * scale), scale = nbins / x_max.  The host checks
// that sigma / (1 - x_max) fits in a cell, so the stencil holds every such pair.
// Shaped particles: the bin of the pair's compression factor by bisection
// over the bin edges e_k = k h with the FP64 overlap contract along the
// scaled separation D (1 - e_k) (overlap is monotone along it for convex
// shapes containing their centres); -1 when the pair does not overlap at
// the last edge.
template <int DIM>
__device__ int sdf_shaped_bin(const Shape2& s2, const Shape3& s3, const double D[3], const double* qi,
                              const double* qj, double h, uint32_t nbins)
{
    auto overlap_at = [&](uint32_t k) {
        const double sc = 1.0 - (double)k * h;
        if (DIM == 2) return overlap2d64<0>(s2, D[0] * sc, D[1] * sc, qi[0], qi[1], qj[0], qj[1]);
        const double Ds[3] = { D[0] * sc, D[1] * sc, D[2] * sc };
        int it = 0;
        return overlap3d64<0>(s3, Ds, qi, qj, &it);
    };
    if (!overlap_at(nbins)) return -1;
    uint32_t lo = 0, hi = nbins;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) / 2;
        if (overlap_at(mid)) hi = mid;
        else lo = mid;
    }
    return (int)lo;
}

__global__ void k_sdf_shaped(Dev dv, int b, const __grid_constant__ Shape2 s2, const __grid_constant__ Shape3 s3,
                             double h, uint32_t nbins, int32_t only_r, unsigned long long* hist)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dv.ntot) return;
    const uint32_t r = dv.rep_of[i];
    if (only_r >= 0 && (int32_t)r != only_r) return;
    const Rep& rp = dv.reps[r];
    const Bufs& B = dv.buf[b];
    const int d3 = dv.dim == 3;
    const int ix = cell_axis(B.px[i], dv.shift[3 * r], rp.L[0], rp.inv_w[0], rp.nc[0]);
    const int iy = cell_axis(B.py[i], dv.shift[3 * r + 1], rp.L[1], rp.inv_w[1], rp.nc[1]);
    const int iz = d3 ? cell_axis(B.pz[i], dv.shift[3 * r + 2], rp.L[2], rp.inv_w[2], rp.nc[2]) : 0;
    const uint32_t ti = B.tag[i];
    const double qi[4] = { B.q0[i], B.q1[i], d3 ? B.q2[i] : 0.0, d3 ? B.q3[i] : 0.0 };
    for (int oz = -d3; oz <= d3; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                const int jx = (ix + ox + rp.nc[0]) % rp.nc[0];
                const int jy = (iy + oy + rp.nc[1]) % rp.nc[1];
                const int jz = d3 ? (iz + oz + rp.nc[2]) % rp.nc[2] : 0;
                const uint32_t cc = rp.cbase + (uint32_t)jx +
                                    (uint32_t)rp.nc[0] * ((uint32_t)jy + (uint32_t)rp.nc[1] * (uint32_t)jz);
                for (uint32_t e = dv.start[cc]; e < dv.start[cc + 1]; ++e) {
                    if (B.tag[e] <= ti) continue;
                    const double D[3] = { min_image(B.px[e] - B.px[i], rp.L[0], rp.halfL[0]),
                                          min_image(B.py[e] - B.py[i], rp.L[1], rp.halfL[1]),
                                          d3 ? min_image(B.pz[e] - B.pz[i], rp.L[2], rp.halfL[2]) : 0.0 };
                    const double qj[4] = { B.q0[e], B.q1[e], d3 ? B.q2[e] : 0.0, d3 ? B.q3[e] : 0.0 };
                    const int bin = d3 ? sdf_shaped_bin<3>(s2, s3, D, qi, qj, h, nbins)
                                       : sdf_shaped_bin<2>(s2, s3, D, qi, qj, h, nbins);
                    if (bin >= 0) atomicAdd(hist + bin, 1ull);
                }
            }
}

__global__ void k_sdf(Dev dv, int b, double sigma, double x_max, double scale, uint32_t nbins, int32_t only_r,
                      unsigned long long* hist)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dv.ntot) return;
    const uint32_t r = dv.rep_of[i];
    if (only_r >= 0 && (int32_t)r != only_r) return;
    const Rep& rp = dv.reps[r];
    const Bufs& B = dv.buf[b];
    const int d3 = dv.dim == 3;
    const int ix = cell_axis(B.px[i], dv.shift[3 * r], rp.L[0], rp.inv_w[0], rp.nc[0]);
    const int iy = cell_axis(B.py[i], dv.shift[3 * r + 1], rp.L[1], rp.inv_w[1], rp.nc[1]);
    const int iz = d3 ? cell_axis(B.pz[i], dv.shift[3 * r + 2], rp.L[2], rp.inv_w[2], rp.nc[2]) : 0;
    const uint32_t ti = B.tag[i];
    for (int oz = -d3; oz <= d3; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                const int jx = (ix + ox + rp.nc[0]) % rp.nc[0];
                const int jy = (iy + oy + rp.nc[1]) % rp.nc[1];
                const int jz = d3 ? (iz + oz + rp.nc[2]) % rp.nc[2] : 0;
                const uint32_t cc = rp.cbase + (uint32_t)jx +
                                    (uint32_t)rp.nc[0] * ((uint32_t)jy + (uint32_t)rp.nc[1] * (uint32_t)jz);
                for (uint32_t e = dv.start[cc]; e < dv.start[cc + 1]; ++e) {
                    if (B.tag[e] <= ti) continue;
                    const double Dx = min_image(B.px[e] - B.px[i], rp.L[0], rp.halfL[0]);
                    const double Dy = min_image(B.py[e] - B.py[i], rp.L[1], rp.halfL[1]);
                    double q2 = Dx * Dx + Dy * Dy;
                    if (d3) {
                        const double Dz = min_image(B.pz[e] - B.pz[i], rp.L[2], rp.halfL[2]);
                        q2 = q2 + Dz * Dz;
                    }
                    const double x = 1.0 - sigma / sqrt(q2);
                    if (!(x >= 0.0) || !(x < x_max)) continue;
                    const int bin = (int)(x * scale);
                    if (bin < (int)nbins) atomicAdd(hist + bin, 1ull);
                }
            }
}

// ---------------------------------------------------------------- checks
// Count overlapping pairs (each unordered pair once: the lower tag counts
// it) of the sorted buffer `b` with the FP64 contract predicate.
template <int NV>
__global__ void k_check2d(Dev dv, Shape2 sh, int b, int32_t only_r, unsigned long long* out)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dv.ntot) return;
    const uint32_t r = dv.rep_of[i];
    if (only_r >= 0 && (int32_t)r != only_r) return;
    const Rep& rp = dv.reps[r];
    const Bufs& B = dv.buf[b];
    const int ix = cell_axis(B.px[i], dv.shift[3 * r], rp.L[0], rp.inv_w[0], rp.nc[0]);
    const int iy = cell_axis(B.py[i], dv.shift[3 * r + 1], rp.L[1], rp.inv_w[1], rp.nc[1]);
    const uint32_t ti = B.tag[i];
    unsigned long long n = 0;
    for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
            const int jx = (ix + ox + rp.nc[0]) % rp.nc[0];
            const int jy = (iy + oy + rp.nc[1]) % rp.nc[1];
            const uint32_t cc = rp.cbase + (uint32_t)jx + (uint32_t)rp.nc[0] * (uint32_t)jy;
            for (uint32_t e = dv.start[cc]; e < dv.start[cc + 1]; ++e) {
                if (B.tag[e] <= ti) continue;
                const double Dx = min_image(B.px[e] - B.px[i], rp.L[0], rp.halfL[0]);
                const double Dy = min_image(B.py[e] - B.py[i], rp.L[1], rp.halfL[1]);
                if (Dx * Dx + Dy * Dy > sh.rc2) continue;
                if (overlap2d64<NV>(sh, Dx, Dy, B.q0[i], B.q1[i], B.q0[e], B.q1[e])) n += 1;
            }
        }
    if (n) atomicAdd(out, n);
}

}  // namespace hpmc
