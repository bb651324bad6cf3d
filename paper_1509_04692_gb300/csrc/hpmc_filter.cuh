// hpmc_filter.cuh -- FP32 side of the certified filter (device).
//
// These routines evaluate the same quantities as the FP64 contract in FP32
// and return a verdict only when it is farther from the threshold than the
// certified margin of hpmc_bounds.h; otherwise they return "uncertain" and
// the caller re-decides in FP64.  Fused multiply-adds are used freely: a
// single rounding is covered by the separate multiply-then-add bound.
#pragma once
#include "hpmc_types.h"

namespace hpmc {

// z' = z * dz(t) with the Cayley rotation dz = ((1 - t^2), 2t) / (1 + t^2).
__device__ __forceinline__ void rotate32(float c, float s, float t, float& co, float& so)
{
    const float tt = __fmul_rn(t, t);
    const float inv = __frcp_rn(__fadd_rn(1.0f, tt));
    const float cd = __fmul_rn(__fsub_rn(1.0f, tt), inv);
    const float sd = __fmul_rn(__fadd_rn(t, t), inv);
    co = __fmaf_rn(c, cd, -__fmul_rn(s, sd));
    so = __fmaf_rn(c, sd, __fmul_rn(s, cd));
}

// One half of the 2D separating-axis test in FP32: B placed in A's frame by
// (cr, sr) and (lx, ly), tested on A's edge normals.
// Returns 0 = some axis certainly separates, 1 = every axis certainly
// overlaps, 2 = neither.
template <int NV>
__device__ __forceinline__ int half32(const Shape2& sh, float E, float cr, float sr, float lx, float ly)
{
    const int nv = NV ? NV : sh.nv;
    float px[NV ? NV : kMaxV2], py[NV ? NV : kMaxV2];
#pragma unroll
    for (int i = 0; i < nv; ++i) {
        px[i] = __fmaf_rn(cr, sh.fvx[i], __fmaf_rn(-sr, sh.fvy[i], lx));
        py[i] = __fmaf_rn(sr, sh.fvx[i], __fmaf_rn(cr, sh.fvy[i], ly));
    }
    bool all_ov = true;
#pragma unroll
    for (int k = 0; k < nv; ++k) {
        float lo = __fmaf_rn(sh.fnx[k], px[0], __fmul_rn(sh.fny[k], py[0]));
        float hi = lo;
#pragma unroll
        for (int i = 1; i < nv; ++i) {
            const float t = __fmaf_rn(sh.fnx[k], px[i], __fmul_rn(sh.fny[k], py[i]));
            lo = fminf(lo, t);
            hi = fmaxf(hi, t);
        }
        const float g = fmaxf(__fsub_rn(lo, sh.fahi[k]), __fsub_rn(sh.falo[k], hi));
        if (g > E) return 0;
        all_ov = all_ov && (g < -E);
    }
    return all_ov ? 1 : 2;
}

// FP32 certified separating-axis test of A (trial, orientation (cA, sA)) and
// B at Delta = (dx, dy) with orientation (cB, sB).  0 separated, 1 overlap,
// 2 uncertain.
template <int NV>
__device__ __forceinline__ int sat32(const Shape2& sh, float E, float dx, float dy, float cA, float sA,
                                     float cB, float sB)
{
    const float cr = __fmaf_rn(cA, cB, __fmul_rn(sA, sB));
    const float sr = __fmaf_rn(cA, sB, -__fmul_rn(sA, cB));
    const float lx = __fmaf_rn(cA, dx, __fmul_rn(sA, dy));
    const float ly = __fmaf_rn(cA, dy, -__fmul_rn(sA, dx));
    const int r1 = half32<NV>(sh, E, cr, sr, lx, ly);
    if (r1 == 0) return 0;
    const float mx = __fmaf_rn(cB, dx, __fmul_rn(sB, dy));
    const float my = __fmaf_rn(cB, dy, -__fmul_rn(sB, dx));
    const int r2 = half32<NV>(sh, E, cr, -sr, -mx, -my);
    if (r2 == 0) return 0;
    return (r1 == 1 && r2 == 1) ? 1 : 2;
}

}  // namespace hpmc
