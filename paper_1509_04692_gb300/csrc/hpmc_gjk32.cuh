// hpmc_gjk32.cuh -- FP32 GJK that certifies the FP64 contract's verdict.
//
// The FP64 contract (overlap3d64 in hpmc_device.cuh) decides overlap by a
// sequence of data-dependent branches (support argmax, Voronoi-region tests,
// sign tests).  This routine performs the same operations in FP32 and carries
// with every value a bound on its distance to the value the FP64 contract
// computes at the same step.  A branch is taken only when the FP32 operands
// are farther apart than their combined bounds, which proves that the FP64
// run takes the same branch; then, by induction, both runs visit the same
// simplices and return the same verdict.  Any branch that cannot be certified
// returns GJK32_UNCERTAIN and the caller re-decides with the FP64 contract.
//
// Bound model per operation (a32, b32 with bounds ea, eb on |a32 - a64|,
// |b32 - b64|; r = fl32(a32 op b32); the FP64 side rounds once too):
//   add/sub: |r - r64| <= ea + eb + (u32 + u64) |r| (1 + ...)
//   mul:     |r - r64| <= |a32| eb + (|b32| + eb) ea + (u32 + u64) |r| (...)
//   div:     |r - r64| <= (|a32| eb + |b32| ea) / (|b32| (|b32| - eb)) + (...)
// All bound arithmetic rounds upward (__f*_ru) and every bound is inflated
// by (1 + 2^-20) and a tiny absolute term, so rounding of the bound
// computation itself cannot make it too small.
#pragma once
#include "hpmc_types.h"

namespace hpmc {

enum : int { GJK32_SEPARATED = 0, GJK32_OVERLAP = 1, GJK32_UNCERTAIN = 2 };

struct Fe { float v, e; };                 // value, bound on |value - FP64 value|
struct Fe3 { Fe x, y, z; };

constexpr float kUr = 0x1.0p-24f + 0x1.0p-40f;   // u32 + u64 (and more), per rounding
constexpr float kInfl = 1.0f + 0x1.0p-20f;
constexpr float kTiny = 1e-30f;

__device__ __forceinline__ float ru_add(float a, float b) { return __fadd_ru(a, b); }
__device__ __forceinline__ float ru_mul(float a, float b) { return __fmul_ru(a, b); }

__device__ __forceinline__ float fin(float e) { return __fadd_ru(__fmul_ru(e, kInfl), kTiny); }

__device__ __forceinline__ Fe fe_add(Fe a, Fe b)
{
    const float r = __fadd_rn(a.v, b.v);
    return { r, fin(ru_add(ru_add(a.e, b.e), ru_mul(kUr, fabsf(r)))) };
}
__device__ __forceinline__ Fe fe_sub(Fe a, Fe b)
{
    const float r = __fsub_rn(a.v, b.v);
    return { r, fin(ru_add(ru_add(a.e, b.e), ru_mul(kUr, fabsf(r)))) };
}
__device__ __forceinline__ Fe fe_mul(Fe a, Fe b)
{
    const float r = __fmul_rn(a.v, b.v);
    const float e = ru_add(ru_add(ru_mul(fabsf(a.v), b.e), ru_mul(ru_add(fabsf(b.v), b.e), a.e)),
                           ru_mul(kUr, fabsf(r)));
    return { r, fin(e) };
}
__device__ __forceinline__ Fe fe_neg(Fe a) { return { -a.v, a.e }; }
// certified signs
__device__ __forceinline__ bool fe_pos(Fe a) { return a.v > a.e; }       // FP64 value > 0
__device__ __forceinline__ bool fe_neg_(Fe a) { return -a.v > a.e; }     // FP64 value < 0
__device__ __forceinline__ bool fe_sure(Fe a) { return fabsf(a.v) > a.e; }

// a / b, requires |b| > eb (checked by the caller through *ok)
__device__ __forceinline__ Fe fe_div(Fe a, Fe b, bool* ok)
{
    const float bb = fabsf(b.v);
    if (!(bb > b.e)) { *ok = false; return { 0.f, 0.f }; }
    const float r = __fdiv_rn(a.v, b.v);
    const float num = ru_add(ru_mul(fabsf(a.v), b.e), ru_mul(bb, a.e));
    const float den = __fmul_rd(bb, __fsub_rd(bb, b.e));
    const float e = ru_add(__fdiv_ru(num, den), ru_mul(kUr, fabsf(r)));
    return { r, fin(e) };
}

__device__ __forceinline__ Fe3 fe3_sub(const Fe3& a, const Fe3& b) { return { fe_sub(a.x, b.x), fe_sub(a.y, b.y), fe_sub(a.z, b.z) }; }
__device__ __forceinline__ Fe3 fe3_neg(const Fe3& a) { return { fe_neg(a.x), fe_neg(a.y), fe_neg(a.z) }; }
// (a0 b0 + a1 b1) + a2 b2, the contract's dot order
__device__ __forceinline__ Fe fe3_dot(const Fe3& a, const Fe3& b)
{
    return fe_add(fe_add(fe_mul(a.x, b.x), fe_mul(a.y, b.y)), fe_mul(a.z, b.z));
}
__device__ __forceinline__ Fe3 fe3_cross(const Fe3& a, const Fe3& b)
{
    return { fe_sub(fe_mul(a.y, b.z), fe_mul(a.z, b.y)), fe_sub(fe_mul(a.z, b.x), fe_mul(a.x, b.z)),
             fe_sub(fe_mul(a.x, b.y), fe_mul(a.y, b.x)) };
}
// a + t * b (component order of the contract)
__device__ __forceinline__ Fe3 fe3_axpy(const Fe3& a, Fe t, const Fe3& b)
{
    return { fe_add(a.x, fe_mul(t, b.x)), fe_add(a.y, fe_mul(t, b.y)), fe_add(a.z, fe_mul(t, b.z)) };
}

// Hamilton product, left-to-right sums as in the contract
__device__ __forceinline__ void fe_qmul(const Fe a[4], const Fe b[4], Fe o[4])
{
    o[0] = fe_sub(fe_sub(fe_sub(fe_mul(a[0], b[0]), fe_mul(a[1], b[1])), fe_mul(a[2], b[2])), fe_mul(a[3], b[3]));
    o[1] = fe_sub(fe_add(fe_add(fe_mul(a[0], b[1]), fe_mul(a[1], b[0])), fe_mul(a[2], b[3])), fe_mul(a[3], b[2]));
    o[2] = fe_add(fe_add(fe_sub(fe_mul(a[0], b[2]), fe_mul(a[1], b[3])), fe_mul(a[2], b[0])), fe_mul(a[3], b[1]));
    o[3] = fe_add(fe_sub(fe_add(fe_mul(a[0], b[3]), fe_mul(a[1], b[2])), fe_mul(a[2], b[1])), fe_mul(a[3], b[0]));
}

// v' = (v + w t) + q_v x t with t = 2 (q_v x v), as the contract
__device__ __forceinline__ Fe3 fe_qrot(const Fe q[4], const Fe3& v)
{
    const Fe two = { 2.0f, 0.0f };
    const Fe tx = fe_mul(two, fe_sub(fe_mul(q[2], v.z), fe_mul(q[3], v.y)));
    const Fe ty = fe_mul(two, fe_sub(fe_mul(q[3], v.x), fe_mul(q[1], v.z)));
    const Fe tz = fe_mul(two, fe_sub(fe_mul(q[1], v.y), fe_mul(q[2], v.x)));
    return { fe_add(fe_add(v.x, fe_mul(q[0], tx)), fe_sub(fe_mul(q[2], tz), fe_mul(q[3], ty))),
             fe_add(fe_add(v.y, fe_mul(q[0], ty)), fe_sub(fe_mul(q[3], tx), fe_mul(q[1], tz))),
             fe_add(fe_add(v.z, fe_mul(q[0], tz)), fe_sub(fe_mul(q[1], ty), fe_mul(q[2], tx))) };
}

// a strictly above b in the FP64 run
__device__ __forceinline__ bool fe_gt_sure(Fe a, Fe b) { return fe_pos(fe_sub(a, b)); }

// Certified support of B - A in direction d: the FP64 run picks the first
// strict maximum of pb.d and the first strict minimum of v.d; certified when
// the chosen index beats every other by more than the bounds.
template <int NV>
__device__ __forceinline__ bool support32(const Shape3& sh, const Fe3* pb, const Fe3* va, const Fe3& d,
                                          Fe3& out)
{
    const int nv = NV ? NV : sh.nv;
    int ib = 0, ia = 0;
    Fe best = fe3_dot(pb[0], d), least = fe3_dot(va[0], d);
#pragma unroll
    for (int i = 1; i < nv; ++i) {
        const Fe t = fe3_dot(pb[i], d);
        if (t.v > best.v) { best = t; ib = i; }
        const Fe u = fe3_dot(va[i], d);
        if (u.v < least.v) { least = u; ia = i; }
    }
    bool ok = true;
#pragma unroll
    for (int i = 0; i < nv; ++i) {
        if (i != ib) ok = ok && fe_gt_sure(best, fe3_dot(pb[i], d));
        if (i != ia) ok = ok && fe_gt_sure(fe3_dot(va[i], d), least);
    }
    out = fe3_sub(pb[ib], va[ia]);
    return ok;
}

// closest point of segment [a, b]; returns mask (a=1, b=2), -1 uncertain
__device__ __forceinline__ int closest_seg32(const Fe3& a, const Fe3& b, Fe3& out)
{
    const Fe3 ab = fe3_sub(b, a);
    const Fe3 ap = fe3_neg(a);
    const Fe tn = fe3_dot(ab, ap);
    if (!fe_sure(tn)) return -1;
    if (tn.v <= 0.f) { out = a; return 1; }
    const Fe den = fe3_dot(ab, ab);
    const Fe dd = fe_sub(tn, den);
    if (!fe_sure(dd)) return -1;
    if (dd.v >= 0.f) { out = b; return 2; }
    bool ok = true;
    const Fe t = fe_div(tn, den, &ok);
    if (!ok) return -1;
    out = fe3_axpy(a, t, ab);
    return 3;
}

// closest point of triangle (a, b, c); mask (a=1, b=2, c=4), 0 degenerate,
// -1 uncertain.  Every branch of the contract's region tests is certified.
__device__ __forceinline__ int closest_tri32(const Fe3& a, const Fe3& b, const Fe3& c, Fe3& out)
{
    const Fe3 ab = fe3_sub(b, a), ac = fe3_sub(c, a), ap = fe3_neg(a);
    const Fe d1 = fe3_dot(ab, ap), d2 = fe3_dot(ac, ap);
    // (d1 <= 0 && d2 <= 0)
    {
        const bool s1 = fe_sure(d1), s2 = fe_sure(d2);
        const bool c1 = d1.v <= 0.f, c2 = d2.v <= 0.f;
        if ((s1 && !c1) || (s2 && !c2)) { /* condition false for sure */ }
        else if (s1 && s2) { out = a; return 1; }
        else return -1;
    }
    const Fe3 bp = fe3_neg(b);
    const Fe d3 = fe3_dot(ab, bp), d4 = fe3_dot(ac, bp);
    // (d3 >= 0 && d4 <= d3)
    {
        const Fe e43 = fe_sub(d4, d3);
        const bool s1 = fe_sure(d3), s2 = fe_sure(e43);
        const bool c1 = d3.v >= 0.f, c2 = e43.v <= 0.f;
        if ((s1 && !c1) || (s2 && !c2)) { }
        else if (s1 && s2) { out = b; return 2; }
        else return -1;
    }
    const Fe vc = fe_sub(fe_mul(d1, d4), fe_mul(d3, d2));
    // (vc <= 0 && d1 >= 0 && d3 <= 0)
    {
        const bool s0 = fe_sure(vc), s1 = fe_sure(d1), s2 = fe_sure(d3);
        const bool c0 = vc.v <= 0.f, c1 = d1.v >= 0.f, c2 = d3.v <= 0.f;
        if ((s0 && !c0) || (s1 && !c1) || (s2 && !c2)) { }
        else if (s0 && s1 && s2) {
            bool ok = true;
            const Fe t = fe_div(d1, fe_sub(d1, d3), &ok);
            if (!ok) return -1;
            out = fe3_axpy(a, t, ab);
            return 3;
        } else return -1;
    }
    const Fe3 cp = fe3_neg(c);
    const Fe d5 = fe3_dot(ab, cp), d6 = fe3_dot(ac, cp);
    // (d6 >= 0 && d5 <= d6)
    {
        const Fe e56 = fe_sub(d5, d6);
        const bool s1 = fe_sure(d6), s2 = fe_sure(e56);
        const bool c1 = d6.v >= 0.f, c2 = e56.v <= 0.f;
        if ((s1 && !c1) || (s2 && !c2)) { }
        else if (s1 && s2) { out = c; return 4; }
        else return -1;
    }
    const Fe vb = fe_sub(fe_mul(d5, d2), fe_mul(d1, d6));
    // (vb <= 0 && d2 >= 0 && d6 <= 0)
    {
        const bool s0 = fe_sure(vb), s1 = fe_sure(d2), s2 = fe_sure(d6);
        const bool c0 = vb.v <= 0.f, c1 = d2.v >= 0.f, c2 = d6.v <= 0.f;
        if ((s0 && !c0) || (s1 && !c1) || (s2 && !c2)) { }
        else if (s0 && s1 && s2) {
            bool ok = true;
            const Fe t = fe_div(d2, fe_sub(d2, d6), &ok);
            if (!ok) return -1;
            out = fe3_axpy(a, t, ac);
            return 5;
        } else return -1;
    }
    const Fe va = fe_sub(fe_mul(d3, d6), fe_mul(d5, d4));
    const Fe e43 = fe_sub(d4, d3), e56 = fe_sub(d5, d6);
    // (va <= 0 && e43 >= 0 && e56 >= 0)
    {
        const bool s0 = fe_sure(va), s1 = fe_sure(e43), s2 = fe_sure(e56);
        const bool c0 = va.v <= 0.f, c1 = e43.v >= 0.f, c2 = e56.v >= 0.f;
        if ((s0 && !c0) || (s1 && !c1) || (s2 && !c2)) { }
        else if (s0 && s1 && s2) {
            bool ok = true;
            const Fe t = fe_div(e43, fe_add(e43, e56), &ok);
            if (!ok) return -1;
            out = fe3_axpy(b, t, fe3_sub(c, b));
            return 6;
        } else return -1;
    }
    const Fe sum = fe_add(fe_add(va, vb), vc);
    if (!fe_sure(sum)) return -1;
    if (!(sum.v > 0.f)) return 0;
    bool ok = true;
    const Fe den = fe_div(Fe{ 1.0f, 0.0f }, sum, &ok);
    if (!ok) return -1;
    const Fe v = fe_mul(vb, den), w = fe_mul(vc, den);
    out = { fe_add(fe_add(a.x, fe_mul(ab.x, v)), fe_mul(ac.x, w)),
            fe_add(fe_add(a.y, fe_mul(ab.y, v)), fe_mul(ac.y, w)),
            fe_add(fe_add(a.z, fe_mul(ab.z, v)), fe_mul(ac.z, w)) };
    return 7;
}

// origin strictly beyond plane (p, q, r) from s: 1 yes, 0 no, -1 uncertain
__device__ __forceinline__ int origin_outside32(const Fe3& p, const Fe3& q, const Fe3& r, const Fe3& s)
{
    const Fe3 n = fe3_cross(fe3_sub(q, p), fe3_sub(r, p));
    const Fe sp = fe3_dot(fe3_neg(p), n);
    const Fe sd = fe3_dot(fe3_sub(s, p), n);
    // (sp > 0 && sd < 0) || (sp < 0 && sd > 0): zero on either side means "no"
    if (!fe_sure(sp) || !fe_sure(sd)) {
        // a certain zero cannot be told apart from a tiny nonzero: uncertain
        return -1;
    }
    return ((sp.v > 0.f) != (sd.v > 0.f)) ? 1 : 0;
}

// reduce the simplex; returns 0 continue, 1 overlap (as the contract), -1 uncertain
__device__ __forceinline__ int gjk_reduce32(Fe3 sp[4], int& n, Fe3& v)
{
    int mask = 0;
    if (n == 2) {
        mask = closest_seg32(sp[0], sp[1], v);
        if (mask < 0) return -1;
    } else if (n == 3) {
        mask = closest_tri32(sp[0], sp[1], sp[2], v);
        if (mask < 0) return -1;
        if (mask == 0) return 1;
    } else {
        bool found = false;
        Fe best = { 0.f, 0.f };
#pragma unroll 1
        for (int f = 0; f < 4; ++f) {
            const int i0 = (f == 3) ? 1 : 0;
            const int i1 = (f <= 1) ? 1 : 2;
            const int i2 = (f == 0) ? 2 : 3;
            const int i3 = 3 - f;
            const int o = origin_outside32(sp[i0], sp[i1], sp[i2], sp[i3]);
            if (o < 0) return -1;
            if (!o) continue;
            Fe3 pt;
            const int m = closest_tri32(sp[i0], sp[i1], sp[i2], pt);
            if (m < 0) return -1;
            if (m == 0) return 1;
            const Fe dd = fe3_dot(pt, pt);
            bool take;
            if (!found) {
                take = true;
            } else {
                const Fe diff = fe_sub(dd, best);
                if (!fe_sure(diff)) return -1;
                take = diff.v < 0.f;
            }
            if (take) {
                found = true;
                best = dd;
                v = pt;
                mask = ((m & 1) ? (1 << i0) : 0) | ((m & 2) ? (1 << i1) : 0) | ((m & 4) ? (1 << i2) : 0);
            }
        }
        if (!found) return 1;
    }
    int m = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k < n && (mask & (1 << k))) {
            if (m != k) sp[m] = sp[k];
            m += 1;
        }
    }
    n = m;
    return 0;
}

// FP32 certified GJK of A (orientation qA, errors eqA) and B at Delta (error
// eD per component) with orientation qB (error eqB): GJK32_SEPARATED /
// GJK32_OVERLAP when certified equal to the FP64 contract, else
// GJK32_UNCERTAIN.  *iters as the contract (kGjkMaxIt + 1 at the cap).
template <int NV>
__device__ __noinline__ int gjk32c(const Shape3& sh, float dx, float dy, float dz, float eD, const float qA[4],
                                   float eqA, const float qB[4], float eqB, int* iters)
{
    const int nv = NV ? NV : sh.nv;
    const Fe qAc[4] = { { qA[0], eqA }, { -qA[1], eqA }, { -qA[2], eqA }, { -qA[3], eqA } };
    const Fe qBe[4] = { { qB[0], eqB }, { qB[1], eqB }, { qB[2], eqB }, { qB[3], eqB } };
    Fe qr[4];
    fe_qmul(qAc, qBe, qr);
    const Fe3 D = { { dx, eD }, { dy, eD }, { dz, eD } };
    const Fe3 l = fe_qrot(qAc, D);
    Fe3 pb[NV ? NV : kMaxV3], va[NV ? NV : kMaxV3];
#pragma unroll
    for (int i = 0; i < nv; ++i) {
        // fv = fl32(v): |fv - v| <= u32 |fv| (inflated)
        const Fe3 v = { { sh.fv[i][0], fin(ru_mul(fabsf(sh.fv[i][0]), kUr)) },
                        { sh.fv[i][1], fin(ru_mul(fabsf(sh.fv[i][1]), kUr)) },
                        { sh.fv[i][2], fin(ru_mul(fabsf(sh.fv[i][2]), kUr)) } };
        va[i] = v;
        const Fe3 r = fe_qrot(qr, v);
        pb[i] = { fe_add(r.x, l.x), fe_add(r.y, l.y), fe_add(r.z, l.z) };
    }
    // d = -l, or (-1, 0, 0) when l is exactly zero in the FP64 run
    Fe3 d = fe3_neg(l);
    if (!fe_sure(l.x) && !fe_sure(l.y) && !fe_sure(l.z)) return GJK32_UNCERTAIN;
    Fe3 sp[4], v;
    int n = 1;
    if (!support32<NV>(sh, pb, va, d, sp[0])) return GJK32_UNCERTAIN;
    v = sp[0];
#pragma unroll 1
    for (int it = 0; it < kGjkMaxIt; ++it) {
        *iters = it + 1;
        const Fe vv = fe3_dot(v, v);
        if (!fe_pos(vv)) return GJK32_UNCERTAIN;     // FP64 vv could be 0
        Fe3 w;
        if (!support32<NV>(sh, pb, va, fe3_neg(v), w)) return GJK32_UNCERTAIN;
        const Fe vw = fe3_dot(v, w);
        if (!fe_sure(vw)) return GJK32_UNCERTAIN;
        if (vw.v > 0.f) return GJK32_SEPARATED;
        sp[n] = w;
        n += 1;
        const int rr = gjk_reduce32(sp, n, v);
        if (rr < 0) return GJK32_UNCERTAIN;
        if (rr == 1) return GJK32_OVERLAP;
    }
    *iters = kGjkMaxIt + 1;
    return GJK32_OVERLAP;
}

}  // namespace hpmc
