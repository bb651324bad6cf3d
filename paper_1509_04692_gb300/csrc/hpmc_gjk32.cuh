// hpmc_gjk32.cuh -- FP32 GJK with certificates about the exact shapes.
//
// The FP64 contract (overlap3d64 in hpmc_device.cuh) breaks exact support
// ties by vertex index; near GJK's convergence ties are the rule for
// polytopes (the search direction becomes a face normal or an edge cross), and
// which of the tied vertices FP64 rounding picks cannot be reproduced in FP32.
// So the FP32 path does not mimic the FP64 run; it runs GJK in FP32 and then
// proves a verdict about the exact shapes (the exact transform of the FP64
// contract's inputs) with margin tau:
//  * overlap: the origin lies inside the tetrahedron of four exact vertex
//    differences of B - A, farther than tau from each face.  Then B - A
//    contains the origin at depth > tau, every FP64 support query has v.w <
//    0, so the FP64 GJK cannot answer "separated" (its cap counts as overlap):
//    it answers overlap.
//  * separated: some direction n has every vertex of B above every vertex of
//    A by more than tau |n|.  The FP64 closest-point GJK then answers
//    "separated": its distance estimate decreases to the positive separation
//    and the test v.w > 0 fires; this relies on GJK's termination for
//    polytopes separated far above its rounding (tau = 1e-9 of the shape
//    size, rounding ~1e-13), checked on random near-contact pairs by the
//    tests rather than proved.
// Anything not certified is re-decided by the FP64 contract.  All bound
// arithmetic rounds upward (__f*_ru) and bounds are inflated slightly.
#pragma once
#include "hpmc_types.h"

namespace hpmc {

// verdicts; every value >= GJK32_UNCERTAIN means "not certified" and names why
enum : int {
    GJK32_SEPARATED = 0,
    GJK32_OVERLAP = 1,
    GJK32_UNCERTAIN = 2,        // converged apart, gap within the bound
    GJK32_UNC_INSIDE = 3,       // enclosed, origin within the bound of a face
    GJK32_UNC_DEGENERATE = 4,   // flat simplex or zero direction
    GJK32_UNC_CAP = 5           // iteration cap
};

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

// ---------------------------------------------------------------- FP32 GJK
// Plain FP32 GJK with the contract's steps; every simplex point remembers the
// vertex pair (ib, ia) it came from so that the result can be certified.
struct G32 {
    float x, y, z;
};
__device__ __forceinline__ G32 g_sub(G32 a, G32 b) { return { a.x - b.x, a.y - b.y, a.z - b.z }; }
__device__ __forceinline__ G32 g_neg(G32 a) { return { -a.x, -a.y, -a.z }; }
// Products and sums in fused multiply-adds: each result is rounded at most
// as often as with separate operations, so the certificates' bounds, which
// count one rounding per operation, cover them.
__device__ __forceinline__ float g_dot(G32 a, G32 b) { return __fmaf_rn(a.z, b.z, __fmaf_rn(a.y, b.y, a.x * b.x)); }
__device__ __forceinline__ G32 g_cross(G32 a, G32 b)
{
    return { __fmaf_rn(a.y, b.z, -(a.z * b.y)), __fmaf_rn(a.z, b.x, -(a.x * b.z)), __fmaf_rn(a.x, b.y, -(a.y * b.x)) };
}
__device__ __forceinline__ G32 g_axpy(G32 a, float t, G32 b) { return { a.x + t * b.x, a.y + t * b.y, a.z + t * b.z }; }

struct SPt {
    G32 p;
    int ib, ia;
};

// vertex i of A (its own frame): the shape's FP32 copy, read from the kernel
// parameter (constant bank) instead of a register array
__device__ __forceinline__ G32 vA(const Shape3& sh, int i) { return G32{ sh.fv[i][0], sh.fv[i][1], sh.fv[i][2] }; }

template <int NV>
__device__ __forceinline__ SPt g_support(int nv, const G32* pb, const Shape3& sh, G32 d)
{
    int ib = 0, ia = 0;
    float best = g_dot(pb[0], d), least = g_dot(vA(sh, 0), d);
    auto step = [&](int i) {
        const float t = g_dot(pb[i], d);
        if (t > best) { best = t; ib = i; }
        const float u = g_dot(vA(sh, i), d);
        if (u < least) { least = u; ia = i; }
    };
    if constexpr (NV >= 16) {
        // many vertices: a partly unrolled loop keeps the body small
#pragma unroll 4
        for (int i = 1; i < NV; ++i) step(i);
    } else {
#pragma unroll
        for (int i = 1; i < (NV ? NV : kMaxV3); ++i) {
            if (!NV && i >= nv) break;
            step(i);
        }
    }
    return { g_sub(pb[ib], vA(sh, ia)), ib, ia };
}

// The same query for a centrally symmetric shape (fv ordered in pairs k,
// k + NV / 2) from the first half: the partner's pb . d is 2 l.d - pb_k . d
// and its vA . d is -vA_k . d, up to rounding, which only the searches use
// (the certificates scan every vertex).
template <int NV>
__device__ __forceinline__ SPt g_support_sym(const G32* pb, const Shape3& sh, G32 l, G32 d)
{
    constexpr int H = NV / 2;
    const float c2 = 2.0f * g_dot(l, d);
    int ib = 0, ia = 0;
    float best = g_dot(pb[0], d), least = g_dot(vA(sh, 0), d);
    if (c2 - best > best) { best = c2 - best; ib = H; }
    if (-least < least) { least = -least; ia = H; }
#pragma unroll
    for (int k = 1; k < H; ++k) {
        const float t = g_dot(pb[k], d), tp = c2 - t;
        const float u = g_dot(vA(sh, k), d);
        if (t > best) { best = t; ib = k; }
        if (tp > best) { best = tp; ib = k + H; }
        if (u < least) { least = u; ia = k; }
        if (-u < least) { least = -u; ia = k + H; }
    }
    return { g_sub(pb[ib], vA(sh, ia)), ib, ia };
}

// the support query of the searches
template <int NV>
__device__ __forceinline__ SPt g_support_q(int nv, const G32* pb, const Shape3& sh, G32 l, G32 d)
{
    if constexpr (NV >= 16)
        if (sh.sym) return g_support_sym<NV>(pb, sh, l, d);
    return g_support<NV>(nv, pb, sh, d);
}

__device__ __forceinline__ int g_closest_seg(G32 a, G32 b, G32& out)
{
    const G32 ab = g_sub(b, a), ap = g_neg(a);
    const float tn = g_dot(ab, ap);
    if (tn <= 0.f) { out = a; return 1; }
    const float den = g_dot(ab, ab);
    if (tn >= den) { out = b; return 2; }
    out = g_axpy(a, tn / den, ab);
    return 3;
}

__device__ __forceinline__ int g_closest_tri(G32 a, G32 b, G32 c, G32& out)
{
    const G32 ab = g_sub(b, a), ac = g_sub(c, a), ap = g_neg(a);
    const float d1 = g_dot(ab, ap), d2 = g_dot(ac, ap);
    if (d1 <= 0.f && d2 <= 0.f) { out = a; return 1; }
    const G32 bp = g_neg(b);
    const float d3 = g_dot(ab, bp), d4 = g_dot(ac, bp);
    if (d3 >= 0.f && d4 <= d3) { out = b; return 2; }
    const float vc = d1 * d4 - d3 * d2;
    if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) { out = g_axpy(a, d1 / (d1 - d3), ab); return 3; }
    const G32 cp = g_neg(c);
    const float d5 = g_dot(ab, cp), d6 = g_dot(ac, cp);
    if (d6 >= 0.f && d5 <= d6) { out = c; return 4; }
    const float vb = d5 * d2 - d1 * d6;
    if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) { out = g_axpy(a, d2 / (d2 - d6), ac); return 5; }
    const float va = d3 * d6 - d5 * d4;
    const float e43 = d4 - d3, e56 = d5 - d6;
    if (va <= 0.f && e43 >= 0.f && e56 >= 0.f) { out = g_axpy(b, e43 / (e43 + e56), g_sub(c, b)); return 6; }
    const float sum = (va + vb) + vc;
    if (!(sum > 0.f)) return 0;
    const float den = 1.0f / sum;
    const float v = vb * den, w = vc * den;
    out = { (a.x + ab.x * v) + ac.x * w, (a.y + ab.y * v) + ac.y * w, (a.z + ab.z * v) + ac.z * w };
    return 7;
}

__device__ __forceinline__ bool g_outside(G32 p, G32 q, G32 r, G32 s)
{
    const G32 n = g_cross(g_sub(q, p), g_sub(r, p));
    const float sp = g_dot(g_neg(p), n), sd = g_dot(g_sub(s, p), n);
    return (sp > 0.f && sd < 0.f) || (sp < 0.f && sd > 0.f);
}

// 0 continue, 1 origin inside the tetrahedron, 2 degenerate
__device__ __forceinline__ int g_reduce(SPt sp[4], int& n, G32& v)
{
    int mask = 0;
    if (n == 2) {
        mask = g_closest_seg(sp[0].p, sp[1].p, v);
    } else if (n == 3) {
        mask = g_closest_tri(sp[0].p, sp[1].p, sp[2].p, v);
        if (mask == 0) return 2;
    } else {
        bool found = false;
        float best = 0.f;
#pragma unroll 1
        for (int f = 0; f < 4; ++f) {
            const int i0 = (f == 3) ? 1 : 0, i1 = (f <= 1) ? 1 : 2, i2 = (f == 0) ? 2 : 3, i3 = 3 - f;
            if (!g_outside(sp[i0].p, sp[i1].p, sp[i2].p, sp[i3].p)) continue;
            G32 pt;
            const int m = g_closest_tri(sp[i0].p, sp[i1].p, sp[i2].p, pt);
            if (m == 0) return 2;
            const float dd = g_dot(pt, pt);
            if (!found || dd < best) {
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

// ------------------------------------------------------------ certificates
// Separation: along direction nrm, every vertex of B (in A's frame) lies above
// every vertex of A by more than tau |nrm| once all FP32 errors are added.
template <int NV>
__device__ __forceinline__ bool cert_separated(int nv, const G32* pb, const Shape3& sh, G32 nrm, float e_pb,
                                               float e_va, float tau)
{
    float minB = g_dot(pb[0], nrm), maxA = g_dot(vA(sh, 0), nrm);
    float P = 0.f, V = 0.f;
    auto step = [&](int i) {
        minB = fminf(minB, g_dot(pb[i], nrm));
        maxA = fmaxf(maxA, g_dot(vA(sh, i), nrm));
        P = fmaxf(P, fmaxf(fabsf(pb[i].x), fmaxf(fabsf(pb[i].y), fabsf(pb[i].z))));
        V = fmaxf(V, fmaxf(fabsf(vA(sh, i).x), fmaxf(fabsf(vA(sh, i).y), fabsf(vA(sh, i).z))));
    };
    if constexpr (NV >= 16) {
#pragma unroll 4
        for (int i = 0; i < NV; ++i) step(i);
    } else {
#pragma unroll
        for (int i = 0; i < (NV ? NV : kMaxV3); ++i) {
            if (!NV && i >= nv) break;
            step(i);
        }
    }
    const float n1 = __fadd_ru(__fadd_ru(fabsf(nrm.x), fabsf(nrm.y)), fabsf(nrm.z));
    const float gap = minB - maxA;
    // |dot32 - dot_exact| <= |n|_1 (e_vertex + 4 u P); the gap's own rounding
    const float eg = __fmul_ru(n1, __fadd_ru(__fadd_ru(e_pb, e_va), __fmul_ru(4.0f * kUr, __fadd_ru(P, V))));
    const float bound = __fadd_ru(__fadd_ru(eg, __fmul_ru(2.0f * kUr, fabsf(gap))), __fmul_ru(tau, n1));
    return gap > fin(bound);
}

// Overlap: the origin lies strictly inside the tetrahedron of the four exact
// vertex differences, farther than tau from each face plane.
// The test on four points W[k] of B - A given with their error bounds (the
// exact points, which the test is about, lie within them).
__device__ __forceinline__ bool cert_inside_pts(const Fe3 W[4], float tau)
{
#pragma unroll 1
    for (int f = 0; f < 4; ++f) {
        const int i0 = (f == 3) ? 1 : 0, i1 = (f <= 1) ? 1 : 2, i2 = (f == 0) ? 2 : 3, i3 = 3 - f;
        const Fe3 nn = fe3_cross(fe3_sub(W[i1], W[i0]), fe3_sub(W[i2], W[i0]));
        const Fe so = fe3_dot(fe3_neg(W[i0]), nn);
        const Fe sd = fe3_dot(fe3_sub(W[i3], W[i0]), nn);
        if (!fe_sure(so) || !fe_sure(sd)) return false;
        if ((so.v > 0.f) != (sd.v > 0.f)) return false;        // origin outside this face
        // distance to the plane: (|so| - e_so) / |n|_2 > tau, |n|_2 <= |n|_1 + 3 e_n
        const float n1 = __fadd_ru(__fadd_ru(__fadd_ru(fabsf(nn.x.v), nn.x.e), __fadd_ru(fabsf(nn.y.v), nn.y.e)),
                                   __fadd_ru(fabsf(nn.z.v), nn.z.e));
        if (!(__fsub_rd(fabsf(so.v), so.e) > __fmul_ru(tau, n1))) return false;
    }
    return true;
}

__device__ __forceinline__ Fe3 fe3_vertex_diff(const G32* pb, const Shape3& sh, const SPt& q, float e_pb, float e_va)
{
    const G32 b = pb[q.ib], a = vA(sh, q.ia);
    return fe3_sub(Fe3{ { b.x, e_pb }, { b.y, e_pb }, { b.z, e_pb } }, Fe3{ { a.x, e_va }, { a.y, e_va }, { a.z, e_va } });
}

// the tetrahedron of four exact vertex differences
__device__ __forceinline__ bool cert_inside(const G32* pb, const Shape3& sh, const SPt sp[4], float e_pb, float e_va,
                                            float tau)
{
    Fe3 W[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) W[k] = fe3_vertex_diff(pb, sh, sp[k], e_pb, e_va);
    return cert_inside_pts(W, tau);
}

// GJK stops at the first tetrahedron that encloses the origin, which may
// have the origin next to one of its faces although the origin lies deep
// inside B - A.  Expansion (one step of the polytope expansion used for
// penetration depths, a few times): take the face nearest the origin, add
// the support point w beyond it, and move to whichever of the three
// tetrahedra (w, opposite vertex, face edge) encloses the origin; certify it.
template <int NV>
__device__ __noinline__ bool expand_inside(int nv, const G32* pb, const Shape3& sh, SPt sp[4], float e_pb, float e_va,
                                           float tau)
{
#pragma unroll 1
    for (int rep = 0; rep < 4; ++rep) {
        // face of the current tetrahedron nearest the origin (plain FP32)
        int fbest = 0;
        float dbest = 0.f;
        G32 nbest = { 0.f, 0.f, 0.f };
#pragma unroll 1
        for (int f = 0; f < 4; ++f) {
            const int i0 = (f == 3) ? 1 : 0, i1 = (f <= 1) ? 1 : 2, i2 = (f == 0) ? 2 : 3, i3 = 3 - f;
            G32 n = g_cross(g_sub(sp[i1].p, sp[i0].p), g_sub(sp[i2].p, sp[i0].p));
            if (g_dot(n, g_sub(sp[i3].p, sp[i0].p)) > 0.f) n = g_neg(n);       // outward
            const float nn = g_dot(n, n);
            if (!(nn > 0.f)) return false;
            const float h = g_dot(n, sp[i0].p);                                 // > 0: origin inside
            const float dd = h * fabsf(h) / nn;
            if (f == 0 || dd < dbest) { dbest = dd; fbest = f; nbest = n; }
        }
        const int i0 = (fbest == 3) ? 1 : 0, i1 = (fbest <= 1) ? 1 : 2, i2 = (fbest == 0) ? 2 : 3, i3 = 3 - fbest;
        const SPt w = g_support<NV>(nv, pb, sh, nbest);
        const float hw = g_dot(nbest, w.p), hf = g_dot(nbest, sp[i0].p);
        if (!(hw > hf + 1e-6f * fabsf(hf) + 1e-30f)) return false;              // face on the boundary of B - A
        const SPt T[3][4] = { { w, sp[i3], sp[i0], sp[i1] }, { w, sp[i3], sp[i1], sp[i2] },
                              { w, sp[i3], sp[i2], sp[i0] } };
        int pick = -1;
#pragma unroll 1
        for (int t = 0; t < 3 && pick < 0; ++t) {
            bool in = true;
#pragma unroll 1
            for (int f = 0; f < 4 && in; ++f) {
                const int j0 = (f == 3) ? 1 : 0, j1 = (f <= 1) ? 1 : 2, j2 = (f == 0) ? 2 : 3, j3 = 3 - f;
                in = !g_outside(T[t][j0].p, T[t][j1].p, T[t][j2].p, T[t][j3].p);
            }
            if (in) pick = t;
        }
        if (pick < 0) return false;
#pragma unroll
        for (int k = 0; k < 4; ++k) sp[k] = T[pick][k];
        if (cert_inside(pb, sh, sp, e_pb, e_va, tau)) return true;
    }
    return false;
}

// B placed in A's frame in FP32 (A with orientation qA, B at Delta with
// orientation qB): its centre l and its vertices pb.  Quaternions as (w, x,
// y, z) in a float4's (x, y, z, w).
template <int NV>
__device__ __forceinline__ void gjk32_setup(const Shape3& sh, float dx, float dy, float dz, float4 qA, float4 qB,
                                            G32& l, G32* pb)
{
    const int nv = NV ? NV : sh.nv;
    // qr = conj(qA) qB, l = rot(conj(qA), Delta), pb = rot(qr, v) + l
    const float a0 = qA.x, a1 = -qA.y, a2 = -qA.z, a3 = -qA.w;
    const float b0 = qB.x, b1 = qB.y, b2 = qB.z, b3 = qB.w;
    const float r0 = ((a0 * b0 - a1 * b1) - a2 * b2) - a3 * b3;
    const float r1 = ((a0 * b1 + a1 * b0) + a2 * b3) - a3 * b2;
    const float r2 = ((a0 * b2 - a1 * b3) + a2 * b0) + a3 * b1;
    const float r3 = ((a0 * b3 + a1 * b2) - a2 * b1) + a3 * b0;
    // (fused multiply-adds: no more roundings than the operations the
    // vertex bound counts)
    auto rot = [](float w, float x, float y, float z, G32 v) {
        const float tx = 2.0f * __fmaf_rn(y, v.z, -(z * v.y));
        const float ty = 2.0f * __fmaf_rn(z, v.x, -(x * v.z));
        const float tz = 2.0f * __fmaf_rn(x, v.y, -(y * v.x));
        return G32{ __fmaf_rn(w, tx, v.x) + __fmaf_rn(y, tz, -(z * ty)), __fmaf_rn(w, ty, v.y) + __fmaf_rn(z, tx, -(x * tz)),
                    __fmaf_rn(w, tz, v.z) + __fmaf_rn(x, ty, -(y * tx)) };
    };
    l = rot(a0, a1, a2, a3, G32{ dx, dy, dz });
    if (NV >= 16 && sh.sym) {
        // rot is odd in v, exactly: the partner k + nv / 2 of vertex k is
        // l - rot(v_k), the same FP32 value as rot(-v_k) + l
        constexpr int H = NV / 2;
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const G32 rr = rot(r0, r1, r2, r3, vA(sh, k));
            pb[k] = G32{ rr.x + l.x, rr.y + l.y, rr.z + l.z };
            pb[k + H] = G32{ l.x - rr.x, l.y - rr.y, l.z - rr.z };
        }
    } else if constexpr (NV >= 16) {
#pragma unroll 4
        for (int i = 0; i < NV; ++i) {
            const G32 rr = rot(r0, r1, r2, r3, vA(sh, i));
            pb[i] = G32{ rr.x + l.x, rr.y + l.y, rr.z + l.z };
        }
    } else {
#pragma unroll
        for (int i = 0; i < (NV ? NV : kMaxV3); ++i) {
            if (!NV && i >= nv) break;
            const G32 rr = rot(r0, r1, r2, r3, vA(sh, i));
            pb[i] = G32{ rr.x + l.x, rr.y + l.y, rr.z + l.z };
        }
    }
}

// FP32 GJK + certificate from B's vertices pb in A's frame and B's centre l
// there: GJK32_SEPARATED / GJK32_OVERLAP when certified about the exact
// shapes with margin tau (where the FP64 contract decides the same),
// GJK32_UNCERTAIN (or a more specific reason >= 2) otherwise.
template <int NV>
__device__ __forceinline__ int gjk32_run(int nv, const G32* pb, const Shape3& sh, G32 l, float e_pb, float e_va,
                                         float tau)
{
    // the centre line first: well-separated pairs are certified without GJK
    if (cert_separated<NV>(nv, pb, sh, l, e_pb, e_va, tau)) return GJK32_SEPARATED;
    G32 d = g_neg(l);
    if (d.x == 0.f && d.y == 0.f && d.z == 0.f) d.x = -1.0f;
    SPt sp[4];
    int n = 1;
    sp[0] = g_support_q<NV>(nv, pb, sh, l, d);
    G32 v = sp[0].p;
    bool tried = false;   // a separating direction failed its certificate
#pragma unroll 1
    for (int it = 0; it < kGjkMaxIt; ++it) {
        const float vv = g_dot(v, v);
        if (vv == 0.f) return GJK32_UNC_DEGENERATE;
        const SPt w = g_support_q<NV>(nv, pb, sh, l, g_neg(v));
        const float vw = g_dot(v, w.p);
        if (vw > 0.f) {
            // v separates in FP32.  Certify it; if the gap is within the
            // bound, keep iterating towards the closest point (the largest
            // gap any direction can show) until the distance estimate stalls.
            if (cert_separated<NV>(nv, pb, sh, v, e_pb, e_va, tau)) return GJK32_SEPARATED;
            if (tried && __fsub_rn(vv, vw) <= __fmul_rn(1e-6f, vv)) return GJK32_UNCERTAIN;
            tried = true;
        }
        bool dup = false;
#pragma unroll
        for (int k = 0; k < 4; ++k) dup |= (k < n) && sp[k].ib == w.ib && sp[k].ia == w.ia;
        if (dup) return vw > 0.f ? GJK32_UNCERTAIN : GJK32_UNC_DEGENERATE;
        sp[n] = w;
        n += 1;
        const int rr = g_reduce(sp, n, v);
        if (rr == 1) {
            if (cert_inside(pb, sh, sp, e_pb, e_va, tau)) return GJK32_OVERLAP;
            return expand_inside<NV>(nv, pb, sh, sp, e_pb, e_va, tau) ? GJK32_OVERLAP : GJK32_UNC_INSIDE;
        }
        if (rr == 2) return GJK32_UNC_DEGENERATE;
    }
    return GJK32_UNC_CAP;
}

// the same from Delta and the two orientations
template <int NV>
__device__ __forceinline__ int gjk32_cert(const Shape3& sh, float dx, float dy, float dz, float4 qA, float4 qB,
                                          float e_pb, float e_va, float tau)
{
    G32 l;
    G32 pb[NV ? NV : kMaxV3];
    gjk32_setup<NV>(sh, dx, dy, dz, qA, qB, l, pb);
    return gjk32_run<NV>(NV ? NV : sh.nv, pb, sh, l, e_pb, e_va, tau);
}

// Boxes (Shape3::box: vertices (+-h0, +-h1, +-h2)): the separating-axis
// test decides a pair exactly, since two boxes are disjoint iff one of 15
// axes separates them: A's face normals e_k, B's face normals u_j (B's axes
// in A's frame, the columns of the rotation matrix M of qr = conj(qA) qB)
// and the 9 edge crosses e_i x u_j.  Along an axis n the centre distance
// |l.n| (l = rot(conj(qA), Delta)) is compared with the two half extents
// sum_k h_k |n_k| and sum_m h_m |n.u_m|, the latter from M's orthonormal
// identities (u_j.u_m = delta_jm, e_i x u_j . u_m = +-M[i][k]).  With s(n) =
// |l.n| - extent_A - extent_B and s_max the largest s of the 15:
//  * s_max > e_sep: the exact boxes are apart along that axis by more than
//    the FP32 error and the separation floor (host: box_sat_margins);
//  * s_max < -e_ov: every exact candidate axis shows an overlap deeper than
//    tau, so the exact boxes intersect and their Minkowski difference holds
//    the origin at depth > tau (its facet normals are among the candidates),
//    where the FP64 GJK answers overlap;
//  * otherwise uncertain (within the error band of contact, or a degenerate
//    edge cross): the FP64 contract decides.
// Branch-free: 15 axes, about 200 FP32 operations, no vertex loop.
__device__ __forceinline__ int box32_sat(const Shape3& sh, float dx, float dy, float dz, float4 qA, float4 qB,
                                         float e_sep, float e_ov)
{
    const float a0 = qA.x, a1 = -qA.y, a2 = -qA.z, a3 = -qA.w;
    const float b0 = qB.x, b1 = qB.y, b2 = qB.z, b3 = qB.w;
    const float w = ((a0 * b0 - a1 * b1) - a2 * b2) - a3 * b3;
    const float x = ((a0 * b1 + a1 * b0) + a2 * b3) - a3 * b2;
    const float y = ((a0 * b2 - a1 * b3) + a2 * b0) + a3 * b1;
    const float z = ((a0 * b3 + a1 * b2) - a2 * b1) + a3 * b0;
    // l = rot(conj(qA), Delta), the same evaluation as the certified GJK
    // (fused multiply-adds throughout: no more roundings than the
    // operations the margins count)
    const float tx = 2.0f * __fmaf_rn(a2, dz, -(a3 * dy));
    const float ty = 2.0f * __fmaf_rn(a3, dx, -(a1 * dz));
    const float tz = 2.0f * __fmaf_rn(a1, dy, -(a2 * dx));
    const float l[3] = { __fmaf_rn(a0, tx, dx) + __fmaf_rn(a2, tz, -(a3 * ty)),
                         __fmaf_rn(a0, ty, dy) + __fmaf_rn(a3, tx, -(a1 * tz)),
                         __fmaf_rn(a0, tz, dz) + __fmaf_rn(a1, ty, -(a2 * tx)) };
    // M[k][j] = component k of u_j = R(qr) e_j
    float M[3][3];
    M[0][0] = 1.0f - 2.0f * __fmaf_rn(y, y, z * z);
    M[1][1] = 1.0f - 2.0f * __fmaf_rn(x, x, z * z);
    M[2][2] = 1.0f - 2.0f * __fmaf_rn(x, x, y * y);
    M[1][0] = 2.0f * __fmaf_rn(x, y, w * z);
    M[0][1] = 2.0f * __fmaf_rn(x, y, -(w * z));
    M[2][0] = 2.0f * __fmaf_rn(x, z, -(w * y));
    M[0][2] = 2.0f * __fmaf_rn(x, z, w * y);
    M[2][1] = 2.0f * __fmaf_rn(y, z, w * x);
    M[1][2] = 2.0f * __fmaf_rn(y, z, -(w * x));
    float A[3][3];   // |M|
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j) A[k][j] = fabsf(M[k][j]);
    const float h[3] = { sh.bh[0], sh.bh[1], sh.bh[2] };
    float smax = -3.0e38f;
    // A's faces e_k
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float eb = __fmaf_rn(h[2], A[k][2], __fmaf_rn(h[1], A[k][1], h[0] * A[k][0]));
        smax = fmaxf(smax, (fabsf(l[k]) - h[k]) - eb);
    }
    // B's faces u_j
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float c = __fmaf_rn(l[2], M[2][j], __fmaf_rn(l[1], M[1][j], l[0] * M[0][j]));
        const float ea = __fmaf_rn(h[2], A[2][j], __fmaf_rn(h[1], A[1][j], h[0] * A[0][j]));
        smax = fmaxf(smax, (fabsf(c) - ea) - h[j]);
    }
    // edge crosses e_i x u_j; (i, i1, i2) and (j, j1, j2) cyclic
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
            const float c = __fmaf_rn(l[i2], M[i1][j], -(l[i1] * M[i2][j]));
            const float ea = __fmaf_rn(h[i1], A[i2][j], h[i2] * A[i1][j]);
            const float eb = __fmaf_rn(h[j1], A[i][j2], h[j2] * A[i][j1]);
            smax = fmaxf(smax, (fabsf(c) - ea) - eb);
        }
    }
    if (smax > e_sep) return GJK32_SEPARATED;
    if (-smax > e_ov) return GJK32_OVERLAP;
    return GJK32_UNCERTAIN;
}

}  // namespace hpmc
