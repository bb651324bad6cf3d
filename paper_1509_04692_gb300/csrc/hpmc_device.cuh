// hpmc_device.cuh -- device core: Philox streams and the FP64 decision
// contract (trial moves, cell rule, separating-axis and GJK overlap tests).
//
// Everything in this file is the library's own statement of the rules both
// the CPU oracle and the kernels follow; it shares no code with the oracle.
// The translation unit is compiled with -fmad=false, so every FP64 expression
// below rounds once per operation, in the written (left-to-right) order,
// exactly like the IEEE host arithmetic it is compared against.
#pragma once
#include <cstdint>
#include "hpmc_types.h"

namespace hpmc {

// Programmatic dependent launch (sm_90 and later).  The rebuild kernels are
// launched with programmatic stream serialisation: each sweep kernel first
// lets the next kernel of the stream be scheduled (its blocks become
// resident and wait), then waits until the previous kernel has completed and
// its memory is visible.  Nothing is read or written before the wait, so the
// order of the stream is kept; what is saved is the launch latency between
// the short rebuild kernels (24 -> 16 us per sweep of 4096 particles).  In a
// kernel launched without the attribute (the first set kernel of a sweep)
// the wait returns at once.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// The set kernels after the first of a sweep are launched with the same
// attribute but only wait: no set kernel lets the next kernel be scheduled
// before its blocks exit (waiting blocks beside a running set kernel
// measured slower), so what overlaps is the next launch's setup with the
// drain of this one.
__device__ __forceinline__ void pdl_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds, each two
// 32x32->64 multiplies whose halves are xored with the other counter words
// and the round key; the key advances by the golden-ratio / sqrt(3) Weyl
// constants between rounds.
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Random words of one trial move (Sec. 2.5: one stream per trial move):
// counter (cell, lo32(sweep), hi32(sweep) << 16 | k, 1 << 24 | set << 16 | block).
__device__ __forceinline__ uint4 move_block(uint64_t seed, uint64_t sweep, uint32_t set,
                                            uint32_t cell, uint32_t k, uint32_t block)
{
    return philox(make_uint4(cell, (uint32_t)sweep, ((uint32_t)(sweep >> 32) << 16) | k,
                             (1u << 24) | (set << 16) | block),
                  (uint32_t)seed, (uint32_t)(seed >> 32));
}

__device__ __forceinline__ uint4 shift_block(uint64_t seed, uint64_t sweep, uint32_t block)
{
    return philox(make_uint4(0u, (uint32_t)sweep, (uint32_t)(sweep >> 32) << 16, (2u << 24) | block),
                  (uint32_t)seed, (uint32_t)(seed >> 32));
}

// u in [0, 1) from the 53 top bits of (a << 32 | b); exact.
__device__ __forceinline__ double u53(uint32_t a, uint32_t b)
{
    const unsigned long long m = (((unsigned long long)a << 32) | b) >> 11;
    return __ull2double_rn(m) * 0x1.0p-53;
}

// 2*u53(a, b) - 1 scaled by 2^53: the integer j = 2k - 2^53 with
// k = (a << 32 | b) >> 11, |j| <= 2^53, so (double)j is exact.  For a factor f,
// fl((f * 2^-53) * j) equals fl(f * (2*u53 - 1)) bit for bit (the power-of-two
// scaling of f is exact), with one integer-to-double conversion instead of
// the conversion, scaling, doubling and subtraction of the direct form.
__device__ __forceinline__ double pm53(uint32_t a, uint32_t b)
{
    const long long k = (long long)((((unsigned long long)a << 32) | b) >> 11);
    return __ll2double_rn(2 * k - (1LL << 53));
}

// Periodic wrap of a coordinate moved by less than L, with the sign and
// upper-bound tests done on the bit pattern (IEEE order of non-negative
// doubles is the order of their bit patterns); same results as wrap_pos.
__device__ __forceinline__ double wrap_pos_bits(double x, double L)
{
    const long long b = __double_as_longlong(x);
    if (b < 0 && b != (long long)0x8000000000000000ULL) x = x + L;   // x < 0 (not -0)
    if (__double_as_longlong(x) >= __double_as_longlong(L)) x = x - L;
    return x;
}

// y = x - s (+ L when negative) with the sign test on the bit pattern
__device__ __forceinline__ double cell_coord_bits(double x, double s, double L)
{
    double y = x - s;
    const long long b = __double_as_longlong(y);
    if (b < 0 && b != (long long)0x8000000000000000ULL) y = y + L;
    return y;
}

// FP32 stand-in for 2*u53(a, b) - 1 built from the 24 top bits of a; exact
// in FP32 and within 2^-23 of the FP64 value.
__device__ __forceinline__ float m24(uint32_t a)
{
    return __fmul_rn(2.0f, __uint2float_rn(a >> 8) * 0x1.0p-24f) - 1.0f;
}

// --------------------------------------------------------- contract: cells
__device__ __forceinline__ int cell_axis(double x, double s, double L, double inv_w, int nc)
{
    double y = x - s;
    if (y < 0.0) y = y + L;
    int i = (int)(y * inv_w);
    if (i >= nc) i = nc - 1;
    return i;
}

__device__ __forceinline__ double wrap_pos(double x, double L)
{
    if (x < 0.0) x = x + L;
    if (x >= L) x = x - L;
    return x;
}

__device__ __forceinline__ double min_image(double d, double L, double halfL)
{
    if (d > halfL) d = d - L;
    else if (d < -halfL) d = d + L;
    return d;
}

// ------------------------------------------------- contract: trial moves
// 2D translation + Cayley rotation from the words r1..r6 of a select.
struct Trial2 { double x, y, c, s; };

__device__ __forceinline__ Trial2 propose2d(const Rep& rp, double x, double y, double c, double s,
                                            uint32_t r1, uint32_t r2, uint32_t r3, uint32_t r4,
                                            uint32_t r5, uint32_t r6)
{
    // d * (2 u53 - 1) etc., see pm53
    const double dx = rp.d_s * pm53(r1, r2);
    const double dy = rp.d_s * pm53(r3, r4);
    const double t = rp.tau_s * pm53(r5, r6);
    Trial2 o;
    o.x = wrap_pos_bits(x + dx, rp.L[0]);
    o.y = wrap_pos_bits(y + dy, rp.L[1]);
    const double tt = t * t;
    const double inv = 1.0 / (1.0 + tt);
    const double cd = (1.0 - tt) * inv;
    const double sd = (t + t) * inv;
    const double c1 = c * cd - s * sd;
    const double s1 = c * sd + s * cd;
    const double n2 = c1 * c1 + s1 * s1;
    const double f = 1.5 - 0.5 * n2;
    o.c = c1 * f;
    o.s = s1 * f;
    return o;
}

// Hamilton product a * b, sums left to right.
__device__ __forceinline__ void qmul(const double a[4], const double b[4], double o[4])
{
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// rotate v by unit quaternion q: t = 2 (q_v x v); v' = (v + w t) + q_v x t
__device__ __forceinline__ void qrot(const double q[4], const double v[3], double o[3])
{
    const double tx = 2.0 * (q[2] * v[2] - q[3] * v[1]);
    const double ty = 2.0 * (q[3] * v[0] - q[1] * v[2]);
    const double tz = 2.0 * (q[1] * v[1] - q[2] * v[0]);
    o[0] = (v[0] + q[0] * tx) + (q[2] * tz - q[3] * ty);
    o[1] = (v[1] + q[0] * ty) + (q[3] * tx - q[1] * tz);
    o[2] = (v[2] + q[0] * tz) + (q[1] * ty - q[2] * tx);
}

struct Trial3 { double x[3]; double q[4]; };

// 3D translation + rotation dq = (1, v) / sqrt(1 + v.v) from words r1..r12.
// orientation step of the contract: dq = (1, v) / sqrt(1 + v.v) with
// v = tau (2u - 1) per component from words r[7..12]
__device__ __forceinline__ void orient_step3(const Rep& rp, const uint32_t* r, double dq[4])
{
    const double v0 = rp.tau_s * pm53(r[7], r[8]);
    const double v1 = rp.tau_s * pm53(r[9], r[10]);
    const double v2 = rp.tau_s * pm53(r[11], r[12]);
    const double vv = (v0 * v0 + v1 * v1) + v2 * v2;
    const double inv = 1.0 / sqrt(1.0 + vv);
    dq[0] = inv; dq[1] = v0 * inv; dq[2] = v1 * inv; dq[3] = v2 * inv;
}

// trial orientation of the contract: q' = renorm(q (x) dq)
__device__ __forceinline__ void orient_apply3(const double q[4], const double dq[4], double o[4])
{
    double q1[4];
    qmul(q, dq, q1);
    const double n2 = ((q1[0] * q1[0] + q1[1] * q1[1]) + q1[2] * q1[2]) + q1[3] * q1[3];
    const double f = 1.5 - 0.5 * n2;
    o[0] = q1[0] * f; o[1] = q1[1] * f; o[2] = q1[2] * f; o[3] = q1[3] * f;
}

// Component i of qmul(a, b) with the contract's operations: a0 b_i first,
// then a_j b_(i^j) for j = 1, 2, 3 in order, the sign of each term folded
// into a_j (negation is exact, and x - y rounds as x + (-y)).
__device__ __forceinline__ double qmul_component(const double a[4], const double* b, int i)
{
    const int neg = (0x2147 >> (4 * i)) & 7;          // i: 0 -> 7, 1 -> 4, 2 -> 1, 3 -> 2
    double acc = a[0] * b[i];
    acc = acc + ((neg & 1) ? -a[1] : a[1]) * b[i ^ 1];
    acc = acc + ((neg & 2) ? -a[2] : a[2]) * b[i ^ 2];
    acc = acc + ((neg & 4) ? -a[3] : a[3]) * b[i ^ 3];
    return acc;
}

__device__ __forceinline__ void propose3d_orient(const Rep& rp, const double q[4], const uint32_t* r, double o[4])
{
    double dq[4];
    orient_step3(rp, r, dq);
    orient_apply3(q, dq, o);
}

__device__ __forceinline__ Trial3 propose3d(const Rep& rp, const double x[3], const double q[4],
                                            const uint32_t* r)
{
    Trial3 o;
    const double dx = rp.d_s * pm53(r[1], r[2]);
    const double dy = rp.d_s * pm53(r[3], r[4]);
    const double dz = rp.d_s * pm53(r[5], r[6]);
    o.x[0] = wrap_pos_bits(x[0] + dx, rp.L[0]);
    o.x[1] = wrap_pos_bits(x[1] + dy, rp.L[1]);
    o.x[2] = wrap_pos_bits(x[2] + dz, rp.L[2]);
    propose3d_orient(rp, q, r, o.q);
    return o;
}

// ------------------------------------- contract: 2D separating axes, FP64
// B placed in A's frame by rotation (cr, sr) and offset (lx, ly); the edge
// normals of A separate when A's interval and B's projections do not meet.
template <int NV>
__device__ __forceinline__ bool sat_half64(const Shape2& sh, double cr, double sr, double lx, double ly)
{
    const int nv = NV ? NV : sh.nv;
    double px[NV ? NV : kMaxV2], py[NV ? NV : kMaxV2];
#pragma unroll
    for (int i = 0; i < nv; ++i) {
        px[i] = (cr * sh.vx[i] - sr * sh.vy[i]) + lx;
        py[i] = (sr * sh.vx[i] + cr * sh.vy[i]) + ly;
    }
#pragma unroll
    for (int k = 0; k < nv; ++k) {
        double lo = sh.nx[k] * px[0] + sh.ny[k] * py[0];
        double hi = lo;
#pragma unroll
        for (int i = 1; i < nv; ++i) {
            const double t = sh.nx[k] * px[i] + sh.ny[k] * py[i];
            lo = t < lo ? t : lo;
            hi = t > hi ? t : hi;
        }
        if (sh.ahi[k] < lo || hi < sh.alo[k]) return true;
    }
    return false;
}

// One axis of D: half hf = 0 tests A's normal k with B placed in A's frame,
// hf = 1 tests B's normal k with A placed in B's frame; the operations are
// those sat_half64 performs for that axis, so D(...) separates iff some
// (hf, k) returns true here.
template <int NV>
__device__ __forceinline__ bool axis_separates64(const Shape2& sh, int hf, int k, double Dx, double Dy,
                                                 double cA, double sA, double cB, double sB)
{
    const int nv = NV ? NV : sh.nv;
    const double cr = cA * cB + sA * sB;
    const double sr = cA * sB - sA * cB;
    double cc, ss, lx, ly;
    if (hf == 0) {
        cc = cr; ss = sr;
        lx = cA * Dx + sA * Dy;
        ly = cA * Dy - sA * Dx;
    } else {
        cc = cr; ss = -sr;
        lx = -(cB * Dx + sB * Dy);
        ly = -(cB * Dy - sB * Dx);
    }
    double lo = 0.0, hi = 0.0;
#pragma unroll
    for (int i = 0; i < (NV ? NV : kMaxV2); ++i) {
        if (!NV && i >= nv) break;
        const double px = (cc * sh.vx[i] - ss * sh.vy[i]) + lx;
        const double py = (ss * sh.vx[i] + cc * sh.vy[i]) + ly;
        const double t = sh.nx[k] * px + sh.ny[k] * py;
        lo = (i == 0 || t < lo) ? t : lo;
        hi = (i == 0 || t > hi) ? t : hi;
    }
    return sh.ahi[k] < lo || hi < sh.alo[k];
}

// D(Delta, zA, zB): true = overlap (touching counts), false = separated.
template <int NV>
__device__ __forceinline__ bool overlap2d64(const Shape2& sh, double Dx, double Dy,
                                            double cA, double sA, double cB, double sB)
{
    if (NV == 0 && sh.round) return (Dx * Dx + Dy * Dy) <= sh.rc2;      // disks
    const double cr = cA * cB + sA * sB;
    const double sr = cA * sB - sA * cB;
    const double lx = cA * Dx + sA * Dy;
    const double ly = cA * Dy - sA * Dx;
    if (sat_half64<NV>(sh, cr, sr, lx, ly)) return false;
    const double mx = cB * Dx + sB * Dy;
    const double my = cB * Dy - sB * Dx;
    if (sat_half64<NV>(sh, cr, -sr, -mx, -my)) return false;
    return true;
}

// ------------------------------------------------ contract: 3D GJK, FP64
__device__ __forceinline__ double dot3(const double a[3], const double b[3])
{
    return (a[0] * b[0] + a[1] * b[1]) + a[2] * b[2];
}
__device__ __forceinline__ void cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ void sub3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
__device__ __forceinline__ void neg3(const double a[3], double o[3])
{
    o[0] = -a[0]; o[1] = -a[1]; o[2] = -a[2];
}
__device__ __forceinline__ void cpy3(const double a[3], double o[3])
{
    o[0] = a[0]; o[1] = a[1]; o[2] = a[2];
}

// Support of B - A in direction d (B's vertices pb already in A's frame):
// first argmax of pb.d minus first argmin of v.d.
template <int NV>
__device__ __forceinline__ void support3(const Shape3& sh, const double (*pb)[3],
                                         const double d[3], double out[3])
{
    const int nv = NV ? NV : sh.nv;
    int ib = 0, ia = 0;
    double best = dot3(pb[0], d);
    double least = dot3(sh.v[0], d);
#pragma unroll
    for (int i = 1; i < nv; ++i) {
        const double t = dot3(pb[i], d);
        if (t > best) { best = t; ib = i; }
        const double u = dot3(sh.v[i], d);
        if (u < least) { least = u; ia = i; }
    }
    sub3(pb[ib], sh.v[ia], out);
}

// closest point of segment [a, b] to the origin; feature mask (a=1, b=2)
__device__ __forceinline__ int closest_seg(const double a[3], const double b[3], double out[3])
{
    double ab[3], ap[3];
    sub3(b, a, ab);
    neg3(a, ap);
    const double tn = dot3(ab, ap);
    if (tn <= 0.0) { cpy3(a, out); return 1; }
    const double den = dot3(ab, ab);
    if (tn >= den) { cpy3(b, out); return 2; }
    const double t = tn / den;
    out[0] = a[0] + t * ab[0];
    out[1] = a[1] + t * ab[1];
    out[2] = a[2] + t * ab[2];
    return 3;
}

// closest point of triangle (a, b, c) to the origin by Voronoi regions;
// feature mask (a=1, b=2, c=4); 0 = degenerate face
__device__ __forceinline__ int closest_tri(const double a[3], const double b[3], const double c[3],
                                           double out[3])
{
    double ab[3], ac[3], ap[3], bp[3], cp[3];
    sub3(b, a, ab);
    sub3(c, a, ac);
    neg3(a, ap);
    const double d1 = dot3(ab, ap);
    const double d2 = dot3(ac, ap);
    if (d1 <= 0.0 && d2 <= 0.0) { cpy3(a, out); return 1; }
    neg3(b, bp);
    const double d3 = dot3(ab, bp);
    const double d4 = dot3(ac, bp);
    if (d3 >= 0.0 && d4 <= d3) { cpy3(b, out); return 2; }
    const double vc = d1 * d4 - d3 * d2;
    if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
        const double t = d1 / (d1 - d3);
        out[0] = a[0] + t * ab[0]; out[1] = a[1] + t * ab[1]; out[2] = a[2] + t * ab[2];
        return 3;
    }
    neg3(c, cp);
    const double d5 = dot3(ab, cp);
    const double d6 = dot3(ac, cp);
    if (d6 >= 0.0 && d5 <= d6) { cpy3(c, out); return 4; }
    const double vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
        const double t = d2 / (d2 - d6);
        out[0] = a[0] + t * ac[0]; out[1] = a[1] + t * ac[1]; out[2] = a[2] + t * ac[2];
        return 5;
    }
    const double va = d3 * d6 - d5 * d4;
    const double e43 = d4 - d3, e56 = d5 - d6;
    if (va <= 0.0 && e43 >= 0.0 && e56 >= 0.0) {
        const double t = e43 / (e43 + e56);
        double bc[3];
        sub3(c, b, bc);
        out[0] = b[0] + t * bc[0]; out[1] = b[1] + t * bc[1]; out[2] = b[2] + t * bc[2];
        return 6;
    }
    const double sum = (va + vb) + vc;
    if (!(sum > 0.0)) return 0;
    const double den = 1.0 / sum;
    const double v = vb * den, w = vc * den;
    out[0] = (a[0] + ab[0] * v) + ac[0] * w;
    out[1] = (a[1] + ab[1] * v) + ac[1] * w;
    out[2] = (a[2] + ab[2] * v) + ac[2] * w;
    return 7;
}

// origin strictly on the other side of plane (p, q, r) from s
__device__ __forceinline__ bool origin_outside(const double p[3], const double q[3],
                                               const double r[3], const double s[3])
{
    double pq[3], pr[3], ps[3], po[3], n[3];
    sub3(q, p, pq);
    sub3(r, p, pr);
    cross3(pq, pr, n);
    neg3(p, po);
    sub3(s, p, ps);
    const double sp = dot3(po, n);
    const double sd = dot3(ps, n);
    return (sp > 0.0 && sd < 0.0) || (sp < 0.0 && sd > 0.0);
}

// reduce the simplex to the feature nearest the origin; true = overlap
__device__ __forceinline__ bool gjk_reduce(double sp[4][3], int& n, double v[3])
{
    int mask = 0;
    if (n == 2) {
        mask = closest_seg(sp[0], sp[1], v);
    } else if (n == 3) {
        mask = closest_tri(sp[0], sp[1], sp[2], v);
        if (mask == 0) return true;
    } else {
        bool found = false;
        double best = 0.0;
#pragma unroll 1
        for (int f = 0; f < 4; ++f) {
            // faces {0,1,2} opp 3, {0,1,3} opp 2, {0,2,3} opp 1, {1,2,3} opp 0
            const int i0 = (f == 3) ? 1 : 0;
            const int i1 = (f <= 1) ? 1 : 2;
            const int i2 = (f == 0) ? 2 : 3;
            const int i3 = 3 - f;
            if (!origin_outside(sp[i0], sp[i1], sp[i2], sp[i3])) continue;
            double pt[3];
            const int m = closest_tri(sp[i0], sp[i1], sp[i2], pt);
            if (m == 0) return true;
            const double dd = dot3(pt, pt);
            if (!found || dd < best) {
                found = true;
                best = dd;
                cpy3(pt, v);
                mask = ((m & 1) ? (1 << i0) : 0) | ((m & 2) ? (1 << i1) : 0) | ((m & 4) ? (1 << i2) : 0);
            }
        }
        if (!found) return true;
    }
    int m = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k < n && (mask & (1 << k))) {
            if (m != k) cpy3(sp[k], sp[m]);
            m += 1;
        }
    }
    n = m;
    return false;
}

// D(Delta, qA, qB) for convex polyhedra (closest-point GJK with boolean
// exits).  Returns true for overlap; *iters = support evaluations after the
// first (kGjkMaxIt + 1 when the cap is reached).
template <int NV>
__device__ __noinline__ bool overlap3d64(const Shape3& sh, const double D[3], const double qA[4],
                                         const double qB[4], int* iters)
{
    if (NV == 0 && sh.round) {                                          // spheres
        *iters = 0;
        return ((D[0] * D[0] + D[1] * D[1]) + D[2] * D[2]) <= sh.rc2;
    }
    const double qAc[4] = { qA[0], -qA[1], -qA[2], -qA[3] };
    double qr[4], l[3];
    qmul(qAc, qB, qr);
    qrot(qAc, D, l);
    double pb[NV ? NV : kMaxV3][3];
    const int nv = NV ? NV : sh.nv;
#pragma unroll
    for (int i = 0; i < nv; ++i) {
        double r[3];
        qrot(qr, sh.v[i], r);
        pb[i][0] = r[0] + l[0];
        pb[i][1] = r[1] + l[1];
        pb[i][2] = r[2] + l[2];
    }
    double d[3];
    neg3(l, d);
    if (d[0] == 0.0 && d[1] == 0.0 && d[2] == 0.0) d[0] = -1.0;
    double sp[4][3], v[3];
    int n = 1;
    support3<NV>(sh, pb, d, sp[0]);
    cpy3(sp[0], v);
#pragma unroll 1
    for (int it = 0; it < kGjkMaxIt; ++it) {
        *iters = it + 1;
        const double vv = dot3(v, v);
        if (vv == 0.0) return true;
        double nv3[3], w[3];
        neg3(v, nv3);
        support3<NV>(sh, pb, nv3, w);
        if (dot3(v, w) > 0.0) return false;
        cpy3(w, sp[n]);
        n += 1;
        if (gjk_reduce(sp, n, v)) return true;
    }
    *iters = kGjkMaxIt + 1;
    return true;
}

}  // namespace hpmc
