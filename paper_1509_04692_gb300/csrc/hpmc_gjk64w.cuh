// hpmc_gjk64w.cuh -- the FP64 GJK of the contract (overlap3d64, Sec. 2.3 /
// Eq. 2) evaluated by a whole warp.
//
// The FP32-filtered 3D kernels re-decide the rare pairs their certified GJK
// leaves uncertain with the FP64 test.  On one lane that test is a chain of
// about a thousand FP64 instructions, and on this GPU each FP64 warp
// instruction occupies the sub-partition's FP64 pipe for the same time
// however few lanes are active, so one re-check held its warp for tens of
// microseconds.  Here the 32 lanes of the warp share the independent parts
// of the same computation: the four components of the relative rotation, the
// three of the offset, one vertex of B per lane placed in A's frame, the
// support's dot products one vertex per lane with an exact argmax/argmin
// reduction, and the four faces of a tetrahedral simplex one per lane.  Every
// FP64 value is produced by the operations, in the order, that overlap3d64
// uses, so the verdict is identical; the scalar steps (the simplex of up to
// four points, the GJK loop) are computed redundantly by all lanes.
//
// Call convergently from all 32 lanes of a warp with the same arguments; the
// verdict is returned on every lane.
#pragma once
#include "hpmc_device.cuh"

namespace hpmc {

// Integer key with the order of a finite double (-0 keyed as +0, since the
// FP64 comparisons treat them as equal).
__device__ __forceinline__ long long dkey(double x)
{
    long long b = __double_as_longlong(x);
    if (b == (long long)0x8000000000000000ull) b = 0;
    return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}

__device__ __forceinline__ double sel3(int c, double a0, double a1, double a2)
{
    return c == 0 ? a0 : (c == 1 ? a1 : a2);
}

__device__ __forceinline__ double sel4(int c, double a0, double a1, double a2, double a3)
{
    return c == 0 ? a0 : (c == 1 ? a1 : (c == 2 ? a2 : a3));
}

__device__ __forceinline__ void shfl3(const double a[3], int src, double o[3])
{
    o[0] = __shfl_sync(0xffffffffu, a[0], src);
    o[1] = __shfl_sync(0xffffffffu, a[1], src);
    o[2] = __shfl_sync(0xffffffffu, a[2], src);
}

// Reduction step keeping the larger key, the smaller index on equal keys
// (the first index of the maximum, as a sequential strict > scan keeps).
__device__ __forceinline__ void argmax_step(long long& k, int& i, int o)
{
    const long long k2 = __shfl_xor_sync(0xffffffffu, k, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
    if (k2 > k || (k2 == k && i2 < i)) { k = k2; i = i2; }
}

// Support of B - A in direction d (support3's result).  half: lanes 0..15
// hold pb_i, lanes 16..31 hold A's vertex v_i (nv <= 16); otherwise every
// lane i < nv holds both.
template <int NV>
__device__ __forceinline__ void support_w(const Shape3& sh, int nv, bool half, int lane, const double pb[3],
                                          const double va[3], const double d[3], double out[3])
{
    int ib, ia;
    if (half) {
        const int vi = lane & 15;
        const bool lo = lane < 16;
        const double* P = lo ? pb : va;
        const double t = dot3(P, d);
        long long k = vi < nv ? (lo ? dkey(t) : ~dkey(t)) : (long long)0x8000000000000000ull;
        int i = vi < nv ? vi : 64;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) argmax_step(k, i, o);
        ib = __shfl_sync(0xffffffffu, i, 0);
        ia = __shfl_sync(0xffffffffu, i, 16);
    } else {
        const double t = dot3(pb, d);
        const double u = dot3(va, d);
        long long kb = lane < nv ? dkey(t) : (long long)0x8000000000000000ull;
        long long ka = lane < nv ? ~dkey(u) : (long long)0x8000000000000000ull;
        int jb = lane < nv ? lane : 64, ja = jb;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            argmax_step(kb, jb, o);
            argmax_step(ka, ja, o);
        }
        ib = jb;
        ia = ja;
    }
    double p[3];
    shfl3(pb, ib, p);
    out[0] = p[0] - sh.v[ia][0];
    out[1] = p[1] - sh.v[ia][1];
    out[2] = p[2] - sh.v[ia][2];
}

// gjk_reduce with the tetrahedron's faces evaluated one per lane (face
// f = lane & 3); the smaller simplices are reduced by every lane alike.
__device__ __forceinline__ bool gjk_reduce_w(double sp[4][3], int& n, double v[3], int lane)
{
    int mask = 0;
    if (n == 2) {
        mask = closest_seg(sp[0], sp[1], v);
    } else if (n == 3) {
        mask = closest_tri(sp[0], sp[1], sp[2], v);
        if (mask == 0) return true;
    } else {
        // faces {0,1,2} opp 3, {0,1,3} opp 2, {0,2,3} opp 1, {1,2,3} opp 0
        const int f = lane & 3;
        double P0[3], P1[3], P2[3], P3[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            P0[a] = f == 3 ? sp[1][a] : sp[0][a];
            P1[a] = f <= 1 ? sp[1][a] : sp[2][a];
            P2[a] = f == 0 ? sp[2][a] : sp[3][a];
            P3[a] = sel4(f, sp[3][a], sp[2][a], sp[1][a], sp[0][a]);
        }
        const bool out = origin_outside(P0, P1, P2, P3);
        int m = -1;
        double pt[3] = { 0.0, 0.0, 0.0 };
        long long key = 0x7fffffffffffffffll;
        if (out) {
            m = closest_tri(P0, P1, P2, pt);
            if (m != 0) key = dkey(dot3(pt, pt));
        }
        const unsigned bout = __ballot_sync(0xffffffffu, out) & 0xfu;
        const unsigned bdeg = __ballot_sync(0xffffffffu, out && m == 0) & 0xfu;
        if (bdeg) return true;                        // the scan stops at a degenerate face
        if (!bout) return true;
        // first face of the smallest distance among those the origin is outside
        long long k = ~key;
        int fi = out ? f : 64;
        argmax_step(k, fi, 2);
        argmax_step(k, fi, 1);
        const int fb = __shfl_sync(0xffffffffu, fi, 0);
        const int mb = __shfl_sync(0xffffffffu, m, fb);
        shfl3(pt, fb, v);
        const int j0 = (fb == 3) ? 1 : 0;
        const int j1 = (fb <= 1) ? 1 : 2;
        const int j2 = (fb == 0) ? 2 : 3;
        mask = ((mb & 1) ? (1 << j0) : 0) | ((mb & 2) ? (1 << j1) : 0) | ((mb & 4) ? (1 << j2) : 0);
    }
    // keep the points of the nearest feature, in order
    double nsp[4][3];
    int m = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool keep = k < n && (mask & (1 << k));
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (keep && m == j) {
#pragma unroll
                for (int a = 0; a < 3; ++a) nsp[j][a] = sp[k][a];
            }
        }
        m += keep ? 1 : 0;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (j < m)
#pragma unroll
            for (int a = 0; a < 3; ++a) sp[j][a] = nsp[j][a];
    n = m;
    return false;
}

// overlap3d64 by a warp: same verdict and the same *iters.
template <int NV>
__device__ __noinline__ bool overlap3d64_warp(const Shape3& sh, const double D[3], const double qA[4],
                                              const double qB[4], int* iters)
{
    const int lane = threadIdx.x & 31;
    if (NV == 0 && sh.round) {                                          // spheres
        *iters = 0;
        return ((D[0] * D[0] + D[1] * D[1]) + D[2] * D[2]) <= sh.rc2;
    }
    const int nv = NV ? NV : sh.nv;
    const double qAc[4] = { qA[0], -qA[1], -qA[2], -qA[3] };
    // qr = qAc (x) qB: component c of the Hamilton product on lane c (mod 4),
    // a0 b_c first, then a_j b_(c^j) for j = 1, 2, 3 with qmul's signs
    double qr[4];
    {
        const int c = lane & 3;
        const int neg = (0x2147 >> (4 * c)) & 7;
        const double b_c = sel4(c, qB[0], qB[1], qB[2], qB[3]);
        const double b_c1 = sel4(c ^ 1, qB[0], qB[1], qB[2], qB[3]);
        const double b_c2 = sel4(c ^ 2, qB[0], qB[1], qB[2], qB[3]);
        const double b_c3 = sel4(c ^ 3, qB[0], qB[1], qB[2], qB[3]);
        double acc = qAc[0] * b_c;
        acc = acc + ((neg & 1) ? -qAc[1] : qAc[1]) * b_c1;
        acc = acc + ((neg & 2) ? -qAc[2] : qAc[2]) * b_c2;
        acc = acc + ((neg & 4) ? -qAc[3] : qAc[3]) * b_c3;
#pragma unroll
        for (int k = 0; k < 4; ++k) qr[k] = __shfl_sync(0xffffffffu, acc, k);
    }
    // l = rot(qAc, D) (qrot's operations), component c = lane mod 3 per lane
    double l[3];
    {
        const int c = lane % 3;
        const double qa = sel3(c, qAc[2], qAc[3], qAc[1]);   // q[1 + (c+1)%3]
        const double qb = sel3(c, qAc[3], qAc[1], qAc[2]);   // q[1 + (c+2)%3]
        const double t = 2.0 * (qa * sel3(c, D[2], D[0], D[1]) - qb * sel3(c, D[1], D[2], D[0]));
        const double t0 = __shfl_sync(0xffffffffu, t, 0);
        const double t1 = __shfl_sync(0xffffffffu, t, 1);
        const double t2 = __shfl_sync(0xffffffffu, t, 2);
        const double o = (sel3(c, D[0], D[1], D[2]) + qAc[0] * sel3(c, t0, t1, t2)) +
                         (qa * sel3(c, t2, t0, t1) - qb * sel3(c, t1, t2, t0));
        l[0] = __shfl_sync(0xffffffffu, o, 0);
        l[1] = __shfl_sync(0xffffffffu, o, 1);
        l[2] = __shfl_sync(0xffffffffu, o, 2);
    }
    // B's vertex vi in A's frame (pb_vi = rot(qr, v_vi) + l) and A's vertex vi
    const bool half = nv <= 16;
    const int vi = half ? (lane & 15) : lane;
    double pb[3], va[3];
    {
        const int vc = vi < nv ? vi : 0;
        va[0] = sh.v[vc][0]; va[1] = sh.v[vc][1]; va[2] = sh.v[vc][2];
        double r[3];
        qrot(qr, va, r);
        pb[0] = r[0] + l[0];
        pb[1] = r[1] + l[1];
        pb[2] = r[2] + l[2];
    }
    double d[3];
    neg3(l, d);
    if (d[0] == 0.0 && d[1] == 0.0 && d[2] == 0.0) d[0] = -1.0;
    double sp[4][3], v[3];
    int n = 1;
    support_w<NV>(sh, nv, half, lane, pb, va, d, sp[0]);
    cpy3(sp[0], v);
#pragma unroll 1
    for (int it = 0; it < kGjkMaxIt; ++it) {
        *iters = it + 1;
        const double vv = dot3(v, v);
        if (vv == 0.0) return true;
        double nv3[3], w[3];
        neg3(v, nv3);
        support_w<NV>(sh, nv, half, lane, pb, va, nv3, w);
        if (dot3(v, w) > 0.0) return false;
        cpy3(w, sp[n]);
        n += 1;
        if (gjk_reduce_w(sp, n, v, lane)) return true;
    }
    *iters = kGjkMaxIt + 1;
    return true;
}

// Boxes (Shape3::box): an FP64 separating-axis certificate tried before the
// warp GJK on the pairs the FP32 test leaves uncertain.  The 15 axes of two
// boxes decide their overlap exactly, and FP64 rounding moves the 15 values
// by ~1e-14 of the size, so almost every pair of that FP32 band is decided
// here: s_max > sep (the exact boxes apart by more than 4e-6 2R along an
// axis, where the FP64 GJK answers "separated") or s_max < -ov (every
// candidate axis overlapping deeper than tau, where it answers overlap).
// Only pairs within that band of contact reach the GJK, whose verdict there
// no geometric test reproduces.
//
// Lanes share the work: lane c computes qr component c (c < 4), l component
// c (c < 3) and entry c of B's axes M[r][j] = (R(qr) e_j)_r (c < 9); lane a
// < 15 then takes axis a (A's faces e_k, B's faces u_j, the crosses e_i x
// u_j) as a vector n and evaluates s = |l.n| - sum_k h_k |n_k| - sum_j h_j
// |n.u_j| (B's extent along n from its edge vectors u_j, no orthonormality
// assumed); a max-reduction gives s_max on every lane.  Returns 0
// (separated), 1 (overlap) or 2 (left to the GJK).  Call convergently from
// all 32 lanes with the same arguments.
static __device__ __noinline__ int box64_sat_warp(const Shape3& sh, const double D[3], const double qA[4],
                                                  const double qB[4], double sep, double ov)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const double qAc[4] = { qA[0], -qA[1], -qA[2], -qA[3] };
    double qr[4];
    {
        const int c = lane & 3;
        const int neg = (0x2147 >> (4 * c)) & 7;
        double acc = qAc[0] * sel4(c, qB[0], qB[1], qB[2], qB[3]);
        acc = acc + ((neg & 1) ? -qAc[1] : qAc[1]) * sel4(c ^ 1, qB[0], qB[1], qB[2], qB[3]);
        acc = acc + ((neg & 2) ? -qAc[2] : qAc[2]) * sel4(c ^ 2, qB[0], qB[1], qB[2], qB[3]);
        acc = acc + ((neg & 4) ? -qAc[3] : qAc[3]) * sel4(c ^ 3, qB[0], qB[1], qB[2], qB[3]);
#pragma unroll
        for (int k = 0; k < 4; ++k) qr[k] = __shfl_sync(FULL, acc, k);
    }
    double l[3];
    {
        const int c = lane % 3;
        const double qa = sel3(c, qAc[2], qAc[3], qAc[1]);
        const double qb = sel3(c, qAc[3], qAc[1], qAc[2]);
        const double t = 2.0 * (qa * sel3(c, D[2], D[0], D[1]) - qb * sel3(c, D[1], D[2], D[0]));
        const double t0 = __shfl_sync(FULL, t, 0);
        const double t1 = __shfl_sync(FULL, t, 1);
        const double t2 = __shfl_sync(FULL, t, 2);
        const double o = (sel3(c, D[0], D[1], D[2]) + qAc[0] * sel3(c, t0, t1, t2)) +
                         (qa * sel3(c, t2, t0, t1) - qb * sel3(c, t1, t2, t0));
        l[0] = __shfl_sync(FULL, o, 0);
        l[1] = __shfl_sync(FULL, o, 1);
        l[2] = __shfl_sync(FULL, o, 2);
    }
    double M[3][3];
    {
        // entry (r, j) on lane 3 r + j: 1 - 2 (v_i1^2 + v_i2^2) on the
        // diagonal, 2 (v_r v_j +- w v_k) off it (+ when r - j = 1 mod 3)
        const int e = lane % 9, r = e / 3, j = e - 3 * r;
        const double x = qr[1], y = qr[2], z = qr[3];
        double m;
        if (r == j) {
            const double a = sel3((r + 1) % 3, x, y, z), b = sel3((r + 2) % 3, x, y, z);
            m = 1.0 - 2.0 * (a * a + b * b);
        } else {
            const double vr = sel3(r, x, y, z), vj = sel3(j, x, y, z);
            const double wk = qr[0] * sel3(3 - r - j, x, y, z);
            m = ((r - j + 3) % 3 == 1) ? 2.0 * (vr * vj + wk) : 2.0 * (vr * vj - wk);
        }
#pragma unroll
        for (int t = 0; t < 9; ++t) M[t / 3][t % 3] = __shfl_sync(FULL, m, t);
    }
    const double h[3] = { fabs(sh.v[0][0]), fabs(sh.v[0][1]), fabs(sh.v[0][2]) };
    double s = -1.0e300;
    if (lane < 15) {
        double n[3];
        if (lane < 3) {
            n[0] = lane == 0 ? 1.0 : 0.0;
            n[1] = lane == 1 ? 1.0 : 0.0;
            n[2] = lane == 2 ? 1.0 : 0.0;
        } else if (lane < 6) {
            const int j = lane - 3;
            n[0] = sel3(j, M[0][0], M[0][1], M[0][2]);
            n[1] = sel3(j, M[1][0], M[1][1], M[1][2]);
            n[2] = sel3(j, M[2][0], M[2][1], M[2][2]);
        } else {
            // e_i x u_j = (0, -u_z, u_y), (u_z, 0, -u_x), (-u_y, u_x, 0)
            const int i = (lane - 6) / 3, j = (lane - 6) % 3;
            const double u0 = sel3(j, M[0][0], M[0][1], M[0][2]);
            const double u1 = sel3(j, M[1][0], M[1][1], M[1][2]);
            const double u2 = sel3(j, M[2][0], M[2][1], M[2][2]);
            n[0] = sel3(i, 0.0, u2, -u1);
            n[1] = sel3(i, -u2, 0.0, u0);
            n[2] = sel3(i, u1, -u0, 0.0);
        }
        const double c = (l[0] * n[0] + l[1] * n[1]) + l[2] * n[2];
        const double ea = (h[0] * fabs(n[0]) + h[1] * fabs(n[1])) + h[2] * fabs(n[2]);
        double eb = 0.0;
#pragma unroll
        for (int j = 0; j < 3; ++j) eb = eb + h[j] * fabs((n[0] * M[0][j] + n[1] * M[1][j]) + n[2] * M[2][j]);
        s = (fabs(c) - ea) - eb;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(FULL, s, o));
    if (s > sep) return 0;
    if (-s > ov) return 1;
    return 2;
}

}  // namespace hpmc
