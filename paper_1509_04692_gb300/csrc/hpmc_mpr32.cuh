// hpmc_mpr32.cuh -- FP32 portal refinement with certificates, for convex
// polyhedra whose local origin is interior (Shape3::mpr).
//
// Sec. 2.3 names XenoCollide, a Minkowski portal refinement, as the GPU's
// overlap test for general convex shapes.  Here it is the FP32 filter's
// search step, written from that scheme: in B - A (A's frame) start from
// the interior point v0 = l (B's centre minus A's), find a portal triangle
// of support points that the ray from v0 towards the origin crosses, then
// replace one portal vertex at a time by the support point along the
// portal's outward normal n until
//   * the origin lies on v0's side of the portal: it is inside the
//     tetrahedron (v0, v1, v2, v3), a "hit";
//   * a support point along n stays below the origin: -n separates, a "miss";
//   * the portal stops moving (the boundary runs next to the origin) or the
//     iteration cap is reached.
// Every iteration is one support query along a direction plus a few cross
// products and sign tests, with the query at a single place in the loop, so
// the lanes of a warp (one pair each) run their iterations together instead
// of following the case analysis of GJK's simplex one lane at a time.
//
// The verdicts are certified about the exact shapes as in hpmc_gjk32.cuh: a
// miss by cert_separated along -n, a hit by the tetrahedron test with v0's
// exact value within e_pb of l (the exact centres are interior points of
// the exact shapes, so the exact tetrahedron lies in the exact B - A).  A
// verdict that fails its certificate, and every unfinished search, goes to
// the certified GJK; what that leaves uncertain goes to the FP64 contract.
#pragma once
#include "hpmc_gjk32.cuh"

namespace hpmc {

constexpr int kMprMaxIt = 32;

template <int NV>
__device__ __forceinline__ int mpr32_cert(const Shape3& sh, float dx, float dy, float dz, float4 qA, float4 qB,
                                          float e_pb, float e_va, float tau)
{
    const int nv = NV ? NV : sh.nv;
    G32 l;
    G32 pb[NV ? NV : kMaxV3];
    gjk32_setup<NV>(sh, dx, dy, dz, qA, qB, l, pb);
    // (the first iteration's query along -l tests the centre line: a miss
    // there is certified along l like GJK's first step)
    const G32 v0 = l;
    // a move of the portal below this is no progress (lengths scale with 2R)
    const float tol = 1e-6f * sqrtf(sh.frc2);
    SPt s[3];
    s[0] = s[1] = s[2] = SPt{ G32{ 0.f, 0.f, 0.f }, 0, 0 };
    G32 n = g_neg(v0);
    int phase = 0;        // 0: first portal point, 1: second, 2: portal discovery, 3: refinement
    int res = 0;          // 1 hit, 2 miss (-n separates), 3 no progress
    if (v0.x == 0.f && v0.y == 0.f && v0.z == 0.f) res = 3;
#pragma unroll 1
    for (int it = 0; it < kMprMaxIt && res == 0; ++it) {
        if (phase == 3) {
            n = g_cross(g_sub(s[1].p, s[0].p), g_sub(s[2].p, s[0].p));
            if (g_dot(n, s[0].p) >= 0.f) {
                res = 1;
                break;
            }
        }
        const SPt p = g_support_q<NV>(nv, pb, sh, l, n);
        if (g_dot(p.p, n) <= 0.f) {
            res = 2;
            break;
        }
        if (phase == 0) {
            s[0] = p;
            n = g_cross(p.p, v0);
            if (n.x == 0.f && n.y == 0.f && n.z == 0.f) res = 3;     // origin on the line v0 v1
            phase = 1;
        } else if (phase == 1) {
            s[1] = p;
            n = g_cross(g_sub(s[0].p, v0), g_sub(p.p, v0));
            if (g_dot(n, v0) > 0.f) {
                const SPt t = s[0];
                s[0] = s[1];
                s[1] = t;
                n = g_neg(n);
            }
            phase = 2;
        } else if (phase == 2) {
            if (g_dot(g_cross(s[0].p, p.p), v0) < 0.f) {
                s[1] = p;
                n = g_cross(g_sub(s[0].p, v0), g_sub(p.p, v0));
            } else if (g_dot(g_cross(p.p, s[1].p), v0) < 0.f) {
                s[0] = p;
                n = g_cross(g_sub(p.p, v0), g_sub(s[1].p, v0));
            } else {
                s[2] = p;
                phase = 3;
            }
        } else {
            const float n1 = (fabsf(n.x) + fabsf(n.y)) + fabsf(n.z);
            if (g_dot(g_sub(p.p, s[2].p), n) <= tol * n1) {
                res = 3;
                break;
            }
            // the new portal: the one of the three around p that the ray
            // from v0 towards the origin crosses
            const G32 x = g_cross(p.p, v0);
            if (g_dot(s[0].p, x) > 0.f) {
                if (g_dot(s[1].p, x) > 0.f) s[0] = p;
                else s[2] = p;
            } else {
                if (g_dot(s[2].p, x) > 0.f) s[1] = p;
                else s[0] = p;
            }
        }
    }
    if (res == 2) {
        if (cert_separated<NV>(nv, pb, sh, g_neg(n), e_pb, e_va, tau)) return GJK32_SEPARATED;
    } else if (res == 1) {
        Fe3 W[4];
        W[0] = Fe3{ { v0.x, e_pb }, { v0.y, e_pb }, { v0.z, e_pb } };
#pragma unroll
        for (int k = 0; k < 3; ++k) W[k + 1] = fe3_vertex_diff(pb, sh, s[k], e_pb, e_va);
        if (cert_inside_pts(W, tau)) return GJK32_OVERLAP;
    }
    return gjk32_run<NV>(nv, pb, sh, l, e_pb, e_va, tau);
}

}  // namespace hpmc
