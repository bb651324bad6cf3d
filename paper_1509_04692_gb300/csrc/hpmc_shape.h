// hpmc_shape.h -- shape constants of the overlap tests (host only).
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

#include "../../include/hpmc.h"
#include "hpmc_types.h"

namespace hpmc {

// Shape constants of the overlap tests from the local-frame vertices:
// circumradius R, cull threshold (2R)^2, polygon edge normals and A's own
// projection intervals (2D), FP32 copies.  Validates the vertex list
// (2D: convex, counter-clockwise).  Host only.
inline double shape_inradius(int dim, const double* v, uint32_t nv);

inline int build_shapes(int dim, const double* verts, uint32_t nv, Shape2& s2, Shape3& s3, double& Rc,
                        double& rc2)
{
    if (dim != 2 && dim != 3) return HPMC_ERR_INVALID_ARG;
    if (nv == 0) {
        // disks / spheres of radius verts[0]: the shape is its circumsphere
        if (!verts || !std::isfinite(verts[0]) || !(verts[0] > 0.0)) return HPMC_ERR_INVALID_ARG;
        Rc = verts[0];
        const double dcut = Rc + Rc;
        rc2 = dcut * dcut;
        s2 = Shape2{};
        s3 = Shape3{};
        s2.round = s3.round = 1;
        s2.rc2 = s3.rc2 = rc2;
        s2.frc2 = s3.frc2 = (float)rc2;
        return 0;
    }
    if (dim == 2 && (nv < 3 || nv > (uint32_t)kMaxV2)) return HPMC_ERR_INVALID_ARG;
    if (dim == 3 && (nv < 4 || nv > (uint32_t)kMaxV3)) return HPMC_ERR_INVALID_ARG;
    if (!verts) return HPMC_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < nv * (uint32_t)dim; ++i)
        if (!std::isfinite(verts[i])) return HPMC_ERR_INVALID_ARG;
    double r2 = 0.0;
    for (uint32_t i = 0; i < nv; ++i) {
        const double* v = verts + (size_t)i * dim;
        double q = v[0] * v[0] + v[1] * v[1];
        if (dim == 3) q = q + v[2] * v[2];
        if (q > r2) r2 = q;
    }
    Rc = std::sqrt(r2);
    if (!(Rc > 0.0)) return HPMC_ERR_INVALID_ARG;
    const double dcut = Rc + Rc;
    rc2 = dcut * dcut;
    if (dim == 2) {
        // convex and counter-clockwise: strictly left turns everywhere
        for (uint32_t i = 0; i < nv; ++i) {
            const double* p0 = verts + 2 * i;
            const double* p1 = verts + 2 * ((i + 1) % nv);
            const double* p2 = verts + 2 * ((i + 2) % nv);
            const double cr = (p1[0] - p0[0]) * (p2[1] - p1[1]) - (p1[1] - p0[1]) * (p2[0] - p1[0]);
            if (!(cr > 0.0)) return HPMC_ERR_INVALID_ARG;
        }
        Shape2& s = s2;
        s = Shape2{};
        s.nv = (int)nv;
        for (uint32_t k = 0; k < nv; ++k) {
            s.vx[k] = verts[2 * k];
            s.vy[k] = verts[2 * k + 1];
        }
        for (uint32_t k = 0; k < nv; ++k) {
            const uint32_t k1 = (k + 1) % nv;
            s.nx[k] = s.vy[k1] - s.vy[k];
            s.ny[k] = s.vx[k] - s.vx[k1];
            double lo = 0.0, hi = 0.0;
            for (uint32_t i = 0; i < nv; ++i) {
                const double t = s.nx[k] * s.vx[i] + s.ny[k] * s.vy[i];
                if (i == 0 || t < lo) lo = t;
                if (i == 0 || t > hi) hi = t;
            }
            s.alo[k] = lo;
            s.ahi[k] = hi;
        }
        for (uint32_t k = 0; k < nv; ++k) {
            s.fvx[k] = (float)s.vx[k]; s.fvy[k] = (float)s.vy[k];
            s.fnx[k] = (float)s.nx[k]; s.fny[k] = (float)s.ny[k];
            s.falo[k] = (float)s.alo[k]; s.fahi[k] = (float)s.ahi[k];
        }
        s.rc2 = rc2;
        s.frc2 = (float)rc2;
    } else {
        Shape3& s = s3;
        s = Shape3{};
        s.nv = (int)nv;
        for (uint32_t k = 0; k < nv; ++k)
            for (int a = 0; a < 3; ++a) {
                s.v[k][a] = verts[3 * k + a];
                s.fv[k][a] = (float)verts[3 * k + a];
            }
        s.rc2 = rc2;
        s.frc2 = (float)rc2;
        s.mpr = shape_inradius(3, verts, nv) > 1e-3 * Rc ? 1 : 0;
        // central symmetry (every vertex's negation is a vertex too): the FP32
        // copies the filter scans are reordered into pairs k, k + nv / 2; the
        // filter's certificates do not depend on the order, and the FP64
        // contract keeps the given one
        if (nv >= 2 && nv % 2 == 0) {
            bool ok = true;
            uint32_t h = 0;
            int used[kMaxV3] = {};
            int rep[kMaxV3 / 2], par[kMaxV3 / 2];
            for (uint32_t i = 0; i < nv && ok; ++i) {
                if (used[i]) continue;
                int j = -1;
                for (uint32_t k = i + 1; k < nv; ++k)
                    if (!used[k] && s.v[k][0] == -s.v[i][0] && s.v[k][1] == -s.v[i][1] && s.v[k][2] == -s.v[i][2]) {
                        j = (int)k;
                        break;
                    }
                if (j < 0) ok = false;
                else {
                    used[i] = used[j] = 1;
                    rep[h] = (int)i;
                    par[h] = j;
                    h += 1;
                }
            }
            if (ok && 2 * h == nv) {
                s.sym = 1;
                for (uint32_t k = 0; k < h; ++k)
                    for (int a = 0; a < 3; ++a) {
                        s.fv[k][a] = (float)s.v[rep[k]][a];
                        s.fv[k + h][a] = (float)s.v[par[k]][a];
                    }
            }
        }
        // a box centred on the origin and aligned with the local axes: every
        // vertex is (+-h0, +-h1, +-h2) and all 8 sign patterns occur
        if (nv == 8) {
            double h[3] = { 0.0, 0.0, 0.0 };
            for (uint32_t k = 0; k < 8; ++k)
                for (int a = 0; a < 3; ++a) h[a] = std::fmax(h[a], std::fabs(s.v[k][a]));
            unsigned seen = 0;
            bool ok = h[0] > 0.0 && h[1] > 0.0 && h[2] > 0.0;
            for (uint32_t k = 0; k < 8 && ok; ++k) {
                unsigned pat = 0;
                for (int a = 0; a < 3; ++a) {
                    if (std::fabs(s.v[k][a]) != h[a]) ok = false;
                    if (s.v[k][a] > 0.0) pat |= 1u << a;
                }
                seen |= 1u << pat;
            }
            if (ok && seen == 0xffu) {
                s.box = 1;
                for (int a = 0; a < 3; ++a) s.bh[a] = (float)h[a];
            }
        }
    }
    return 0;
}

// Inradius about the local origin: the distance from the origin to the
// nearest facet plane (2D: edge line), or 0 when the origin is not strictly
// inside.  A ball of this radius lies inside the shape, so two shapes whose
// centres are closer than twice it overlap whatever their orientations.
// 3D facets are found by brute force over vertex triples (nv <= 32).
inline double shape_inradius(int dim, const double* v, uint32_t nv)
{
    if (nv == 0) return v[0];                 // disk / sphere
    double best = INFINITY;
    if (dim == 2) {
        for (uint32_t k = 0; k < nv; ++k) {
            const double* p0 = v + 2 * k;
            const double* p1 = v + 2 * ((k + 1) % nv);
            const double nx = p1[1] - p0[1], ny = p0[0] - p1[0];      // outward (CCW)
            const double nn = std::sqrt(nx * nx + ny * ny);
            best = std::fmin(best, (nx * p0[0] + ny * p0[1]) / nn);
        }
    } else {
        double scale = 0.0;
        for (uint32_t i = 0; i < 3 * nv; ++i) scale = std::fmax(scale, std::fabs(v[i]));
        for (uint32_t i = 0; i < nv; ++i)
            for (uint32_t j = i + 1; j < nv; ++j)
                for (uint32_t k = j + 1; k < nv; ++k) {
                    const double* a = v + 3 * i;
                    const double* b = v + 3 * j;
                    const double* c = v + 3 * k;
                    const double u[3] = { b[0] - a[0], b[1] - a[1], b[2] - a[2] };
                    const double w[3] = { c[0] - a[0], c[1] - a[1], c[2] - a[2] };
                    double n[3] = { u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0] };
                    const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
                    if (!(nn > 1e-9 * scale * scale)) continue;
                    for (double& x : n) x /= nn;
                    const double d0 = n[0] * a[0] + n[1] * a[1] + n[2] * a[2];
                    int above = 0, below = 0;
                    for (uint32_t m = 0; m < nv; ++m) {
                        const double t = n[0] * v[3 * m] + n[1] * v[3 * m + 1] + n[2] * v[3 * m + 2] - d0;
                        if (t > 1e-9 * scale) above += 1;
                        if (t < -1e-9 * scale) below += 1;
                    }
                    if (above && below) continue;               // not a supporting plane
                    best = std::fmin(best, std::fabs(d0) * ((above ? -d0 : d0) > 0.0 ? 1.0 : -1.0));
                }
    }
    return best > 0.0 && std::isfinite(best) ? best : 0.0;
}

}  // namespace hpmc
