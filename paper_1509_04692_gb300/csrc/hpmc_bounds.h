// hpmc_bounds.h -- certified margins of the FP32 filter (host only).
//
// The FP32 form evaluates every decision of a trial move (in-cell test,
// circumsphere cull, separating-axis test) in FP32 on cell-relative
// coordinates, and only trusts an FP32 verdict when it is farther from the
// decision threshold than a bound E on |FP32 value - FP64 contract value|.
// Such a verdict provably equals the FP64 contract's verdict; anything closer
// is re-decided in FP64.  E comes from a forward error analysis: each
// quantity carries (m, e) = (bound on |exact value|, bound on |computed -
// exact|) and every operation propagates them with the standard model
// |fl(a op b) - (a op b)| <= u |a op b|, u = 2^-24 (FP32) or 2^-53 (FP64).
// A fused multiply-add rounds once, so the bound of a separate multiply and
// add also covers it.  Every margin is then doubled.
#pragma once
#include <algorithm>
#include <cmath>

namespace hpmc {

constexpr double kU32 = 0x1.0p-24;
constexpr double kU64 = 0x1.0p-53;

struct EV {
    double m, e;
};

inline EV ev_mul(EV a, EV b, double u)
{
    return { a.m * b.m, a.m * b.e + b.m * a.e + a.e * b.e + u * (a.m + a.e) * (b.m + b.e) };
}

inline EV ev_add(EV a, EV b, double u)
{
    return { a.m + b.m, a.e + b.e + u * (a.m + a.e + b.m + b.e) };
}

struct Margins {
    double e_rel;      // stored FP32 cell-relative coordinate vs exact
    double e_delta;    // FP32 translation vs FP64 translation
    double e_rho;      // FP32 trial relative coordinate vs the FP64 trial's
    double e_in;       // in-cell certification margin
    double e_dlt;      // |Delta32 - Delta64| per component
    double e_cull;     // circumsphere cull margin on |Delta|^2
    double e_ori;      // FP32 trial orientation vs the FP64 contract's, per component
    double e_sat;      // separating-axis gap margin (2D) / support margin (3D)
};

// Geometry-independent parts: w = largest cell width, L = largest box side,
// d = translation half-width, tau = tan(a / 2), dim = 2 or 3.
inline Margins base_margins(int dim, double w, double L, double d, double tau, double rc2)
{
    Margins g{};
    // rel64 = fl(fl(x - s [+ L]) - fl(i * w)): three FP64 roundings of
    // magnitude <= L; then the cast to FP32 of a value in [0, w].
    g.e_rel = 1.01 * kU32 * w + 4.0 * kU64 * L;
    // delta32 = fl32(fl32(d) * m24) with |m24 - (2 u53 - 1)| <= 2^-23
    g.e_delta = d * (kU32 + 2.0 * kU32 + kU32) + kU64 * d;
    // rel'32 = fl32(rel32 + delta32); the FP64 trial x' = fl(x + delta64)
    // (+-L) adds one FP64 rounding of magnitude <= L.
    g.e_rho = g.e_rel + g.e_delta + kU64 * L + kU32 * (w + d);
    // the FP64 cell index floor(fl(fl(y') * nc / L)) moves a wall by at most a
    // few FP64 ulps of L
    g.e_in = 2.0 * (g.e_rho + 8.0 * kU64 * L);
    // Delta32 = fl32(fl32(rel_B + o w32) - rel'32); Delta64 = fl(x_B - x') (+-L)
    const double e_P = g.e_rel + kU32 * w + 2.0 * kU32 * w;
    g.e_dlt = e_P + g.e_rho + 3.0 * kU32 * w + 2.0 * kU64 * L;
    // |Delta|^2 of a stencil neighbour of an in-cell trial: |Delta_a| < 2 w
    const double dm = 2.0 * w + g.e_dlt;
    const double QM = dim * dm * dm;
    const double e_q32 = (dim + 1) * kU32 * QM;
    const double e_q64 = (dim + 1) * kU64 * QM;
    const double e_diff = dim * g.e_dlt * (2.0 * dm + g.e_dlt);
    g.e_cull = 2.0 * (e_q32 + e_q64 + e_diff) + 4.0 * kU32 * rc2;
    // FP32 trial orientation: t32 = fl32(tau32 * m24), |t32 - t64| <= 4 u32 tau;
    // the rotation is 2-Lipschitz in t; the FP32 Cayley map and complex product
    // add ~15 u32; the FP64 contract's own rounding and renormalisation add
    // less than 1e-15.  (3D: quaternion product of 4 terms, same order.)
    const double e_t = 4.0 * kU32 * tau;
    g.e_ori = 2.0 * ((dim == 2 ? 16.0 : 24.0) * kU32 + 4.0 * e_t + 3e-15);
    return g;
}

// 2D separating-axis gap margin.  vm = max |vertex component|, nm = max
// |normal component|, am = max |alo|, |ahi|, R = circumradius.
inline double sat2_margin(const Margins& g, double R, double vm, double nm, double am)
{
    const double zm = 1.0 + 1e-6;
    const double dm = 2.0 * R * (1.0 + 1e-9) + g.e_dlt;
    auto gap_err = [&](double u, bool fp32) {
        const double eA = fp32 ? g.e_ori : 0.0;
        const double eB = fp32 ? kU32 * zm + 1e-15 : 0.0;
        const double eD = fp32 ? g.e_dlt : 0.0;
        const double ev_ = fp32 ? kU32 * vm : 0.0;
        const double en_ = fp32 ? kU32 * nm : 0.0;
        const double ea_ = fp32 ? kU32 * am : 0.0;
        EV cA{ zm, eA }, cB{ zm, eB }, D{ dm, eD }, v{ vm, ev_ }, n{ nm, en_ }, a{ am, ea_ };
        double worst = 0.0;
        for (int half = 0; half < 2; ++half) {
            const EV& c0 = half == 0 ? cA : cB;   // frame of the tested edge normals
            EV cr = ev_add(ev_mul(cA, cB, u), ev_mul(cA, cB, u), u);
            EV l = ev_add(ev_mul(c0, D, u), ev_mul(c0, D, u), u);
            EV p = ev_add(ev_add(ev_mul(cr, v, u), ev_mul(cr, v, u), u), l, u);
            EV dot = ev_add(ev_mul(n, p, u), ev_mul(n, p, u), u);
            EV gap = fp32 ? ev_add(dot, a, u) : dot;
            worst = std::max(worst, gap.e);
        }
        return worst;
    };
    const double e32 = gap_err(kU32, true);
    const double e64 = gap_err(kU64, false);
    return 2.0 * (e32 + e64);
}

// 3D: bound on |pb32 - pb| per component for B's vertices moved into A's
// frame (qr = conj(qA) qB, l = rot(conj(qA), Delta), pb = rot(qr, v) + l),
// where pb is the exact transform of the FP64 contract's inputs and pb32 the
// FP32 evaluation from the FP32 inputs.  vm = max |vertex component|.
inline double gjk3_vertex_margin(const Margins& g, double R, double vm)
{
    // Magnitudes use what the operations preserve (unit quaternions, norm
    // preserving rotations) instead of the generic model, which would
    // overestimate the rotated vectors a hundredfold.
    const double u = kU32 * 1.0001;
    const double ea = g.e_ori, eb = kU32 * 1.000001 + 1e-15;   // quaternion component errors
    // qr = conj(qA) qB: each component a signed sum of four products with
    // sum |a_i b_j| <= |a| |b| <= 1 (plus slack); sum |a_i| <= 2 for unit a
    const double e_qr = 2.0 * (ea + eb) + 2.0 * ea * eb + 4.0 * u * 1.000001;
    // rot(q, x) for |x|_2 <= X, component errors ex, quaternion errors eq:
    // t = 2 q_v x x (|t| <= 2X); o = (x + w t) + q_v x t (|o| <= 5X before the
    // cancellations of an exact rotation)
    auto rot_err = [&](double X, double ex, double eq) {
        const double e_cross1 = 2.0 * (ex + X * eq + ex * eq) + 3.0 * u * X;   // q_v x x, per component
        const double et = 2.0 * e_cross1;                                      // times 2 (exact)
        const double T = 2.0 * X * 1.000001;
        const double e_wt = et + T * eq + et * eq + u * T;                     // w t
        const double e_s1 = ex + e_wt + u * 3.0 * X;                           // x + w t
        const double e_cross2 = 2.0 * (et + T * eq + et * eq) + 3.0 * u * T;   // q_v x t
        return e_s1 + e_cross2 + u * 5.0 * X;
    };
    const double X_D = 2.0 * R * (1.0 + 1e-9) + 2.0 * g.e_dlt;
    const double e_l = rot_err(X_D, g.e_dlt, ea);
    const double X_v = std::sqrt(3.0) * vm;
    const double e_rv = rot_err(X_v, kU32 * vm, e_qr);
    const double e_pb = e_rv + e_l + u * (X_v + X_D) * 5.0;
    return 2.0 * e_pb;
}

}  // namespace hpmc
