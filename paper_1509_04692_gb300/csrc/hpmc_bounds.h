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

// rot(q, x) as the 3D kernels evaluate it in FP32 (t = 2 q_v x x, o = (x +
// w t) + q_v x t), |x|_2 <= X, component errors ex, quaternion component
// errors eq, per-rounding unit u: bound on the output components' error.
inline double rot3_err(double X, double ex, double eq, double u)
{
    const double e_cross1 = 2.0 * (ex + X * eq + ex * eq) + 3.0 * u * X;   // q_v x x, per component
    const double et = 2.0 * e_cross1;                                      // times 2 (exact)
    const double T = 2.0 * X * 1.000001;
    const double e_wt = et + T * eq + et * eq + u * T;                     // w t
    const double e_s1 = ex + e_wt + u * 3.0 * X;                           // x + w t
    const double e_cross2 = 2.0 * (et + T * eq + et * eq) + 3.0 * u * T;   // q_v x t
    return e_s1 + e_cross2 + u * 5.0 * X;
}

// 3D boxes (half extents h): margins of the certified separating-axis test
// (box32_sat).  The FP32 test sees l = rot(conj(qA), Delta) with per-component
// error e_l and B's axes M (the closed-form rotation matrix of qr = conj(qA)
// qB) with per-entry error e_u.  Along one of its axes n (the FP32 vector) it
// computes s = |l.n| - sum_k h_k |n_k| - extent_B, extent_B from M's
// orthonormal identities.  E_sep bounds |s - s*(n)|, s*(n) the same quantity
// for the exact boxes along the same n; E_ov adds |s*(n) - s*(n*)| for the
// exact candidate axis n* the FP32 n stands for (|n - n*|_1 <= 3 e_u, times
// the Lipschitz constant of s* in the 1-norm).  Returned, doubled, with:
//   sep = 2 E_sep + 4e-6 2R |n|_2: s > sep leaves the exact boxes more than
//         4e-6 2R apart along n, far outside the zone near contact where the
//         FP64 GJK may answer overlap for separated shapes;
//   ov  = 2 E_ov + tau |n|_2: -s > ov on all 15 axes gives every exact
//         candidate axis an overlap deeper than tau, so the exact boxes
//         intersect at depth > tau, where the FP64 GJK answers overlap.
struct BoxMargins {
    double sep, ov;
};

inline BoxMargins box_sat_margins(const Margins& g, double R, const double h[3], double tau)
{
    const double u = kU32 * 1.0001;
    const double r3 = std::sqrt(3.0);
    const double ea = g.e_ori, eb = kU32 * 1.000001 + 1e-15;   // quaternion component errors
    const double e_qr = 2.0 * (ea + eb) + 2.0 * ea * eb + 4.0 * u * 1.000001;
    const double X_D = 2.0 * R * (1.0 + 1e-9) + 2.0 * g.e_dlt;          // |Delta| of a culled pair
    const double e_l = rot3_err(X_D, g.e_dlt, ea, u);
    // entries 2(ab +- cd) and 1 - 2(a^2 + b^2) of components within e_qr
    const double e_u = 8.0 * e_qr * (1.0 + e_qr) + 8.0 * u;
    const double e64 = 1e-12;       // the FP64 quaternions' departure from a rotation (~1e-15)
    const double N1 = r3 * (1.0 + 2.0 * e_u);                           // |n|_1 of any axis
    const double N2 = 1.0 + 2.0 * e_u;                                  // |n|_2 of any axis
    const double Lm = (X_D + r3 * e_l) * N2;                            // |l.n|
    const double hsum = h[0] + h[1] + h[2];
    const double hmax = std::max(h[0], std::max(h[1], h[2]));
    const double e_c = N1 * e_l + 3.0 * u * Lm;                         // l.n
    const double e_A = 4.01 * u * hmax * N1;                            // sum h_k |n_k|, h rounded to FP32
    const double e_B = hsum * ((1.0 + r3) * e_u * 1.001 + e64 + 5.0 * u * (1.0 + e_u));
    const double e_s = 2.0 * u * (Lm + 2.0 * hsum * N2) * 1.001;        // the two subtractions
    const double E_sep = e_c + e_A + e_B + e_s;
    const double E_ov = E_sep + (X_D + hmax + hsum) * 3.0 * (e_u + e64) * 1.001;
    return { 2.0 * E_sep + 4e-6 * 2.0 * R * N2, 2.0 * E_ov + tau * N2 };
}

// The same test in FP64 (box64_sat_warp) on the FP64 contract's inputs
// themselves: only its own roundings (unit u64) separate its values from the
// exact ones, plus the departure of the FP64 quaternions from unit length
// (~1e-15, taken as 1e-12) in the face normals of B.  Returned like
// box_sat_margins: sep = 2 E + 4e-6 2R |n|_2, ov = 2 (E + Lipschitz term) +
// tau |n|_2; both are the floors to within ~1e-11 of the size.
inline BoxMargins box_sat_margins64(double R, const double h[3], double tau)
{
    const double u = kU64 * 1.01;
    const double r3 = std::sqrt(3.0);
    const double e_qr = 4.0 * u * 1.000001;
    const double X_D = 2.0 * R * (1.0 + 1e-9);
    const double e_l = rot3_err(X_D, 0.0, 0.0, u);
    const double e_u = 8.0 * e_qr * (1.0 + e_qr) + 8.0 * u;
    const double e64 = 1e-12;
    const double N1 = r3 * (1.0 + 2.0 * e_u + e64);
    const double N2 = 1.0 + 2.0 * e_u + e64;
    const double Lm = (X_D + r3 * e_l) * N2;
    const double hsum = h[0] + h[1] + h[2];
    const double hmax = std::max(h[0], std::max(h[1], h[2]));
    const double e_c = N1 * e_l + 3.0 * u * Lm;
    const double e_A = 3.0 * u * hmax * N1;
    const double e_B = hsum * (N1 * e_u + 6.0 * u * N1 * N2);
    const double e_s = 2.0 * u * (Lm + 2.0 * hsum * N1);
    const double E = e_c + e_A + e_B + e_s;
    const double lip = (X_D + hmax + hsum * N2) * 3.0 * (e_u + e64) * 1.001;
    return { 2.0 * E + 4e-6 * 2.0 * R * N2, 2.0 * (E + lip) + tau * N2 };
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
    auto rot_err = [&](double X, double ex, double eq) { return rot3_err(X, ex, eq, u); };
    const double X_D = 2.0 * R * (1.0 + 1e-9) + 2.0 * g.e_dlt;
    const double e_l = rot_err(X_D, g.e_dlt, ea);
    const double X_v = std::sqrt(3.0) * vm;
    const double e_rv = rot_err(X_v, kU32 * vm, e_qr);
    const double e_pb = e_rv + e_l + u * (X_v + X_D) * 5.0;
    return 2.0 * e_pb;
}

}  // namespace hpmc
