// pressure.cu -- pressure of hard particles from the scale-distribution
// histogram (Sec. 4 of Anderson, Irrgang & Glotzer: the volume-perturbation
// estimator, extended to particles with shape).  Host code only.
//
// Compressing every position by the factor (1 - x), shapes unchanged, makes
// a pair touch at some x*.  With h(x) the number of pairs per unit x and per
// configuration whose x* lies at x, the probability that a compression by a
// small x creates an overlap is h(0) x while the volume shrinks by dim x V,
// which gives beta P / rho = 1 + h(0) / (dim N).  h(0) is extrapolated from
// the histogram that hpmc_sdf accumulates: weighted least squares of log h
// on the bin centres (Poisson weights: the standard error of log n is
// 1 / sqrt(n)), a polynomial of the given degree evaluated at x = 0.
#include <cmath>
#include <vector>

#include "../../include/hpmc.h"

namespace {

// Least squares min |A c - b| by Householder QR (A: m x n, column-major
// copy), then the (0, 0) entry of (A^T A)^-1 from R.  Returns false when A
// is rank deficient.
bool lsq_qr(std::vector<double> A, std::vector<double> b, int m, int n, std::vector<double>& c, double& cov00)
{
    auto at = [&](int i, int j) -> double& { return A[(size_t)j * m + i]; };
    for (int k = 0; k < n; ++k) {
        double nrm = 0.0;
        for (int i = k; i < m; ++i) nrm += at(i, k) * at(i, k);
        nrm = std::sqrt(nrm);
        if (!(nrm > 0.0)) return false;
        const double alpha = at(k, k) > 0.0 ? -nrm : nrm;
        // v = x - alpha e_k, stored in place below the diagonal
        std::vector<double> v(m - k);
        for (int i = k; i < m; ++i) v[i - k] = at(i, k);
        v[0] -= alpha;
        double vv = 0.0;
        for (double t : v) vv += t * t;
        if (!(vv > 0.0)) return false;
        for (int j = k; j < n; ++j) {
            double s = 0.0;
            for (int i = k; i < m; ++i) s += v[i - k] * at(i, j);
            s = 2.0 * s / vv;
            for (int i = k; i < m; ++i) at(i, j) -= s * v[i - k];
        }
        double s = 0.0;
        for (int i = k; i < m; ++i) s += v[i - k] * b[i];
        s = 2.0 * s / vv;
        for (int i = k; i < m; ++i) b[i] -= s * v[i - k];
    }
    // back substitution R c = (Q^T b)[0..n)
    c.assign(n, 0.0);
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int j = k + 1; j < n; ++j) s -= at(k, j) * c[j];
        if (!(std::fabs(at(k, k)) > 0.0)) return false;
        c[k] = s / at(k, k);
    }
    // (A^T A)^-1 = R^-1 R^-T; its (0, 0) entry is the squared norm of row 0 of R^-1
    std::vector<double> Ri((size_t)n * n, 0.0);            // upper triangular inverse, row-major
    for (int k = n - 1; k >= 0; --k) {
        Ri[(size_t)k * n + k] = 1.0 / at(k, k);
        for (int j = k + 1; j < n; ++j) {
            double s = 0.0;
            for (int l = k + 1; l <= j; ++l) s += at(k, l) * Ri[(size_t)l * n + j];
            Ri[(size_t)k * n + j] = -s / at(k, k);
        }
    }
    cov00 = 0.0;
    for (int j = 0; j < n; ++j) cov00 += Ri[j] * Ri[j];
    return true;
}

}  // namespace

extern "C" int hpmc_pressure(const uint64_t* hist, uint32_t nbins, uint64_t n_samples, double x_max, uint64_t N,
                             double volume, int dim, int deg, double sigma, hpmc_pressure_t* out)
{
    if (!hist || !out || nbins == 0 || n_samples == 0 || N == 0 || (dim != 2 && dim != 3) || deg < 0 ||
        deg > 8 || !(x_max > 0.0) || !std::isfinite(x_max) || !(volume > 0.0) || !std::isfinite(volume) ||
        !(sigma > 0.0) || !std::isfinite(sigma))
        return HPMC_ERR_INVALID_ARG;
    const double dx = x_max / (double)nbins;
    const int n = deg + 1;
    std::vector<double> A, b;
    std::vector<uint32_t> rows;
    for (uint32_t k = 0; k < nbins; ++k) {
        if (hist[k] == 0) continue;                           // log 0: an empty bin carries no weight
        rows.push_back(k);
    }
    const int m = (int)rows.size();
    if (m <= n) return HPMC_ERR_INVALID_ARG;                 // too few populated bins
    A.assign((size_t)m * n, 0.0);
    b.assign(m, 0.0);
    for (int i = 0; i < m; ++i) {
        const double cnt = (double)hist[rows[i]];
        const double w = std::sqrt(cnt);
        // the polynomial in z = x / x_max (well conditioned columns); its
        // value at z = 0 is the value at x = 0
        const double z = ((double)rows[i] + 0.5) / (double)nbins;
        double p = 1.0;
        for (int j = 0; j < n; ++j) {
            A[(size_t)j * m + i] = w * p;
            p *= z;
        }
        b[i] = w * std::log(cnt / ((double)n_samples * dx));
    }
    std::vector<double> c;
    double cov00 = 0.0;
    if (!lsq_qr(A, b, m, n, c, cov00)) return HPMC_ERR_INVALID_ARG;
    const double h0 = std::exp(c[0]);
    const double dh0 = h0 * std::sqrt(cov00);
    const double bpr = 1.0 + h0 / ((double)dim * (double)N);
    const double rho = (double)N / volume;
    const double ref = dim == 2 ? sigma * sigma : M_PI / 6.0 * sigma * sigma * sigma;
    out->h0 = h0;
    out->h0_err = dh0;
    out->beta_P_over_rho = bpr;
    out->beta_P_over_rho_err = dh0 / ((double)dim * (double)N);
    out->P_star = bpr * rho * ref;
    out->P_star_err = out->beta_P_over_rho_err * rho * ref;
    return 0;
}
