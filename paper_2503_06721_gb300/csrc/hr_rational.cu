// hr_rational.cu -- rational approximations for the RHMC (Sec. 4.3.2): the
// best relative approximation of degree (n, n)
//
//     r(x) = c prod_k (x + z_k) / (x + p_k)  ~  x^(-alpha)   on [lo, hi],
//
// returned in partial fractions r(x) = a0 + sum_k a_k / (x + p_k), whose
// poles p_k are the shifts of one multi-shift inversion.  The paper computes
// such coefficients with the Remez algorithm and stores them in a table; this
// is a Remez exchange written for this library.  Host code only.
//
// By Chebyshev's alternation theorem the best approximation is the one whose
// relative error e(x) = r(x) x^alpha - 1 takes its largest magnitude E at
// 2n + 2 points with alternating signs.  Each exchange step:
//   1. levels the error on the current reference points x_j: Newton's method
//      on  log(r(x_j) x_j^alpha) = log(1 + (-1)^j E)  for the 2n + 2 unknowns
//      (log c, log z_k, log p_k, E).  In these variables the equations are
//      smooth sums of log(x_j + t) and the Jacobian columns t / (x_j + t) are
//      well scaled over many decades of x, unlike a polynomial basis;
//   2. finds the local extrema of e on [lo, hi] (a grid clustered towards
//      both ends, as Chebyshev points are, refined by golden-section search)
//      and takes 2n + 2 alternating ones as the next reference.
// It stops when the largest |e| equals the levelled |E| to 1e-8 (or to the
// double-precision floor of evaluating r).  The degree is reached by
// continuation: degree 4 (or n) from log-spaced, interlaced poles and zeros,
// then each next degree from the previous solution's poles, zeros and
// reference points resampled in log position.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hr_internal.cuh"

namespace hr {
namespace {

struct Ratl {
    double lc;                 // log c
    std::vector<double> z, p;  // zeros and poles of r on the negative axis: x + z_k, x + p_k
};

// log(r(x) x^alpha)
double log_rel(const Ratl &r, double x, double alpha)
{
    double s = r.lc + alpha * std::log(x);
    for (double t : r.z) s += std::log(x + t);
    for (double t : r.p) s -= std::log(x + t);
    return s;
}
double rel_err(const Ratl &r, double x, double alpha) { return std::expm1(log_rel(r, x, alpha)); }

// solves A d = b (m x m, row-major) by Gaussian elimination with partial pivoting
bool solve(std::vector<double> &A, std::vector<double> &b, int m)
{
    for (int k = 0; k < m; k++) {
        int piv = k;
        for (int i = k + 1; i < m; i++)
            if (std::fabs(A[(size_t)i * m + k]) > std::fabs(A[(size_t)piv * m + k])) piv = i;
        if (A[(size_t)piv * m + k] == 0.0 || !std::isfinite(A[(size_t)piv * m + k])) return false;
        if (piv != k) {
            for (int j = 0; j < m; j++) std::swap(A[(size_t)k * m + j], A[(size_t)piv * m + j]);
            std::swap(b[k], b[piv]);
        }
        for (int i = k + 1; i < m; i++) {
            const double f = A[(size_t)i * m + k] / A[(size_t)k * m + k];
            if (f == 0.0) continue;
            for (int j = k; j < m; j++) A[(size_t)i * m + j] -= f * A[(size_t)k * m + j];
            b[i] -= f * b[k];
        }
    }
    for (int k = m - 1; k >= 0; k--) {
        double s = b[k];
        for (int j = k + 1; j < m; j++) s -= A[(size_t)k * m + j] * b[j];
        b[k] = s / A[(size_t)k * m + k];
    }
    return true;
}

// step 1: levels the error on the reference xr (2n + 2 points); keeps the
// iterate with the smallest residual
void level(const std::vector<double> &xr, double alpha, Ratl &r, double &E)
{
    const int n = (int)r.z.size(), m = 2 * n + 2;
    std::vector<double> th(m), best;
    th[0] = r.lc;
    for (int k = 0; k < n; k++) {
        th[1 + k] = std::log(r.z[k]);
        th[1 + n + k] = std::log(r.p[k]);
    }
    th[m - 1] = E;
    double best_res = INFINITY;
    std::vector<double> J((size_t)m * m), F(m);
    Ratl cur = r;
    for (int it = 0; it < 60; it++) {
        cur.lc = th[0];
        for (int k = 0; k < n; k++) {
            cur.z[k] = std::exp(th[1 + k]);
            cur.p[k] = std::exp(th[1 + n + k]);
        }
        const double e = th[m - 1];
        double res = 0;
        bool ok = std::fabs(e) < 0.5;
        for (int j = 0; j < m && ok; j++) {
            const double s = (j & 1) ? -1.0 : 1.0;
            F[j] = -(log_rel(cur, xr[j], alpha) - std::log1p(s * e));
            res = std::max(res, std::fabs(F[j]));
            double *row = &J[(size_t)j * m];
            row[0] = 1.0;
            for (int k = 0; k < n; k++) {
                row[1 + k] = cur.z[k] / (xr[j] + cur.z[k]);
                row[1 + n + k] = -cur.p[k] / (xr[j] + cur.p[k]);
            }
            row[m - 1] = -s / (1.0 + s * e);
        }
        if (!ok || !std::isfinite(res)) break;
        if (res < best_res) {
            best_res = res;
            best = th;
        }
        if (res < 1e-14) break;
        if (!solve(J, F, m)) break;
        double big = 0;
        for (int q = 0; q < m - 1; q++) big = std::max(big, std::fabs(F[q]));
        const double damp = big > 0.5 ? 0.5 / big : 1.0;   // at most a factor e^0.5 per step
        for (int q = 0; q < m; q++) th[q] += damp * F[q];
    }
    if (best.empty()) return;
    r.lc = best[0];
    for (int k = 0; k < n; k++) {
        r.z[k] = std::exp(best[1 + k]);
        r.p[k] = std::exp(best[1 + n + k]);
    }
    E = best[m - 1];
}

// step 2: alternating extrema of e on [lo, hi] in t = log x; returns false
// unless exactly 2n + 2 remain after merging equal-sign neighbours
bool extrema(const Ratl &r, double alpha, double lo, double hi, std::vector<double> &xe, double &D)
{
    const int n = (int)r.z.size();
    const int M = 64 * (2 * n + 2);
    const double t0 = std::log(lo), L = std::log(hi / lo);
    std::vector<double> t(M), e(M);
    for (int i = 0; i < M; i++) {
        t[i] = t0 + L * 0.5 * (1.0 - std::cos(M_PI * i / (M - 1)));
        e[i] = rel_err(r, std::exp(t[i]), alpha);
    }
    std::vector<double> pt, pv;
    const double g = 0.5 * (std::sqrt(5.0) - 1.0);
    for (int i = 0; i < M; i++) {
        if (i == 0 || i == M - 1) {
            pt.push_back(t[i]);
            pv.push_back(e[i]);
            continue;
        }
        if ((e[i] - e[i - 1]) * (e[i + 1] - e[i]) > 0) continue;
        // golden-section search for the extremum of sign(e[i]) * e on [t_{i-1}, t_{i+1}]
        const double sg = e[i] >= 0 ? 1.0 : -1.0;
        double a = t[i - 1], b = t[i + 1];
        for (int it = 0; it < 50; it++) {
            const double u1 = b - g * (b - a), u2 = a + g * (b - a);
            if (sg * rel_err(r, std::exp(u1), alpha) > sg * rel_err(r, std::exp(u2), alpha))
                b = u2;
            else
                a = u1;
        }
        const double u = 0.5 * (a + b);
        pt.push_back(u);
        pv.push_back(rel_err(r, std::exp(u), alpha));
    }
    std::vector<double> kt, kv;
    for (size_t q = 0; q < pt.size(); q++) {
        if (!kv.empty() && (pv[q] >= 0) == (kv.back() >= 0)) {
            if (std::fabs(pv[q]) > std::fabs(kv.back())) {
                kt.back() = pt[q];
                kv.back() = pv[q];
            }
        } else {
            kt.push_back(pt[q]);
            kv.push_back(pv[q]);
        }
    }
    size_t first = 0, last = kt.size();
    while (last - first > (size_t)(2 * n + 2)) {
        if (std::fabs(kv[first]) < std::fabs(kv[last - 1]))
            first++;
        else
            last--;
    }
    if (last - first != (size_t)(2 * n + 2)) return false;
    D = 0;
    xe.assign(2 * n + 2, 0.0);
    for (size_t q = first; q < last; q++) {
        xe[q - first] = std::exp(kt[q]);
        D = std::max(D, std::fabs(kv[q]));
    }
    for (int i = 0; i < M; i++) D = std::max(D, std::fabs(e[i]));
    return std::isfinite(D);
}

// exchange steps at fixed degree until the levelled error is the largest one
bool exchange(double alpha, double lo, double hi, Ratl &r, std::vector<double> &xr, double &D)
{
    // levelled to 1e-8 relative (or the rounding floor of evaluating r);
    // if that is out of reach, to 1e-4 after the last step
    double E = 0;
    bool loose = false;
    for (int it = 0; it < 40; it++) {
        level(xr, alpha, r, E);
        std::vector<double> xe;
        if (!extrema(r, alpha, lo, hi, xe, D)) return loose;
        loose = D - std::fabs(E) <= 1e-4 * D + 1e-13;
        xr = xe;
        if (D - std::fabs(E) <= 1e-8 * D + 2e-14) return true;
    }
    return loose;
}

double log_c_at_centre(const Ratl &r, double alpha, double lo, double hi)
{
    Ratl t = r;
    t.lc = 0;
    return -log_rel(t, std::sqrt(lo * hi), alpha);
}

}  // namespace

hr_status rational_remez(double alpha, int n, double lo, double hi, double *a0, double *res, double *poles,
                         double *max_rel_err)
{
    const int n0 = std::min(n, 4);
    const double L = std::log(hi / lo);
    Ratl r;
    // degree n0: 2 n0 log-spaced points, poles and zeros interlaced (a pole
    // first for a decreasing power, alpha > 0; a zero first for alpha < 0)
    for (int i = 0; i < 2 * n0; i++) {
        const double t = lo * std::exp(L * (i + 0.5) / (2 * n0));
        const bool pole = (alpha > 0) == ((i & 1) == 0);
        (pole ? r.p : r.z).push_back(t);
    }
    r.lc = log_c_at_centre(r, alpha, lo, hi);
    std::vector<double> xr(2 * n0 + 2);
    for (int j = 0; j < 2 * n0 + 2; j++) xr[j] = lo * std::exp(L * 0.5 * (1.0 - std::cos(M_PI * j / (2 * n0 + 1))));
    double D = 0;
    if (!exchange(alpha, lo, hi, r, xr, D)) {
        set_error("hr_rational_approx: the Remez exchange did not converge at degree %d", n0);
        return HR_ERR_NOT_CONVERGED;
    }
    for (int m = n0 + 1; m <= n; m++) {
        // next degree: resample the sorted poles and zeros (log position
        // against index) to 2m points, and the reference to 2m + 2
        std::vector<double> all(r.z);
        all.insert(all.end(), r.p.begin(), r.p.end());
        std::sort(all.begin(), all.end());
        const int k = (int)all.size();
        Ratl q;
        for (int i = 0; i < 2 * m; i++) {
            const double s = (double)i * (k - 1) / (2 * m - 1);
            const int i0 = std::min((int)s, k - 2);
            const double f = s - i0;
            const double t = std::exp((1 - f) * std::log(all[i0]) + f * std::log(all[i0 + 1]));
            const bool pole = (alpha > 0) == ((i & 1) == 0);
            (pole ? q.p : q.z).push_back(t);
        }
        q.lc = log_c_at_centre(q, alpha, lo, hi);
        std::vector<double> x2(2 * m + 2);
        const int kx = (int)xr.size();
        for (int j = 0; j < 2 * m + 2; j++) {
            const double s = (double)j * (kx - 1) / (2 * m + 1);
            const int j0 = std::min((int)s, kx - 2);
            const double f = s - j0;
            x2[j] = std::exp((1 - f) * std::log(xr[j0]) + f * std::log(xr[j0 + 1]));
        }
        x2.front() = lo;
        x2.back() = hi;
        r = q;
        xr = x2;
        if (!exchange(alpha, lo, hi, r, xr, D)) {
            set_error("hr_rational_approx: the Remez exchange did not converge at degree %d (of %d) on [%g, %g]",
                      m, n, lo, hi);
            return HR_ERR_NOT_CONVERGED;
        }
    }
    // partial fractions: a0 = c, a_k = c prod_j (z_j - p_k) / prod_{j != k} (p_j - p_k)
    std::vector<int> order(n);
    for (int k = 0; k < n; k++) order[k] = k;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return r.p[a] < r.p[b]; });
    const double c = std::exp(r.lc);
    *a0 = c;
    for (int q = 0; q < n; q++) {
        const int k = order[q];
        double v = c;
        for (int j = 0; j < n; j++) {
            v *= r.z[j] - r.p[k];
            if (j != k) v /= r.p[j] - r.p[k];
        }
        res[q] = v;
        poles[q] = r.p[k];
    }
    *max_rel_err = D;
    return HR_OK;
}

}  // namespace hr

extern "C" hr_status hr_rational_approx(double alpha, int n, double lo, double hi, double *a0, double *res,
                                        double *poles, double *max_rel_err)
{
    if (!a0 || !res || !poles || !max_rel_err || n < 1 || n > 64 || !(lo > 0) || !(hi > lo) || !std::isfinite(hi) ||
        !(std::fabs(alpha) > 0 && std::fabs(alpha) < 1)) {
        hr::set_error("hr_rational_approx: need 0 < |alpha| < 1, 1 <= n <= 64, 0 < lo < hi and output arrays");
        return HR_ERR_INVALID;
    }
    return hr::rational_remez(alpha, n, lo, hi, a0, res, poles, max_rel_err);
}
