// Default force-split parameters, computed on the host in FP64.
//
// Sec. 2.4, Eq. (fitform): the residual filtered grid force between two unit
// masses is F_grid(r) = tanh(br)/r^2 - (b/r)/cosh^2(br) + c r (1 + d r^2) e^{-d r^2}
//                       + e (1 + f r^2 + g r^4 + l r^6) e^{-h r^2},
// b=.72 c=.01 d=.27 e=1e-4 f=360 g=100 h=.67 l=17.
// Sec. 3.1, Eq. (force): f_SR(s) = (s+eps)^(-3/2) - P5(s), P5 a fifth-order
// polynomial in s = r.r standing in for the grid force.  The paper prints no
// P5 coefficients, r_cut or eps; the library's defaults are:
//   r_cut: the root of r^2 F_grid(r) = 1 near three grid cells (where the
//          fitted grid force meets Newton; Sec. 2.3 matches at three cells);
//   P5:    least squares of F_grid(r)/r on a uniform grid of r in [1e-3, r_cut]
//          with residuals weighted by r^3 (error relative to 1/r^2), under the
//          constraint P5(r_cut^2) = F_grid(r_cut)/r_cut (f_SR(r_cut^2) = 0 at
//          eps = 0), solved by Householder QR in u = s / r_cut^2;
//   eps:   2.5e-4 grid units^2;  G: 1.
#include <cmath>
#include <vector>

#include "../../include/hacc.h"

namespace {

double f_grid(double r) {
    const double b = 0.72, c = 0.01, d = 0.27, e = 1e-4, f = 360.0, g = 100.0, h = 0.67, l = 17.0;
    const double br = b * r, r2 = r * r;
    const double ch = std::cosh(br);
    return std::tanh(br) / r2 - (b / r) / (ch * ch) + c * r * (1.0 + d * r2) * std::exp(-d * r2) +
           e * (1.0 + f * r2 + g * r2 * r2 + l * r2 * r2 * r2) * std::exp(-h * r2);
}

double r_cut_root() {
    double lo = 2.5, hi = 3.5;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid * mid * f_grid(mid) - 1.0 < 0.0) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

// min || A x - b ||_2 for an m x n matrix A (row-major, m >= n) by Householder QR.
std::vector<double> lstsq_qr(std::vector<double> A, std::vector<double> b, int m, int n) {
    for (int k = 0; k < n; ++k) {
        double norm = 0.0;
        for (int i = k; i < m; ++i) norm += A[(size_t)i * n + k] * A[(size_t)i * n + k];
        norm = std::sqrt(norm);
        double akk = A[(size_t)k * n + k];
        double alpha = akk > 0 ? -norm : norm;
        std::vector<double> v(m - k);
        for (int i = k; i < m; ++i) v[i - k] = A[(size_t)i * n + k];
        v[0] -= alpha;
        double vnorm2 = 0.0;
        for (double x : v) vnorm2 += x * x;
        if (vnorm2 == 0.0) continue;
        for (int j = k; j < n; ++j) {
            double dot = 0.0;
            for (int i = k; i < m; ++i) dot += v[i - k] * A[(size_t)i * n + j];
            double s = 2.0 * dot / vnorm2;
            for (int i = k; i < m; ++i) A[(size_t)i * n + j] -= s * v[i - k];
        }
        double dot = 0.0;
        for (int i = k; i < m; ++i) dot += v[i - k] * b[i];
        double s = 2.0 * dot / vnorm2;
        for (int i = k; i < m; ++i) b[i] -= s * v[i - k];
    }
    std::vector<double> x(n);
    for (int k = n - 1; k >= 0; --k) {
        double acc = b[k];
        for (int j = k + 1; j < n; ++j) acc -= A[(size_t)k * n + j] * x[j];
        x[k] = acc / A[(size_t)k * n + k];
    }
    return x;
}

}  // namespace

extern "C" hacc_status hacc_split_default(hacc_split *out) {
    if (!out) return HACC_EINVAL;
    const double rc = r_cut_root();
    const int m = 40001, nunk = 5;
    const double rmin = 1e-3;
    const double yc = f_grid(rc) / rc;
    std::vector<double> A((size_t)m * nunk), b(m);
    for (int i = 0; i < m; ++i) {
        double r = rmin + (rc - rmin) * i / (m - 1);
        double u = (r * r) / (rc * rc);
        double w = r * r * r;
        double uk = 1.0;
        for (int k = 1; k <= nunk; ++k) {
            uk *= u;
            A[(size_t)i * nunk + (k - 1)] = (uk - 1.0) * w;
        }
        b[i] = (f_grid(r) / r - yc) * w;
    }
    std::vector<double> d = lstsq_qr(A, b, m, nunk);
    double d0 = yc;
    for (double x : d) d0 -= x;
    double scale = 1.0;
    out->poly[0] = d0;
    for (int k = 1; k <= 5; ++k) {
        scale *= rc * rc;
        out->poly[k] = d[k - 1] / scale;
    }
    out->r_cut = (float)rc;
    out->eps = 2.5e-4f;
    out->G = 1.0f;
    return HACC_OK;
}
