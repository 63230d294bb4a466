// Layer design on the host: the predicted amplitude of the residual wave a layer lets
// back into the physical domain, from the one-edge decay rate of the discrete PML
// (eq:IntroDecayRate, Sec. 1.1.2) and its cumulative product (Sec. 1.1.4).
//
// For an edge with damping s (times h) a discrete wave exp(-i w t + i k h j) crossing the
// edge is multiplied by
//     rho(s, k, w) = (2 + i (s/(w h)) (1 - e^{-i k h})) / (2 + i (s/(w h)) (1 - e^{+i k h}))
// (s here is sigma * h, so s/(w h) is sigma / w).  A layer truncated periodically, as in
// this library, passes the wave once through every layer edge before it re-enters the
// physical domain: factor prod_e |rho(s_e, k, w)|.  A layer backed by a reflecting wall
// returns the reflected wave (wave number -conj(k)) through the same edges: factor
// prod_e |rho(s_e, k, w)| / |rho(s_e, -conj(k), w)|.
#include <cmath>
#include <complex>
#include <vector>

#include "pml.h"

namespace pml {
void set_global_error(const char *msg);
}

namespace {

using cd = std::complex<double>;

cd rho(double s, cd kh, double wh)
{
    const cd i(0.0, 1.0);
    const cd q = i * (s / wh);
    return (2.0 + q * (1.0 - std::exp(-i * kh))) / (2.0 + q * (1.0 - std::exp(i * kh)));
}

double factor(int m, const double *s, cd kh, double wh, int backed)
{
    double f = 1.0;
    for (int e = 0; e < m; ++e) {
        f *= std::abs(rho(s[e], kh, wh));
        if (backed) f /= std::abs(rho(s[e], -std::conj(kh), wh));
    }
    return f;
}

pml_status bad(const char *msg)
{
    pml::set_global_error(msg);
    return PML_EINVAL;
}

}  // namespace

extern "C" pml_status pml_residual_factor(int m, const double *sigma_h, double kh_re, double kh_im, double omega_h,
                                          int backed, double *out)
{
    if (m < 0 || (m > 0 && !sigma_h) || !out) return bad("pml_residual_factor: bad arguments");
    if (!(omega_h != 0.0) || !std::isfinite(omega_h)) return bad("pml_residual_factor: omega_h must be finite and nonzero");
    for (int e = 0; e < m; ++e)
        if (!(sigma_h[e] >= 0.0) || !std::isfinite(sigma_h[e]))
            return bad("pml_residual_factor: damping values must be finite and >= 0");
    *out = factor(m, sigma_h, cd(kh_re, kh_im), omega_h, backed);
    return PML_OK;
}

extern "C" pml_status pml_design_width(int kind, double sigma_max_h, double order, double cos_min, double omega_h_max,
                                       double eps, int backed, int w_max, int *w_out, double *worst_out)
{
    if (!w_out || !worst_out) return bad("pml_design_width: NULL output");
    if (kind != PML_SIGMA_CONSTANT && kind != PML_SIGMA_POWER)
        return bad("pml_design_width: kind must be PML_SIGMA_CONSTANT or PML_SIGMA_POWER");
    if (!(sigma_max_h > 0.0) || !(cos_min > 0.0 && cos_min <= 1.0) || !(omega_h_max > 0.0 && omega_h_max <= 2.0) ||
        !(eps > 0.0) || w_max < 1 || !(order > 0.0))
        return bad("pml_design_width: need sigma_max_h > 0, 0 < cos_min <= 1, 0 < omega_h_max <= 2, eps > 0, "
                   "order > 0, w_max >= 1");
    // sweep: omega h in (0, omega_h_max], normal wave number k h = cos(theta) omega h with
    // cos(theta) in [cos_min, 1] (theta = arccos(Re(k)/omega), the paper's incidence angle)
    const int NW = 64, NC = 16;
    *w_out = -1;
    *worst_out = 1.0;
    for (int w = 1; w <= w_max; ++w) {
        // the edges a wave crosses in one pass: depths 1..w on one side, w-1..1 on the other
        std::vector<double> s;
        for (int d = 1; d <= w; ++d) s.push_back(kind == PML_SIGMA_CONSTANT ? sigma_max_h : sigma_max_h * std::pow(double(d) / w, order));
        for (int d = w - 1; d >= 1; --d) s.push_back(kind == PML_SIGMA_CONSTANT ? sigma_max_h : sigma_max_h * std::pow(double(d) / w, order));
        double worst = 0.0;
        for (int a = 1; a <= NW; ++a) {
            const double wh = omega_h_max * a / NW;
            for (int b = 0; b <= NC; ++b) {
                const double c = cos_min + (1.0 - cos_min) * b / NC;
                const double f = factor(int(s.size()), s.data(), cd(c * wh, 0.0), wh, backed);
                if (f > worst) worst = f;
            }
        }
        *worst_out = worst;
        if (worst <= eps) {
            *w_out = w;
            return PML_OK;
        }
    }
    return PML_OK;   // *w_out = -1: no width up to w_max meets eps (*worst_out is that of w_max)
}
