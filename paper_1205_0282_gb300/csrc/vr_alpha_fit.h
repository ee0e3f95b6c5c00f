// Host-side fit of the opacity correction alpha(a) = 1 - (1 - a)^r (r = step in
// voxels) used by the ray-march kernels: alpha = a * Q(a) with Q a Chebyshev
// interpolant of (1 - (1 - a)^r) / a, converted to powers of t = 2a/split - 1.
// Two fits: a short one for small opacities (the common case) and a longer one up
// to `split`; above it the kernels use the exponential form.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstring>

namespace vr {

inline double alpha_over_a(double a, double r) {
    if (a == 0.0) return r;
    return -std::expm1(r * std::log1p(-a)) / a;
}

// Fit `terms` coefficients on [0, split]; returns the maximum error of Q on a
// dense grid (evaluated in double).
inline double fit_alpha_terms(double r, double split, int terms, float* coeff) {
    const int m = terms;
    double c[32] = {}, mono[32] = {}, tkm1[32] = {}, tk[32] = {}, tkp1[32] = {};
    for (int j = 0; j < m; ++j) {
        double s = 0;
        for (int k = 0; k < m; ++k) {
            const double th = M_PI * (k + 0.5) / m;
            s += alpha_over_a((std::cos(th) + 1.0) * 0.5 * split, r) * std::cos(j * th);
        }
        c[j] = 2.0 * s / m;
    }
    c[0] *= 0.5;
    // Chebyshev -> monomial: T_0 = 1, T_1 = t, T_{k+1} = 2t T_k - T_{k-1}
    tkm1[0] = 1.0;
    if (m > 1) tk[1] = 1.0;
    for (int j = 0; j < m; ++j) {
        const double* T = (j == 0) ? tkm1 : tk;
        for (int q = 0; q < m; ++q) mono[q] += c[j] * T[q];
        if (j >= 1) {
            for (int q = 0; q < m; ++q) tkp1[q] = (q > 0 ? 2.0 * tk[q - 1] : 0.0) - tkm1[q];
            std::memcpy(tkm1, tk, sizeof(tk));
            std::memcpy(tk, tkp1, sizeof(tk));
        }
    }
    double err = 0;
    for (int g = 0; g <= 4000; ++g) {
        const double a = split * g / 4000.0, t = 2.0 * a / split - 1.0;
        double q = 0;
        for (int k = m - 1; k >= 0; --k) q = q * t + mono[k];
        err = std::max(err, std::fabs(q - alpha_over_a(a, r)));
    }
    for (int k = 0; k < m; ++k) coeff[k] = (float)mono[k];
    return err;
}

// Largest split from `splits` whose fit error is below tol (the last one otherwise).
template <int N>
inline double fit_alpha(double r, const double (&splits)[N], int terms, float* coeff, double tol) {
    for (int k = 0; k < N; ++k)
        if (fit_alpha_terms(r, splits[k], terms, coeff) < tol || k == N - 1) return splits[k];
    return splits[N - 1];
}

}  // namespace vr
