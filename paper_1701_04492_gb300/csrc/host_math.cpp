// host_math.cpp -- FP64 host arithmetic of the planning stage.
//
//  * Bessel functions J_n(z) of integer order by their power series.
//  * The coefficients a_pr of eq. (2.6) (Lemma A.1, eq. (A.1)).
//  * The rank rule: the smallest K whose dropped terms sum to <= eps (the
//    triangle-inequality bound in the proof of Lemma A.1), capped by Table 2.1.
//  * Twiddle factors exp(-2 pi i m / n) with exact argument reduction.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "nufft_internal.h"

namespace nufft {

// J_n(z) = sum_m (-1)^m (z/2)^(2m+n) / (m! (m+n)!), n >= 0 (NIST 10.2.2).  The
// arguments here satisfy |z| <= pi/4, where the terms fall below 1e-17 of the
// first within a dozen steps.  Negative orders use J_{-n} = (-1)^n J_n.
double bessel_j_int(int n, double z) {
    if (n < 0) return (n & 1) ? -bessel_j_int(-n, z) : bessel_j_int(-n, z);
    const double h = 0.5 * z;
    double term = 1.0;
    for (int i = 1; i <= n; ++i) term *= h / i;
    double sum = term;
    const double h2 = h * h;
    for (int m = 1; m < 200; ++m) {
        term *= -h2 / (double(m) * double(m + n));
        sum += term;
        if (std::fabs(term) <= 1e-18 * std::fabs(sum)) break;
    }
    return sum;
}

// alpha[p*K + r] with a_pr = i^r alpha_pr:
// alpha_pr = 4 J_{(p+r)/2}(-gamma pi/2) J_{(r-p)/2}(-gamma pi/2) if p - r is even, else 0.
void chebyshev_alpha(int K, double gamma, double *alpha) {
    const double z = -gamma * M_PI / 2.0;
    for (int p = 0; p < K; ++p)
        for (int r = 0; r < K; ++r)
            alpha[p * K + r] = ((p - r) % 2 == 0)
                                   ? 4.0 * bessel_j_int((p + r) / 2, z) * bessel_j_int((r - p) / 2, z)
                                   : 0.0;
}

// sum of w_p w_r |a_pr| over p >= K or r >= K (w_0 = 1/2, else 1): a bound on
// ||A - A_K||_max since |T_p| <= 1 on [-1, 1] and |exp(i theta)| = 1.
double tail_bound(int K, double gamma) {
    constexpr int PT = 64;   // terms beyond are below 1e-60 for gamma <= 1/2
    std::vector<double> a(PT * PT);
    chebyshev_alpha(PT, gamma, a.data());
    std::vector<double> dropped;
    for (int p = 0; p < PT; ++p)
        for (int r = 0; r < PT; ++r)
            if (p >= K || r >= K) {
                const double w = (p == 0 ? 0.5 : 1.0) * (r == 0 ? 0.5 : 1.0);
                dropped.push_back(w * std::fabs(a[p * PT + r]));
            }
    std::sort(dropped.begin(), dropped.end());
    double s = 0.0;
    for (double v : dropped) s += v;
    return s;
}

// Table 2.1, double row.
static int table_double_rank(double gamma) {
    if (gamma <= 0.0) return 1;
    if (gamma <= 1.0 / 32) return 8;
    if (gamma <= 1.0 / 16) return 9;
    if (gamma <= 1.0 / 8) return 11;
    if (gamma <= 1.0 / 4) return 13;
    return 16;
}

int choose_rank(double eps, double gamma) {
    if (gamma == 0.0) return 1;   // A is all ones (section 2.1.2)
    const int cap = table_double_rank(gamma);
    for (int K = 1; K <= cap; ++K)
        if (tail_bound(K, gamma) <= eps) return K;
    return cap;
}

// exp(-2 pi i m / n) for 0 <= m < n.  The angle 2 pi m/n is split into the octant
// o = floor(8m/n) and a remainder, so the library cos/sin only see [0, pi/4].
void twiddle(int64_t n, int64_t m, double *c, double *s) {
    m %= n;
    if (m < 0) m += n;
    const int64_t a = 8 * m;
    const int64_t o = a / n;                 // octant 0..7
    const int64_t rem = a - o * n;           // angle within the octant = (pi/4) rem/n
    double phi;
    bool odd = (o & 1) != 0;
    if (!odd) phi = (M_PI / 4.0) * (double(rem) / double(n));
    else phi = (M_PI / 4.0) * (double(n - rem) / double(n));
    const double cp = std::cos(phi), sp = std::sin(phi);
    // theta = o*pi/4 + (pi/4) rem/n; reconstruct cos(theta), sin(theta)
    double ct, st;
    switch (o) {
        case 0: ct = cp;  st = sp;  break;   // theta = phi
        case 1: ct = sp;  st = cp;  break;   // theta = pi/2 - phi
        case 2: ct = -sp; st = cp;  break;   // theta = pi/2 + phi
        case 3: ct = -cp; st = sp;  break;   // theta = pi - phi
        case 4: ct = -cp; st = -sp; break;   // theta = pi + phi
        case 5: ct = -sp; st = -cp; break;   // theta = 3pi/2 - phi
        case 6: ct = sp;  st = -cp; break;   // theta = 3pi/2 + phi
        default: ct = cp; st = -sp; break;   // theta = 2pi - phi
    }
    *c = ct;
    *s = -st;   // exp(-i theta)
}

}  // namespace nufft

// ---- host-only entry points (no GPU call) -----------------------------------------

extern "C" int nufft_rank(double eps, double gamma, int *K) {
    if (!K || !(eps > 0.0 && eps < 1.0) || !(gamma >= 0.0 && gamma <= 0.5)) return NUFFT_EINVAL;
    *K = nufft::choose_rank(eps, gamma);
    return NUFFT_OK;
}

extern "C" int nufft_lowrank_coeffs(int K, double gamma, double *alpha) {
    if (!alpha || K < 1 || K > 64 || !(gamma >= 0.0 && gamma <= 0.5)) return NUFFT_EINVAL;
    nufft::chebyshev_alpha(K, gamma, alpha);
    return NUFFT_OK;
}
