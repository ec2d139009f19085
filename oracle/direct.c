/* The nonuniform DFT by its definition, eq. (1.2) of arXiv:1701.04492, in FP64.
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, smoke() and the CPU baseline of the
 * benchmark, never by the product library.
 *
 *   nudft2   f_j = sum_k c_k exp(-2 pi i x_j k)          j < M, k < N  (type II)
 *   nudft2h  c_k = sum_j g_j exp(+2 pi i x_j k)          the adjoint A^H g
 *   nudft2d  f_j = sum_k (-2 pi i k) c_k exp(-2 pi i x_j k)   (d f_j / d x_j)
 *   nudft2_2d f_j = sum_{k1<m,k2<n} C[k1][k2] exp(-2 pi i (k1 x_j + k2 y_j))  (eq. (4.1))
 *   nudft2h_at     c_k for a list of frequencies k: the adjoint sum at chosen outputs
 *   nudft2h_2d_at  C[k1][k2] = sum_j g_j exp(+2 pi i (k1 x_j + k2 y_j)) for a list of
 *                  (k1, k2): the adjoint of eq. (4.1) at chosen outputs
 *
 * The phase x_j k is reduced modulo 1 exactly: with Q = 2^32, x (mod 1) =
 * (s + r) / Q where s = floor(Q x) is an integer and r in [0,1) is exact (Q is a
 * power of two), so x k = (s k mod Q) / Q + r k / Q with an exact integer part and
 * a small remainder.  The naive product x_j * k would carry an absolute phase error
 * of order N * 1e-16.  Sums are Neumaier-compensated.  Complex data is interleaved
 * (re, im).
 */
#include <math.h>
#include <stdint.h>

static const double TWO_PI = 6.283185307179586476925286766559;
static const double Q = 4294967296.0; /* 2^32 */

typedef struct { double s, c; } acc_t; /* Neumaier sum and compensation */

static inline void acc_add(acc_t *a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}

/* x mod 1 split as (s + r)/Q with integer s in [0, Q) and r in [0, 1). */
static inline void split_x(double x, uint64_t *s, double *r) {
    double xf = x - floor(x);          /* exact for |x| < 2^52 */
    double qx = xf * Q;                /* exact: Q is a power of two */
    double fs = floor(qx);
    *s = (uint64_t)fs;
    *r = qx - fs;
    if (*s >= (uint64_t)Q) { *s -= (uint64_t)Q; }
}

/* The fraction of x k in [0, 1), from the split of x. */
static inline double frac_xk(uint64_t s, double r, int64_t k) {
    uint64_t ip = (s * (uint64_t)k) & 0xffffffffULL;   /* (s k) mod Q, exact */
    double th = ((double)ip + r * (double)k) / Q;       /* r k < k <= 2^31 */
    return th - floor(th);
}

void nudft2(int64_t N, int64_t M, const double *x, const double *c, double *f) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < M; ++j) {
        uint64_t s; double r;
        split_x(x[j], &s, &r);
        acc_t re = {0, 0}, im = {0, 0};
        for (int64_t k = 0; k < N; ++k) {
            double th = TWO_PI * frac_xk(s, r, k);
            double cs = cos(th), sn = -sin(th);         /* exp(-i th) */
            double cr = c[2 * k], ci = c[2 * k + 1];
            acc_add(&re, cr * cs);
            acc_add(&re, -ci * sn);
            acc_add(&im, cr * sn);
            acc_add(&im, ci * cs);
        }
        f[2 * j] = re.s + re.c;
        f[2 * j + 1] = im.s + im.c;
    }
}

void nudft2h(int64_t N, int64_t M, const double *x, const double *g, double *c) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < N; ++k) {
        acc_t re = {0, 0}, im = {0, 0};
        for (int64_t j = 0; j < M; ++j) {
            uint64_t s; double r;
            split_x(x[j], &s, &r);
            double th = TWO_PI * frac_xk(s, r, k);
            double cs = cos(th), sn = sin(th);          /* exp(+i th) */
            double gr = g[2 * j], gi = g[2 * j + 1];
            acc_add(&re, gr * cs);
            acc_add(&re, -gi * sn);
            acc_add(&im, gr * sn);
            acc_add(&im, gi * cs);
        }
        c[2 * k] = re.s + re.c;
        c[2 * k + 1] = im.s + im.c;
    }
}

void nudft2d(int64_t N, int64_t M, const double *x, const double *c, double *f) {
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < M; ++j) {
        uint64_t s; double r;
        split_x(x[j], &s, &r);
        acc_t re = {0, 0}, im = {0, 0};
        for (int64_t k = 0; k < N; ++k) {
            double th = TWO_PI * frac_xk(s, r, k);
            double cs = cos(th), sn = -sin(th);
            /* (-2 pi i k) c_k = (2 pi k ci, -2 pi k cr) */
            double w = TWO_PI * (double)k;
            double cr = w * c[2 * k + 1], ci = -w * c[2 * k];
            acc_add(&re, cr * cs);
            acc_add(&re, -ci * sn);
            acc_add(&im, cr * sn);
            acc_add(&im, ci * cs);
        }
        f[2 * j] = re.s + re.c;
        f[2 * j + 1] = im.s + im.c;
    }
}

void nudft2_2d(int64_t m, int64_t n, int64_t M, const double *x, const double *y,
               const double *C, double *f) {
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < M; ++j) {
        uint64_t sx, sy; double rx, ry;
        split_x(x[j], &sx, &rx);
        split_x(y[j], &sy, &ry);
        acc_t re = {0, 0}, im = {0, 0};
        for (int64_t k1 = 0; k1 < m; ++k1) {
            double a = frac_xk(sx, rx, k1);
            for (int64_t k2 = 0; k2 < n; ++k2) {
                double th = a + frac_xk(sy, ry, k2);
                th = TWO_PI * (th - floor(th));
                double cs = cos(th), sn = -sin(th);
                const double *cc = C + 2 * (k1 * n + k2);
                acc_add(&re, cc[0] * cs);
                acc_add(&re, -cc[1] * sn);
                acc_add(&im, cc[0] * sn);
                acc_add(&im, cc[1] * cs);
            }
        }
        f[2 * j] = re.s + re.c;
        f[2 * j + 1] = im.s + im.c;
    }
}

void nudft2h_at(int64_t nk, const int64_t *ks, int64_t M, const double *x, const double *g, double *c) {
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < nk; ++q) {
        const int64_t k = ks[q];
        acc_t re = {0, 0}, im = {0, 0};
        for (int64_t j = 0; j < M; ++j) {
            uint64_t s; double r;
            split_x(x[j], &s, &r);
            double th = TWO_PI * frac_xk(s, r, k);
            double cs = cos(th), sn = sin(th);          /* exp(+i th) */
            double gr = g[2 * j], gi = g[2 * j + 1];
            acc_add(&re, gr * cs);
            acc_add(&re, -gi * sn);
            acc_add(&im, gr * sn);
            acc_add(&im, gi * cs);
        }
        c[2 * q] = re.s + re.c;
        c[2 * q + 1] = im.s + im.c;
    }
}

void nudft2h_2d_at(int64_t nk, const int64_t *k1s, const int64_t *k2s, int64_t M, const double *x,
                   const double *y, const double *g, double *C) {
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < nk; ++q) {
        const int64_t k1 = k1s[q], k2 = k2s[q];
        acc_t re = {0, 0}, im = {0, 0};
        for (int64_t j = 0; j < M; ++j) {
            uint64_t sx, sy; double rx, ry;
            split_x(x[j], &sx, &rx);
            split_x(y[j], &sy, &ry);
            double th = frac_xk(sx, rx, k1) + frac_xk(sy, ry, k2);
            th = TWO_PI * (th - floor(th));
            double cs = cos(th), sn = sin(th);          /* exp(+i th) */
            double gr = g[2 * j], gi = g[2 * j + 1];
            acc_add(&re, gr * cs);
            acc_add(&re, -gi * sn);
            acc_add(&im, gr * sn);
            acc_add(&im, gi * cs);
        }
        C[2 * q] = re.s + re.c;
        C[2 * q + 1] = im.s + im.c;
    }
}
