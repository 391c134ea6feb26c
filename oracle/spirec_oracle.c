/*
 * spirec_oracle.c -- plain, slow, FP64 CPU oracle for regularized spiral-MRI
 * reconstruction (Boubertakh, Giovannelli, De Cesare, Herment, "Regularized
 * Reconstruction of MR Images from Spiral Acquisitions").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header or table with the CUDA path.
 *
 * Everything here is the direct definition written out, in double precision,
 * with the paper's notation:
 *   f[n][m]  complex N x N image, row-major f[n*N+m]; n pairs with ky, m with kx
 *            (section 2, Eq. ModDirect: r_nm = [n, m], phase kx*m + ky*n).
 *   s_l      complex data, l = 0..L-1, k-space point (kx_l, ky_l) in [-0.5,0.5]^2.
 *   H        (Hf)_l = (1/N) sum_{n,m} f[n][m] exp(+i 2 pi (kx_l m + ky_l n))
 *            (Eq. ModDirect; the paper calls H the inverse Fourier matrix).
 * Complex arrays are interleaved (re, im) doubles.
 *
 * Readings of the paper taken here:
 *  - phi acts on the complex modulus: phi(|z|) (section 3.3 states Huber for
 *    real x only).
 *  - the difference sums of Omega_1 have a free boundary: N(N-1) differences
 *    per direction, no wrap (section 3.3).
 *  - the gradient is dJ/dRe f + i dJ/dIm f, which gives 2 f*G - 2D for the
 *    data term (section 3.4 and Appendix B).
 *  - the "hyperbolic" phi is 2a(sqrt(a^2+r^2)-a); the paper does not define it.
 *  - the Polak-Ribiere line search is three majorize-minimize steps on
 *    h(t) = J(f + t d); the paper names the method (section 3.3) and the cost of
 *    one gradient and three criterion evaluations per iteration (section 4.2)
 *    but not the line search.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

enum { PHI_HUBER = 0, PHI_HYPERBOLIC = 1, PHI_QUADRATIC = 2 };

/* ---------------------------------------------------------------- phases */

/* exp(sign * i 2 pi theta), theta in cycles.  theta is reduced to
 * [-0.5, 0.5] by subtracting the nearest integer before the trig call, so the
 * argument of cos/sin never exceeds pi (the exact range reduction the
 * interpolation-free model needs, section 2). */
static void phasor(double theta, double sign, double* re, double* im)
{
    double r = theta - nearbyint(theta);
    double a = 2.0 * OR_PI * r;
    *re = cos(a);
    *im = sign * sin(a);
}

/* ------------------------------------------------- forward model, Eq. ModDirect */

/* y = H f: y_l = (1/N) sum_{n,m} f[n][m] exp(+i2pi(kx_l m + ky_l n)). */
void oracle_forward(int32_t N, int64_t L, const double* kx, const double* ky,
                    const double* f, double* y)
{
    const double inv = 1.0 / (double)N;
#pragma omp parallel for schedule(static)
    for (int64_t l = 0; l < L; ++l) {
        double acc_re = 0.0, acc_im = 0.0;
        for (int32_t n = 0; n < N; ++n) {
            for (int32_t m = 0; m < N; ++m) {
                double er, ei;
                phasor(kx[l] * (double)m + ky[l] * (double)n, +1.0, &er, &ei);
                const double fr = f[2 * ((int64_t)n * N + m)];
                const double fi = f[2 * ((int64_t)n * N + m) + 1];
                acc_re += fr * er - fi * ei;
                acc_im += fr * ei + fi * er;
            }
        }
        y[2 * l] = inv * acc_re;
        y[2 * l + 1] = inv * acc_im;
    }
}

/* x = H^H r: x[n][m] = (1/N) sum_l r_l exp(-i2pi(kx_l m + ky_l n)).  With r = s
 * this is the matrix D of Eq. AnnMatGD (Appendix A). */
static void adjoint_pixel(int32_t N, int64_t L, const double* kx, const double* ky,
                          const double* r, int32_t n, int32_t m, double* out)
{
    double acc_re = 0.0, acc_im = 0.0;
    for (int64_t l = 0; l < L; ++l) {
        double er, ei;
        phasor(kx[l] * (double)m + ky[l] * (double)n, -1.0, &er, &ei);
        acc_re += r[2 * l] * er - r[2 * l + 1] * ei;
        acc_im += r[2 * l] * ei + r[2 * l + 1] * er;
    }
    out[0] = acc_re / (double)N;
    out[1] = acc_im / (double)N;
}

void oracle_adjoint(int32_t N, int64_t L, const double* kx, const double* ky,
                    const double* r, double* x)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < (int64_t)N * N; ++p)
        adjoint_pixel(N, L, kx, ky, r, (int32_t)(p / N), (int32_t)(p % N), &x[2 * p]);
}

/* D at P sampled pixels (n_i, m_i): one output at a time, for checks at sizes
 * where the full adjoint is too slow. */
void oracle_adjoint_at(int32_t N, int64_t L, const double* kx, const double* ky,
                       const double* r, int64_t P, const int32_t* n, const int32_t* m,
                       double* out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < P; ++i)
        adjoint_pixel(N, L, kx, ky, r, n[i], m[i], &out[2 * i]);
}

/* ------------------------------------------------------- G, Eq. AnnMatG */

/* G_{u,v} = (1/N^2) sum_l exp(+i2pi(kx_l u + ky_l v)); u is the kx (column)
 * lag, v the ky (row) lag. */
static void gram_entry(int32_t N, int64_t L, const double* kx, const double* ky,
                       int32_t u, int32_t v, double* out)
{
    double acc_re = 0.0, acc_im = 0.0;
    for (int64_t l = 0; l < L; ++l) {
        double er, ei;
        phasor(kx[l] * (double)u + ky[l] * (double)v, +1.0, &er, &ei);
        acc_re += er;
        acc_im += ei;
    }
    out[0] = acc_re / ((double)N * N);
    out[1] = acc_im / ((double)N * N);
}

/* Full (2N-1) x (2N-1) G, stored G[(v+N-1)*(2N-1) + (u+N-1)]. */
void oracle_gram(int32_t N, int64_t L, const double* kx, const double* ky, double* G)
{
    const int32_t W = 2 * N - 1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < (int64_t)W * W; ++p) {
        const int32_t v = (int32_t)(p / W) - (N - 1);
        const int32_t u = (int32_t)(p % W) - (N - 1);
        gram_entry(N, L, kx, ky, u, v, &G[2 * p]);
    }
}

void oracle_gram_at(int32_t N, int64_t L, const double* kx, const double* ky,
                    int64_t P, const int32_t* u, const int32_t* v, double* out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < P; ++i)
        gram_entry(N, L, kx, ky, u[i], v[i], &out[2 * i]);
}

/* ----------------------------------------- Toeplitz-form pieces, Appendix A/B */

/* Summation bounds of Appendix A: m(w) = max(w, 0), M(w) = N-1 + min(w, 0). */
static int32_t lag_lo(int32_t w) { return w >= 0 ? w : 0; }
static int32_t lag_hi(int32_t N, int32_t w) { return w >= 0 ? N - 1 : N - 1 + w; }

/* Image correlation C_{u,v} = sum_{n,m} f[n][m] conj(f[n-v][m-u]) over the
 * bounds m(.), M(.) (Appendix A, with u the column lag and v the row lag).
 * Stored like G. */
void oracle_autocorr(int32_t N, const double* f, double* C)
{
    const int32_t W = 2 * N - 1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < (int64_t)W * W; ++p) {
        const int32_t v = (int32_t)(p / W) - (N - 1);
        const int32_t u = (int32_t)(p % W) - (N - 1);
        double acc_re = 0.0, acc_im = 0.0;
        for (int32_t n = lag_lo(v); n <= lag_hi(N, v); ++n) {
            for (int32_t m = lag_lo(u); m <= lag_hi(N, u); ++m) {
                const double ar = f[2 * ((int64_t)n * N + m)];
                const double ai = f[2 * ((int64_t)n * N + m) + 1];
                const double br = f[2 * ((int64_t)(n - v) * N + (m - u))];
                const double bi = -f[2 * ((int64_t)(n - v) * N + (m - u)) + 1];
                acc_re += ar * br - ai * bi;
                acc_im += ar * bi + ai * br;
            }
        }
        C[2 * p] = acc_re;
        C[2 * p + 1] = acc_im;
    }
}

/* (T x)[n][m] = sum_{n',m'} x[n'][m'] conj(G_{m-m', n-n'}): the product H^H H x
 * written with the lags of G (Appendix B; the column lag m-m' is G's first
 * index, the kx lag). */
void oracle_toeplitz_apply(int32_t N, const double* G, const double* x, double* Tx)
{
    const int32_t W = 2 * N - 1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < (int64_t)N * N; ++p) {
        const int32_t n = (int32_t)(p / N), m = (int32_t)(p % N);
        double acc_re = 0.0, acc_im = 0.0;
        for (int32_t n2 = 0; n2 < N; ++n2) {
            for (int32_t m2 = 0; m2 < N; ++m2) {
                const int64_t g = (int64_t)(n - n2 + N - 1) * W + (m - m2 + N - 1);
                const double gr = G[2 * g], gi = -G[2 * g + 1];
                const double xr = x[2 * ((int64_t)n2 * N + m2)];
                const double xi = x[2 * ((int64_t)n2 * N + m2) + 1];
                acc_re += gr * xr - gi * xi;
                acc_im += gr * xi + gi * xr;
            }
        }
        Tx[2 * p] = acc_re;
        Tx[2 * p + 1] = acc_im;
    }
}

/* --------------------------------------------- penalties, section 3.3 */

/* phi_alpha(r) for r = |z| >= 0.
 *   Huber (section 3.3):  r^2 if r <= alpha, else 2 alpha r - alpha^2.
 *   hyperbolic (not in the paper): 2 alpha (sqrt(alpha^2 + r^2) - alpha).
 *   quadratic (Hunt, section 3.3): r^2. */
double oracle_phi(int32_t kind, double alpha, double r)
{
    switch (kind) {
    case PHI_HUBER:
        return r <= alpha ? r * r : 2.0 * alpha * r - alpha * alpha;
    case PHI_HYPERBOLIC:
        return 2.0 * alpha * (sqrt(alpha * alpha + r * r) - alpha);
    default:
        return r * r;
    }
}

/* b(r) = phi'(r) / r, the weight of the half-quadratic majorant; finite at 0. */
double oracle_phi_weight(int32_t kind, double alpha, double r)
{
    switch (kind) {
    case PHI_HUBER:
        return r <= alpha ? 2.0 : 2.0 * alpha / r;
    case PHI_HYPERBOLIC:
        return 2.0 * alpha / sqrt(alpha * alpha + r * r);
    default:
        return 2.0;
    }
}

typedef struct {
    double lambda1, alpha1, lambda0, alpha0;
    int32_t kind;
} oracle_reg;

static double cabs2(double re, double im) { return sqrt(re * re + im * im); }

/* R(f) = lambda1 Omega1(f) + lambda0 Omega0(f):
 *   Omega1 = sum_{n<N-1,m} phi(|f[n+1][m]-f[n][m]|) + sum_{n,m<N-1} phi(|f[n][m+1]-f[n][m]|)
 *   Omega0 = sum_{n,m} phi(|f[n][m]|). */
double oracle_penalty(int32_t N, const double* f, const oracle_reg* reg)
{
    double o1 = 0.0, o0 = 0.0;
    for (int32_t n = 0; n < N; ++n) {
        for (int32_t m = 0; m < N; ++m) {
            const int64_t p = (int64_t)n * N + m;
            if (n + 1 < N) {
                const int64_t q = p + N;
                o1 += oracle_phi(reg->kind, reg->alpha1,
                                 cabs2(f[2 * q] - f[2 * p], f[2 * q + 1] - f[2 * p + 1]));
            }
            if (m + 1 < N) {
                const int64_t q = p + 1;
                o1 += oracle_phi(reg->kind, reg->alpha1,
                                 cabs2(f[2 * q] - f[2 * p], f[2 * q + 1] - f[2 * p + 1]));
            }
            o0 += oracle_phi(reg->kind, reg->alpha0, cabs2(f[2 * p], f[2 * p + 1]));
        }
    }
    return reg->lambda1 * o1 + reg->lambda0 * o0;
}

/* Adds the gradient of R to g.  For an edge from pixel p to pixel q with
 * z = f_q - f_p, d phi(|z|) = b(|z|) z, added at q and subtracted at p. */
void oracle_penalty_grad(int32_t N, const double* f, const oracle_reg* reg, double* g)
{
    for (int32_t n = 0; n < N; ++n) {
        for (int32_t m = 0; m < N; ++m) {
            const int64_t p = (int64_t)n * N + m;
            for (int dir = 0; dir < 2; ++dir) {
                int64_t q;
                if (dir == 0) {
                    if (n + 1 >= N) continue;
                    q = p + N;
                } else {
                    if (m + 1 >= N) continue;
                    q = p + 1;
                }
                const double zr = f[2 * q] - f[2 * p], zi = f[2 * q + 1] - f[2 * p + 1];
                const double w = reg->lambda1 * oracle_phi_weight(reg->kind, reg->alpha1, cabs2(zr, zi));
                g[2 * q] += w * zr;
                g[2 * q + 1] += w * zi;
                g[2 * p] -= w * zr;
                g[2 * p + 1] -= w * zi;
            }
            const double w0 = reg->lambda0 *
                              oracle_phi_weight(reg->kind, reg->alpha0, cabs2(f[2 * p], f[2 * p + 1]));
            g[2 * p] += w0 * f[2 * p];
            g[2 * p + 1] += w0 * f[2 * p + 1];
        }
    }
}

/* ------------------------------------------- criterion, Eq. CritLS + R */

/* J(f) = ||s - H f||^2 + R(f), written out directly (no D, no G). */
double oracle_objective(int32_t N, int64_t L, const double* kx, const double* ky,
                        const double* s, const double* f, const oracle_reg* reg)
{
    double* y = (double*)malloc(sizeof(double) * 2 * (size_t)L);
    oracle_forward(N, L, kx, ky, f, y);
    double ls = 0.0;
    for (int64_t l = 0; l < L; ++l) {
        const double dr = s[2 * l] - y[2 * l], di = s[2 * l + 1] - y[2 * l + 1];
        ls += dr * dr + di * di;
    }
    free(y);
    return ls + oracle_penalty(N, f, reg);
}

/* grad J(f) = 2 H^H (H f - s) + grad R(f).  Also returns the data part g_ls and
 * J(f), both from the same forward product. */
static double gradient_parts(int32_t N, int64_t L, const double* kx, const double* ky,
                             const double* s, const double* f, const oracle_reg* reg,
                             double* g, double* g_ls, double* y)
{
    oracle_forward(N, L, kx, ky, f, y);
    double ls = 0.0;
    for (int64_t l = 0; l < L; ++l) {
        y[2 * l] -= s[2 * l];
        y[2 * l + 1] -= s[2 * l + 1];
        ls += y[2 * l] * y[2 * l] + y[2 * l + 1] * y[2 * l + 1];
    }
    oracle_adjoint(N, L, kx, ky, y, g_ls);
    const int64_t P = (int64_t)N * N;
    for (int64_t i = 0; i < 2 * P; ++i) {
        g_ls[i] *= 2.0;
        g[i] = g_ls[i];
    }
    oracle_penalty_grad(N, f, reg, g);
    return ls + oracle_penalty(N, f, reg);
}

void oracle_gradient(int32_t N, int64_t L, const double* kx, const double* ky,
                     const double* s, const double* f, const oracle_reg* reg, double* g)
{
    const int64_t P = (int64_t)N * N;
    double* g_ls = (double*)malloc(sizeof(double) * 2 * (size_t)P);
    double* y = (double*)malloc(sizeof(double) * 2 * (size_t)L);
    gradient_parts(N, L, kx, ky, s, f, reg, g, g_ls, y);
    free(g_ls);
    free(y);
}

/* ------------------------------------------------ line search helpers */

/* Penalty part of h'(t) and of the majorant curvature for the step f + t d:
 *   num += sum_e lambda b(|z_e + t w_e|) Re(conj(z_e + t w_e) w_e)
 *   den += sum_e lambda b(|z_e + t w_e|) |w_e|^2
 * over the edge differences (Omega1) and the pixels (Omega0). */
static void penalty_line_terms(int32_t N, const double* f, const double* d, double t,
                               const oracle_reg* reg, double* num, double* den)
{
    double a = 0.0, b = 0.0;
    for (int32_t n = 0; n < N; ++n) {
        for (int32_t m = 0; m < N; ++m) {
            const int64_t p = (int64_t)n * N + m;
            for (int dir = 0; dir < 2; ++dir) {
                int64_t q;
                if (dir == 0) {
                    if (n + 1 >= N) continue;
                    q = p + N;
                } else {
                    if (m + 1 >= N) continue;
                    q = p + 1;
                }
                const double zr = f[2 * q] - f[2 * p], zi = f[2 * q + 1] - f[2 * p + 1];
                const double wr = d[2 * q] - d[2 * p], wi = d[2 * q + 1] - d[2 * p + 1];
                const double xr = zr + t * wr, xi = zi + t * wi;
                const double wt = reg->lambda1 * oracle_phi_weight(reg->kind, reg->alpha1, cabs2(xr, xi));
                a += wt * (xr * wr + xi * wi);
                b += wt * (wr * wr + wi * wi);
            }
            const double zr = f[2 * p], zi = f[2 * p + 1];
            const double wr = d[2 * p], wi = d[2 * p + 1];
            const double xr = zr + t * wr, xi = zi + t * wi;
            const double wt = reg->lambda0 * oracle_phi_weight(reg->kind, reg->alpha0, cabs2(xr, xi));
            a += wt * (xr * wr + xi * wi);
            b += wt * (wr * wr + wi * wi);
        }
    }
    *num += a;
    *den += b;
}

static double re_dot(int64_t n, const double* a, const double* b)
{
    double acc = 0.0;
    for (int64_t i = 0; i < n; ++i) acc += a[2 * i] * b[2 * i] + a[2 * i + 1] * b[2 * i + 1];
    return acc;
}

/* ------------------------------------------------------------ minimiser */

/* Pseudo-conjugate gradient with the Polak-Ribiere correction (section 3.3):
 *   g0 = grad J(x0), d0 = -g0
 *   per iteration:
 *     h(t) = J(f + t d) = J_LS(f) + q1 t + q2 t^2 + R(f + t d),
 *       q1 = Re<d, g_ls>, q2 = ||H d||^2;
 *     three majorize-minimize steps from t = 0:
 *       t <- t - h'(t) / (2 q2 + sum lambda b(|z + t w|) |w|^2);
 *     f <- f + t d; g' = grad J(f);
 *     beta = max(0, Re<g', g' - g> / <g, g>); d <- -g' + beta d;
 *     if Re<g', d> >= 0 then d <- -g'   (restart on a non-descent direction).
 * J_hist[0] = J(x0), J_hist[k+1] = J after iteration k; t_hist[k] the step. */
int oracle_solve(int32_t N, int64_t L, const double* kx, const double* ky,
                 const double* s, const oracle_reg* reg, const double* x0,
                 int32_t iters, double* x_out, double* J_hist, double* t_hist)
{
    const int64_t P = (int64_t)N * N;
    double* f = (double*)malloc(sizeof(double) * 2 * (size_t)P);
    double* g = (double*)malloc(sizeof(double) * 2 * (size_t)P);
    double* gn = (double*)malloc(sizeof(double) * 2 * (size_t)P);
    double* g_ls = (double*)malloc(sizeof(double) * 2 * (size_t)P);
    double* d = (double*)malloc(sizeof(double) * 2 * (size_t)P);
    double* y = (double*)malloc(sizeof(double) * 2 * (size_t)L);
    if (!f || !g || !gn || !g_ls || !d || !y) {
        free(f); free(g); free(gn); free(g_ls); free(d); free(y);
        return -2;
    }
    memcpy(f, x0, sizeof(double) * 2 * (size_t)P);

    double J = gradient_parts(N, L, kx, ky, s, f, reg, g, g_ls, y);
    if (J_hist) J_hist[0] = J;
    for (int64_t i = 0; i < 2 * P; ++i) d[i] = -g[i];

    for (int32_t k = 0; k < iters; ++k) {
        /* q2 = ||H d||^2, q1 = Re<d, g_ls> */
        oracle_forward(N, L, kx, ky, d, y);
        double q2 = 0.0;
        for (int64_t l = 0; l < L; ++l) q2 += y[2 * l] * y[2 * l] + y[2 * l + 1] * y[2 * l + 1];
        const double q1 = re_dot(P, d, g_ls);

        double t = 0.0;
        for (int j = 0; j < 3; ++j) {
            double num = q1 + 2.0 * q2 * t, den = 2.0 * q2;
            penalty_line_terms(N, f, d, t, reg, &num, &den);
            if (den > 0.0) t -= num / den;
        }
        if (t_hist) t_hist[k] = t;
        for (int64_t i = 0; i < 2 * P; ++i) f[i] += t * d[i];

        J = gradient_parts(N, L, kx, ky, s, f, reg, gn, g_ls, y);
        if (J_hist) J_hist[k + 1] = J;

        const double gg_old = re_dot(P, g, g);
        double num_b = 0.0;
        for (int64_t i = 0; i < 2 * P; ++i) num_b += gn[i] * (gn[i] - g[i]);
        double beta = gg_old > 0.0 ? num_b / gg_old : 0.0;
        if (beta < 0.0) beta = 0.0;
        for (int64_t i = 0; i < 2 * P; ++i) d[i] = -gn[i] + beta * d[i];
        if (re_dot(P, gn, d) >= 0.0)
            for (int64_t i = 0; i < 2 * P; ++i) d[i] = -gn[i];
        memcpy(g, gn, sizeof(double) * 2 * (size_t)P);
    }
    memcpy(x_out, f, sizeof(double) * 2 * (size_t)P);
    free(f); free(g); free(gn); free(g_ls); free(d); free(y);
    return 0;
}

/* Number of OpenMP threads the oracle runs on (1 without OpenMP). */
#ifdef _OPENMP
#include <omp.h>
int oracle_num_threads(void) { return omp_get_max_threads(); }
#else
int oracle_num_threads(void) { return 1; }
#endif
