/*
 * ks_oracle.c -- plain, slow FP64 reference for the adjoint-descent step of the
 * Jacobian-free variational method for connecting orbits (Ashtari & Schneider,
 * arXiv 2301.11704), applied to the Kuramoto-Sivashinsky equation (KSE).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * Every routine is written as the plain definition (naive DFT sums, the two
 * explicit trig sums that define the rational-Chebyshev derivative, explicit
 * loops over sections and modes), in FP64, with OpenMP only over independent
 * sections or modes.
 *
 * Conventions (Sec. V.C.1 "Spectral discretization"):
 *   N   Fourier modes / grid points per time section, x_n = n L / N.
 *   M   interior rational-Chebyshev sections; P = M + 1; rows m = 0..P.
 *       Row 0 is s -> +inf (u_+), row P is s -> -inf (u_-)   (eq. t_grid).
 *   A section is stored spectrally as N/2 complex coefficients u^_j,
 *   j = 0..N/2-1; u^_{-j} = conj(u^_j) for a real field; the Nyquist
 *   coefficient j = -N/2 is held at zero.
 *   A curve is a row-major array [P+1][N/2] of complex coefficients.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define KO_PI 3.14159265358979323846264338327950288

int ko_version(void) { return 1; }

int ko_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Fourier direction (Sec. V.C.1)                                            */
/* ------------------------------------------------------------------------ */

/* wavenumber k_j = 2 pi j / L */
static double kwave(int j, double L) { return 2.0 * KO_PI * (double)j / L; }

/* Table of e^{+2 pi i t / N}, t = 0..N-1; every phase of a transform is
 * looked up by the exact integer t = (j n mod N). */
static cplx *phase_table(int N)
{
    cplx *tab = malloc(sizeof(cplx) * N);
    for (int t = 0; t < N; ++t) {
        double a = 2.0 * KO_PI * (double)t / (double)N;
        tab[t] = cos(a) + I * sin(a);
    }
    return tab;
}

static int imod(long a, long n)
{
    long r = a % n;
    return (int)(r < 0 ? r + n : r);
}

/* Forward transform of one real section:
 *   u^_j = (1/N) sum_n u_n exp(-2 pi i j n / N),   j = 0..N/2-1.
 * Inverse of the expansion u(x_n) = sum_j u^_j exp(i j 2 pi x_n / L). */
void ko_fwd(int N, const double *u, cplx *uh)
{
    cplx *ph = phase_table(N);
    for (int j = 0; j < N / 2; ++j) {
        cplx acc = 0.0;
        for (int n = 0; n < N; ++n)
            acc += u[n] * conj(ph[imod((long)j * n, N)]);
        uh[j] = acc / (double)N;
    }
    free(ph);
}

/* Inverse transform: u(x_n) = sum_{j=-N/2}^{N/2-1} u^_j exp(i j 2 pi n / N)
 * with u^_{-j} = conj(u^_j) and the Nyquist coefficient u^_{-N/2} = 0. */
void ko_inv(int N, const cplx *uh, double *u)
{
    cplx *ph = phase_table(N);
    for (int n = 0; n < N; ++n) {
        cplx acc = 0.0;
        for (int j = -N / 2 + 1; j <= N / 2 - 1; ++j) {
            cplx c = (j >= 0) ? uh[j] : conj(uh[-j]);
            acc += c * ph[imod((long)j * n, N)];
        }
        u[n] = creal(acc);
    }
    free(ph);
}

/* KSE right-hand side (eq. KSE with nu = 1), pseudo-spectrally:
 *   f = -u u_x - u_xx - u_xxxx,  u u_x written as (1/2) d/dx (u^2),
 *   d^q/dx^q -> (i k_j)^q  (Hadamard product with D_x^(q)).
 * The product u^2 is formed on the grid x_n. */
void ko_rhs(int N, double L, const cplx *uh, cplx *fh)
{
    double *u = malloc(sizeof(double) * N);
    cplx *wh = malloc(sizeof(cplx) * (N / 2));
    ko_inv(N, uh, u);
    for (int n = 0; n < N; ++n) u[n] = u[n] * u[n];
    ko_fwd(N, u, wh);
    for (int j = 0; j < N / 2; ++j) {
        double k = kwave(j, L);
        cplx ik = I * k;
        /* -(1/2)(ik) w^  - (ik)^2 u^  - (ik)^4 u^ */
        fh[j] = -0.5 * ik * wh[j] - (ik * ik) * uh[j] - (ik * ik * ik * ik) * uh[j];
    }
    free(u);
    free(wh);
}

/* Directional derivative of f at u along v (App. A, eq. KSE_directional_derivative,
 * spatial part):  Df(u) v = -d/dx (u v) - v_xx - v_xxxx. */
void ko_jac_apply(int N, double L, const cplx *uh, const cplx *vh, cplx *out)
{
    double *u = malloc(sizeof(double) * N);
    double *v = malloc(sizeof(double) * N);
    cplx *ph = malloc(sizeof(cplx) * (N / 2));
    ko_inv(N, uh, u);
    ko_inv(N, vh, v);
    for (int n = 0; n < N; ++n) u[n] = u[n] * v[n];
    ko_fwd(N, u, ph);
    for (int j = 0; j < N / 2; ++j) {
        cplx ik = I * kwave(j, L);
        out[j] = -ik * ph[j] - (ik * ik) * vh[j] - (ik * ik * ik * ik) * vh[j];
    }
    free(u);
    free(v);
    free(ph);
}

/* Spatial part of the adjoint operator (eq. KSE_G / App. A):
 *   (Df(u))^T r = u r_x - r_xx - r_xxxx. */
void ko_jac_adjoint_apply(int N, double L, const cplx *uh, const cplx *rh, cplx *out)
{
    double *u = malloc(sizeof(double) * N);
    double *rx = malloc(sizeof(double) * N);
    cplx *tmp = malloc(sizeof(cplx) * (N / 2));
    ko_inv(N, uh, u);
    for (int j = 0; j < N / 2; ++j) tmp[j] = I * kwave(j, L) * rh[j];
    ko_inv(N, tmp, rx);
    for (int n = 0; n < N; ++n) u[n] = u[n] * rx[n];
    ko_fwd(N, u, tmp);
    for (int j = 0; j < N / 2; ++j) {
        cplx ik = I * kwave(j, L);
        out[j] = tmp[j] - (ik * ik) * rh[j] - (ik * ik * ik * ik) * rh[j];
    }
    free(u);
    free(rx);
    free(tmp);
}

/* ------------------------------------------------------------------------ */
/* Temporal direction: rational Chebyshev functions (Sec. IV)               */
/* ------------------------------------------------------------------------ */

/* c-bar of eq. c_bar */
static double cbar(int j, int P) { return (j == 0 || j == P) ? 2.0 : 1.0; }

/* cos(pi t / P) and sin(pi t / P) looked up by the integer t = (m k mod 2P) */
static double cos_idx(long t, int P) { return cos(KO_PI * (double)imod(t, 2L * P) / (double)P); }
static double sin_idx(long t, int P) { return sin(KO_PI * (double)imod(t, 2L * P) / (double)P); }

/* The same values tabulated for t = 0..2P-1 (index with imod(m k, 2P)). */
typedef struct { double *c, *s; int P; } trig_tab;
static trig_tab trig_table(int P)
{
    trig_tab t;
    t.P = P;
    t.c = malloc(sizeof(double) * 2 * P);
    t.s = malloc(sizeof(double) * 2 * P);
    for (int i = 0; i < 2 * P; ++i) { t.c[i] = cos_idx(i, P); t.s[i] = sin_idx(i, P); }
    return t;
}
static void trig_free(trig_tab t) { free(t.c); free(t.s); }
#define TC(tb, i) ((tb).c[imod((i), 2L * (tb).P)])
#define TS(tb, i) ((tb).s[imod((i), 2L * (tb).P)])

/* Collocation grid (eq. t_grid, eq. Rational_domain):
 *   theta_m = m pi / (M+1),  s_m = s0 + S cot(theta_m),  m = 1..M,
 *   s_0 = +inf, s_{M+1} = -inf.
 * Quadrature weights for integrals over s (trapezoid rule in theta mapped
 * to s, ds = -S / sin^2(theta) dtheta):  w_m = (pi/(M+1)) S / sin^2(theta_m)
 * for interior m; the end weights are 0 (the integrands used vanish there). */
void ko_grid(int M, double S, double s0, double *theta, double *s, double *w)
{
    int P = M + 1;
    for (int m = 0; m <= P; ++m) {
        double th = KO_PI * (double)m / (double)P;
        if (theta) theta[m] = th;
        if (m == 0 || m == P) {
            if (s) s[m] = (m == 0) ? INFINITY : -INFINITY;
            if (w) w[m] = 0.0;
        } else {
            double sn = sin_idx(m, P), cs = cos_idx(m, P);
            if (s) s[m] = s0 + S * cs / sn;
            if (w) w[m] = (KO_PI / (double)P) * S / (sn * sn);
        }
    }
}

/* Expansion coefficients (eq. rational_coeffs):
 *   c_k = 2/((M+1) cbar_k) sum_{m=0}^{M+1} q(s_m)/cbar_m cos(m k pi/(M+1)). */
void ko_dt_coeffs(int M, const double *q, double *c)
{
    int P = M + 1;
    trig_tab tb = trig_table(P);
    for (int k = 0; k <= P; ++k) {
        double acc = 0.0;
        for (int m = 0; m <= P; ++m) acc += q[m] / cbar(m, P) * TC(tb, (long)m * k);
        c[k] = 2.0 / ((double)P * cbar(k, P)) * acc;
    }
    trig_free(tb);
}

/* Differentiation along s (eq. rational_diff_matrix), evaluated as its two
 * sums: first the coefficients c_k of eq. rational_coeffs, then
 *   (D_t q)_j = (1/S) sin^2(j pi/(M+1)) sum_{k=0}^{M+1} k c_k sin(k j pi/(M+1)).
 * Equal to the matrix of eq. rational_diff_matrix applied to q. */
void ko_dt_apply(int M, double S, const double *q, double *d)
{
    int P = M + 1;
    double *c = malloc(sizeof(double) * (P + 1));
    trig_tab tb = trig_table(P);
    ko_dt_coeffs(M, q, c);
    for (int j = 0; j <= P; ++j) {
        double acc = 0.0;
        for (int k = 0; k <= P; ++k) acc += (double)k * c[k] * TS(tb, (long)k * j);
        double sj = TS(tb, j);
        d[j] = sj * sj / S * acc;
    }
    trig_free(tb);
    free(c);
}

/* Transpose of eq. rational_diff_matrix, factor by factor:
 *   (D_t^T y)_m = 2/(S (M+1) cbar_m) sum_k (k / cbar_k) cos(m k pi/(M+1))
 *                  * [ sum_j sin^2(j pi/(M+1)) sin(k j pi/(M+1)) y_j ]. */
void ko_dtT_apply(int M, double S, const double *y, double *z)
{
    int P = M + 1;
    double *b = malloc(sizeof(double) * (P + 1));
    trig_tab tb = trig_table(P);
    for (int k = 0; k <= P; ++k) {
        double acc = 0.0;
        for (int j = 0; j <= P; ++j) {
            double sj = TS(tb, j);
            acc += sj * sj * TS(tb, (long)k * j) * y[j];
        }
        b[k] = acc;
    }
    for (int m = 0; m <= P; ++m) {
        double acc = 0.0;
        for (int k = 0; k <= P; ++k) acc += (double)k / cbar(k, P) * TC(tb, (long)m * k) * b[k];
        z[m] = 2.0 / (S * (double)P * cbar(m, P)) * acc;
    }
    trig_free(tb);
    free(b);
}

/* The matrix of eq. rational_diff_matrix, entry by entry (O(M^3); tests only). */
void ko_dt_matrix(int M, double S, double *D)
{
    int P = M + 1;
    trig_tab tb = trig_table(P);
    for (int j = 0; j <= P; ++j) {
        double sj = TS(tb, j);
        for (int m = 0; m <= P; ++m) {
            double acc = 0.0;
            for (int k = 0; k <= P; ++k)
                acc += (double)k / (cbar(m, P) * cbar(k, P)) * TC(tb, (long)m * k) * TS(tb, (long)k * j);
            D[(long)j * (P + 1) + m] = 2.0 / (S * (double)P) * sj * sj * acc;
        }
    }
    trig_free(tb);
}

/* Row j of the matrix of eq. rational_diff_matrix, each entry by its explicit
 * k-sum (O(M^2) per row; used to check sampled sections of large curves). */
void ko_dt_row(int M, double S, int j, double *row)
{
    int P = M + 1;
    trig_tab tb = trig_table(P);
    double sj = TS(tb, j);
#pragma omp parallel for schedule(static)
    for (int m = 0; m <= P; ++m) {
        double acc = 0.0;
        for (int k = 0; k <= P; ++k)
            acc += (double)k / (cbar(m, P) * cbar(k, P)) * TC(tb, (long)m * k) * TS(tb, (long)k * j);
        row[m] = 2.0 / (S * (double)P) * sj * sj * acc;
    }
    trig_free(tb);
}

/* Apply D_t (or D_t^T) to every real and imaginary column of a curve. */
static void curve_dt(int M, int N, double S, const cplx *X, cplx *Y, int transpose)
{
    int P = M + 1, H = N / 2;
#pragma omp parallel
    {
        double *q = calloc(P + 1, sizeof(double));
        double *d = calloc(P + 1, sizeof(double));
        double *e = calloc(P + 1, sizeof(double));
#pragma omp for schedule(static)
        for (int j = 0; j < H; ++j) {
            for (int m = 0; m <= P; ++m) q[m] = creal(X[(long)m * H + j]);
            if (transpose) ko_dtT_apply(M, S, q, d); else ko_dt_apply(M, S, q, d);
            for (int m = 0; m <= P; ++m) q[m] = cimag(X[(long)m * H + j]);
            if (transpose) ko_dtT_apply(M, S, q, e); else ko_dt_apply(M, S, q, e);
            for (int m = 0; m <= P; ++m) Y[(long)m * H + j] = d[m] + I * e[m];
        }
        free(q);
        free(d);
        free(e);
    }
}

/* ------------------------------------------------------------------------ */
/* The curve: residual, adjoint, cost (Sec. II, III, V.A, V.C)              */
/* ------------------------------------------------------------------------ */

/* Residual (eq. residual_definition, eq. KSE_residual):
 *   r = f(u) - lambda dU/ds,   dU/ds = D_t u^ (left multiplication, Sec. V.C.1).
 * lambda = 1 is the method as published; lambda scales the s-derivative.
 * Rows 0 and M+1 of r are identically zero (asymptotic conditions, Sec. III).
 * Dtu (optional) receives D_t u^ without the lambda factor. */
void ko_curve_residual(int M, int N, double L, double S, double lambda,
                       const cplx *U, cplx *R, cplx *Dtu)
{
    int P = M + 1, H = N / 2;
    cplx *D = malloc(sizeof(cplx) * (long)(P + 1) * H);
    curve_dt(M, N, S, U, D, 0);
#pragma omp parallel
    {
        cplx *fh = malloc(sizeof(cplx) * H);
#pragma omp for schedule(static)
        for (int m = 0; m <= P; ++m) {
            ko_rhs(N, L, U + (long)m * H, fh);
            for (int j = 0; j < H; ++j) {
                cplx r = fh[j] - lambda * D[(long)m * H + j];
                R[(long)m * H + j] = (m == 0 || m == P) ? 0.0 : r;
            }
        }
        free(fh);
    }
    if (Dtu) memcpy(Dtu, D, sizeof(cplx) * (long)(P + 1) * H);
    free(D);
}

/* Residual of the f(u) part only for each section: used to check that the
 * end sections are equilibria, f(u_+-) = 0 (eq. connecting_orbit_def). */
void ko_curve_rhs(int M, int N, double L, const cplx *U, cplx *F)
{
    int P = M + 1, H = N / 2;
#pragma omp parallel for schedule(static)
    for (int m = 0; m <= P; ++m) ko_rhs(N, L, U + (long)m * H, F + (long)m * H);
}

/* Linearisation of the residual along G (eq. directional_derivative,
 * eq. KSE_directional_derivative):  L(u;G) = Df(u) G - lambda D_t G,
 * zero at the end rows. */
void ko_curve_linearised(int M, int N, double L, double S, double lambda,
                         const cplx *U, const cplx *G, cplx *out)
{
    int P = M + 1, H = N / 2;
    cplx *D = malloc(sizeof(cplx) * (long)(P + 1) * H);
    curve_dt(M, N, S, G, D, 0);
#pragma omp parallel
    {
        cplx *t = malloc(sizeof(cplx) * H);
#pragma omp for schedule(static)
        for (int m = 0; m <= P; ++m) {
            ko_jac_apply(N, L, U + (long)m * H, G + (long)m * H, t);
            for (int j = 0; j < H; ++j) {
                cplx v = t[j] - lambda * D[(long)m * H + j];
                out[(long)m * H + j] = (m == 0 || m == P) ? 0.0 : v;
            }
        }
        free(t);
    }
    free(D);
}

/* Adjoint operator and descent direction (eq. KSE_G):
 *   L^dagger(u;r) = lambda dr/ds + u r_x - r_xx - r_xxxx,   G = -L^dagger.
 * mode 0 (as published): the s-term is lambda D_t r.
 * mode 1 (exact adjoint of the discretised residual under the quadrature
 *   inner product <a,b>_W = dx sum_m w_m sum_n a b):  the s-term is
 *   -lambda W^{-1} D_t^T W r.
 * G vanishes at the end rows (Sec. III, Sec. V.C.1).  A (optional) receives
 * the spatial part (Df)^T r. */
void ko_curve_adjoint(int M, int N, double L, double S, double lambda, int mode,
                      const cplx *U, const cplx *R, cplx *G, cplx *A)
{
    int P = M + 1, H = N / 2;
    cplx *E = malloc(sizeof(cplx) * (long)(P + 1) * H);
    if (mode == 0) {
        curve_dt(M, N, S, R, E, 0);
        for (long i = 0; i < (long)(P + 1) * H; ++i) E[i] *= lambda;
    } else {
        double *w = malloc(sizeof(double) * (P + 1));
        cplx *Y = malloc(sizeof(cplx) * (long)(P + 1) * H);
        ko_grid(M, S, 0.0, NULL, NULL, w);
        for (int m = 0; m <= P; ++m)
            for (int j = 0; j < H; ++j)
                Y[(long)m * H + j] = (m == 0 || m == P) ? 0.0 : w[m] * R[(long)m * H + j];
        curve_dt(M, N, S, Y, E, 1);
        for (int m = 0; m <= P; ++m)
            for (int j = 0; j < H; ++j)
                E[(long)m * H + j] = (m == 0 || m == P) ? 0.0 : -lambda * E[(long)m * H + j] / w[m];
        free(w);
        free(Y);
    }
#pragma omp parallel
    {
        cplx *a = malloc(sizeof(cplx) * H);
#pragma omp for schedule(static)
        for (int m = 0; m <= P; ++m) {
            ko_jac_adjoint_apply(N, L, U + (long)m * H, R + (long)m * H, a);
            for (int j = 0; j < H; ++j) {
                long i = (long)m * H + j;
                if (A) A[i] = a[j];
                G[i] = (m == 0 || m == P) ? 0.0 : -(a[j] + E[i]);
            }
        }
        free(a);
    }
    free(E);
}

/* Squared spatial norm of one section on the grid: |q|^2 = dx sum_n q_n^2
 * (the norm |.| of eq. J_arc, integral over Omega as the grid sum). */
static double section_norm2(int N, double L, const cplx *qh)
{
    double *q = malloc(sizeof(double) * N);
    ko_inv(N, qh, q);
    double acc = 0.0;
    for (int n = 0; n < N; ++n) acc += q[n] * q[n];
    free(q);
    return acc * (L / (double)N);
}

static double section_dot(int N, double L, const cplx *ah, const cplx *bh)
{
    double *a = malloc(sizeof(double) * N);
    double *b = malloc(sizeof(double) * N);
    ko_inv(N, ah, a);
    ko_inv(N, bh, b);
    double acc = 0.0;
    for (int n = 0; n < N; ++n) acc += a[n] * b[n];
    free(a);
    free(b);
    return acc * (L / (double)N);
}

/* Scalars of one evaluation, with the quadrature w_m over s (ko_grid) and
 * the grid sum over x:
 *   out[0] J^2     = sum_m w_m |r_m|^2                    (eq. cost_function_general)
 *   out[1] J_arc   = sum_m w_m |r_m| |lambda d_m| / sum_m w_m |lambda d_m|   (eq. J_arc)
 *   out[2] dJ^2/dlambda = -2 sum_m w_m <d_m, r_m>          (d = D_t u)
 *   out[3] |G|_W^2 = sum_m w_m |G_m|^2   (only if G != NULL, else 0)
 *   out[4] |lambda D_t u|_W  (the scale of the s-derivative, for J_rel)
 */
void ko_curve_scalars(int M, int N, double L, double S, double lambda,
                      const cplx *R, const cplx *Dtu, const cplx *G, double *out)
{
    int P = M + 1, H = N / 2;
    double *w = malloc(sizeof(double) * (P + 1));
    double *rr = calloc(P + 1, sizeof(double));
    double *dd = calloc(P + 1, sizeof(double));
    double *dr = calloc(P + 1, sizeof(double));
    double *gg = calloc(P + 1, sizeof(double));
    ko_grid(M, S, 0.0, NULL, NULL, w);
#pragma omp parallel for schedule(static)
    for (int m = 1; m <= M; ++m) {
        rr[m] = section_norm2(N, L, R + (long)m * H);
        dd[m] = section_norm2(N, L, Dtu + (long)m * H);
        dr[m] = section_dot(N, L, Dtu + (long)m * H, R + (long)m * H);
        if (G) gg[m] = section_norm2(N, L, G + (long)m * H);
    }
    double J2 = 0, num = 0, den = 0, dl = 0, G2 = 0, D2 = 0;
    for (int m = 1; m <= M; ++m) {
        J2 += w[m] * rr[m];
        num += w[m] * sqrt(rr[m]) * fabs(lambda) * sqrt(dd[m]);
        den += w[m] * fabs(lambda) * sqrt(dd[m]);
        dl += w[m] * dr[m];
        G2 += w[m] * gg[m];
        D2 += w[m] * lambda * lambda * dd[m];
    }
    out[0] = J2;
    out[1] = den > 0 ? num / den : 0.0;
    out[2] = -2.0 * dl;
    out[3] = G2;
    out[4] = sqrt(D2);
    free(w);
    free(rr);
    free(dd);
    free(dr);
    free(gg);
}

/* |X|_W^2 = sum_{m=1}^{M} w_m |X_m|^2 over the interior rows. */
double ko_curve_norm2_W(int M, int N, double L, double S, const cplx *X)
{
    int P = M + 1, H = N / 2;
    double *w = malloc(sizeof(double) * (P + 1));
    double *xx = calloc(P + 1, sizeof(double));
    ko_grid(M, S, 0.0, NULL, NULL, w);
#pragma omp parallel for schedule(static)
    for (int m = 1; m <= M; ++m) xx[m] = section_norm2(N, L, X + (long)m * H);
    double acc = 0.0;
    for (int m = 1; m <= M; ++m) acc += w[m] * xx[m];
    free(w);
    free(xx);
    return acc;
}

/* ------------------------------------------------------------------------ */
/* Full-linear-implicit stepping (Sec. V.C.3)                                */
/* ------------------------------------------------------------------------ */
/*
 * The paper steps the descent by semi-implicit forward Euler, treating the
 * terms of G that are linear in u implicitly.  On the interior rows the linear
 * part of the paper's G (eq. KSE_G with r of eq. KSE_residual) is
 *     Lin_j u = (lambda^2 Dt~^2 - a_j^2) u,    a_j = k_j^4 - k_j^2,
 * per spatial mode j, where Dt~ is the interior block (rows and columns
 * 1..M) of the matrix of eq. rational_diff_matrix: the end rows of u are
 * fixed and r's end rows are zero.  The step
 *     (I - dtau Lin_j) u_new = u + dtau (G(u) - Lin_j u)
 * is taken in its equivalent increment form
 *     (I (1 + dtau a_j^2) - dtau lambda^2 Dt~^2) delta_j = dtau G_j,
 *     u_new = u + delta,
 * by an LU factorisation with partial pivoting of each mode's M x M matrix
 * (factored once per (dtau, lambda)).  With the discrete adjoint the same
 * operator is applied to its G.
 */
typedef struct {
    int M, H;
    double L, dtau, lambda;
    double *D2;   /* Dt~^2, M x M row-major */
    double *F;    /* H LU factors, M x M each */
    int *piv;     /* H x M row interchanges */
} implicit_ops;

static implicit_ops *implicit_new(int M, int H, double L, double S)
{
    int P = M + 1;
    implicit_ops *im = calloc(1, sizeof(implicit_ops));
    im->M = M; im->H = H; im->L = L; im->dtau = -1.0; im->lambda = 0.0;
    double *Dfull = malloc(sizeof(double) * (size_t)(P + 1) * (P + 1));
    ko_dt_matrix(M, S, Dfull);
    im->D2 = calloc((size_t)M * M, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < M; ++i)
        for (int k = 0; k < M; ++k) {
            double acc = 0.0;
            for (int l = 0; l < M; ++l)
                acc += Dfull[(long)(i + 1) * (P + 1) + (l + 1)] * Dfull[(long)(l + 1) * (P + 1) + (k + 1)];
            im->D2[(long)i * M + k] = acc;
        }
    free(Dfull);
    im->F = malloc(sizeof(double) * (size_t)H * M * M);
    im->piv = malloc(sizeof(int) * (size_t)H * M);
    return im;
}

static void implicit_free(implicit_ops *im)
{
    if (!im) return;
    free(im->D2); free(im->F); free(im->piv); free(im);
}

/* Gaussian elimination with partial pivoting, in place: the multipliers below
 * the diagonal, U on and above it, piv[c] the row swapped into row c. */
static void lu_factor(int n, double *A, int *piv)
{
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[(long)r * n + c]) > fabs(A[(long)p * n + c])) p = r;
        piv[c] = p;
        if (p != c)
            for (int k = 0; k < n; ++k) {
                double t = A[(long)c * n + k];
                A[(long)c * n + k] = A[(long)p * n + k];
                A[(long)p * n + k] = t;
            }
        for (int r = c + 1; r < n; ++r) {
            double f = A[(long)r * n + c] / A[(long)c * n + c];
            A[(long)r * n + c] = f;
            for (int k = c + 1; k < n; ++k) A[(long)r * n + k] -= f * A[(long)c * n + k];
        }
    }
}

/* Solves with the factors of lu_factor: row interchanges, L y = b, U x = y. */
static void lu_apply(int n, const double *A, const int *piv, double *b)
{
    for (int c = 0; c < n; ++c) {
        double t = b[c]; b[c] = b[piv[c]]; b[piv[c]] = t;
    }
    for (int r = 0; r < n; ++r) {
        double acc = b[r];
        for (int c = 0; c < r; ++c) acc -= A[(long)r * n + c] * b[c];
        b[r] = acc;
    }
    for (int r = n - 1; r >= 0; --r) {
        double acc = b[r];
        for (int k = r + 1; k < n; ++k) acc -= A[(long)r * n + k] * b[k];
        b[r] = acc / A[(long)r * n + r];
    }
}

static void implicit_update(implicit_ops *im, double dtau, double lambda, const cplx *G, cplx *U)
{
    const int M = im->M, H = im->H;
    if (im->dtau != dtau || im->lambda != lambda) {
#pragma omp parallel for schedule(dynamic)
        for (int j = 0; j < H; ++j) {
            double a = pow(kwave(j, im->L), 4) - pow(kwave(j, im->L), 2);
            double *A = im->F + (size_t)j * M * M;
            for (int i = 0; i < M; ++i)
                for (int k = 0; k < M; ++k)
                    A[(long)i * M + k] = (i == k ? 1.0 + dtau * a * a : 0.0) - dtau * lambda * lambda * im->D2[(long)i * M + k];
            lu_factor(M, A, im->piv + (size_t)j * M);
        }
        im->dtau = dtau;
        im->lambda = lambda;
    }
#pragma omp parallel for schedule(dynamic)
    for (int j = 0; j < H; ++j) {
        double *re = malloc(sizeof(double) * M), *imv = malloc(sizeof(double) * M);
        for (int i = 0; i < M; ++i) {
            cplx g = G[(long)(i + 1) * H + j];
            re[i] = dtau * creal(g);
            imv[i] = dtau * cimag(g);
        }
        lu_apply(M, im->F + (size_t)j * M * M, im->piv + (size_t)j * M, re);
        lu_apply(M, im->F + (size_t)j * M * M, im->piv + (size_t)j * M, imv);
        for (int i = 0; i < M; ++i) U[(long)(i + 1) * H + j] += re[i] + I * imv[i];
        free(re);
        free(imv);
    }
}

/* ------------------------------------------------------------------------ */
/* Descent in fictitious time (Sec. III, Sec. V.C.3)                         */
/* ------------------------------------------------------------------------ */

/* Semi-implicit forward Euler for du/dtau = G (Sec. V.C.3).
 * scheme 0: the term of G that is linear in u and diagonal in Fourier space,
 * -A^2 u with A = d_xx + d_xxxx (symbol a_j = k_j^4 - k_j^2), is taken at the
 * new level, the rest of G at the old level:
 *   u^{n+1} = [u^n + dtau (G(u^n) + a_j^2 u^n)] / (1 + dtau a_j^2)
 * for the interior rows; the end rows stay at u_+-.
 * scheme 1: every linear term of G at the new level (implicit_update above).
 * conv: 0 stop when J_arc < tol, 1 when J < tol, 2 when J/|lambda D_t u|_W < tol;
 * tol <= 0 never stops early.
 * hist (optional) [nsteps+1][6]: (step, tau, J, J_arc, |G|_W, lambda) of the
 * state each step starts from.
 * out[0..4]: J, J_arc, dJ^2/dlambda, |G|_W, lambda of the final state
 * (the cost and lambda-gradient of the returned state; |G| of the last step).
 * Returns the number of updates applied. */
long ko_curve_descend(int M, int N, double L, double S, double lambda, int lambda_free,
                      double dtau, double dtau_lambda, int mode, int scheme, long nsteps, double tol,
                      int conv, cplx *U, double *hist, double *out)
{
    int P = M + 1, H = N / 2;
    long sz = (long)(P + 1) * H;
    cplx *R = malloc(sizeof(cplx) * sz);
    cplx *D = malloc(sizeof(cplx) * sz);
    cplx *G = malloc(sizeof(cplx) * sz);
    double sc[5] = {0, 0, 0, 0, 0}, gnorm = 0.0;
    long step = 0;
    implicit_ops *im = (scheme == 1) ? implicit_new(M, H, L, S) : NULL;
    for (;;) {
        ko_curve_residual(M, N, L, S, lambda, U, R, D);
        ko_curve_scalars(M, N, L, S, lambda, R, D, NULL, sc);
        double J = sqrt(sc[0]);
        if (hist) {
            double *h = hist + 6 * step;
            h[0] = (double)step; h[1] = dtau * (double)step; h[2] = J;
            h[3] = sc[1]; h[4] = gnorm; h[5] = lambda;
        }
        double crit = (conv == 0) ? sc[1] : (conv == 1) ? J : (sc[4] > 0 ? J / sc[4] : J);
        if (step >= nsteps || (tol > 0 && crit < tol)) break;
        ko_curve_adjoint(M, N, L, S, lambda, mode, U, R, G, NULL);
        gnorm = sqrt(ko_curve_norm2_W(M, N, L, S, G));
        if (im) {
            implicit_update(im, dtau, lambda, G, U);
        } else {
            for (int m = 1; m <= M; ++m)
                for (int j = 0; j < H; ++j) {
                    double a = pow(kwave(j, L), 4) - pow(kwave(j, L), 2);
                    long i = (long)m * H + j;
                    U[i] = (U[i] + dtau * (G[i] + a * a * U[i])) / (1.0 + dtau * a * a);
                }
        }
        if (lambda_free) lambda -= dtau_lambda * sc[2];
        ++step;
    }
    out[0] = sqrt(sc[0]);
    out[1] = sc[1];
    out[2] = sc[2];
    out[3] = gnorm;
    out[4] = lambda;
    free(R);
    free(D);
    free(G);
    implicit_free(im);
    return step;
}

/* One full-linear-implicit update of the interior rows, for tests of a single
 * step: U += delta with (I (1 + dtau a_j^2) - dtau lambda^2 Dt~^2) delta_j = dtau G_j. */
void ko_implicit_update(int M, int N, double L, double S, double dtau, double lambda, const cplx *G, cplx *U)
{
    implicit_ops *im = implicit_new(M, N / 2, L, S);
    implicit_update(im, dtau, lambda, G, U);
    implicit_free(im);
}

/* ------------------------------------------------------------------------ */
/* Initial curve (Sec. V.C.2)                                                */
/* ------------------------------------------------------------------------ */

/* Trial curve, on the grid x_n, for the interior rows (eq. KSE_initial_curve):
 *   u0(x,s) = 1/2[(1+tanh s) u_+ + (1-tanh s) u_-] + a exp(-s^2) v(x)
 *             + sum_p amps[p] sin((p+1) theta) vp[p](x)
 * The last sum is a smooth perturbation that vanishes at both ends; the
 * paper's own choice is npert = 0.  Rows 0 and M+1 are u_+ and u_-.
 * Inputs are physical sections of length N; the result is spectral. */
void ko_curve_init(int M, int N, double S, double s0, const double *up, const double *um,
                   double a, const double *v, int npert, const double *amps,
                   const double *vp, cplx *U)
{
    int P = M + 1, H = N / 2;
    double *s = malloc(sizeof(double) * (P + 1));
    double *th = malloc(sizeof(double) * (P + 1));
    ko_grid(M, S, s0, th, s, NULL);
    double *row = malloc(sizeof(double) * N);
    for (int m = 0; m <= P; ++m) {
        for (int n = 0; n < N; ++n) {
            if (m == 0) { row[n] = up[n]; continue; }
            if (m == P) { row[n] = um[n]; continue; }
            double t = tanh(s[m]);
            double val = 0.5 * ((1.0 + t) * up[n] + (1.0 - t) * um[n]);
            if (v && a != 0.0) val += a * exp(-s[m] * s[m]) * v[n];
            for (int p = 0; p < npert; ++p) val += amps[p] * sin_idx((long)(p + 1) * m, P) * vp[(long)p * N + n];
            row[n] = val;
        }
        ko_fwd(N, row, U + (long)m * H);
    }
    free(s);
    free(th);
    free(row);
}

/* ------------------------------------------------------------------------ */
/* End-point equilibria (Sec. V.D: E_1, E_2, E_3 are inversion symmetric)    */
/* ------------------------------------------------------------------------ */

/* LU factorisation with partial pivoting and solve, A (n x n, row-major) is
 * overwritten; returns 0 on success, -1 if singular. */
static int lu_solve(int n, double *A, double *b)
{
    int *piv = malloc(sizeof(int) * n);
    for (int i = 0; i < n; ++i) piv[i] = i;
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[(long)r * n + c]) > fabs(A[(long)p * n + c])) p = r;
        if (A[(long)p * n + c] == 0.0) { free(piv); return -1; }
        if (p != c) {
            for (int k = 0; k < n; ++k) {
                double t = A[(long)c * n + k];
                A[(long)c * n + k] = A[(long)p * n + k];
                A[(long)p * n + k] = t;
            }
            double t = b[c]; b[c] = b[p]; b[p] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[(long)r * n + c] / A[(long)c * n + c];
            A[(long)r * n + c] = f;
            for (int k = c + 1; k < n; ++k) A[(long)r * n + k] -= f * A[(long)c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double acc = b[r];
        for (int k = r + 1; k < n; ++k) acc -= A[(long)r * n + k] * b[k];
        b[r] = acc / A[(long)r * n + r];
    }
    free(piv);
    return 0;
}

/* Sine coefficients c_j (j = 1..N/2-1) of an odd field from its spectrum:
 * q(x) = sum_j c_j sin(k_j x)  <=>  q^_j = -i c_j / 2. */
static void odd_spec(int N, const double *b, cplx *uh)
{
    uh[0] = 0.0;
    for (int j = 1; j < N / 2; ++j) uh[j] = -0.5 * I * b[j - 1];
}

static double odd_residual(int N, double L, const double *b, double *F)
{
    int H = N / 2;
    cplx *uh = malloc(sizeof(cplx) * H), *fh = malloc(sizeof(cplx) * H);
    odd_spec(N, b, uh);
    ko_rhs(N, L, uh, fh);
    double nf = 0.0;
    for (int j = 1; j < H; ++j) {
        F[j - 1] = -2.0 * cimag(fh[j]);
        if (fabs(F[j - 1]) > nf) nf = fabs(F[j - 1]);
    }
    free(uh);
    free(fh);
    return nf;
}

/* Damped Newton iteration for f(u) = 0 inside the inversion-symmetric
 * (odd) subspace u = sum_{j=1}^{N/2-1} b_j sin(k_j x).  The Jacobian is built
 * column by column from the explicit linearisation Df(u) (ko_jac_apply); the
 * step is halved until the max-norm of the residual decreases.
 * Returns the iteration count (or -1 if the solve failed); *resnorm gets the
 * final max-norm of the sine coefficients of f. */
int ko_newton_odd(int N, double L, double *b, int maxit, double tol, double *resnorm)
{
    int n = N / 2 - 1, H = N / 2;
    double *F = malloc(sizeof(double) * n), *Ft = malloc(sizeof(double) * n);
    double *Jm = malloc(sizeof(double) * (long)n * n), *d = malloc(sizeof(double) * n);
    double *bt = malloc(sizeof(double) * n);
    cplx *uh = malloc(sizeof(cplx) * H), *vh = malloc(sizeof(cplx) * H), *o = malloc(sizeof(cplx) * H);
    int it = 0, rc = -1;
    double nf = odd_residual(N, L, b, F);
    for (it = 0; it < maxit; ++it) {
        if (nf < tol) { rc = it; break; }
        odd_spec(N, b, uh);
        for (int l = 0; l < n; ++l) {
            for (int j = 0; j < H; ++j) vh[j] = 0.0;
            vh[l + 1] = -0.5 * I;
            ko_jac_apply(N, L, uh, vh, o);
            for (int j = 0; j < n; ++j) Jm[(long)j * n + l] = -2.0 * cimag(o[j + 1]);
        }
        for (int j = 0; j < n; ++j) d[j] = -F[j];
        if (lu_solve(n, Jm, d) != 0) break;
        double alpha = 1.0, nt = nf;
        for (int h = 0; h < 40; ++h) {
            for (int j = 0; j < n; ++j) bt[j] = b[j] + alpha * d[j];
            nt = odd_residual(N, L, bt, Ft);
            if (nt < nf) break;
            alpha *= 0.5;
        }
        if (!(nt < nf)) break;
        memcpy(b, bt, sizeof(double) * n);
        memcpy(F, Ft, sizeof(double) * n);
        nf = nt;
    }
    if (rc < 0 && nf < tol) rc = it;
    if (resnorm) *resnorm = nf;
    free(F); free(Ft); free(Jm); free(d); free(bt); free(uh); free(vh); free(o);
    return rc;
}

/* Jacobian Df(u) restricted to the zero-mean subspace (Sec. V.B), as a real
 * (N-2) x (N-2) matrix in the coordinates (Re u^_1..Re u^_{N/2-1},
 * Im u^_1..Im u^_{N/2-1}); row-major. */
void ko_jacobian_zero_mean(int N, double L, const cplx *uh, double *Jm)
{
    int H = N / 2, n = N - 2;
    cplx *vh = malloc(sizeof(cplx) * H), *o = malloc(sizeof(cplx) * H);
    for (int l = 0; l < n; ++l) {
        for (int j = 0; j < H; ++j) vh[j] = 0.0;
        if (l < H - 1) vh[l + 1] = 1.0; else vh[l - (H - 1) + 1] = I;
        ko_jac_apply(N, L, uh, vh, o);
        for (int j = 1; j < H; ++j) {
            Jm[(long)(j - 1) * n + l] = creal(o[j]);
            Jm[(long)(j - 1 + H - 1) * n + l] = cimag(o[j]);
        }
    }
    free(vh);
    free(o);
}

/* ------------------------------------------------------------------------ */
/* Time stepping of the KSE itself (for the trajectory check)               */
/* ------------------------------------------------------------------------ */

static void ks_nonlinear(int N, double L, const cplx *uh, cplx *out)
{
    double *u = malloc(sizeof(double) * N);
    ko_inv(N, uh, u);
    for (int n = 0; n < N; ++n) u[n] = u[n] * u[n];
    ko_fwd(N, u, out);
    for (int j = 0; j < N / 2; ++j) out[j] *= -0.5 * I * kwave(j, L);
    free(u);
}

static void project_sym(int N, cplx *uh, int sym)
{
    for (int j = 0; j < N / 2; ++j) {
        if (sym & 1) uh[j] = I * cimag(uh[j]);          /* odd: u(-x) = -u(x) */
        if ((sym & 2) && (j % 2 == 1)) uh[j] = 0.0;     /* period L/2 */
    }
}

/* Integrate du/dt = f(u) (eq. KSE) from t to t + T with the integrating-factor
 * fourth-order Runge-Kutta scheme (the linear part k^2 - k^4 integrated
 * exactly), in ceil(T/dt) equal steps.  sym: bit 0 keeps u odd, bit 1 keeps
 * it L/2-periodic (projection after every step). */
void ko_ks_integrate(int N, double L, cplx *uh, double T, double dt, int sym)
{
    int H = N / 2;
    long nst = (long)ceil(T / dt);
    if (nst < 1) nst = 1;
    double h = T / (double)nst;
    cplx *E = malloc(sizeof(cplx) * H), *E2 = malloc(sizeof(cplx) * H);
    cplx *a = malloc(sizeof(cplx) * H), *b = malloc(sizeof(cplx) * H);
    cplx *c = malloc(sizeof(cplx) * H), *d = malloc(sizeof(cplx) * H), *t = malloc(sizeof(cplx) * H);
    for (int j = 0; j < H; ++j) {
        double k = kwave(j, L);
        E[j] = exp((k * k - k * k * k * k) * h / 2.0);
        E2[j] = E[j] * E[j];
    }
    for (long s = 0; s < nst; ++s) {
        ks_nonlinear(N, L, uh, a);
        for (int j = 0; j < H; ++j) { a[j] *= h; t[j] = E[j] * (uh[j] + a[j] / 2.0); }
        ks_nonlinear(N, L, t, b);
        for (int j = 0; j < H; ++j) { b[j] *= h; t[j] = E[j] * uh[j] + b[j] / 2.0; }
        ks_nonlinear(N, L, t, c);
        for (int j = 0; j < H; ++j) { c[j] *= h; t[j] = E2[j] * uh[j] + E[j] * c[j]; }
        ks_nonlinear(N, L, t, d);
        for (int j = 0; j < H; ++j) {
            d[j] *= h;
            uh[j] = E2[j] * uh[j] + (E2[j] * a[j] + 2.0 * E[j] * (b[j] + c[j]) + d[j]) / 6.0;
        }
        if (sym) project_sym(N, uh, sym);
    }
    free(E); free(E2); free(a); free(b); free(c); free(d); free(t);
}
