/*
 * ksconn.h -- C ABI of the GB300 (sm_103a) adjoint-descent library for
 * connecting orbits of the Kuramoto-Sivashinsky equation (KSE), after
 * Ashtari & Schneider, "Jacobian-Free Variational Method for Constructing
 * Connecting Orbits in Nonlinear Dynamical Systems" (arXiv 2301.11704).
 *
 * One curve u(x, s) joins two equilibria u_- (s -> -inf) and u_+ (s -> +inf).
 * It is discretised with N Fourier modes in x (Sec. V.C.1) and M + 2
 * rational-Chebyshev sections in s (eq. t_grid; N_s = M + 2 counts both end
 * sections).  One descent step evaluates, for every curve point at once,
 *   f(u)           the KSE right-hand side            (eq. KSE, nu = 1)
 *   r = f - l D_t u  the residual                      (eq. residual_definition, eq. KSE_residual)
 *   G = -L^dagger(u; r) the adjoint descent direction  (eq. KSE_G)
 *   J^2, J_arc     the cost and its arc-length form   (eq. cost_function_general, eq. J_arc)
 * and advances u by semi-implicit Euler in fictitious time (Sec. V.C.3).
 * l (lambda) scales the s-derivative; l = 1 is the published method.
 *
 * Conventions shared by every entry point
 *  - All functions return ks_status; KS_OK is 0.  No function throws, exits or
 *    prints.  On failure ks_last_error() returns a message for the calling
 *    thread; outputs are then unspecified, and the curve stays usable unless
 *    the status is KS_ECUDA (a failed CUDA call; the CUDA context may be lost).
 *  - Device pointers ("_dev") point to memory of the current CUDA device,
 *    allocated by the caller.  Every buffer the library uses lives in the
 *    caller's workspace; the one exception is the one-time set-up of
 *    KS_SCHEME_IMPLICIT (ks_curve_create / ks_batch_create), whose eigensolver
 *    allocates and frees temporary device memory before create returns.
 *    Host pointers ("_host" or scalar outputs) are ordinary host memory.
 *  - Physical curve arrays are row-major [N_s][N] in the storage type of the
 *    curve (double for KS_FP64, float for the others); row m is section s_m,
 *    row 0 is s = +inf (u_+), row N_s-1 is s = -inf (u_-); column n is x_n = n L / N.
 *  - Work is issued on the caller's CUDA stream (cudaStream_t passed as void*;
 *    NULL = legacy default stream).  Functions that return host scalars
 *    synchronise that stream; the others are asynchronous.
 *  - A curve handle is not thread safe; distinct handles are independent.
 */
#ifndef KSCONN_H
#define KSCONN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KS_OK = 0,
    KS_EINVAL = 1,            /* bad argument (sizes, null pointers, ranges) */
    KS_ENOMEM = 2,            /* caller workspace smaller than ks_curve_workspace_bytes() */
    KS_ECUDA = 3,             /* a CUDA runtime call failed */
    KS_ETIMEOUT = 4,          /* a device-side bounded wait expired */
    KS_ENONFINITE = 5,        /* J or G became NaN/Inf; the descent stopped */
    KS_ENOTCONV = 6,          /* nsteps exhausted before the tolerance was met */
    KS_ENOTEQUILIBRIUM = 7,   /* an end section is not an equilibrium (|f(u)| too large) */
    KS_ENOTIMPL = 8
} ks_status;

/* Arithmetic of the curve's fields and transforms; J, J_arc, dJ^2/dlambda,
 * |G|, the lambda update and the convergence test are FP64 in every precision.
 * KS_FP64:   FP64 storage and transforms.
 * KS_FP32:   FP32 storage, FP32 transforms (FFTs in x and s).
 * KS_BF16X2, KS_BF16X3: FP32 storage; the x-transforms of every section (one
 *            forward or backward DFT per section, Sec. V.C.1: four per row phase)
 *            as dense products with the N x N DFT matrices on the tensor cores,
 *            each FP32 operand split into two (BF16X2, about 2^-17 relative) or
 *            three (BF16X3, about FP32 rounding) BF16 parts with FP32
 *            accumulation; the s-transforms as in KS_FP32.  N must be 64, 128
 *            or 256; single curves only (batches take KS_FP64 or KS_FP32); the
 *            persistent launch form (launch = 1) does not apply. */
typedef enum { KS_FP64 = 0, KS_FP32 = 1, KS_BF16X2 = 2, KS_BF16X3 = 3 } ks_precision;

/* s-term of the adjoint (eq. KSE_G).
 * KS_ADJ_PAPER:    +lambda D_t r, the continuous adjoint discretised, as published.
 * KS_ADJ_DISCRETE: -lambda W^-1 D_t^T W r, the exact adjoint of the discretised
 *                  residual under the quadrature inner product (W = diag(w_m)),
 *                  so that G is exactly the negative W-gradient of J^2. */
typedef enum { KS_ADJ_PAPER = 0, KS_ADJ_DISCRETE = 1 } ks_adjoint;

/* Convergence measure compared with `tol` in ks_curve_descend.
 * KS_CONV_JARC: J_arc (eq. J_arc; the published criterion is J_arc < 1e-12).
 * KS_CONV_J:    J = sqrt(J^2).
 * KS_CONV_JREL: J / |lambda D_t u|_W (scale-free; the FP32 criterion). */
typedef enum { KS_CONV_JARC = 0, KS_CONV_J = 1, KS_CONV_JREL = 2 } ks_conv;

/* Time stepping of the descent du/dtau = G, semi-implicit forward Euler
 * (Sec. V.C.3: the terms of G linear in u at the new level, the rest at the old).
 * KS_SCHEME_IMEX: the diagonal term -a_j^2 u (a_j = k_j^4 - k_j^2):
 *   u += dtau G / (1 + dtau a_j^2); stable while dtau rho(lambda^2 D_t^2) < 2.
 * KS_SCHEME_IMPLICIT: every linear term, (lambda^2 D~^2 - a_j^2) u with D~ the
 *   interior block of D_t (eq. rational_diff_matrix):
 *   (I (1 + dtau a_j^2) - dtau lambda^2 D~^2) delta_j = dtau G_j, u += delta,
 *   applied as V (dtau / (1 + dtau (a_j^2 - lambda^2 mu))) V^-1 in the
 *   eigenbases of D~^2 restricted to its even and odd parts under s -> -s
 *   (computed once at create, in FP64, by cuSOLVER's nonsymmetric eigensolver,
 *   which the library opens at run time: create fails with KS_ECUDA if it is
 *   missing, KS_EINVAL if an eigenvalue is complex or positive).  Single
 *   curves, launch = 0, N_s <= 16384; the set-up temporarily allocates device
 *   memory of about 5 (N_s / 2)^2 doubles besides the workspace. */
typedef enum { KS_SCHEME_IMEX = 0, KS_SCHEME_IMPLICIT = 1 } ks_scheme;

/* Bits of ks_params.symmetry (Sec. V.B). */
enum { KS_SYM_ODD = 1, KS_SYM_HALF_PERIOD = 2, KS_SYM_SINE = 4 };

typedef struct {
    double L;            /* domain length, > 0 (Sec. V: x in [0, L)) */
    int32_t nx;          /* N: Fourier modes = grid points per section; power of two, 8..256 */
    int32_t ns;          /* N_s = M + 2 sections including both ends; 3 <= N_s <= 65536 */
    double S;            /* map scale S > 0 (eq. Rational_domain) */
    double s0;           /* map centre s0 (eq. Rational_domain) */
    double lambda;       /* scale of the s-derivative; 1 = the published method */
    int32_t lambda_free; /* 1: lambda descends along -dJ^2/dlambda with step dtau_lambda */
    double dtau;         /* fictitious time step > 0 (Sec. V.C.3) */
    double dtau_lambda;  /* step of the lambda update (used when lambda_free) */
    int32_t precision;   /* ks_precision: storage and transform arithmetic; reductions are FP64 */
    int32_t adjoint;     /* ks_adjoint */
    int32_t conv;        /* ks_conv */
    int32_t check_ends;  /* 1: ks_curve_create fails with KS_ENOTEQUILIBRIUM when an end
                            section has |f(u)|_2 > 1e-8 (1 + |u|_2); 0: no check */
    int32_t symmetry;    /* symmetric subspace held exactly (Sec. V.B; the dynamics preserves it):
                            bit 0: every section odd, u(-x) = -u(x) (real parts of u^ zero);
                            bit 1: every section L/2-periodic (odd Fourier modes zero);
                            bit 2 (KS_SYM_SINE, with bit 0 only): sine storage: every stored
                            field keeps only Im u^_j, N_x/2 words per section instead of N_x,
                            and every s-contraction runs on those N_x/2 columns (half the
                            bytes and half the s-side work of bit 0 alone; same results to
                            rounding).  Inputs and outputs of the entry points keep the
                            physical layout.  Needs N_x >= 16, precision KS_FP64 or KS_FP32
                            (the FFT row phase), scheme KS_SCHEME_IMEX, launch = 0 and
                            s_transform 0, 1, 2, 4 or 5 (auto applies its rule to the
                            N_x/2 stored columns); batched curves take it curve by curve.
                            0 = none.  Values above 7, and bit 2 without bit 0, are
                            invalid. */
    int32_t s_transform; /* how D_t is applied along s (same result to rounding):
                            0 auto: for a single curve the form measured fastest on GB300 for its
                            size: from N_s = 684 on (FFT length >= 4096) a four-step FFT form:
                            in FP32 the clustered one (5) at N_x <= 64 up to N_s = 5462 and at
                            N_x = 128 up to N_s = 2731, else the three-launch one (4); in FP64
                            the clustered one at N_x <= 16 up to N_s = 1366, the one-CTA form
                            at N_x = 256 while it fits (N_s <= 1366), else the three-launch one;
                            below N_s = 684 dense, or in FP64 the one-CTA FFT form at N_x >= 64
                            or N_s <= 128; above the four-step limit dense (on the tensor cores
                            for FP32 when N_s >= 8192, or N_s >= 4096 at N_x >= 128); in a
                            batch the one-CTA FFT form wherever it fits;
                            1 dense contraction generated from the O(N_s) cot table;
                            2 FFT convolution (N_s <= 21846; one CTA per mode up to N_s = 2731
                            FP32 / 1366 FP64, the four-step form above);
                            3 dense contraction on the tensor cores (FP32 storage only: each
                            FP32 operand split exactly into three TF32 parts, six products,
                            FP32 accumulation per 32 sections, FP32 sums across them);
                            4 FFT convolution in the four-step form (transform length F = F1 F2
                            from 4096 to 65536: 684 <= N_s <= 21846), which 2 and auto use
                            above one CTA's limit: three launches through a scratch array;
                            5 the same four-step form in one launch: a cluster of 8 CTAs per
                            one or two Fourier modes holds their intermediate array in
                            distributed shared memory (same N_s range as 4, in FP64 up to
                            N_s = 10923: F <= 32768) */
    int32_t launch;      /* how a single curve's descent steps are launched (same results):
                            0 three kernels per step, chained by programmatic dependent
                            launch and replayed from a CUDA graph;
                            1 one persistent cooperative kernel for many steps, with
                            grid-wide barriers between the phases of a step (dense form
                            only, else as 0; measured slower than 0 on GB300).
                            Batches ignore it. */
    int32_t scheme;      /* ks_scheme (time stepping); the workspace grows by
                            2 (ceil(M/2)^2 + floor(M/2)^2) + 16 M N storage words + 8 M bytes
                            for KS_SCHEME_IMPLICIT */
} ks_params;

/* Scalars of the state most recently evaluated (cost, gradient or descent). */
typedef struct {
    double J;            /* sqrt(J^2), J^2 = sum_m w_m |r_m|^2 (eq. cost_function_general) */
    double J_arc;        /* eq. J_arc */
    double dJ2_dlambda;  /* -2 sum_m w_m <D_t u_m, r_m> */
    double G_norm;       /* |G|_W of the last gradient evaluated */
    double Dnorm;        /* |lambda D_t u|_W, for J / Dnorm */
    double lambda;       /* current lambda */
    double tau;          /* fictitious time reached */
    int64_t step;        /* descent steps applied since create / set_state */
    int32_t converged;   /* 1 once the tolerance of the last descend was met */
    int32_t status;      /* ks_status of the device-side checks (KS_OK or KS_ENONFINITE) */
} ks_scalars;

typedef struct ks_curve ks_curve;

/* Thread-local message of the last failure on this thread ("" if none). */
const char *ks_last_error(void);

/* Library version, (major << 16) | minor. */
int32_t ks_version(void);

/* Bytes of device workspace a curve with these parameters needs (0 if the
 * parameters are invalid; ks_last_error() says why).  The workspace holds the
 * spectral state, its s-derivative, the residual, the adjoint, the
 * rational-Chebyshev tables (O(N_s)), the Fourier tables and the FP64
 * reduction buffers: about 6 N_s N storage words in total.  No O(N_s^2)
 * matrix is stored: D_t is generated from an O(N_s) table on the fly. */
size_t ks_curve_workspace_bytes(const ks_params *p);

/* Length of the FFT that a single curve with parameters p applies D_t with
 * (s_transform rule above), or 0 when it uses the dense contraction.  -1 when
 * p is invalid (message in ks_last_error). */
int32_t ks_curve_fft_length(const ks_params *p);

/* The form a single curve with parameters p applies D_t in, as an s_transform
 * code with `auto` resolved: 1 dense, 2 FFT with one CTA per mode, 3 dense on the
 * tensor cores, 4 four-step FFT in three launches, 5 four-step FFT in one
 * clustered launch.  -1 when p is invalid (message in ks_last_error). */
int32_t ks_curve_s_form(const ks_params *p);

/* Creates a curve (Sec. V.C.1-2).
 *  p            parameters (copied).
 *  u_plus_host  [N] physical u_+ (s -> +inf), u_minus_host [N] physical u_- (s -> -inf).
 *  u_init_dev   [N_s][N] physical initial curve in the storage type, or NULL
 *               for the trial curve of eq. KSE_initial_curve with a = 0
 *               (use ks_curve_init_trial for a != 0 or a perturbation).
 *               Rows 0 and N_s-1 of u_init_dev are replaced by u_+ and u_-.
 *  workspace_dev, workspace_bytes: caller memory, >= ks_curve_workspace_bytes(p),
 *               256-byte aligned; owned by the caller, used until ks_curve_destroy.
 *  stream       cudaStream_t for all work of this curve (may be changed with
 *               ks_curve_set_stream).
 *  out          receives the handle.
 * The handle holds host metadata, a pinned host copy of the device scalars
 * (cudaMallocHost, freed by ks_curve_destroy) and, for the FFT row phase from
 * N_s = 2048 on, the tensor maps of the row phase's TMA tile loads.
 * Errors: KS_EINVAL, KS_ENOMEM, KS_ECUDA, KS_ENOTEQUILIBRIUM (check_ends = 1).
 * Synchronises the stream. */
ks_status ks_curve_create(const ks_params *p, const double *u_plus_host, const double *u_minus_host,
                          const void *u_init_dev, void *workspace_dev, size_t workspace_bytes,
                          void *stream, ks_curve **out);

ks_status ks_curve_set_stream(ks_curve *c, void *stream);

/* Re-initialises the interior sections with the trial curve (eq. KSE_initial_curve):
 *   u0(x, s_m) = 1/2[(1 + tanh s_m) u_+ + (1 - tanh s_m) u_-] + a exp(-s_m^2) v(x)
 *               + sum_{p=1}^{npert} amps[p-1] sin(p theta_m) vp[p-1](x).
 * The last sum is a perturbation that vanishes at both ends (npert = 0 gives the
 * published form).  v_host [N] may be NULL when a = 0; vp_host is [npert][N];
 * npert <= 16.  Resets step, tau and lambda (to p->lambda).  Synchronises. */
ks_status ks_curve_init_trial(ks_curve *c, double a, const double *v_host, int32_t npert,
                              const double *amps_host, const double *vp_host);

/* Residual r = f(u) - lambda D_t u of the current state, physical [N_s][N] in
 * the storage type (eq. KSE_residual); rows 0 and N_s-1 are 0.  Also refreshes
 * J, J_arc, dJ2_dlambda and Dnorm of ks_curve_scalars.  Asynchronous. */
ks_status ks_curve_residual(ks_curve *c, void *r_dev);

/* J^2 (eq. cost_function_general) and J_arc (eq. J_arc) of the current state
 * into host doubles (either may be NULL).  Synchronises. */
ks_status ks_curve_cost(ks_curve *c, double *J2, double *J_arc);

/* Gradient of the current state into g_dev, physical [N_s][N], storage type.
 *  euclidean = 0: the descent direction G = -L^dagger(u; r) of the curve's
 *                 adjoint mode (eq. KSE_G); rows 0 and N_s-1 are 0.
 *  euclidean = 1: dJ^2/du_{m,n} of the discretised cost J^2 = sum_m w_m |r_m|^2
 *                 with respect to the interior grid values, = -2 dx w_m G_DISCRETE;
 *                 rows 0 and N_s-1 are 0 (the end sections are fixed).
 *  dJ2_dlambda (host, may be NULL) receives dJ^2/dlambda.  Synchronises when
 *  dJ2_dlambda is not NULL. */
ks_status ks_curve_gradient(ks_curve *c, int32_t euclidean, void *g_dev, double *dJ2_dlambda);

/* Runs up to nsteps descent steps (Sec. III, Sec. V.C.3) on the device:
 * each step evaluates r and G of the current state and applies
 *   u <- [u + dtau (G + a_j^2 u)] / (1 + dtau a_j^2),  a_j = k_j^4 - k_j^2,
 * to the interior sections (the term -A^2 u of G, A = d_xx + d_xxxx, implicit),
 * and, when lambda_free, lambda <- lambda - dtau_lambda dJ^2/dlambda.
 * Stops early once the convergence measure of p->conv falls below tol
 * (tol <= 0: never).  steps_done, J, J_arc (host, may be NULL) receive the
 * steps applied and the cost of the final state.  Returns KS_ENOTCONV when
 * tol > 0 was not reached, KS_ENONFINITE if the cost became NaN/Inf.
 * Synchronises. */
ks_status ks_curve_descend(ks_curve *c, int64_t nsteps, double tol, int64_t *steps_done, double *J,
                           double *J_arc);

/* Enqueues `nsteps` descent steps without synchronising or checking the
 * tolerance on the host (the device still stops at convergence to tol).
 * For timing loops and CUDA-graph capture by the caller. */
ks_status ks_curve_descend_async(ks_curve *c, int64_t nsteps, double tol);

/* Host copy of the scalars of the most recent evaluation.  Synchronises. */
ks_status ks_curve_scalars(ks_curve *c, ks_scalars *out);

/* Current state, physical [N_s][N] in the storage type (may be NULL), plus
 * lambda and tau (host, may be NULL).  Synchronises when lambda or tau is
 * requested. */
ks_status ks_curve_get_state(ks_curve *c, void *u_dev, double *lambda, double *tau);

/* Replaces the state (all rows, including the end sections) from a physical
 * [N_s][N] array in the storage type, with lambda and tau; step is reset to 0.
 * The array is transformed in FP64 (FP32 storage: double-float arithmetic,
 * about 44 bits) and rounded per coefficient to the storage type.
 * Asynchronous. */
ks_status ks_curve_set_state(ks_curve *c, const void *u_dev, double lambda, double tau);

/* Device time of the descent steps, measured with CUDA events recorded on the
 * curve's stream around each kernel.  Three-kernel steps (launch = 1, or the
 * FFT form) are timed per phase:
 *   phase 0: row phase (f, residual, spatial adjoint, cost reductions)
 *   phase 1: s-phase with the descent update (D_t r, G, u update, |G|^2)
 *   phase 2: s-phase D_t u of the new state;
 * launches of the persistent step kernel are timed whole (step_*).
 * ks_curve_profile(c, max_steps) starts recording for up to max_steps steps or
 * persistent launches (max_steps = 0 stops and releases the events);
 * ks_curve_profile_read synchronises and returns the accumulated milliseconds
 * and launch counts. */
typedef struct {
    double ms[3];            /* kernel-per-phase steps: milliseconds per phase (rows, update,
                                D_t u); the clustered four-step form applies D_t u inside the
                                update launch and reports no third phase */
    int64_t launches[3];
    double step_ms;          /* persistent step kernel: milliseconds of its launches */
    int64_t step_launches;   /* its launches */
    int64_t step_steps;      /* steps those launches were asked to run */
    double pass_ms[2][3];    /* three-launch four-step form (s_transform 4): milliseconds of
                                passes 1, 2, 3 of the update (row 0) and of D_t u (row 1) */
    int64_t pass_launches[2][3];
    double impl_ms;          /* KS_SCHEME_IMPLICIT: milliseconds of the increment's two
                                products (part of phase 1) */
    int64_t impl_launches;   /* steps they were timed for */
} ks_profile;

ks_status ks_curve_profile(ks_curve *c, int32_t max_steps);
ks_status ks_curve_profile_read(ks_curve *c, ks_profile *out);

/* ------------------------------------------------------------------------
 * Batches: many independent curves (uneven N_s, N and L, one precision and
 * one adjoint mode) descending together.  Each phase of a step is one launch
 * over the (curve, block) work items of all curves, and the steps are
 * replayed from a captured CUDA graph; every curve keeps its own gates,
 * reductions and convergence test (the method of Sec. III applied per curve).
 * Arrays indexed by curve have nb entries; u_plus_host / u_minus_host / vp_host
 * concatenate the curves' sections in curve order.
 * ------------------------------------------------------------------------ */
typedef struct ks_batch ks_batch;

/* Device workspace of a batch (0 for invalid parameters). */
size_t ks_batch_workspace_bytes(int32_t nb, const ks_params *params);

/* Creates a batch with the trial curves of eq. KSE_initial_curve (a = 0).
 * Same conventions as ks_curve_create; synchronises the stream. */
ks_status ks_batch_create(int32_t nb, const ks_params *params, const double *u_plus_host,
                          const double *u_minus_host, void *workspace_dev, size_t workspace_bytes,
                          void *stream, ks_batch **out);

/* Trial curves with npert perturbation modes per curve (see ks_curve_init_trial):
 * amps_host [nb][npert], vp_host the curves' [npert][N_i] fields concatenated. */
ks_status ks_batch_init_trial(ks_batch *b, int32_t npert, const double *amps_host, const double *vp_host);

/* Up to nsteps steps of every curve; a curve stops once its own convergence
 * measure is below tol.  steps_done, J, J_arc (host, nb entries each, may be
 * NULL).  KS_ENOTCONV if some curve missed tol > 0.  Synchronises. */
ks_status ks_batch_descend(ks_batch *b, int64_t nsteps, double tol, int64_t *steps_done, double *J,
                           double *J_arc);
ks_status ks_batch_descend_async(ks_batch *b, int64_t nsteps, double tol);

/* Scalars of every curve (out: nb entries).  Synchronises. */
ks_status ks_batch_scalars(ks_batch *b, ks_scalars *out);

/* Physical state of curve i, [N_s,i][N_i] in the storage type.  Asynchronous. */
ks_status ks_batch_get_state(ks_batch *b, int32_t i, void *u_dev);

/* Tunes the batch's launch shapes by timing `steps` real descent steps of every
 * curve per candidate (the timed steps count in each curve's step counter and
 * tau), one knob after the other, keeping the fastest:
 *   1. sections per CTA of the row phase: 8 or 16;
 *   2. for each transform length F of the four-step curves (the batched FFT form
 *      from F = 1024 on), the split F = F1 F2 of its line transforms: 32 x 32;
 *      64 x 32 or 32 x 64; 64 x 64, 128 x 32 or 32 x 128; 128 x 64 (the kernel
 *      spectrum and twiddles are recomputed for the split);
 *   3. for dense-form curves with N >= 64, the s-phase tile width: 64 or 32 columns.
 * *chosen (may be NULL) receives the sections per row CTA; ks_batch_get_tuning
 * reports every choice.  Synchronises. */
ks_status ks_batch_autotune(ks_batch *b, int32_t steps, int32_t *chosen);

typedef struct {
    int32_t row_sections;   /* sections per row-phase CTA */
    int32_t dense_tile;     /* s-phase tile width of dense-form curves (0: per-curve default) */
    int32_t nlen;           /* transform lengths of the four-step curves (at most 8 listed) */
    int32_t F[8], F1[8];    /* each length F and its split F = F1 (F / F1) */
    double ms_per_step;     /* a batch step with these choices, as the autotuner timed it (0 before) */
} ks_batch_tuning;

/* The batch's current launch-shape choices (defaults before ks_batch_autotune). */
ks_status ks_batch_get_tuning(ks_batch *b, ks_batch_tuning *out);

ks_status ks_batch_destroy(ks_batch *b);

/* Allocation-free cost evaluation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory, such as a host
 * program that owns every device allocation and hands this library only its
 * input and output buffers, a time-critical loop that must not pay cudaMalloc's
 * synchronisation and latency, or a process whose device memory is reserved up
 * front.  It computes J^2 and J_arc (eq. cost_function_general, eq. J_arc) of
 * a curve without a handle and without a workspace:
 *   p        parameters, same rules as ks_curve_workspace_bytes; p->launch is
 *            ignored (the evaluation runs kernel by kernel).  The scratch the
 *            curve needs, ks_curve_workspace_bytes(p) with p->launch = 0, must
 *            not exceed KS_NOALLOC_SCRATCH_BYTES, else KS_ENOMEM with a message.
 *   u_dev    [N_s][N] physical curve in the storage type (rows 0 and N_s-1
 *            are the end sections u_+ and u_-).
 *   out_dev  device doubles [2] receiving J^2 and J_arc; both are NaN when a
 *            bounded device-side wait of the evaluation gave up (the results
 *            of that launch are invalid; ks_curve_cost reports the same event
 *            as KS_ETIMEOUT).
 *   stream   cudaStream_t (NULL = legacy default stream); asynchronous.
 * The scratch is one static device array of KS_NOALLOC_SCRATCH_BYTES, held on
 * every device that loads the library until the process exits.  Every call
 * looks up that array's device address in the current device's context (the
 * first call on a device also loads the library's module there); make the
 * first call on a device before any stream capture.  All calls share the array
 * and it keeps the last call's contents (each call clears what must start at
 * zero): calls that overlap on the GPU race and give wrong results.
 * No device memory is allocated or freed. */
#define KS_NOALLOC_SCRATCH_BYTES (32u << 20)
ks_status ks_cost_noalloc(const ks_params *p, const void *u_dev, double *out_dev, void *stream);

/* Test hook for the failure path of the device-side bounded waits; the paper has
 * no counterpart.  The kernels that wait on an mbarrier (the split-BF16 row
 * phase, the FFT form with one CTA per mode, the tensor-core contraction) spin
 * at most `cycles` clock cycles in their first wait of a launch (0 restores the
 * default, about 2^31 cycles; a negative value makes that wait give up at once).
 * A wait that gives up sets the curve's error word, lets the copies and
 * products already in flight finish (with the default bound), frees its tensor
 * memory and returns; every later call that reads the curve's scalars returns
 * KS_ETIMEOUT until ks_curve_init_trial re-initialises the curve (which also
 * restores the default bound).  Asynchronous. */
ks_status ks_curve_debug_wait_limit(ks_curve *c, int64_t cycles);

/* Releases the handle (host memory only; the workspace stays the caller's). */
ks_status ks_curve_destroy(ks_curve *c);

#ifdef __cplusplus
}
#endif

#endif /* KSCONN_H */
