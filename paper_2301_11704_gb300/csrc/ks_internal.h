// ks_internal.h -- declarations shared by the kernels (ks_kernels.cu) and the
// C-ABI host code (ks_capi.cu).  Not part of the public interface.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda.h>   // CUtensorMap (the tensor maps are encoded through the runtime's driver entry point)
#include <cuda_runtime.h>

#include "../../include/ksconn.h"

namespace ks {

// Structured s-direction contraction (D_t or W^-1 D_t^T W applied to the
// columns of a curve): DT_BM output sections x BN real columns per CTA, DT_BK
// sections of the contraction per shared-memory stage, the contraction split
// over `ksplit` CTAs when the tiles alone cannot fill the GPU.
constexpr int DT_BM = 32;
constexpr int DT_BK = 32;
constexpr int DT_THREADS = 256;
constexpr int DT_TARGET_CTAS = 256;   // split the contraction until about this many CTAs run
constexpr int DT_MIN_KCHUNK = 64;     // but keep at least this many sections per split
constexpr int DT_MAX_SPLIT = 8;       // the splits of one tile form one thread-block cluster

// Tensor-core form of the dense s-contraction (FP32 storage): 128 output
// sections per CTA, stages of TC_KC sections, split over up to DT_MAX_SPLIT CTAs
// of a cluster.
constexpr int TC_M = 128;
constexpr int TC_KC = 32;
constexpr int TC_THREADS = 256;

// FFT form of the s-contraction: one CTA per Fourier mode (a column pair), the
// convolution of length F (a power of two >= 3 (N_s - 1)) in shared memory.
constexpr int SC_THREADS = 512;
constexpr int SC_FMAX_F32 = 8192;
constexpr int SC_FMAX_F64 = 4096;
// FFT length for a curve, 0 if above the single-CTA limit of the precision.
inline int fft_size(int ns, int prec)
{
    int F = 16;
    while (F < 3 * (ns - 1)) F <<= 1;
    return F <= (prec ? SC_FMAX_F32 : SC_FMAX_F64) ? F : 0;
}

// Four-step form for longer transforms (single curves): F = F1 F2 with line
// FFTs of F1, F2 <= 256 points by one warp each and one pass through a scratch
// buffer in between; up to F4_FMAX.
constexpr int F4_FMAX = 65536;
constexpr int F4_FMIN = 4096;             // 64 x 64
constexpr int F4B_FMIN = 1024;            // 32 x 32: the one-CTA-per-mode variant of batched curves
constexpr int F4B_FMAX_F32 = 8192;        // 128 x 64
constexpr int F4B_FMAX_F64 = 4096;        // 64 x 64
constexpr int F4_THREADS = 256;           // 8 warps, one line each
constexpr int F4C_CS = 8;                 // clustered four-step form: CTAs per cluster (portable size)
constexpr size_t F4C_SMEM_MAX = 224 * 1024;   // its dynamic shared memory per CTA (of 227 KB)
// F = F1 F2 with F1 = F2 or 2 F2
inline void f4_split(int F, int &F1, int &F2)
{
    int lg = 0;
    while ((1 << lg) < F) ++lg;
    F1 = 1 << ((lg + 1) / 2);
    F2 = F / F1;
}
// dynamic shared memory of the clustered form: line twiddles, the CTA's rows
// [mpc][F1/cs][F2] and its tile [mpc][F2/cs][F1 + pad] (complex values)
inline size_t f4c_bytes(int prec, int F1, int F2, int mpc, int cs)
{
    const size_t cb = prec ? 8 : 16;
    const size_t lt = (size_t)F1 + (prec ? 2 : 1);
    return ((size_t)F1 + F2 + 16 + (size_t)mpc * (F1 / cs) * F2 + (size_t)mpc * (F2 / cs) * lt) * cb;
}
inline bool f4c_fits(int prec, int F1, int F2) { return f4c_bytes(prec, F1, F2, 1, F4C_CS) <= F4C_SMEM_MAX; }
// The sizes where the clustered form is the fastest measured on GB300 (FP32:
// N_x <= 64 up to F = 16384, N_x = 128 up to F = 8192; FP64: N_x <= 16 at
// F = 4096).  Descent steps there apply the update and D_t u in one launch; the
// fused kernel's registers allow one wave of clusters at these sizes only.
inline bool f4c_fused(int prec, int nx, int F)
{
    return prec ? ((nx <= 64 && F <= 16384) || (nx <= 128 && F <= 8192)) : (nx <= 16 && F == 4096);
}
// modes per cluster: two FP32 modes (16-byte row segments) once there are enough
// modes to fill the GPU and their rows fit, else one
inline int f4c_mpc(int prec, int nx, int F1, int F2)
{
    return (prec && nx >= 128 && f4c_bytes(prec, F1, F2, 2, F4C_CS) <= F4C_SMEM_MAX) ? 2 : 1;
}
// Four-step length for a curve: above the single-CTA limit, or from F4_FMIN on
// when asked for (any = 1); 0 outside the range.
inline int fft4_size(int ns, int prec, int any = 0)
{
    int F = 16;
    while (F < 3 * (ns - 1)) F <<= 1;
    const int lo = any ? F4_FMIN : 2 * (prec ? SC_FMAX_F32 : SC_FMAX_F64);
    return (F >= lo && F <= F4_FMAX) ? F : 0;
}

// Length of the three-launch four-step form for a single curve.  D_t is applied
// there as two convolutions of the column z_m (m <= P, not its symmetric
// extension): a Toeplitz part with lags in [-P, P] and a Hankel part with lags
// in [0, 2P], so a power of two F >= 2P + 1 suffices (F >= 3P for the extended
// sequence of the other FFT forms): F in [fmin, F4_FMAX], 0 outside.  The
// batched one-CTA-per-mode variant uses the same split from F4B_FMIN on.
inline int fft4h_size(int ns, int fmin = F4_FMIN)
{
    int F = fmin;
    while (F < 2 * (ns - 1) + 1) F <<= 1;
    return F <= F4_FMAX ? F : 0;
}

// Form of the s-contraction: dense, FFT with one CTA per mode, four-step FFT in
// three launches, four-step FFT in one clustered launch.
enum SForm { SF_DENSE = 0, SF_FFT1 = 1, SF_FFT4 = 2, SF_FFT4C = 3 };

// Form that `auto` picks for a single curve (nx: the contraction's columns, N_x
// or N_x/2 in sine storage): the fastest measured on GB300 (20
// graph-replayed steps, N_x from 8 to 256, N_s from 256 to 16384).  From
// N_s = 684 on (F >= 4096) a four-step form wins: in FP32 the clustered one-launch
// form up to F = 16384 at N_x <= 64 and up to F = 8192 at N_x = 128 (15-30 %
// ahead: fewer launches and no scratch), the three-launch form elsewhere; in FP64,
// where the transforms' arithmetic dominates, the clustered form only at
// F = 4096, N_x <= 16, and the one-CTA form at N_x = 256 while it fits.  Below
// N_s = 684 the dense form, except the one-CTA FFT form in FP64 at N_x >= 64 or
// N_s <= 128.
inline int auto_form(int ns, int nx, int prec)
{
    const bool f1 = fft_size(ns, prec) > 0;
    const int F = fft4_size(ns, prec, 1);
    if (F) {
        int F1 = 0, F2 = 0;
        f4_split(F, F1, F2);
        if (f4c_fused(prec, nx, F) && f4c_fits(prec, F1, F2)) return SF_FFT4C;
        if (!prec && nx >= 256 && f1) return SF_FFT1;
        return SF_FFT4;
    }
    if (!prec && f1 && (nx >= 64 || ns <= 128)) return SF_FFT1;
    return SF_DENSE;
}

// Where `auto` puts a dense-form FP32 curve on the tensor cores: the sizes where
// it measured faster than the SIMT contraction on GB300 (one step, L2 flushed,
// N_x in {32, 64, 128, 256}, N_s from 1024 to 16384: by 7-20 %).
inline bool tc_preferred(int ns, int nx)
{
    return nx >= 32 && (ns >= 8192 || (nx >= 128 && ns >= 4096));
}

// Storage in FP32 (KS_FP32 and the split-BF16 forms) rather than FP64.
inline int storage32(int precision) { return precision != KS_FP64 ? 1 : 0; }
// Parts of the split-BF16 x-transforms on the tensor cores (0: FFT row phase).
inline int xtc_of(int precision) { return precision == KS_BF16X3 ? 3 : (precision == KS_BF16X2 ? 2 : 0); }

// Sections handled per CTA by the row (x-direction) kernels: two rows per warp,
// packed into one complex FFT.
constexpr int ROWS_WARPS = 4;
constexpr int ROWS_PER_CTA = 2 * ROWS_WARPS;
// Single curves from this N_s on load the row phase's tiles of U and D_t U by
// TMA (measured on GB300: 1-2% faster row phase at N_s = 4096 and 16384; at
// N_s = 1024, 128 CTAs, 5-8% slower than per-lane loads, which are kept there).
constexpr int ROWS_TMA_MIN_NS = 2048;

constexpr int MAX_PERT = 16;

// Persistent descent step (one cooperative launch for many steps of a single
// curve in the dense form): CTA size, warps per row unit, largest grid.
constexpr int PS_THREADS = 256;
constexpr int PS_WARPS = PS_THREADS / 32;
constexpr int PS_MAX_CTAS = 1024;

// Device-resident scalars of one curve.  Written only by device code during a
// descent (single writer per field: the last CTA of a kernel), read by the host
// after a stream synchronisation.
struct DevScalars {
    double J2, Jarc, dJdl, Dnorm, G2;   // of the last evaluated state
    double lambda, lambda_next, tau;
    double f2_plus, f2_minus;           // |f(u_+)|^2, |f(u_-)|^2 (spatial norm)
    double u2_plus, u2_minus;           // |u_+|^2, |u_-|^2
    double tol, dtau, dtau_lambda;
    long long step, limit;
    int done, active, status, conv;
    int lambda_free;
    int err;                            // nonzero: a bounded wait in a kernel gave up (launch invalid)
    long long wait_cycles;              // bound of the first mbarrier wait of a kernel (0: about 2^31
                                        // cycles; < 0: give up at once, a test of the error path)
    unsigned int cnt_rows, cnt_gemm;    // arrival counters of the last-CTA reductions
    unsigned long long bar;             // arrivals at the persistent step's grid barriers
};

// Cycles a kernel's first bounded wait may spin for this curve (the waits that
// follow a failed one, which wait for copies still in flight, keep the full bound).
constexpr long long WAIT_CYCLES = 1ll << 31;
__host__ __device__ inline long long wait_bound(const DevScalars &s) { return s.wait_cycles ? s.wait_cycles : WAIT_CYCLES; }

// Gates of the kernels of one descent step:
//   rows kernel:   skip when done or step >= limit (clears `active`)
//   gemm kernels:  skip when !active
enum RowsMode { ROWS_STEP = 0, ROWS_EVAL = 1 };
// GM_STEP (clustered four-step form only): GM_UPDATE, then GM_STORE of the
// updated state in the same launch.
// The three-launch four-step form on the Toeplitz and Hankel parts (single
// curves, f4h) chains a step's two contractions: GM_UPDATE_F is GM_UPDATE whose
// third pass also runs the first pass of D_t u of the updated columns (the same
// CTA lines and scratch locations), GM_STORE_P23 the rest of that D_t u.
enum GemmMode { GM_STORE = 0, GM_UPDATE = 1, GM_GRAD = 2, GM_STEP = 3, GM_UPDATE_F = 4, GM_STORE_P23 = 5 };

// Offsets into the caller's workspace.
struct Layout {
    size_t off_chat, off_ftw;          // FFT form: kernel spectrum [F], twiddles [F] (complex)
    size_t off_f4s;                    // four-step form: scratch [N/2][F] (complex)
    int F;                             // 0: dense contraction
    size_t off_U, off_D, off_R, off_A, off_G, off_X;
    size_t off_rowsc, off_bpart, off_tile, off_tcnt, off_part, off_gpart;
    size_t off_cot, off_sig, off_tau, off_sw, off_twr, off_w;
    size_t off_twid, off_twid64, off_kj, off_aj, off_prec, off_ends, off_pert, off_sc;
    size_t total;
    int bn, tiles_r, tiles_c, ksplit, kchunk, row_blocks;
    int tc, tc_bn, tc_tiles_r, tc_tiles_c, tc_ksplit, tc_kchunk;   // tensor-core form (tc = 1)
    int f4, F1, F2;                    // four-step FFT form (f4 = 1): F = F1 F2
    int f4c;                           // its clustered one-launch variant: cluster size (0: three passes)
    int f4b;                           // its one-CTA-per-mode variant (batched curves; F1 F2 in shared memory)
    int f4h;                           // the three-launch form on the Toeplitz and Hankel parts (F >= 2P + 1)
    int xtc;                           // split-BF16 tensor-core row phase: parts per operand (0: FFT row phase)
    size_t off_xdft;                   // its DFT matrices, split into BF16 parts
    int impl;                          // full-linear-implicit stepping: its eigenbases (0: IMEX)
    size_t off_iv, off_ivi, off_imu;   // V (even block, then odd), V^-1 likewise, eigenvalues (FP64)
    size_t off_isc;                    // the split partials of its two products
    size_t off_ivtc;                   // V^-1 and V as tensor-core operands
    int ivtc;                          // 1: that region exists (single curves, FP32 storage, N >= 32)
    int isplits;                       // K chunks they hold
    int hs;                            // sine storage (odd sections): rows of N/2 words, Im u^_j at j
    int w;                             // stored words per section: N, or N/2 with sine storage
};

// Tensor maps of a single curve's fields U and D_t U for the row phase's tile
// loads (TMA): 2D [N_s][W] in the storage type, box W x ROWS_PER_CTA.
struct RowMaps {
    CUtensorMap u, d;
};

struct CurveDev {
    int ns, nx, P, prec;   // prec: 0 = double, 1 = float
    int sym;               // symmetry bits 0 and 1 of ks_params (coefficients held at zero)
    int hs;                // sine storage: every field row holds Im u^_j at column j (odd sections)
    int W;                 // words per stored row: nx, or nx / 2 with sine storage
    double L, S, s0;
    void *U, *D, *R, *A, *G;
    void *X;               // FP64 physical scratch [N_s][N]
    double *rowsc;         // [N_s][4] row sums (end rows: |u|^2, |f|^2)
    double *bpart;         // [row_blocks][5] per-CTA partial sums of the row phase
    double *tile;          // [tiles] per-tile |G|^2 partials
    unsigned *tcnt;        // [tiles] split arrival counters (zero between launches)
    void *part;            // persistent step: [ksplit][N_s][N] split partial sums (else null)
    double *gpart;         // persistent step: [PS_MAX_CTAS] per-CTA |G|^2 partials
    int bn, tiles_r, tiles_c, ksplit, kchunk, row_blocks;
    int tc, tc_bn, tc_tiles_r, tc_tiles_c, tc_ksplit, tc_kchunk;   // tensor-core form (tc = 1)
    int f4, F1, F2;                    // four-step FFT form (f4 = 1): F = F1 F2
    int f4c;                           // its clustered one-launch variant: cluster size (0: three passes)
    int f4b;                           // its one-CTA-per-mode variant (batched curves; F1 F2 in shared memory)
    int f4h;                           // the three-launch form on the Toeplitz and Hankel parts: the
                                       // spectra of both ([k1][k2] each, Toeplitz first) in chat
    int xtc;               // split-BF16 tensor-core row phase: parts per operand (2 or 3; 0: FFT row phase)
    void *xdft;            // its DFT matrices C (inverse) and E (forward), three BF16 parts, operand layout
    int impl;              // full-linear-implicit stepping (Sec. V.C.3): the eigenbases of the
                           // interior D_t^2 in its even and odd parts under s -> -s
    int ine, ino;          // their sizes: ceil(M/2), floor(M/2)
    void *iv, *ivi;        // V_e [ine][ine] then V_o [ino][ino], row-major (storage type); V^-1 alike
    double *imu;           // eigenvalues: ine of the even part, then ino of the odd part
    void *isc;             // split partials of the increment's products: 2 isplits [M][N]
    void *ivtc;            // V^-1 and V as split-BF16 tensor-core operands (FP32 storage, N >= 32; else null)
    int isplits;           // K chunks those partials hold (IMP_SPLIT_MAX; 1 for batched curves)
    int F;                 // FFT length of the s-contraction (0: dense form)
    void *chat, *ftw;      // FFT form: kernel spectrum / F and twiddles (complex, storage type);
                           // four-step form: spectrum stored [k1][k2] for k = k1 + F1 k2 (both
                           // scrambled), twiddles W_F^p [F] then W_F^(n2 k1) as [n2][k1] and [k1][n2]
    void *f4s;             // four-step form: scratch [N/2][F1][F2] (complex, storage type)
    void *cot, *sig, *tau, *sw, *twr;
    double *w;
    void *twid, *twid64, *kj, *aj, *prec_imex;
    double *ends, *pert;
    DevScalars *sc;
    const RowMaps *rowmaps;   // host pointer: U and D tile maps of a single curve's row phase (else null)
};

// A curve whose step chains its two contractions (GM_UPDATE_F, GM_STORE_P23).
inline bool f4h_chained(const CurveDev &c) { return c.f4 && c.f4h && !c.f4c && !c.f4b && !c.impl; }

// allow_split = 0 lays a curve out without split contractions (batched curves
// get their parallelism from the batch); bn = 0 picks the column tile width.
// hs = 1 lays the fields out in sine storage (rows of nx / 2 words).
Layout make_layout(int ns, int nx, int prec, int allow_split = 1, int bn = 0, int s_transform = 0,
                   int persistent = 0, int xtc = 0, int impl = 0, int hs = 0);
// Layout of a single curve with parameters p (persistent: room for the
// persistent step's partials when p asks for that launch form).
inline Layout curve_layout(const ks_params *p, int persistent)
{
    const int xtc = xtc_of(p->precision);   // the persistent step has its own (FFT) row phase
    return make_layout(p->ns, p->nx, storage32(p->precision), 1, 0, p->s_transform, persistent && !xtc, xtc,
                       p->scheme == KS_SCHEME_IMPLICIT, (p->symmetry & KS_SYM_SINE) ? 1 : 0);
}
// Pointers of a curve whose workspace starts at `base` (256-byte aligned).
CurveDev bind_layout(const ks_params *p, const Layout &l, void *base);
// Encodes the row phase's tensor maps of U and D (FFT row phase); the caller keeps
// *m alive while c.rowmaps points to it.
cudaError_t make_row_maps(const CurveDev &c, RowMaps *m);

// ks_capi.cu: parameter rules of the entry points, and the thread-local
// message returned by ks_last_error().
ks_status check_params(const ks_params *p);
ks_status report_error(ks_status s, const char *fmt, ...);

// ---- launchers (ks_kernels.cu); all enqueue on `st`, return the launch error
cudaError_t launch_setup(const CurveDev &c, double dtau, cudaStream_t st);
// Resets the scalars and the split arrival counters (which must start at zero).
cudaError_t launch_scalars_init(const CurveDev &c, double lambda, int lambda_free, double dtau,
                                double dtau_lambda, int conv, cudaStream_t st);
cudaError_t launch_set_limit(const CurveDev &c, long long nsteps, double tol, cudaStream_t st);
cudaError_t launch_set_lambda_tau(const CurveDev &c, double lambda, double tau, cudaStream_t st);
cudaError_t launch_set_wait_cycles(const CurveDev &c, long long cycles, cudaStream_t st);
// Trial curve (eq. KSE_initial_curve) into the FP64 scratch X.
cudaError_t launch_trial(const CurveDev &c, double a, int has_v, int npert, cudaStream_t st);
// X = (double) in  (a physical curve in the storage type)
cudaError_t launch_widen(const CurveDev &c, const void *in, cudaStream_t st);
// rows 0 and P of X = u_+ and u_-
cudaError_t launch_set_ends(const CurveDev &c, cudaStream_t st);
// spectral state = forward transform of X, computed in FP64 and rounded per
// coefficient to the storage type
cudaError_t launch_row_fwd_x(const CurveDev &c, void *spec, int keep_ends, cudaStream_t st);
// spectral state = forward transform of a physical curve given in the storage
// type: FP64 storage in FP64; FP32 storage in double-float arithmetic (about 44
// bits on the FP32 pipes, ks_dfloat.cuh), rounded per coefficient to FP32 as the
// FP64 transform of launch_row_fwd_x
cudaError_t launch_row_fwd(const CurveDev &c, const void *phys, void *spec, cudaStream_t st);
// spec -> phys; scale_mode 0: plain; 1: Euclidean gradient scaling -2 dx w_m
// and zero end rows.
cudaError_t launch_row_inv(const CurveDev &c, const void *spec, void *phys, int scale_mode, cudaStream_t st);
// Arming of the step limit by the first row phase of a descent call (instead of a
// separate kernel): limit = step + nsteps, the convergence tolerance, done and
// status cleared; `on` = 0 reads them from the scalars as set before.
struct StepArm {
    long long nsteps;
    double tol;
    int on;
};
cudaError_t launch_rows(const CurveDev &c, int mode, cudaStream_t st, StepArm arm = StepArm{0, 0.0, 0});
// Structured contraction along s.  op 0: D_t (columns scaled by tau, rows by
// sigma), op 1: W^-1 D_t^T W.  mode GM_STORE writes D_t U into D (gated when
// `gate`), GM_UPDATE applies the descent update to U, GM_GRAD writes G.
// pass_ev (may be null): for the three-launch four-step form, two events
// recorded on `st` after its first and second pass (per-pass timing).
cudaError_t launch_dt(const CurveDev &c, int mode, int discrete, int gate, cudaStream_t st,
                      cudaEvent_t *pass_ev = nullptr);
// Tensor-core form of the dense contraction (ks_tc.cu; c.tc set): the same
// modes and epilogue as the dense kernel.
cudaError_t launch_dt_tc(const CurveDev &c, int mode, int discrete, int gate, cudaStream_t st);

// Four-step FFT form (ks_fft4.cu; c.f4 set): set-up of the kernel spectrum and
// the s-contraction in the modes of launch_dt.
cudaError_t launch_setup_f4(const CurveDev &c, cudaStream_t st);
cudaError_t launch_f4(const CurveDev &c, int mode, int discrete, int gate, cudaStream_t st,
                      cudaEvent_t *pass_ev = nullptr);
// The one-CTA-per-mode four-step form: over the modes of one curve, or over the
// (curve, mode) items of a batch whose curves share F.
cudaError_t launch_f4b(const CurveDev &c, int mode, int discrete, int gate, cudaStream_t st);
cudaError_t launch_f4b_batch(int prec, int F1, int F2, const CurveDev *cv, const int2 *items, int nitems, int mode,
                             int discrete, int gate, cudaStream_t st);
// The splits F = F1 F2 the one-CTA-per-mode four-step form runs a length in (the
// first is the default of f4_split).
inline int f4b_splits(int F, int prec, int (&F1s)[3])
{
    int n = 0;
    int d1 = 0, d2 = 0;
    f4_split(F, d1, d2);
    F1s[n++] = d1;
    for (int f1 = 32; f1 <= 128; f1 <<= 1) {
        const int f2 = F / f1;
        if (f1 == d1 || f2 < 32 || f2 > 128 || f1 * f2 != F) continue;
        if (F == 8192 && !(prec && f1 == 128)) continue;   // F = 8192: 128 x 64, FP32 only
        if (n < 3) F1s[n++] = f1;
    }
    return n;
}

// Split-BF16 tensor-core row phase (ks_rows_tc.cu; c.xtc set): bytes of its DFT
// matrices, their set-up, and the row phase with the modes of launch_rows.
size_t xdft_bytes(int nx);
cudaError_t launch_setup_xdft(const CurveDev &c, cudaStream_t st);

// ---- full-linear-implicit stepping (ks_implicit.cu)
// Bytes of the eigenbases of a curve with N_s sections in the storage type, and
// of the split partials of the increment's two products (at most IMP_SPLIT_MAX
// K chunks each).
constexpr int IMP_SPLIT_MAX = 8;
size_t implicit_bytes(int ns, int prec);
size_t implicit_scratch_bytes(int ns, int nx, int prec, int splits);
// Work items of a batched curve's increment: (curve, bx, by, parity) of each
// product, (curve, bx, nbx, 0) of the finishing pass.
void implicit_batch_items(const CurveDev &c, int curve, std::vector<int4> &prod, std::vector<int4> &fin);
cudaError_t launch_implicit_batch(int prec, const CurveDev *cv, const int4 *prod, int nprod, const int4 *fin, int nfin,
                                  cudaStream_t st);
// ks_implicit_tc.cu: the two products on the tensor cores (single curves, FP32
// storage, N >= 32): operand bytes, their set-up, and one product (which = 0:
// forward, 1: back) writing the split partials.
size_t implicit_tc_bytes(int ns);
cudaError_t launch_setup_implicit_tc(const CurveDev &c, cudaStream_t st);
cudaError_t launch_implicit_tc(const CurveDev &c, int splits, int gate, cudaStream_t st, int which);
// One-time set-up: eigendecomposition of the interior D_t^2 (FP64, cuSOLVER,
// opened at run time), stored in the curve's workspace.  Synchronous.
ks_status setup_implicit(const CurveDev &c, cudaStream_t st);
// The increment of one step from G (written by the GM_GRAD contraction):
// U += V (dtau / (1 + dtau (a_j^2 - lambda^2 mu))) V^-1 G per parity, then the
// step's bookkeeping (step, tau, lambda); gated like the contractions.
cudaError_t launch_implicit_update(const CurveDev &c, int gate, cudaStream_t st);
cudaError_t launch_rows_tc(const CurveDev &c, int mode, cudaStream_t st, StepArm arm);

// Persistent step (ks_step.cu): nsteps descent steps of a dense-form curve
// (c.part set) in one cooperative launch; stops early with the curve's gates.
cudaError_t launch_step_persistent(const CurveDev &c, int discrete, long long nsteps, cudaStream_t st);

// ---- batched launches over (curve, block) work items; cv is a device array of curves
// warps: 4 or 8 per CTA (2 sections per warp); the items' blocks and each curve's
// row_blocks must use the same width.
cudaError_t launch_rows_batch(int prec, int N, int warps, const CurveDev *cv, const int2 *items, int nitems, int mode,
                              cudaStream_t st);
cudaError_t launch_dt_batch(int prec, int bn, const CurveDev *cv, const int4 *items, int nitems, int mode,
                            int discrete, int gate, cudaStream_t st);
cudaError_t launch_set_limit_batch(const CurveDev *cv, int nb, long long nsteps, double tol, cudaStream_t st);
// FFT-form s-contraction over (curve, mode) items; smem sized for F_max
cudaError_t launch_sconv_batch(int prec, int F_max, const CurveDev *cv, const int2 *items, int nitems, int mode,
                               int discrete, int gate, cudaStream_t st);

}  // namespace ks
