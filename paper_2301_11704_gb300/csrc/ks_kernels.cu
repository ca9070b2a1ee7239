// ks_kernels.cu -- sm_103a kernels of one adjoint-descent step for a curve of
// KSE states (Ashtari & Schneider, arXiv 2301.11704).
//
// Data layout (every field): row-major [N_s][N] real words of the storage type T.
// Row m holds section s_m spectrally: N/2 complex Fourier coefficients
// u^_{m,j}, j = 0..N/2-1, interleaved (re, im); the Nyquist coefficient is not
// stored (held at zero) and Im u^_{m,0} = 0.  Row 0 is s = +inf, row N_s-1 is
// s = -inf (eq. t_grid).  Sine storage (odd sections, symmetry bit 2): rows of
// N/2 words, Im u^_{m,j} at column j (the real parts are zero).
//
// One descent step is three kernels:
//   k_rows  (x-direction, one warp per pair of sections): f(u), r = f - l D_t u,
//           the spatial adjoint (Df)^T r = u r_x - r_xx - r_xxxx, FP64 row sums,
//           and in its last CTA the FP64 cost, J_arc, dJ^2/dl and the
//           convergence decision.
//   k_dt    (s-direction): e = l D_t r^ (or -l W^-1 D_t^T W r^), G = -(A + e)
//           and the semi-implicit update of u, FP64 |G|^2; then
//   k_dt    again: D_t u of the new state, kept for the next step.
// D_t (eq. rational_diff_matrix) is never stored: its entries are
//   D_{j,m} = sigma_j (cot[(j+m) mod 2P] + cot[(j-m) mod 2P]) tau_m,
//   sigma_j = -(-1)^j sin^2(j pi/P) / (2S),  tau_m = (-1)^m / cbar_m,
//   cot[t] = cot(pi t / (2P)), cot[0] = 0,  P = M + 1,
// the closed form of the k-sum in eq. rational_diff_matrix, generated per tile
// from an O(N_s) table.
#include <cmath>
#include <map>
#include <type_traits>
#include <utility>

#include <cooperative_groups.h>

#include "ks_device.cuh"
#include "ks_dfloat.cuh"

namespace ks {

// ---------------------------------------------------------------------------
// Layout of the workspace
// ---------------------------------------------------------------------------
static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

Layout make_layout(int ns, int nx, int prec, int allow_split, int bn, int s_transform, int persistent, int xtc,
                   int impl, int hs)
{
    Layout l{};
    size_t b = prec ? 4 : 8;
    // sine storage: every field row and every s-contraction has nx / 2 columns
    // (the Fourier tables and the physical scratch keep nx)
    l.hs = hs ? 1 : 0;
    const int w = hs ? nx / 2 : nx;
    l.w = w;
    // s_transform 0 (auto): a single curve (allow_split) takes the measured rule,
    // batched curves the one-CTA FFT form wherever it fits
    int form = SF_DENSE;
    // batched curves: the FFT form with one CTA per mode wherever it fits, its
    // four-step variant (register line transforms) from F = 1024 on
    // (F >= 2P + 1 there, so FP64 curves up to N_s = 2048 fit its 4096 points)
    bool batched_f4 = false;
    if (!allow_split && (s_transform == 0 || s_transform == 2)) {
        const int f1 = fft_size(ns, prec), fh = fft4h_size(ns, F4B_FMIN);
        if (f1 && f1 < F4B_FMIN) form = SF_FFT1;
        else if (fh && fh <= (prec ? F4B_FMAX_F32 : F4B_FMAX_F64)) {
            form = SF_FFT4;
            batched_f4 = true;
        } else if (f1) form = SF_FFT1;
    }
    else if (s_transform == 0) form = auto_form(ns, w, prec);   // by the contraction's columns
    else if (s_transform == 2) form = fft_size(ns, prec) ? SF_FFT1 : (fft4_size(ns, prec) ? SF_FFT4 : SF_DENSE);
    else if (s_transform == 4) form = fft4_size(ns, prec, 1) ? SF_FFT4 : SF_DENSE;
    else if (s_transform == 5) form = fft4_size(ns, prec, 1) ? SF_FFT4C : SF_DENSE;
    if (form == SF_FFT1) l.F = fft_size(ns, prec);
    // the three-launch form of a single curve and the batched one-CTA-per-mode
    // form: Toeplitz and Hankel parts, F >= 2P + 1
    const bool f4h = form == SF_FFT4 && fft4h_size(ns, batched_f4 ? F4B_FMIN : F4_FMIN) > 0;
    if (form == SF_FFT4 || form == SF_FFT4C) {   // the four-step form
        l.F = f4h ? fft4h_size(ns, batched_f4 ? F4B_FMIN : F4_FMIN) : fft4_size(ns, prec, 1);
        l.f4 = 1;
        l.f4h = f4h ? 1 : 0;
        f4_split(l.F, l.F1, l.F2);
        l.f4c = (form == SF_FFT4C && f4c_fits(prec, l.F1, l.F2)) ? F4C_CS : 0;
        l.f4b = batched_f4 ? 1 : 0;
    }
    size_t field = al256((size_t)ns * w * b);
    // tiling and split of the s-contraction (over the w stored columns)
    l.bn = bn ? bn : (w >= 64 ? 64 : 32);
    l.tiles_r = (ns + DT_BM - 1) / DT_BM;
    l.tiles_c = (w + l.bn - 1) / l.bn;
    int tiles = l.tiles_r * l.tiles_c;
    int tiles_max = l.tiles_r * ((w + 31) / 32);        // buffers sized for the narrowest tiles
    if (tiles_max < w / 2) tiles_max = w / 2;            // the FFT form has one CTA per column pair
    int ks = (allow_split && tiles < DT_TARGET_CTAS) ? DT_TARGET_CTAS / tiles : 1;
    int kmax = ns / DT_MIN_KCHUNK;
    if (ks > kmax) ks = kmax;
    if (ks > DT_MAX_SPLIT) ks = DT_MAX_SPLIT;
    if (ks < 1) ks = 1;
    int kc = (ns + ks - 1) / ks;
    kc = (kc + DT_BK - 1) / DT_BK * DT_BK;
    l.kchunk = kc;
    l.ksplit = (ns + kc - 1) / kc;
    l.row_blocks = (ns + ROWS_PER_CTA - 1) / ROWS_PER_CTA;
    // tensor-core form of the dense contraction: FP32 storage, single curves,
    // asked for (s_transform 3) or picked by the measured rule (auto)
    if (prec && allow_split && !hs && l.F == 0 && (s_transform == 3 || (s_transform == 0 && tc_preferred(ns, nx)))) {
        l.tc = 1;
        l.tc_bn = nx >= 64 ? 64 : (nx >= 32 ? 32 : 16);
        l.tc_tiles_c = (nx + l.tc_bn - 1) / l.tc_bn;
        l.tc_tiles_r = (ns + TC_M - 1) / TC_M;
        const int tt = l.tc_tiles_c * l.tc_tiles_r;
        int tks = tt < DT_TARGET_CTAS ? DT_TARGET_CTAS / tt : 1;
        if (tks > ns / DT_MIN_KCHUNK) tks = ns / DT_MIN_KCHUNK;
        if (tks > DT_MAX_SPLIT) tks = DT_MAX_SPLIT;
        if (tks < 1) tks = 1;
        int tkc = (ns + tks - 1) / tks;
        tkc = (tkc + TC_KC - 1) / TC_KC * TC_KC;
        l.tc_kchunk = tkc;
        l.tc_ksplit = (ns + tkc - 1) / tkc;
    }
    size_t off = 0;
    l.off_U = off; off += field;
    l.off_D = off; off += field;
    l.off_R = off; off += field;
    l.off_A = off; off += field;
    l.off_G = off; off += field;
    l.off_X = off; off += al256((size_t)ns * nx * 8);   // physical scratch, always FP64
    l.off_rowsc = off; off += al256((size_t)ns * 4 * 8);
    l.off_bpart = off; off += al256((size_t)l.row_blocks * 5 * 8);
    size_t ntile = (size_t)tiles_max * DT_MAX_SPLIT;                   // either contraction form
    if (l.f4 && ntile < (size_t)(l.F2 / 8) * (w / 2)) ntile = (size_t)(l.F2 / 8) * (w / 2);   // four-step CTAs
    l.off_tile = off; off += al256(ntile * 8);
    l.off_tcnt = off; off += al256((size_t)tiles_max * 4);
    // the persistent step's split partials and per-CTA |G|^2 partials (single
    // curves in the dense form that asked for it)
    const bool persist = persistent && allow_split && !hs && l.F == 0;
    l.off_part = off; off += persist ? al256((size_t)l.ksplit * ns * nx * b) : 0;
    l.off_gpart = off; off += persist ? al256((size_t)PS_MAX_CTAS * 8) : 0;
    int P = ns - 1;
    l.off_cot = off; off += al256((size_t)2 * P * b);
    l.off_sig = off; off += al256((size_t)ns * b);
    l.off_tau = off; off += al256((size_t)ns * b);
    l.off_sw = off; off += al256((size_t)ns * b);
    l.off_twr = off; off += al256((size_t)ns * b);
    l.off_w = off; off += al256((size_t)ns * 8);
    l.off_twid = off; off += al256((size_t)nx * b);   // N/2 complex
    l.off_twid64 = off; off += al256((size_t)nx * 8); // N/2 complex, FP64
    l.off_kj = off; off += al256((size_t)(nx / 2) * b);
    l.off_aj = off; off += al256((size_t)(nx / 2) * b);
    l.off_prec = off; off += al256((size_t)(nx / 2) * b);
    l.off_ends = off; off += al256((size_t)2 * nx * 8);
    l.off_pert = off; off += al256((size_t)(nx + MAX_PERT + MAX_PERT * nx) * 8);
    l.off_sc = off; off += al256(sizeof(DevScalars));
    l.off_chat = off; off += l.F ? al256((size_t)l.F * 2 * b * (l.f4h ? 2 : 1)) : 0;
    l.off_ftw = off; off += l.F ? al256((size_t)l.F * (l.f4 ? 3 : 1) * 2 * b) : 0;   // four-step: + step twiddles
    // the three-launch form's scratch (also the FP64 set-up scratch, 32 F bytes);
    // the one-CTA-per-mode variant needs the set-up's only
    l.off_f4s = off; off += l.f4 ? al256(l.f4b ? (size_t)32 * l.F : (size_t)(w / 2) * l.F * 2 * b) : 0;
    // the split-BF16 row phase's DFT matrices
    l.xtc = xtc;
    l.off_xdft = off; off += xtc ? al256(xdft_bytes(nx)) : 0;
    // the implicit step's eigenbases (V and V^-1 of both parts) and eigenvalues
    l.impl = impl;
    const size_t ne = (size_t)(ns - 1) / 2, no = (size_t)(ns - 2) / 2;   // ceil(M/2), floor(M/2)
    l.off_iv = off; off += impl ? al256((ne * ne + no * no) * b) : 0;
    l.off_ivi = off; off += impl ? al256((ne * ne + no * no) * b) : 0;
    l.off_imu = off; off += impl ? al256((ne + no) * 8) : 0;
    l.isplits = allow_split ? IMP_SPLIT_MAX : 1;
    l.off_isc = off; off += impl ? al256(implicit_scratch_bytes(ns, nx, prec, l.isplits)) : 0;
    l.ivtc = (impl && prec && allow_split && nx >= 32) ? 1 : 0;
    l.off_ivtc = off; off += l.ivtc ? al256(implicit_tc_bytes(ns)) : 0;
    l.total = off;
    return l;
}

CurveDev bind_layout(const ks_params *p, const Layout &l, void *base)
{
    CurveDev d{};
    char *b = (char *)base;
    d.ns = p->ns;
    d.nx = p->nx;
    d.P = p->ns - 1;
    d.prec = storage32(p->precision);
    d.sym = p->symmetry & 3;
    d.hs = l.hs;
    d.W = l.w;
    d.L = p->L;
    d.S = p->S;
    d.s0 = p->s0;
    d.U = b + l.off_U;
    d.D = b + l.off_D;
    d.R = b + l.off_R;
    d.A = b + l.off_A;
    d.G = b + l.off_G;
    d.X = b + l.off_X;
    d.rowsc = (double *)(b + l.off_rowsc);
    d.bpart = (double *)(b + l.off_bpart);
    d.tile = (double *)(b + l.off_tile);
    d.tcnt = (unsigned *)(b + l.off_tcnt);
    d.part = l.off_gpart > l.off_part ? (void *)(b + l.off_part) : nullptr;
    d.gpart = l.off_gpart > l.off_part ? (double *)(b + l.off_gpart) : nullptr;
    d.bn = l.bn;
    d.tiles_r = l.tiles_r;
    d.tiles_c = l.tiles_c;
    d.ksplit = l.ksplit;
    d.kchunk = l.kchunk;
    d.row_blocks = l.row_blocks;
    d.F = l.F;
    d.tc = l.tc;
    d.tc_bn = l.tc_bn;
    d.tc_tiles_r = l.tc_tiles_r;
    d.tc_tiles_c = l.tc_tiles_c;
    d.tc_ksplit = l.tc_ksplit;
    d.tc_kchunk = l.tc_kchunk;
    d.chat = l.F ? (void *)(b + l.off_chat) : nullptr;
    d.ftw = l.F ? (void *)(b + l.off_ftw) : nullptr;
    d.f4s = l.f4 ? (void *)(b + l.off_f4s) : nullptr;
    d.f4 = l.f4;
    d.F1 = l.F1;
    d.F2 = l.F2;
    d.f4c = l.f4c;
    d.f4b = l.f4b;
    d.f4h = l.f4h;
    d.xtc = l.xtc;
    d.xdft = l.xtc ? (void *)(b + l.off_xdft) : nullptr;
    d.impl = l.impl;
    d.ine = (p->ns - 1) / 2;
    d.ino = (p->ns - 2) / 2;
    d.iv = l.impl ? (void *)(b + l.off_iv) : nullptr;
    d.ivi = l.impl ? (void *)(b + l.off_ivi) : nullptr;
    d.imu = l.impl ? (double *)(b + l.off_imu) : nullptr;
    d.isc = l.impl ? (void *)(b + l.off_isc) : nullptr;
    d.isplits = l.isplits;
    d.ivtc = l.ivtc ? (void *)(b + l.off_ivtc) : nullptr;
    d.cot = b + l.off_cot;
    d.sig = b + l.off_sig;
    d.tau = b + l.off_tau;
    d.sw = b + l.off_sw;
    d.twr = b + l.off_twr;
    d.w = (double *)(b + l.off_w);
    d.twid = b + l.off_twid;
    d.twid64 = b + l.off_twid64;
    d.kj = b + l.off_kj;
    d.aj = b + l.off_aj;
    d.prec_imex = b + l.off_prec;
    d.ends = (double *)(b + l.off_ends);
    d.pert = (double *)(b + l.off_pert);
    d.sc = (DevScalars *)(b + l.off_sc);
    return d;
}

// ---------------------------------------------------------------------------
// Set-up: rational-Chebyshev tables (eq. t_grid, eq. c_bar, eq. rational_diff_matrix),
// quadrature weights and Fourier tables, all evaluated in FP64 from integer indices.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_setup(CurveDev c, double dtau)
{
    const int P = c.P, ns = c.ns, H = c.nx / 2;
    T *cot = (T *)c.cot, *sig = (T *)c.sig, *tau = (T *)c.tau, *sw = (T *)c.sw, *twr = (T *)c.twr;
    cpx<T> *twid = (cpx<T> *)c.twid;
    T *kj = (T *)c.kj, *aj = (T *)c.aj, *pr = (T *)c.prec_imex;
    int total = max(2 * P, max(ns, H));
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        if (i < 2 * P) {
            double v = 0.0;
            if (i != 0) {
                double s, co;
                sincospi((double)i / (2.0 * P), &s, &co);
                v = co / s;
            }
            cot[i] = (T)v;
        }
        if (i < ns) {
            double s, co;
            sincospi((double)i / (double)P, &s, &co);
            double sn2 = s * s;
            double sgn = (i & 1) ? -1.0 : 1.0;
            bool end = (i == 0 || i == P);
            double cb = end ? 2.0 : 1.0;
            sig[i] = (T)(-sgn * sn2 / (2.0 * c.S));
            tau[i] = (T)(sgn / cb);
            c.w[i] = end ? 0.0 : (M_PI / (double)P) * c.S / sn2;
            sw[i] = end ? T(0) : (T)(-sgn * M_PI / (2.0 * P));               // sigma_i w_i
            twr[i] = end ? T(0) : (T)(sgn * sn2 * (double)P / (M_PI * c.S));  // tau_i / w_i
        }
        if (i < H) {
            double s, co;
            sincospi(2.0 * (double)i / (double)c.nx, &s, &co);
            twid[i] = {(T)co, (T)(-s)};
            ((cpx<double> *)c.twid64)[i] = {co, -s};
            double k = 2.0 * M_PI * (double)i / c.L;
            double a = k * k * k * k - k * k;
            kj[i] = (T)k;
            aj[i] = (T)a;
            pr[i] = (T)(1.0 / (1.0 + dtau * a * a));
        }
    }
}

__global__ void k_scalars_init(DevScalars *sc, unsigned *tcnt, int ntiles, double lambda, int lambda_free,
                               double dtau, double dtau_lambda, int conv)
{
    for (int i = threadIdx.x; i < ntiles; i += blockDim.x) tcnt[i] = 0u;
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        DevScalars z{};
        z.lambda = lambda;
        z.lambda_next = lambda;
        z.lambda_free = lambda_free;
        z.dtau = dtau;
        z.dtau_lambda = dtau_lambda;
        z.conv = conv;
        z.limit = 0;
        *sc = z;
    }
}

__global__ void k_set_wait_cycles(DevScalars *sc, long long cycles)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) sc->wait_cycles = cycles;
}

__global__ void k_set_limit(DevScalars *sc, long long nsteps, double tol)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        sc->limit = sc->step + nsteps;
        sc->tol = tol;
        sc->done = 0;
        sc->status = 0;
        sc->active = 0;
    }
}

__global__ void k_set_lambda_tau(DevScalars *sc, double lambda, double tau)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        sc->lambda = lambda;
        sc->lambda_next = lambda;
        sc->tau = tau;
        sc->step = 0;
        sc->limit = 0;
        sc->done = 0;
        sc->status = 0;
    }
}

// Trial curve (eq. KSE_initial_curve) on the grid, physical, into X:
//   u0 = 1/2[(1 + tanh s_m) u_+ + (1 - tanh s_m) u_-] + a exp(-s_m^2) v
//        + sum_p amps_p sin(p theta_m) vp_p ;   rows 0 and P are u_+ and u_-.
template <typename T>
__global__ void k_trial(CurveDev c, double a, int has_v, int npert)
{
    const int ns = c.ns, N = c.nx, P = c.P;
    const double *up = c.ends, *um = c.ends + N;
    const double *v = c.pert, *amps = c.pert + N, *vp = c.pert + N + MAX_PERT;
    double *X = (double *)c.X;
    size_t total = (size_t)ns * N;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        int m = (int)(i / N), n = (int)(i % N);
        double val;
        if (m == 0) {
            val = up[n];
        } else if (m == P) {
            val = um[n];
        } else {
            double s, co;
            sincospi((double)m / (double)P, &s, &co);
            double sm = c.s0 + c.S * co / s;
            double t = tanh(sm);
            val = 0.5 * ((1.0 + t) * up[n] + (1.0 - t) * um[n]);
            if (has_v) val += a * exp(-sm * sm) * v[n];
            for (int p = 0; p < npert; ++p) {
                double sp, cp;
                long long idx = ((long long)(p + 1) * m) % (2LL * P);
                sincospi((double)idx / (double)P, &sp, &cp);
                val += amps[p] * sp * vp[(size_t)p * N + n];
            }
        }
        X[i] = val;
    }
}

// X (FP64 physical scratch) = a physical curve given in the storage type.
template <typename T>
__global__ void k_widen(CurveDev c, const T *in)
{
    size_t total = (size_t)c.ns * c.nx;
    double *X = (double *)c.X;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
        X[i] = (double)in[i];
}

// Replaces rows 0 and P of a physical curve with u_+ and u_-.
__global__ void k_set_ends(CurveDev c)
{
    const int N = c.nx, P = c.P;
    double *X = (double *)c.X;
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
        X[n] = c.ends[n];
        X[(size_t)P * N + n] = c.ends[N + n];
    }
}

// ---------------------------------------------------------------------------
// Row transforms (physical <-> spectral), two sections per warp
// ---------------------------------------------------------------------------
// Physical (input type Ti) -> spectral in the compute type Tc, rounded to the
// storage type To per coefficient.
template <typename Ti, typename Tc, typename To, int N>
__global__ void __launch_bounds__(ROWS_WARPS * 32) k_row_fwd(CurveDev c, const Ti *phys, To *spec, int keep_ends)
{
    constexpr int H = N / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<Tc> *tw = (cpx<Tc> *)smem_raw;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cpx<Tc> *B0 = tw + H + warp * 2 * N, *B1 = B0 + N;
    for (int t = threadIdx.x; t < H; t += blockDim.x) {
        if constexpr (std::is_same<Tc, dfloat>::value) {   // from the FP64 table
            const cpx<double> w = ((const cpx<double> *)c.twid64)[t];
            tw[t] = {dfloat(w.x), dfloat(w.y)};
        } else {
            tw[t] = ((const cpx<Tc> *)(sizeof(Tc) == 8 ? c.twid64 : c.twid))[t];
        }
    }
    __syncthreads();
    const int ns = c.ns;
    const int m0 = (blockIdx.x * ROWS_WARPS + warp) * 2, m1 = m0 + 1;
    if (m0 >= ns) return;
    const bool has1 = m1 < ns;
    for (int n = lane; n < N; n += 32)
        B0[n] = {(Tc)phys[(size_t)m0 * N + n], has1 ? (Tc)phys[(size_t)m1 * N + n] : Tc(0)};
    __syncwarp();
    cpx<Tc> *W = warp_fft<Tc, N>(B0, B1, tw, false, lane);
    for (int j = lane; j < H; j += 32) {
        cpx<Tc> A, B;
        get_pair<Tc, N>(W, j, A, B);
        A = project(A, j, c.sym);
        B = project(B, j, c.sym);
        if (!(keep_ends && (m0 == 0 || m0 == c.P))) stm(spec, m0, N, j, cpx<To>{(To)A.x, (To)A.y}, c.hs);
        if (has1 && !(keep_ends && m1 == c.P)) stm(spec, m1, N, j, cpx<To>{(To)B.x, (To)B.y}, c.hs);
    }
}

template <typename T, int N>
__global__ void __launch_bounds__(ROWS_WARPS * 32) k_row_inv(CurveDev c, const T *spec, T *phys, int scale_mode)
{
    constexpr int H = N / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T> *tw = (cpx<T> *)smem_raw;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cpx<T> *B0 = tw + H + warp * 2 * N, *B1 = B0 + N;
    for (int t = threadIdx.x; t < H; t += blockDim.x) tw[t] = ((const cpx<T> *)c.twid)[t];
    __syncthreads();
    const int ns = c.ns, P = c.P;
    const int m0 = (blockIdx.x * ROWS_WARPS + warp) * 2, m1 = m0 + 1;
    if (m0 >= ns) return;
    const bool has1 = m1 < ns;
    for (int j = lane; j < H; j += 32) {
        cpx<T> A = ldm(spec, m0, N, j, c.hs);
        cpx<T> B = has1 ? ldm(spec, m1, N, j, c.hs) : cpx<T>{0, 0};
        put_pair<T, N>(B0, j, A, B);
    }
    if (lane == 0) B0[H] = {0, 0};
    __syncwarp();
    cpx<T> *Z = warp_fft<T, N>(B0, B1, tw, true, lane);
    T f0 = 1, f1 = 1;
    if (scale_mode == 1) {   // Euclidean gradient: -2 dx w_m, zero on the end rows
        const double dx = c.L / (double)N;
        f0 = (m0 == 0 || m0 == P) ? T(0) : (T)(-2.0 * dx * c.w[m0]);
        f1 = (!has1 || m1 == P) ? T(0) : (T)(-2.0 * dx * c.w[m1]);
    }
    for (int n = lane; n < N; n += 32) {
        cpx<T> z = Z[n];
        phys[(size_t)m0 * N + n] = f0 * z.x;
        if (has1) phys[(size_t)m1 * N + n] = f1 * z.y;
    }
}

// use_tm: the CTA's rows of U and D_t U come in by TMA through the tensor maps tm
template <typename T, int N>
__global__ void __launch_bounds__(ROWS_WARPS * 32) k_rows(CurveDev c, int mode, StepArm arm,
                                                          const __grid_constant__ RowMaps tm, int use_tm)
{
    rows_body<T, N>(c, mode, blockIdx.x, gridDim.x, true, arm, use_tm ? &tm : nullptr);
}

// Batched row phase: work item (curve, row block) per CTA; every curve keeps its
// own gates, counters and reductions.
template <typename T, int N, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_rows_batch(const CurveDev *cv, const int2 *items, int mode)
{
    const int2 it = items[blockIdx.x];
    const CurveDev &c = cv[it.x];
    rows_body<T, N, WARPS>(c, mode, it.y, c.row_blocks, true);
}

// ---------------------------------------------------------------------------
// s-direction: structured contraction with D_t (or W^-1 D_t^T W)
// ---------------------------------------------------------------------------
// Y[j][col] = rowscale_j * sum_m (cot[(j+m) mod 2P] + tsign cot[(j-m) mod 2P]) colscale_m X[m][col]
//   D_t:          colscale = tau, rowscale = sigma, tsign = +1
//   W^-1 D_t^T W: colscale = sigma w, rowscale = tau / w, tsign = -1
// CTA (tile_c, tile_r, ks) computes a DT_BM x BN output tile over the sections
// [ks kchunk, (ks+1) kchunk) (DtContract).  With ksplit > 1 the splits of a tile
// form one thread-block cluster: each CTA sums one row band of the tile over the
// splits' partial tiles in split order (distributed shared memory;
// deterministic) and runs the epilogue on it:
//   GM_STORE:  D = Y                                  (D_t u of the new state)
//   GM_UPDATE: e = +l Y (published adjoint) or -l Y (discrete adjoint),
//              G = -(A^ + e) on interior rows, u += dtau G / (1 + dtau a_j^2)
//              (the semi-implicit step of Sec. V.C.3 in its algebraically
//              equivalent increment form), FP64 sum_m w_m |G_m|^2
//   GM_GRAD:   as GM_UPDATE but G is written out instead of updating u.
template <typename T, int BN>
__device__ __forceinline__ void dt_body(const CurveDev &c, int mode, int discrete, int gate, int tile_c, int tile_r,
                                        int ks, int tiles_c, int tiles_r)
{
    namespace cg = cooperative_groups;
    constexpr int BM = DT_BM, TM = 2, TN = BN / 16;
    __shared__ DtTiles<T, BN> sm;
    __shared__ __align__(16) T Pt[BM][BN];       // this split's partial tile (read by the cluster)
    __shared__ double red[DT_THREADS];
    __shared__ int am_last;
    DevScalars *sc = c.sc;
    pdl_wait();
    const int g_active = sc->active;
    const double lam_d = sc->lambda, dtau_d = sc->dtau;

    const int ns = c.ns, N = c.W, P = c.P, hs = c.hs;   // N: the stored columns
    const T *rowscale = (const T *)(discrete ? c.twr : c.sig);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int j0 = tile_r * BM, c0 = tile_c * BN;
    DtContract<T, BN> k;
    k.X = (const T *)(mode == GM_STORE ? c.U : c.R);
    k.cot = (const T *)c.cot;
    k.colscale = (const T *)(discrete ? c.sw : c.tau);
    k.tsign = discrete ? T(-1) : T(1);
    k.N = N;
    k.twoP = 2 * P;
    k.j0 = j0;
    k.c0 = c0;
    k.kbeg = ks * c.kchunk;
    k.kend = min(ns, k.kbeg + c.kchunk);
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int l = 0; l < TN; ++l) acc[i][l] = T(0);
    if (k.kbeg < k.kend) k.fetch(k.kbeg);

    // Outputs this CTA finishes: with splits, the row band [r0, r1) of the tile
    // (slot q = element threadIdx.x + q * DT_THREADS of the band); without, the
    // thread's own accumulators.  Their epilogue operands are prefetched here,
    // before the contraction, so their loads overlap it.
    constexpr int EP = TM * TN;
    const int nsplit = c.ksplit;
    const int rows_per = (BM + nsplit - 1) / nsplit;
    const int r0 = min(BM, ks * rows_per), r1 = min(BM, r0 + rows_per);
    auto slot = [&](int q, int &j, int &col) -> bool {
        if (nsplit > 1) {
            const int e = threadIdx.x + q * DT_THREADS;
            if (e >= (r1 - r0) * BN) return false;
            j = j0 + r0 + e / BN;
            col = c0 + e % BN;
        } else {
            j = j0 + ty * TM + q / TN;
            col = c0 + tx * TN + q % TN;
        }
        return j < ns && col < N;
    };
    const T *Ah = (const T *)c.A, *pr = (const T *)c.prec_imex;
    T pA[EP], pU[EP], pS[EP], pP[EP];
    double pW[EP];
#pragma unroll
    for (int q = 0; q < EP; ++q) {
        int j = 0, col = 0;
        const bool ok = slot(q, j, col);
        pS[q] = ok ? rowscale[j] : T(0);
        pA[q] = (ok && mode != GM_STORE) ? Ah[(size_t)j * N + col] : T(0);
        pU[q] = (ok && mode == GM_UPDATE) ? ((const T *)c.U)[(size_t)j * N + col] : T(0);
        pP[q] = (ok && mode == GM_UPDATE) ? pr[col_mode(col, hs)] : T(0);
        pW[q] = (ok && mode != GM_STORE) ? c.w[j] : 0.0;
    }
    if (gate && !g_active) return;
    k.run(sm, acc);

    // ---- sum of the splits of this tile inside the cluster (distributed shared memory)
    const int ntiles = tiles_c * tiles_r;
    if (nsplit > 1) {
        cg::cluster_group cluster = cg::this_cluster();
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int l = 0; l < TN; ++l) Pt[ty * TM + i][tx * TN + l] = acc[i][l];
        cluster.sync();
        // this CTA's row band, read from every split in split order
        for (int e = threadIdx.x; e < (r1 - r0) * BN; e += DT_THREADS) {
            const int jj = r0 + e / BN, cc = e % BN;
            T t = T(0);
            for (int q = 0; q < nsplit; ++q) {
                const T *rem = cluster.map_shared_rank(&Pt[0][0], q);
                t += rem[jj * BN + cc];
            }
            ((T *)sm.Ks)[e] = t;   // the band's sums, row-major with BN per row
        }
        cluster.sync();           // no CTA leaves while its partial tile may still be read
        __syncthreads();
    }

    // ---- epilogue over the slots (operands prefetched above)
    T *Dout = (T *)c.D;
    const T lam = (T)lam_d, dtau = (T)dtau_d;
    T *U = (T *)c.U, *G = (T *)c.G;
    double partsum = 0.0;
#pragma unroll
    for (int q = 0; q < EP; ++q) {
        int j = 0, col = 0;
        if (!slot(q, j, col)) continue;
        const T y0 = (nsplit > 1) ? ((T *)sm.Ks)[threadIdx.x + q * DT_THREADS] : acc[q / TN][q % TN];
        const T y = pS[q] * y0;
        if (mode == GM_STORE) {
            Dout[(size_t)j * N + col] = y;
            continue;
        }
        const bool interior = (j > 0 && j < P);
        T g = 0;
        if (interior && col_live(col, c.sym, hs)) {
            const T e = discrete ? -lam * y : lam * y;
            g = -(pA[q] + e);
            const double cw = col_weight(col, hs);
            partsum += pW[q] * cw * (double)g * (double)g;
        }
        if (mode == GM_UPDATE) {
            if (interior) U[(size_t)j * N + col] = pU[q] + dtau * pP[q] * g;
        } else {
            G[(size_t)j * N + col] = g;
        }
    }
    if (mode == GM_STORE) return;

    // ---- FP64 |G|^2: per-CTA partial, last CTA of the grid sums them in a fixed order
    partsum = block_sum<DT_THREADS>(partsum, red);
    const int bid = (ks * tiles_r + tile_r) * tiles_c + tile_c, nb = ntiles * nsplit;
    if (threadIdx.x == 0) c.tile[bid] = partsum;
    if (!last_cta_arrive(&sc->cnt_gemm, (unsigned)nb, am_last)) return;
    double t = 0.0;
    for (int b = threadIdx.x; b < nb; b += DT_THREADS) t += __ldcg(c.tile + b);
    t = block_sum<DT_THREADS>(t, red);
    if (threadIdx.x == 0) {
        sc->G2 = c.L * t;
        if (mode == GM_UPDATE) {
            sc->step += 1;
            sc->tau += sc->dtau;
            sc->lambda = sc->lambda_next;
        }
        sc->cnt_gemm = 0;
    }
}

template <typename T, int BN>
__global__ void __launch_bounds__(DT_THREADS) k_dt(CurveDev c, int mode, int discrete, int gate)
{
    dt_body<T, BN>(c, mode, discrete, gate, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y);
}

// Batched s-phase: work item (curve, tile_c, tile_r) per CTA, curves laid out
// without splits (ksplit = 1).
template <typename T, int BN>
__global__ void __launch_bounds__(DT_THREADS) k_dt_batch(const CurveDev *cv, const int4 *items, int mode,
                                                          int discrete, int gate)
{
    const int4 it = items[blockIdx.x];
    const CurveDev &c = cv[it.x];
    dt_body<T, BN>(c, mode, discrete, gate, it.y, it.z, 0, c.tiles_c, c.tiles_r);
}

// ---------------------------------------------------------------------------
// s-direction, FFT form
// ---------------------------------------------------------------------------
// After the column scaling x'_m = colscale_m x_m, the contraction
//   y_j = sum_{m=0}^{P} (cot[(j+m) mod 2P] + tsign cot[(j-m) mod 2P]) x'_m,  j = 0..P,
// is the circular convolution of length 2P of the cot table with the extension
//   z_0 = (1+tsign) x'_0, z_m = tsign x'_m (0<m<P), z_P = (1+tsign) x'_P, z_{2P-m} = x'_m,
// and, as only j <= P is needed, equals the zero-padded circular convolution of
// any length F >= 3P with c_F[t] = cot[t] (0 <= t <= P), c_F[F-t] = cot[2P-t]
// (0 < t < 2P), 0 elsewhere.  With F a power of two:
//   y = IFFT_F( FFT_F(c_F) / F * FFT_F(z) )[0..P],
// two real columns (the real and imaginary parts of one Fourier mode) packed
// into one complex transform (c_F is real).

// Twiddles e^{-2 pi i t / F} (t < F) and the kernel spectrum FFT(c_F)/F, by a
// direct DFT in FP64 over the 3P nonzero entries with integer-indexed phases.
template <typename T>
__global__ void k_setup_fft(CurveDev c)
{
    // FP64 tables per CTA: e^{-2 pi i p / F} (p < F) and cot(pi u / 2P) (u < 2P)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int F = c.F, P = c.P, twoP = 2 * P;
    double2 *w64 = (double2 *)smem_raw;
    double *cot64 = (double *)(w64 + F);
    for (int p = threadIdx.x; p < F; p += blockDim.x) {
        double ps, pc;
        sincospi(2.0 * (double)p / (double)F, &ps, &pc);
        w64[p] = make_double2(pc, ps);
    }
    for (int u = threadIdx.x; u < twoP; u += blockDim.x) {
        double sn, cs;
        sincospi((double)u / (2.0 * P), &sn, &cs);
        cot64[u] = u ? cs / sn : 0.0;
    }
    __syncthreads();
    cpx<T> *ftw = (cpx<T> *)c.ftw, *chat = (cpx<T> *)c.chat;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= F) return;
    ftw[k] = {(T)w64[k].x, (T)(-w64[k].y)};
    double re = 0.0, im = 0.0;
    for (int t = -(twoP - 1); t <= P; ++t) {
        const int u = (t % twoP + twoP) % twoP;
        if (u == 0) continue;
        const double cv = cot64[u];
        const int idx = t >= 0 ? t : F + t;
        const double2 wv = w64[(int)(((long long)k * idx) % F)];
        re += cv * wv.x;
        im -= cv * wv.y;
    }
    chat[k] = {(T)(re / F), (T)(im / F)};
}

// ---- bulk copy global -> shared through an mbarrier (the copy engine; no
// tensor map).  Every wait is bounded: after about one second of polling it
// records the failure in the curve's scalars and the launch is invalid.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Thread-level: arm the barrier for `bytes` and start the copy (both 16-byte aligned,
// bytes a multiple of 16).
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity`; false when the bound ran out (a negative
// bound gives up at once: the error path's test).
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, long long bound = WAIT_CYCLES)
{
    if (bound < 0) return false;
    const long long t0 = clock64();
    while (!mbar_test(bar, parity))
        if (clock64() - t0 > bound) return false;
    return true;
}

// Stockham FFT of runtime length F (a power of two) by the whole CTA: radix-4
// stages, then one radix-2 stage when log2(F) is odd; natural order in and out.
// tw[u] = e^{-2 pi i u / F}, u < F.  Each thread keeps two butterflies in flight
// (all their operands loaded before any result is stored).  Returns the buffer
// holding the result.
template <typename T>
__device__ __forceinline__ void r4_load(const cpx<T> *x, const cpx<T> *tw, int j, int Q, int ns, int step, bool inverse,
                                        cpx<T> (&a)[4])
{
    const int k = j & (ns - 1);
    const int u = k * step;
    cpx<T> w1 = tw[u], w2 = tw[2 * u], w3 = tw[3 * u];
    if (inverse) { w1.y = -w1.y; w2.y = -w2.y; w3.y = -w3.y; }
    a[0] = x[j];
    a[1] = cmul(x[j + Q], w1);
    a[2] = cmul(x[j + 2 * Q], w2);
    a[3] = cmul(x[j + 3 * Q], w3);
}

template <typename T>
__device__ __forceinline__ void r4_store(cpx<T> *y, int j, int ns, bool inverse, const cpx<T> (&a)[4])
{
    const int k = j & (ns - 1);
    const cpx<T> t0 = {a[0].x + a[2].x, a[0].y + a[2].y}, t1 = {a[0].x - a[2].x, a[0].y - a[2].y};
    const cpx<T> t2 = {a[1].x + a[3].x, a[1].y + a[3].y}, t3 = {a[1].x - a[3].x, a[1].y - a[3].y};
    // -i t3 (forward) or +i t3 (inverse)
    const cpx<T> t3r = inverse ? cpx<T>{-t3.y, t3.x} : cpx<T>{t3.y, -t3.x};
    const int o = (j - k) * 4 + k;
    y[o] = {t0.x + t2.x, t0.y + t2.y};
    y[o + ns] = {t1.x + t3r.x, t1.y + t3r.y};
    y[o + 2 * ns] = {t0.x - t2.x, t0.y - t2.y};
    y[o + 3 * ns] = {t1.x - t3r.x, t1.y - t3r.y};
}

template <typename T>
__device__ cpx<T> *block_fft(cpx<T> *x, cpx<T> *y, const cpx<T> *tw, int F, bool inverse)
{
    const int Q = F / 4, B = blockDim.x;
    int ns = 1;
    for (; ns * 4 <= F; ns *= 4) {
        const int step = Q / ns;
        for (int j0 = threadIdx.x; j0 < Q; j0 += 2 * B) {
            const int j1 = j0 + B;
            cpx<T> a0[4], a1[4];
            r4_load(x, tw, j0, Q, ns, step, inverse, a0);
            if (j1 < Q) r4_load(x, tw, j1, Q, ns, step, inverse, a1);
            r4_store(y, j0, ns, inverse, a0);
            if (j1 < Q) r4_store(y, j1, ns, inverse, a1);
        }
        __syncthreads();
        cpx<T> *t = x;
        x = y;
        y = t;
    }
    if (ns < F) {   // ns == F / 2: the last radix-2 stage
        for (int j = threadIdx.x; j < F / 2; j += B) {
            const int k = j & (ns - 1);
            cpx<T> a = x[j], b = x[j + F / 2];
            cpx<T> w = tw[k];
            if (inverse) w.y = -w.y;
            b = cmul(b, w);
            const int o = ((j - k) << 1) + k;
            y[o] = {a.x + b.x, a.y + b.y};
            y[o + ns] = {a.x - b.x, a.y - b.y};
        }
        __syncthreads();
        cpx<T> *t = x;
        x = y;
        y = t;
    }
    return x;
}

// Loads of the FFT-form kernel: the largest per-thread counts (F / threads for the
// spectrum, N_s / threads for the epilogue) fixed by the single-CTA size limits.
template <typename T> struct SconvMax;
template <> struct SconvMax<float> { static constexpr int SPEC = SC_FMAX_F32 / SC_THREADS, EPI = (SC_FMAX_F32 / 3 + 1 + SC_THREADS) / SC_THREADS; };
template <> struct SconvMax<double> { static constexpr int SPEC = SC_FMAX_F64 / SC_THREADS, EPI = (SC_FMAX_F64 / 3 + 1 + SC_THREADS) / SC_THREADS; };

template <typename T>
struct vec2;
template <> struct vec2<float> { using type = float2; };
template <> struct vec2<double> { using type = double2; };

template <typename T>
__device__ __forceinline__ void sconv_body(const CurveDev &c, int mode, int discrete, int gate, int jm, int nmodes)
{
    using V2 = typename vec2<T>::type;
    constexpr int SPEC = SconvMax<T>::SPEC, EPI = SconvMax<T>::EPI, ZCH = 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int F = c.F, P = c.P, N = c.W, ns = c.ns, B = SC_THREADS, t = threadIdx.x;
    cpx<T> *Z = (cpx<T> *)smem_raw, *Wb = Z + F, *tw = Wb + F;   // tw: F entries
    __shared__ double red[SC_THREADS];
    __shared__ int am_last;
    __shared__ unsigned long long bar;
    DevScalars *sc = c.sc;
    const cpx<T> *ftw = (const cpx<T> *)c.ftw, *chat = (const cpx<T> *)c.chat;
    // tables first (written at set-up): the kernel spectrum for the product after
    // the forward transform, and the twiddles by one bulk copy
    cpx<T> ch[SPEC];
#pragma unroll
    for (int i = 0; i < SPEC; ++i)
        if (t + i * B < F) ch[i] = chat[t + i * B];
    const bool bulk = ((reinterpret_cast<uintptr_t>(ftw) & 15) == 0);
    if (bulk && t == 0) {
        mbar_init(&bar, 1);
        bulk_load(tw, ftw, (unsigned)(F * sizeof(cpx<T>)), &bar);
    }
    if (!bulk)
        for (int k = t; k < F; k += B) tw[k] = ftw[k];
    pdl_wait();
    const int g_active = sc->active;
    const double lam_d = sc->lambda, dtau_d = sc->dtau;
    const long long wb = wait_bound(*sc);
    if (gate && !g_active) {
        // the thread that armed the barrier keeps the CTA alive until the copy has landed
        if (bulk && t == 0 && !mbar_wait(&bar, 0)) {
            atomicExch(&sc->err, 1);
            mbar_wait(&bar, 0);
        }
        return;
    }

    const T *X = (const T *)(mode == GM_STORE ? c.U : c.R);
    const T *colscale = (const T *)(discrete ? c.sw : c.tau);
    const T *rowscale = (const T *)(discrete ? c.twr : c.sig);
    const T s = discrete ? T(-1) : T(1);
    // the CTA's column pair (a Fourier mode in full storage, two modes' imaginary
    // parts in sine storage)
    const int ca = 2 * jm, cb = 2 * jm + 1;
    const bool oka = col_live(ca, c.sym, c.hs), okb = col_live(cb, c.sym, c.hs);
    // z of the two columns, packed as za + i zb; the (Re, Im) pair is one vector load
    for (int k0 = t; k0 < F; k0 += ZCH * B) {
        V2 xv[ZCH];
        T cs[ZCH];
        int mm[ZCH];
#pragma unroll
        for (int i = 0; i < ZCH; ++i) {
            const int k = k0 + i * B;
            int m = -1;
            T f = T(1);
            if (k == 0) { m = 0; f = T(1) + s; }
            else if (k < P) { m = k; f = s; }
            else if (k == P) { m = P; f = T(1) + s; }
            else if (k < 2 * P) { m = 2 * P - k; }
            if (f == T(0)) m = -1;
            mm[i] = m;
            cs[i] = f;
            if (m >= 0) {
                xv[i] = *reinterpret_cast<const V2 *>(X + (size_t)m * N + ca);
                cs[i] = f * colscale[m];
            }
        }
#pragma unroll
        for (int i = 0; i < ZCH; ++i) {
            const int k = k0 + i * B;
            if (k >= F) break;
            cpx<T> v = {0, 0};
            if (mm[i] >= 0) {
                v.x = oka ? cs[i] * xv[i].x : T(0);
                v.y = okb ? cs[i] * xv[i].y : T(0);
            }
            Z[k] = v;
        }
    }
    __syncthreads();   // z complete; the barrier's initialisation visible to every thread
    if (bulk && !mbar_wait(&bar, 0, wb)) {
        atomicExch(&sc->err, 1);
        mbar_wait(&bar, 0);   // the copy may still be writing this CTA's shared memory
    }
    cpx<T> *Y = block_fft<T>(Z, Wb, tw, F, false);
    cpx<T> *O = (Y == Z) ? Wb : Z;

    // epilogue operands of the sections j = t + i B, issued before the product
    T *Dout = (T *)c.D, *U = (T *)c.U, *G = (T *)c.G;
    const T *Ah = (const T *)c.A;
    const T pra = ((const T *)c.prec_imex)[col_mode(ca, c.hs)], prb = ((const T *)c.prec_imex)[col_mode(cb, c.hs)];
    T rs[EPI];
    double wj[EPI];
    V2 av[EPI], uv[EPI];
#pragma unroll
    for (int i = 0; i < EPI; ++i) {
        const int j = t + i * B;
        if (j < ns) {
            rs[i] = rowscale[j];
            if (mode != GM_STORE && j > 0 && j < P) {
                wj[i] = c.w[j];
                av[i] = *reinterpret_cast<const V2 *>(Ah + (size_t)j * N + ca);
                if (mode == GM_UPDATE) uv[i] = *reinterpret_cast<const V2 *>(U + (size_t)j * N + ca);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < SPEC; ++i)
        if (t + i * B < F) Y[t + i * B] = cmul(Y[t + i * B], ch[i]);
    __syncthreads();
    Y = block_fft<T>(Y, O, tw, F, true);

    // epilogue over the sections j = 0..P of the two columns
    const T lam = (T)lam_d, dtau = (T)dtau_d;
    const double cw = col_weight(cb, c.hs);   // column a's weight where it is live
    double partsum = 0.0;
#pragma unroll
    for (int i = 0; i < EPI; ++i) {
        const int j = t + i * B;
        if (j >= ns) break;
        const cpx<T> yv = {rs[i] * Y[j].x, rs[i] * Y[j].y};
        if (mode == GM_STORE) {
            *reinterpret_cast<V2 *>(Dout + (size_t)j * N + ca) = V2{oka ? yv.x : T(0), okb ? yv.y : T(0)};
            continue;
        }
        const bool interior = (j > 0 && j < P);
        T ga = 0, gb = 0;
        if (interior) {
            if (oka) ga = -(av[i].x + (discrete ? -lam * yv.x : lam * yv.x));
            if (okb) gb = -(av[i].y + (discrete ? -lam * yv.y : lam * yv.y));
            partsum += wj[i] * cw * (double)(ga * ga + gb * gb);
        }
        if (mode == GM_UPDATE) {
            if (interior)
                *reinterpret_cast<V2 *>(U + (size_t)j * N + ca) = V2{uv[i].x + dtau * pra * ga, uv[i].y + dtau * prb * gb};
        } else {
            *reinterpret_cast<V2 *>(G + (size_t)j * N + ca) = V2{ga, gb};
        }
    }
    if (mode == GM_STORE) return;

    partsum = block_sum<SC_THREADS>(partsum, red);
    if (threadIdx.x == 0) c.tile[jm] = partsum;
    if (!last_cta_arrive(&sc->cnt_gemm, (unsigned)nmodes, am_last)) return;
    double tt = 0.0;
    for (int b2 = threadIdx.x; b2 < nmodes; b2 += SC_THREADS) tt += __ldcg(c.tile + b2);
    tt = block_sum<SC_THREADS>(tt, red);
    if (threadIdx.x == 0) {
        sc->G2 = c.L * tt;
        if (mode == GM_UPDATE) {
            sc->step += 1;
            sc->tau += sc->dtau;
            sc->lambda = sc->lambda_next;
        }
        sc->cnt_gemm = 0;
    }
}

template <typename T>
__global__ void __launch_bounds__(SC_THREADS) k_sconv(CurveDev c, int mode, int discrete, int gate)
{
    sconv_body<T>(c, mode, discrete, gate, blockIdx.x, gridDim.x);
}

template <typename T>
__global__ void __launch_bounds__(SC_THREADS) k_sconv_batch(const CurveDev *cv, const int2 *items, int mode,
                                                            int discrete, int gate)
{
    const int2 it = items[blockIdx.x];
    const CurveDev &c = cv[it.x];
    sconv_body<T>(c, mode, discrete, gate, it.y, c.W / 2);
}

template <typename T>
static size_t sconv_smem(int F)
{
    return (size_t)(3 * F) * sizeof(cpx<T>);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------


static int row_grid(int ns) { return (ns + ROWS_PER_CTA - 1) / ROWS_PER_CTA; }


// Launches a step kernel with programmatic stream serialization (it may start
// while its predecessor finishes; see pdl_wait) and, for cluster_z > 0, thread-block
// clusters of 1 x 1 x cluster_z CTAs.
template <typename... KArgs, typename... Args>
static cudaError_t launch_step_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                      int cluster_z, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    int n = 0;
    attr[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[n].val.programmaticStreamSerializationAllowed = 1;
    ++n;
    if (cluster_z > 0) {
        attr[n].id = cudaLaunchAttributeClusterDimension;
        attr[n].val.clusterDim.x = 1;
        attr[n].val.clusterDim.y = 1;
        attr[n].val.clusterDim.z = cluster_z;
        ++n;
    }
    cfg.attrs = attr;
    cfg.numAttrs = n;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args...);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename T>
static cudaError_t rows_t(const CurveDev &c, int mode, cudaStream_t st, StepArm arm)
{
    static const RowMaps none{};
    const int use_tm = c.rowmaps ? 1 : 0;
    const RowMaps &tm = c.rowmaps ? *c.rowmaps : none;
    return dispatch_n(c.nx, [&](auto nn) {
        constexpr int NN = decltype(nn)::value;
        size_t sm = rows_smem<T>(NN, 3, ROWS_WARPS, use_tm ? c.W : 0);
        cudaError_t e = set_smem(k_rows<T, NN>, sm);
        if (e != cudaSuccess) return e;
        return launch_step_kernel(k_rows<T, NN>, dim3(row_grid(c.ns)), dim3(ROWS_WARPS * 32), sm, st, 0, c, mode, arm,
                                  tm, use_tm);
    });
}

// cuTensorMapEncodeTiled of the CUDA driver API, obtained through the runtime's
// entry-point query (no link against libcuda).
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

cudaError_t make_row_maps(const CurveDev &c, RowMaps *m)
{
    static EncodeTiled enc = nullptr;
    if (!enc) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        enc = (EncodeTiled)fn;
    }
    const size_t b = c.prec ? 4 : 8;
    const cuuint64_t dims[2] = {(cuuint64_t)c.W, (cuuint64_t)c.ns};        // columns, sections
    const cuuint64_t strides[1] = {(cuuint64_t)(c.W * b)};                // bytes between sections
    const cuuint32_t box[2] = {(cuuint32_t)c.W, (cuuint32_t)ROWS_PER_CTA};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt = c.prec ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    void *src[2] = {c.U, c.D};
    CUtensorMap *dst[2] = {&m->u, &m->d};
    for (int i = 0; i < 2; ++i)
        if (enc(dst[i], dt, 2, src[i], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    return cudaSuccess;
}

template <typename Ti, typename Tc, typename To>
static cudaError_t row_fwd_t(const CurveDev &c, const void *phys, void *spec, int keep_ends, cudaStream_t st)
{
    return dispatch_n(c.nx, [&](auto nn) {
        constexpr int NN = decltype(nn)::value;
        size_t sm = rows_smem<Tc>(NN, 2);
        cudaError_t e = set_smem(k_row_fwd<Ti, Tc, To, NN>, sm);
        if (e != cudaSuccess) return e;
        k_row_fwd<Ti, Tc, To, NN><<<row_grid(c.ns), ROWS_WARPS * 32, sm, st>>>(c, (const Ti *)phys, (To *)spec,
                                                                               keep_ends);
        return cudaGetLastError();
    });
}

template <typename T>
static cudaError_t row_inv_t(const CurveDev &c, const void *spec, void *phys, int scale_mode, cudaStream_t st)
{
    return dispatch_n(c.nx, [&](auto nn) {
        constexpr int NN = decltype(nn)::value;
        size_t sm = rows_smem<T>(NN, 2);
        cudaError_t e = set_smem(k_row_inv<T, NN>, sm);
        if (e != cudaSuccess) return e;
        k_row_inv<T, NN><<<row_grid(c.ns), ROWS_WARPS * 32, sm, st>>>(c, (const T *)spec, (T *)phys, scale_mode);
        return cudaGetLastError();
    });
}

cudaError_t launch_setup(const CurveDev &c, double dtau, cudaStream_t st)
{
    int total = 2 * c.P > c.ns ? 2 * c.P : c.ns;
    int grid = (total + 255) / 256;
    if (c.prec) k_setup<float><<<grid, 256, 0, st>>>(c, dtau);
    else k_setup<double><<<grid, 256, 0, st>>>(c, dtau);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && c.xtc) e = launch_setup_xdft(c, st);
    if (e != cudaSuccess || c.F == 0) return e;
    if (c.f4) return launch_setup_f4(c, st);
    const int g2 = (c.F + 255) / 256;
    const size_t sm = (size_t)c.F * sizeof(double2) + (size_t)2 * c.P * sizeof(double);
    if (c.prec) {
        if ((e = set_smem(k_setup_fft<float>, sm)) != cudaSuccess) return e;
        k_setup_fft<float><<<g2, 256, sm, st>>>(c);
    } else {
        if ((e = set_smem(k_setup_fft<double>, sm)) != cudaSuccess) return e;
        k_setup_fft<double><<<g2, 256, sm, st>>>(c);
    }
    return cudaGetLastError();
}

cudaError_t launch_scalars_init(const CurveDev &c, double lambda, int lambda_free, double dtau,
                                double dtau_lambda, int conv, cudaStream_t st)
{
    k_scalars_init<<<1, 256, 0, st>>>(c.sc, c.tcnt, c.tiles_r * c.tiles_c, lambda, lambda_free, dtau, dtau_lambda,
                                      conv);
    return cudaGetLastError();
}

cudaError_t launch_set_wait_cycles(const CurveDev &c, long long cycles, cudaStream_t st)
{
    k_set_wait_cycles<<<1, 32, 0, st>>>(c.sc, cycles);
    return cudaGetLastError();
}

cudaError_t launch_set_limit(const CurveDev &c, long long nsteps, double tol, cudaStream_t st)
{
    k_set_limit<<<1, 32, 0, st>>>(c.sc, nsteps, tol);
    return cudaGetLastError();
}

cudaError_t launch_set_lambda_tau(const CurveDev &c, double lambda, double tau, cudaStream_t st)
{
    k_set_lambda_tau<<<1, 32, 0, st>>>(c.sc, lambda, tau);
    return cudaGetLastError();
}

cudaError_t launch_trial(const CurveDev &c, double a, int has_v, int npert, cudaStream_t st)
{
    size_t total = (size_t)c.ns * c.nx;
    int grid = (int)((total + 255) / 256);
    if (grid > 4096) grid = 4096;
    if (c.prec) k_trial<float><<<grid, 256, 0, st>>>(c, a, has_v, npert);
    else k_trial<double><<<grid, 256, 0, st>>>(c, a, has_v, npert);
    return cudaGetLastError();
}

cudaError_t launch_set_ends(const CurveDev &c, cudaStream_t st)
{
    int grid = (c.nx + 255) / 256;
    k_set_ends<<<grid, 256, 0, st>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_widen(const CurveDev &c, const void *in, cudaStream_t st)
{
    size_t total = (size_t)c.ns * c.nx;
    int grid = (int)((total + 255) / 256);
    if (grid > 4096) grid = 4096;
    if (c.prec) k_widen<float><<<grid, 256, 0, st>>>(c, (const float *)in);
    else k_widen<double><<<grid, 256, 0, st>>>(c, (const double *)in);
    return cudaGetLastError();
}

cudaError_t launch_row_fwd_x(const CurveDev &c, void *spec, int keep_ends, cudaStream_t st)
{
    return c.prec ? row_fwd_t<double, double, float>(c, c.X, spec, keep_ends, st)
                  : row_fwd_t<double, double, double>(c, c.X, spec, keep_ends, st);
}

cudaError_t launch_row_fwd(const CurveDev &c, const void *phys, void *spec, cudaStream_t st)
{
    return c.prec ? row_fwd_t<float, dfloat, float>(c, phys, spec, 0, st)
                  : row_fwd_t<double, double, double>(c, phys, spec, 0, st);
}

cudaError_t launch_row_inv(const CurveDev &c, const void *spec, void *phys, int scale_mode, cudaStream_t st)
{
    return c.prec ? row_inv_t<float>(c, spec, phys, scale_mode, st) : row_inv_t<double>(c, spec, phys, scale_mode, st);
}

cudaError_t launch_rows(const CurveDev &c, int mode, cudaStream_t st, StepArm arm)
{
    if (c.xtc) return launch_rows_tc(c, mode, st, arm);
    return c.prec ? rows_t<float>(c, mode, st, arm) : rows_t<double>(c, mode, st, arm);
}

template <typename T, int BN>
static cudaError_t launch_dt_t(const CurveDev &c, int mode, int discrete, int gate, cudaStream_t st)
{
    return launch_step_kernel(k_dt<T, BN>, dim3(c.tiles_c, c.tiles_r, c.ksplit), dim3(DT_THREADS), 0, st, c.ksplit, c,
                              mode, discrete, gate);
}

template <typename T>
static cudaError_t launch_sconv_t(const CurveDev &c, int mode, int discrete, int gate, cudaStream_t st)
{
    const size_t sm = sconv_smem<T>(c.F);
    cudaError_t e = set_smem(k_sconv<T>, sm);
    if (e != cudaSuccess) return e;
    return launch_step_kernel(k_sconv<T>, dim3(c.W / 2), dim3(SC_THREADS), sm, st, 0, c, mode, discrete, gate);
}

cudaError_t launch_sconv_batch(int prec, int F_max, const CurveDev *cv, const int2 *items, int nitems, int mode,
                               int discrete, int gate, cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    cudaError_t e;
    if (prec) {
        const size_t sm = sconv_smem<float>(F_max);
        if ((e = set_smem(k_sconv_batch<float>, sm)) != cudaSuccess) return e;
        return launch_step_kernel(k_sconv_batch<float>, dim3(nitems), dim3(SC_THREADS), sm, st, 0, cv, items, mode,
                                  discrete, gate);
    } else {
        const size_t sm = sconv_smem<double>(F_max);
        if ((e = set_smem(k_sconv_batch<double>, sm)) != cudaSuccess) return e;
        return launch_step_kernel(k_sconv_batch<double>, dim3(nitems), dim3(SC_THREADS), sm, st, 0, cv, items, mode,
                                  discrete, gate);
    }
}

cudaError_t launch_dt(const CurveDev &c, int mode, int discrete, int gate, cudaStream_t st, cudaEvent_t *pass_ev)
{
    if (c.f4b) return launch_f4b(c, mode, discrete, gate, st);
    if (c.f4) return launch_f4(c, mode, discrete, gate, st, pass_ev);
    if (c.F > 0) return c.prec ? launch_sconv_t<float>(c, mode, discrete, gate, st)
                               : launch_sconv_t<double>(c, mode, discrete, gate, st);
    if (c.tc) return launch_dt_tc(c, mode, discrete, gate, st);
    if (c.bn == 64) return c.prec ? launch_dt_t<float, 64>(c, mode, discrete, gate, st)
                                  : launch_dt_t<double, 64>(c, mode, discrete, gate, st);
    return c.prec ? launch_dt_t<float, 32>(c, mode, discrete, gate, st)
                  : launch_dt_t<double, 32>(c, mode, discrete, gate, st);
}

template <typename T, int W>
static cudaError_t rows_batch_t(int N, const CurveDev *cv, const int2 *items, int nitems, int mode, cudaStream_t st)
{
    return dispatch_n(N, [&](auto nn) {
        constexpr int NN = decltype(nn)::value;
        size_t sm = rows_smem<T>(NN, 3, W);
        cudaError_t e = set_smem(k_rows_batch<T, NN, W>, sm);
        if (e != cudaSuccess) return e;
        return launch_step_kernel(k_rows_batch<T, NN, W>, dim3(nitems), dim3(W * 32), sm, st, 0, cv, items, mode);
    });
}

cudaError_t launch_rows_batch(int prec, int N, int warps, const CurveDev *cv, const int2 *items, int nitems, int mode,
                              cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    if (warps == 8)
        return prec ? rows_batch_t<float, 8>(N, cv, items, nitems, mode, st)
                    : rows_batch_t<double, 8>(N, cv, items, nitems, mode, st);
    if (warps != ROWS_WARPS) return cudaErrorInvalidValue;
    return prec ? rows_batch_t<float, ROWS_WARPS>(N, cv, items, nitems, mode, st)
                : rows_batch_t<double, ROWS_WARPS>(N, cv, items, nitems, mode, st);
}

cudaError_t launch_dt_batch(int prec, int bn, const CurveDev *cv, const int4 *items, int nitems, int mode,
                            int discrete, int gate, cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    const dim3 g(nitems), b(DT_THREADS);
    if (bn == 64)
        return prec ? launch_step_kernel(k_dt_batch<float, 64>, g, b, 0, st, 0, cv, items, mode, discrete, gate)
                    : launch_step_kernel(k_dt_batch<double, 64>, g, b, 0, st, 0, cv, items, mode, discrete, gate);
    return prec ? launch_step_kernel(k_dt_batch<float, 32>, g, b, 0, st, 0, cv, items, mode, discrete, gate)
                : launch_step_kernel(k_dt_batch<double, 32>, g, b, 0, st, 0, cv, items, mode, discrete, gate);
}

__global__ void k_set_limit_batch(const CurveDev *cv, int nb, long long nsteps, double tol)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += gridDim.x * blockDim.x) {
        DevScalars *sc = cv[i].sc;
        sc->limit = sc->step + nsteps;
        sc->tol = tol;
        sc->done = 0;
        sc->status = 0;
        sc->active = 0;
    }
}

cudaError_t launch_set_limit_batch(const CurveDev *cv, int nb, long long nsteps, double tol, cudaStream_t st)
{
    k_set_limit_batch<<<(nb + 127) / 128, 128, 0, st>>>(cv, nb, nsteps, tol);
    return cudaGetLastError();
}

}  // namespace ks
