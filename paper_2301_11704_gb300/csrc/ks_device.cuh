// ks_device.cuh -- device code shared by the translation units of the library:
// complex helpers, the warp-level FFT, reductions, the row phase of one
// evaluation (rows_body) and the staged s-contraction (DtContract).  Without
// device linking every translation unit compiles its own copy.
#pragma once

#include <map>
#include <type_traits>
#include <utility>

#include "ks_internal.h"
#include "ks_tcgen05.cuh"

namespace ks {

template <typename T>
struct cpx {
    T x, y;
};

template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b)
{
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// Programmatic dependent launch.  The step kernels are launched so that a kernel
// is set up while its predecessor in the stream drains (its CTAs start as the
// predecessor's CTAs exit, before the predecessor's completion is flushed):
// before pdl_wait() a kernel reads only the tables written at curve set-up
// (complete long before); pdl_wait() returns once the predecessor has completed
// and its writes are visible; every gate and every field is read after it, and
// no CTA leaves before it.  No kernel triggers its successor early: successor
// CTAs parked on the SMs during a whole kernel slowed graph replay (measured).
// A no-op for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Arrival of a CTA at a grid-wide last-CTA reduction, after the CTA has written
// its partials: a CTA barrier, then one acquire-release atomic add at GPU scope
// by thread 0 (its release covers the CTA's writes ordered before the barrier,
// its acquire makes every earlier arrival's partials visible to the last CTA).
// True in every thread of the CTA that arrives last.
__device__ __forceinline__ bool last_cta_arrive(unsigned *cnt, unsigned n, int &flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(prev) : "l"(cnt) : "memory");
        flag = (prev == n - 1);
    }
    __syncthreads();
    return flag != 0;
}

// ---------------------------------------------------------------------------
// Warp-level FFT on shared memory
// ---------------------------------------------------------------------------
// exp(-2 pi i t / N) for t < N from the half table tw[t], t < N/2
template <typename T, int N>
__device__ __forceinline__ cpx<T> tw_full(const cpx<T> *tw, int t)
{
    const cpx<T> w = tw[t < N / 2 ? t : t - N / 2];
    return t < N / 2 ? w : cpx<T>{-w.x, -w.y};
}

// Stockham FFT of length N by one warp: natural order in and out, no bit
// reversal.  tw[t] = exp(-2 pi i t / N), t < N/2.  Forward uses exp(-...),
// inverse exp(+...); neither scales.  Returns the buffer holding the result (x
// or y); the other one is free scratch.  FP32 and double-float: radix-4 stages,
// then one radix-2 stage when log2(N) is odd (half the stages, each a round
// trip through shared memory, which bounds these transforms: the FP32 row phase
// 10-17% faster at N = 128 and 256, measured on GB300).  FP64: radix 2 (on
// GB300's few FP64 pipes the radix-4 form's twiddle sign selections cost more
// than the stages it saves: its row phase measured 32% slower at N = 64).
template <typename T, int N>
__device__ __forceinline__ cpx<T> *warp_fft(cpx<T> *x, cpx<T> *y, const cpx<T> *tw, bool inverse, int lane)
{
    if constexpr (std::is_same<T, double>::value) {
#pragma unroll
        for (int ns = 1; ns < N; ns <<= 1) {
#pragma unroll
            for (int j = lane; j < N / 2; j += 32) {
                const int k = j & (ns - 1);
                cpx<T> a = x[j], b = x[j + N / 2];
                cpx<T> w = tw[k * (N / (2 * ns))];
                if (inverse) w.y = -w.y;
                b = cmul(b, w);
                const int o = ((j - k) << 1) + k;
                y[o] = {a.x + b.x, a.y + b.y};
                y[o + ns] = {a.x - b.x, a.y - b.y};
            }
            __syncwarp();
            cpx<T> *t = x;
            x = y;
            y = t;
        }
        return x;
    }
    constexpr int Q = N / 4;
    int ns = 1;
#pragma unroll
    for (; ns * 4 <= N; ns *= 4) {
#pragma unroll
        for (int j = lane; j < Q; j += 32) {
            const int k = j & (ns - 1);
            const int u = k * (Q / ns);   // exp(-2 pi i k / 4ns) = tw[u]
            cpx<T> w1 = tw_full<T, N>(tw, u), w2 = tw_full<T, N>(tw, 2 * u), w3 = tw_full<T, N>(tw, 3 * u);
            if (inverse) {
                w1.y = -w1.y;
                w2.y = -w2.y;
                w3.y = -w3.y;
            }
            const cpx<T> a0 = x[j], a1 = cmul(x[j + Q], w1), a2 = cmul(x[j + 2 * Q], w2), a3 = cmul(x[j + 3 * Q], w3);
            const cpx<T> t0 = {a0.x + a2.x, a0.y + a2.y}, t1 = {a0.x - a2.x, a0.y - a2.y};
            const cpx<T> t2 = {a1.x + a3.x, a1.y + a3.y}, t3 = {a1.x - a3.x, a1.y - a3.y};
            // -i t3 (forward) or +i t3 (inverse)
            const cpx<T> t3r = inverse ? cpx<T>{-t3.y, t3.x} : cpx<T>{t3.y, -t3.x};
            const int o = (j - k) * 4 + k;
            y[o] = {t0.x + t2.x, t0.y + t2.y};
            y[o + ns] = {t1.x + t3r.x, t1.y + t3r.y};
            y[o + 2 * ns] = {t0.x - t2.x, t0.y - t2.y};
            y[o + 3 * ns] = {t1.x - t3r.x, t1.y - t3r.y};
        }
        __syncwarp();
        cpx<T> *t = x;
        x = y;
        y = t;
    }
    if (ns < N) {   // ns == N / 2: the last radix-2 stage
#pragma unroll
        for (int j = lane; j < N / 2; j += 32) {
            cpx<T> a = x[j], b = x[j + N / 2];
            cpx<T> w = tw[j];
            if (inverse) w.y = -w.y;
            b = cmul(b, w);
            y[j] = {a.x + b.x, a.y + b.y};
            y[j + N / 2] = {a.x - b.x, a.y - b.y};
        }
        __syncwarp();
        cpx<T> *t = x;
        x = y;
        y = t;
    }
    return x;
}

// Full spectrum of z = a + i b for two real sections given by their half spectra
// (j = 0..N/2-1, Nyquist zero):  Z_j = A_j + i B_j,  Z_{N-j} = conj(A_j) + i conj(B_j).
template <typename T, int N>
__device__ __forceinline__ void put_pair(cpx<T> *Z, int j, cpx<T> A, cpx<T> B)
{
    Z[j] = {A.x - B.y, A.y + B.x};
    if (j > 0) Z[N - j] = {A.x + B.y, B.x - A.y};
}

// Half spectra of two real sections from the FFT W of z = a + i b, with the
// 1/N of the forward transform:  A_j = (W_j + conj W_{N-j}) / 2N,
// B_j = (W_j - conj W_{N-j}) / 2iN.
template <typename T, int N>
__device__ __forceinline__ void get_pair(const cpx<T> *W, int j, cpx<T> &A, cpx<T> &B)
{
    cpx<T> wj = W[j], wn = W[(N - j) & (N - 1)];
    const T h = T(0.5) / T(N);
    A = {(wj.x + wn.x) * h, (wj.y - wn.y) * h};
    B = {(wj.y + wn.y) * h, (wn.x - wj.x) * h};
    if (j == 0) { A.y = 0; B.y = 0; }
}

// Symmetric subspaces (Sec. V.B): bit 0 = odd sections (real parts of every
// coefficient zero), bit 1 = L/2-periodic sections (odd modes zero).
template <typename T>
__device__ __forceinline__ cpx<T> project(cpx<T> v, int j, int sym)
{
    if (sym & 1) v.x = T(0);
    if ((sym & 2) && (j & 1)) v = cpx<T>{0, 0};
    return v;
}

__device__ __forceinline__ bool col_allowed(int col, int sym)
{
    if ((sym & 1) && !(col & 1)) return false;
    if ((sym & 2) && ((col >> 1) & 1)) return false;
    return true;
}

template <typename T>
__device__ __forceinline__ cpx<T> ld2(const T *p, int m, int N, int j)
{
    const T *q = p + (size_t)m * N + 2 * j;
    return {q[0], j == 0 ? T(0) : q[1]};
}

template <typename T>
__device__ __forceinline__ void st2(T *p, int m, int N, int j, cpx<T> v)
{
    T *q = p + (size_t)m * N + 2 * j;
    q[0] = v.x;
    q[1] = (j == 0) ? T(0) : v.y;
}

// Columns of a stored row.  Full storage: Re and Im of mode j at columns 2j and
// 2j + 1 (column 1, the imaginary part of the real mean, is zero).  Sine storage
// (odd sections): Im of mode j at column j, N/2 columns (column 0, the mean's,
// is zero).  Every s-contraction treats its columns alike; only the mode of a
// column (its IMEX factor and norm weight) and whether the subspace keeps it
// depend on the storage.
__device__ __forceinline__ int col_mode(int col, int hs) { return hs ? col : col >> 1; }
__device__ __forceinline__ bool col_live(int col, int sym, int hs)
{
    if (hs) return col != 0 && !((sym & 2) && (col & 1));
    return col != 1 && col_allowed(col, sym);
}
// weight of a column in |q|^2 = L sum_j c_j |q^_j|^2 (c_0 = 1, c_j = 2)
__device__ __forceinline__ int col_weight(int col, int hs) { return col_mode(col, hs) == 0 ? 1 : 2; }

// Mode j of section m of a field of N-point sections in either storage (rows of N
// words, or N/2 in sine storage, whose real parts are zero).
template <typename T>
__device__ __forceinline__ cpx<T> ldm(const T *p, int m, int N, int j, int hs)
{
    if (hs) return {T(0), j == 0 ? T(0) : p[(size_t)m * (N / 2) + j]};
    return ld2(p, m, N, j);
}

template <typename T>
__device__ __forceinline__ void stm(T *p, int m, int N, int j, cpx<T> v, int hs)
{
    if (hs) {
        p[(size_t)m * (N / 2) + j] = (j == 0) ? T(0) : v.y;
        return;
    }
    st2(p, m, N, j, v);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums of five FP64 values over a warp with few FP64 instructions (GB300 issues
// a warp's FP64 instruction at a small fraction of the FP32 rate, whatever the
// number of active lanes): the values (padded to eight) are halved at each of the
// first three butterfly levels, each lane keeping the half its lane bit selects,
// so every lane adds 4 + 2 + 1 values there and then 1 + 1 (9 additions instead
// of 25).  Lane l ends with the total of value (l >> 2) & 7 (same in its four
// lanes).  Fixed order: deterministic.
__device__ __forceinline__ double warp_sum5(const double (&t)[5], int lane)
{
    double v8[8] = {t[0], t[1], t[2], t[3], t[4], 0.0, 0.0, 0.0};
    double v4[4], v2[2];
    const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0, b2 = (lane & 4) != 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const double keep = b4 ? v8[4 + i] : v8[i], give = b4 ? v8[i] : v8[4 + i];
        v4[i] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const double keep = b3 ? v4[2 + i] : v4[i], give = b3 ? v4[i] : v4[2 + i];
        v2[i] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
    }
    const double keep = b2 ? v2[1] : v2[0], give = b2 ? v2[0] : v2[1];
    double v = keep + __shfl_xor_sync(0xffffffffu, give, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v;
}

// Fixed-order block reduction (deterministic for a fixed blockDim).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *red)
{
    red[threadIdx.x] = v;
    __syncthreads();
#pragma unroll
    for (int s = NT / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// Row phase of one evaluation
// ---------------------------------------------------------------------------
// Per section m (two per warp, packed as one complex FFT):
//   u   = IDFT(u^)                      physical section
//   w^  = DFT(u^2) / N
//   f^  = -(1/2) i k w^ - a_j u^        (eq. KSE: -u u_x - u_xx - u_xxxx; a_j = k^4 - k^2)
//   r^  = f^ - l d^                     (eq. KSE_residual; 0 on rows 0 and P)
//   r_x = IDFT(i k r^)
//   A^  = DFT(u r_x) / N - a_j r^       ((Df)^T r = u r_x - r_xx - r_xxxx, eq. KSE_G)
// Row sums (Parseval, FP64): |r_m|^2, |d_m|^2, <d_m, r_m> (interior rows) and
// |u_m|^2, |f_m|^2 (end rows).  The last CTA to finish reduces them over m in a
// fixed order: J^2, J_arc, dJ^2/dl, |l d|_W, the end-section residuals, and
// (step mode) the convergence decision and the next lambda.
// FP64 reduction of the row phase over the per-unit partial sums c.bpart[0..nblk)
// in a fixed order (strided per thread, then a shuffle tree per warp, then the
// warps in order), the scalars derived from them (J^2, J_arc, dJ^2/dl, |l d|_W,
// the end-section residuals) and, in step mode, the convergence decision and
// the next lambda.  Called by every thread of a CTA of NT threads; thread 0
// writes the curve's scalars when `write`.  Returns to every thread 1 when the
// descent goes on (always 1 in evaluation mode).
template <int NT>
__device__ __forceinline__ int rows_finish(const CurveDev &c, int mode, int nblk, bool write,
                                           StepArm arm = StepArm{0, 0.0, 0})
{
    __shared__ double wred[NT / 32][5];
    __shared__ int go;
    DevScalars *sc = c.sc;
    const int P = c.P, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // thread 0's scalars and end-row sums, loaded together with the partials
    double lamd = 0, tol = 0, dtl = 0, u2p = 0, f2p = 0, u2m = 0, f2m = 0;
    int conv = 0, lfree = 0;
    if (threadIdx.x == 0) {
        lamd = sc->lambda;
        tol = arm.on ? arm.tol : sc->tol;
        dtl = sc->dtau_lambda;
        conv = sc->conv;
        lfree = sc->lambda_free;
        u2p = __ldcg(c.rowsc + 0);
        f2p = __ldcg(c.rowsc + 3);
        u2m = __ldcg(c.rowsc + 4 * (size_t)P + 0);
        f2m = __ldcg(c.rowsc + 4 * (size_t)P + 3);
    }
    double t[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblk; b += NT)
#pragma unroll
        for (int q = 0; q < 5; ++q) t[q] += __ldcg(c.bpart + (size_t)b * 5 + q);
    {
        const double ws = warp_sum5(t, lane);
        const int v = (lane >> 2) & 7;
        if ((lane & 3) == 0 && v < 5) wred[warp][v] = ws;
    }
    __syncthreads();
    // the sums over the warps (value q in lane q, the warps in order), then the two
    // square roots in lanes 1 and 2 while lane 0 divides
    __shared__ double rtot[5], rroot[3];
    if (warp == 0) {
        double r = 0.0;
        if (lane < 5)
            for (int w = 0; w < NT / 32; ++w) r += wred[w][lane];
        const double rj2 = __shfl_sync(0xffffffffu, r, 0), rd2 = __shfl_sync(0xffffffffu, r, 4);
        if (lane < 5) rtot[lane] = r;
        if (lane == 1 || lane == 2) rroot[lane] = sqrt(lane == 1 ? rj2 : rd2);
        __syncwarp();
    }
    if (threadIdx.x == 0) {
        const double t_j2 = rtot[0], t_num = rtot[1], t_den = rtot[2], t_dl = rtot[3];
        const double Jarc = t_den > 0 ? t_num / t_den : 0.0, dJdl = -2.0 * t_dl, Dnorm = rroot[2];
        int active = 1;
        if (write) {
            sc->J2 = t_j2;
            sc->Jarc = Jarc;
            sc->dJdl = dJdl;
            sc->Dnorm = Dnorm;
            sc->u2_plus = u2p;
            sc->f2_plus = f2p;
            sc->u2_minus = u2m;
            sc->f2_minus = f2m;
        }
        if (mode == ROWS_STEP) {
            const double J = rroot[1];
            const double crit = conv == 0 ? Jarc : (conv == 1 ? J : (Dnorm > 0 ? J / Dnorm : J));
            int done = 0, bad = 0;
            if (!isfinite(t_j2) || !isfinite(Jarc)) {
                bad = 1;
                done = 1;
                active = 0;
            } else if (tol > 0 && crit < tol) {
                done = 1;
                active = 0;
            }
            if (write) {
                if (bad) sc->status = 5;
                if (done) sc->done = 1;
                sc->active = active;
                sc->lambda_next = lfree ? lamd - dtl * dJdl : lamd;
            }
        }
        if (write) sc->cnt_rows = 0;
        go = active;
    }
    __syncthreads();
    return go;
}

// Shared-memory tiles of the row phase's TMA loads: U and D_t U rows of the CTA,
// [2 WARPS][W] each, 128-byte aligned after the transform buffers.
template <typename T, int N, int WARPS>
__device__ __forceinline__ T *rows_tiles(unsigned char *smem_raw)
{
    const size_t off = (size_t)(N / 2 + WARPS * 3 * N) * sizeof(cpx<T>);
    const unsigned a = tc::su32(smem_raw + off);
    return (T *)(smem_raw + off + ((128u - (a & 127u)) & 127u));
}

// tm (single curves): U and D_t U of the CTA's sections come in as two tiles by
// TMA (one tensor-map copy each, issued by thread 0 once the predecessor's writes
// are visible) instead of per-lane loads; rows past the curve read as zeros.
template <typename T, int N, int WARPS = ROWS_WARPS>
__device__ __forceinline__ void rows_body(const CurveDev &c, int mode, int blk, int nblk, bool tail,
                                          StepArm arm = StepArm{0, 0.0, 0}, const RowMaps *tm = nullptr)
{
    constexpr int H = N / 2;
    constexpr int MPL = (H + 31) / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T> *tw = (cpx<T> *)smem_raw;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cpx<T> *B0 = tw + H + warp * 3 * N, *B1 = B0 + N, *B2 = B1 + N;
    __shared__ double wpart[WARPS][5];
    __shared__ int am_last;
    __shared__ unsigned long long tbar;
    T *tileU = tm ? rows_tiles<T, N, WARPS>(smem_raw) : nullptr;
    T *tileD = tm ? tileU + (size_t)2 * WARPS * c.W : nullptr;
    if (tm && threadIdx.x == 0) {
        tc::bar_init(&tbar, 1);
        tc::fence_bar_init();
    }
    DevScalars *sc = c.sc;
    const int ns = c.ns, P = c.P, hs = c.hs;
    const T *U = (const T *)c.U, *D = (const T *)c.D;
    T *R = (T *)c.R, *A = (T *)c.A;
    const T *kj = (const T *)c.kj, *aj = (const T *)c.aj;
    const int m0 = (blk * WARPS + warp) * 2, m1 = m0 + 1;
    const bool has0 = m0 < ns, has1 = m1 < ns;

    // Every independent global load is issued before the first use: the
    // twiddles and the Fourier tables of the modes this lane owns (before the
    // predecessor has finished), then the gate, lambda and both sections of u and
    // D_t u (one memory round trip).
    const cpx<T> twv = ((int)threadIdx.x < H) ? ((const cpx<T> *)c.twid)[threadIdx.x] : cpx<T>{0, 0};
    cpx<T> ua[MPL], ub[MPL], ra[MPL], rb[MPL], dva[MPL], dvb[MPL];
    T kv[MPL], av[MPL];
#pragma unroll
    for (int i = 0; i < MPL; ++i) {
        const int j = lane + 32 * i;
        kv[i] = (j < H) ? kj[j] : T(0);
        av[i] = (j < H) ? aj[j] : T(0);
    }
    const T wm0 = has0 ? (T)c.w[m0] : T(0), wm1 = has1 ? (T)c.w[m1] : T(0);   // quadrature weights
    for (int t = threadIdx.x + blockDim.x; t < H; t += blockDim.x) tw[t] = ((const cpx<T> *)c.twid)[t];
    if (tm) __syncthreads();   // the barrier's initialisation, before any thread waits on it
    pdl_wait();
    if (tm && threadIdx.x == 0) {
        const unsigned tb = (unsigned)(2 * WARPS * c.W * sizeof(T));   // the whole box, zero-filled past N_s
        tc::expect_tx(&tbar, 2 * tb);
        tc::tensor_g2s_2d(tileU, &tm->u, 0, blk * 2 * WARPS, &tbar);
        tc::tensor_g2s_2d(tileD, &tm->d, 0, blk * 2 * WARPS, &tbar);
    }
    // an armed call starts from the current step with `done` cleared; block 0
    // records the limit for the later kernels before its arrival at the
    // reduction, which orders these writes before the last CTA's
    const int g_done = arm.on ? 0 : sc->done;
    const long long g_step = sc->step, g_limit = arm.on ? g_step + arm.nsteps : sc->limit;
    const double lamd0 = sc->lambda;
    if (arm.on && blk == 0 && threadIdx.x == 0) {
        sc->limit = g_limit;
        sc->tol = arm.tol;
        sc->done = 0;
        sc->status = 0;
    }
    const T *Us = U, *Ds = D;
    int r0 = m0, r1 = m1;
    if (tm) {
        // every thread waits for the tiles (bounded: a wait that gives up records
        // the error, then waits again so that no copy lands after the CTA is gone)
        if (!tc::bar_wait(&tbar, 0, wait_bound(*sc))) {
            atomicExch(&sc->err, 1);
            tc::bar_wait(&tbar, 0);
        }
        Us = tileU;
        Ds = tileD;
        r0 = 2 * warp;
        r1 = r0 + 1;
    }
#pragma unroll
    for (int i = 0; i < MPL; ++i) {
        const int j = lane + 32 * i;
        const bool ok = j < H;
        ua[i] = (ok && has0) ? ldm(Us, r0, N, j, hs) : cpx<T>{0, 0};
        ub[i] = (ok && has1) ? ldm(Us, r1, N, j, hs) : cpx<T>{0, 0};
        dva[i] = (ok && has0) ? ldm(Ds, r0, N, j, hs) : cpx<T>{0, 0};
        dvb[i] = (ok && has1) ? ldm(Ds, r1, N, j, hs) : cpx<T>{0, 0};
    }

    if (mode == ROWS_STEP && (g_done || g_step >= g_limit)) {
        if (blk == 0 && threadIdx.x == 0) sc->active = 0;
        return;
    }
    if ((int)threadIdx.x < H) tw[threadIdx.x] = twv;
    __syncthreads();
    const T lam = (T)lamd0;

    if (has0) {
        const bool in0 = (m0 > 0 && m0 < P), in1 = has1 && (m1 > 0 && m1 < P);
        // sums over the modes of a section, in the storage type (N/2 <= 128 terms);
        // sections are combined in FP64 below
        T s0[5] = {0, 0, 0, 0, 0}, s1[5] = {0, 0, 0, 0, 0};   // nr, nd, ndr, nu, nf
        // spectrum of u_a + i u_b
#pragma unroll
        for (int i = 0; i < MPL; ++i) {
            int j = lane + 32 * i;
            if (j < H) put_pair<T, N>(B0, j, ua[i], ub[i]);
        }
        if (lane == 0) B0[H] = {0, 0};
        __syncwarp();
        cpx<T> *Zu = warp_fft<T, N>(B0, B1, tw, true, lane);     // u_a + i u_b on the grid
        cpx<T> *Q = (Zu == B0) ? B1 : B0;
        for (int n = lane; n < N; n += 32) {
            cpx<T> z = Zu[n];
            B2[n] = z;
            Q[n] = {z.x * z.x, z.y * z.y};
        }
        __syncwarp();
        cpx<T> *Wq = warp_fft<T, N>(Q, Zu, tw, false, lane);     // DFT of u_a^2 + i u_b^2
#pragma unroll
        for (int i = 0; i < MPL; ++i) {
            int j = lane + 32 * i;
            if (j < H) {
                cpx<T> wa, wb;
                get_pair<T, N>(Wq, j, wa, wb);
                const T k = kv[i], a = av[i], hk = T(0.5) * k;
                cpx<T> fa = {hk * wa.y - a * ua[i].x, -hk * wa.x - a * ua[i].y};
                cpx<T> fb = {hk * wb.y - a * ub[i].x, -hk * wb.x - a * ub[i].y};
                const cpx<T> da = dva[i], db = dvb[i];
                ra[i] = in0 ? project(cpx<T>{fa.x - lam * da.x, fa.y - lam * da.y}, j, c.sym) : cpx<T>{0, 0};
                rb[i] = in1 ? project(cpx<T>{fb.x - lam * db.x, fb.y - lam * db.y}, j, c.sym) : cpx<T>{0, 0};
                if (j == 0) { ra[i].y = 0; rb[i].y = 0; fa.y = 0; fb.y = 0; }
                const T cw = (j == 0) ? T(1) : T(2);
                s0[0] += cw * (ra[i].x * ra[i].x + ra[i].y * ra[i].y);
                s0[1] += cw * (da.x * da.x + da.y * da.y);
                s0[2] += cw * (da.x * ra[i].x + da.y * ra[i].y);
                s0[3] += cw * (ua[i].x * ua[i].x + ua[i].y * ua[i].y);
                s0[4] += cw * (fa.x * fa.x + fa.y * fa.y);
                s1[0] += cw * (rb[i].x * rb[i].x + rb[i].y * rb[i].y);
                s1[1] += cw * (db.x * db.x + db.y * db.y);
                s1[2] += cw * (db.x * rb[i].x + db.y * rb[i].y);
                s1[3] += cw * (ub[i].x * ub[i].x + ub[i].y * ub[i].y);
                s1[4] += cw * (fb.x * fb.x + fb.y * fb.y);
            }
        }
        __syncwarp();
        // spectrum of (i k r^_a) + i (i k r^_b) -> r_x on the grid
        cpx<T> *X0 = Wq, *X1 = (Wq == B0) ? B1 : B0;
#pragma unroll
        for (int i = 0; i < MPL; ++i) {
            int j = lane + 32 * i;
            if (j < H) {
                const T k = kv[i];
                put_pair<T, N>(X0, j, cpx<T>{-k * ra[i].y, k * ra[i].x}, cpx<T>{-k * rb[i].y, k * rb[i].x});
            }
        }
        if (lane == 0) X0[H] = {0, 0};
        __syncwarp();
        cpx<T> *Rx = warp_fft<T, N>(X0, X1, tw, true, lane);
        cpx<T> *Y = (Rx == X0) ? X1 : X0;
        for (int n = lane; n < N; n += 32) {
            cpx<T> z = B2[n], q = Rx[n];
            Y[n] = {z.x * q.x, z.y * q.y};
        }
        __syncwarp();
        cpx<T> *Pp = warp_fft<T, N>(Y, Rx, tw, false, lane);     // DFT of u_a r_xa + i u_b r_xb
#pragma unroll
        for (int i = 0; i < MPL; ++i) {
            int j = lane + 32 * i;
            if (j < H) {
                cpx<T> pa, pb;
                get_pair<T, N>(Pp, j, pa, pb);
                const T a = av[i];
                stm(R, m0, N, j, ra[i], hs);
                stm(A, m0, N, j, project(cpx<T>{pa.x - a * ra[i].x, pa.y - a * ra[i].y}, j, c.sym), hs);
                if (has1) {
                    stm(R, m1, N, j, rb[i], hs);
                    stm(A, m1, N, j, project(cpx<T>{pb.x - a * rb[i].x, pb.y - a * rb[i].y}, j, c.sym), hs);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            s0[q] = warp_sum(s0[q]);
            s1[q] = warp_sum(s1[q]);
        }
        {
            // Per-section norms |q_m|^2 = L sum_j c_j |q^_j|^2.  The five section
            // terms are formed in the storage type, one per lane (lanes 5 q + k for
            // section q, term k), the four FP64 row sums in lanes 16 + 4 q + k; one
            // FP64 conversion for the warp, the two sections' terms summed in FP64.
            // (GB300 issues a warp's FP64 instruction at a small fraction of the
            // FP32 rate whatever the active lanes, so the lanes share the work.)
            const double lamd = lamd0;
            const T Lt = (T)c.L, alt = (T)fabs(lamd), l2 = (T)(lamd * lamd);
            const bool is_term = lane < 10, is_row = lane >= 16 && lane < 24;
            const int q = is_term ? lane / 5 : (is_row ? (lane - 16) >> 2 : 0);
            const int k = is_term ? lane % 5 : (lane - 16) & 3;
            T sv[5];
#pragma unroll
            for (int i = 0; i < 5; ++i) sv[i] = q ? s1[i] : s0[i];
            const bool ins = q ? in1 : in0, has = q ? has1 : true;
            const T nr = Lt * sv[0], nd = Lt * sv[1], ndr = Lt * sv[2];
            T val = T(0);
            if (is_term && ins) {
                const T w = q ? wm1 : wm0, sd = sqrt(nd);
                switch (k) {
                case 0: val = w * nr; break;                    // J^2
                case 1: val = w * sqrt(nr) * alt * sd; break;   // J_arc numerator
                case 2: val = w * alt * sd; break;              // J_arc denominator
                case 3: val = w * ndr; break;                   // <d, r>_W
                default: val = w * l2 * nd; break;              // |l d|_W^2
                }
            } else if (is_row) {
                switch (k) {
                case 0: val = ins ? nr : Lt * sv[3]; break;
                case 1: val = nd; break;
                case 2: val = ndr; break;
                default: val = Lt * sv[4]; break;
                }
            }
            const double dv = (double)val;
            const double d1 = __shfl_down_sync(0xffffffffu, dv, 5);
            if (lane < 5) wpart[warp][lane] = dv + d1;
            if (is_row && has) c.rowsc[(size_t)(q ? m1 : m0) * 4 + k] = dv;
        }
    } else if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 5; ++q) wpart[warp][q] = 0.0;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < WARPS; ++w) t += wpart[w][threadIdx.x];
        c.bpart[(size_t)blk * 5 + threadIdx.x] = t;
    }

    if (!tail) return;

    // ---- last CTA: the FP64 reduction over the CTAs' partial sums
    if (!last_cta_arrive(&sc->cnt_rows, (unsigned)nblk, am_last)) return;
    rows_finish<WARPS * 32>(c, mode, nblk, true, arm);
}

// ---------------------------------------------------------------------------
// s-direction: staged contraction with D_t (or W^-1 D_t^T W)
// ---------------------------------------------------------------------------
// Y[j][col] = rowscale_j * sum_m (cot[(j+m) mod 2P] + tsign cot[(j-m) mod 2P]) colscale_m X[m][col]
//   D_t:          colscale = tau, rowscale = sigma, tsign = +1
//   W^-1 D_t^T W: colscale = sigma w, rowscale = tau / w, tsign = -1
// Each stage builds its D_t tile in shared memory from two contiguous windows
// of the cot table (one for j+m, one for j-m).
// Sections per stage of the contraction: 64 in FP32, 32 in FP64 (the stage's
// shared memory stays under the 48 KB of static shared memory).
template <typename T>
struct DtStage {
    static constexpr int BK = sizeof(T) == 4 ? 2 * DT_BK : DT_BK;
};

// Shared-memory stage of the contraction: the D_t tile built from the two cot
// windows, and the scaled X rows of the stage.
template <typename T, int BN, int BK = DtStage<T>::BK>
struct DtTiles {
    static constexpr int WIN = DT_BM + BK - 1;
    __align__(16) T Ks[BK][DT_BM];
    __align__(16) T Xs[BK][BN];
    T Wp[WIN + 1], Wm[WIN + 1];
};

template <typename T>
struct Vec4 {
    T x, y, z, w;
};

// Four consecutive values from a 4-element-aligned address.
template <typename T>
__device__ __forceinline__ Vec4<T> ld4(const T *p)
{
    if constexpr (sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        return {v.x, v.y, v.z, v.w};
    } else {
        const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
        return {a.x, a.y, b.x, b.y};
    }
}

template <typename T>
__device__ __forceinline__ void st4(T *p, Vec4<T> v)
{
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v.x, v.y, v.z, v.w);
    } else {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v.x, v.y);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v.z, v.w);
    }
}

// acc += K X over the sections [kbeg, kend) for the DT_BM x BN output tile at
// (j0, c0), summed over the sections in increasing order: each BK-stage is
// staged through registers (the next stage is fetched while the current one is
// multiplied), four consecutive columns per load (N is a multiple of 8).
// fetch(kbeg) must have been called before run().
template <typename T, int BN, int BK_ = DtStage<T>::BK>
struct DtContract {
    static constexpr int BM = DT_BM, BK = BK_, TM = 2, TN = BN / 16, WIN = BM + BK - 1;
    static constexpr int VPR = BN / 4;               // four-column slots per stage row
    static constexpr int RPP = DT_THREADS / VPR;     // stage rows per pass of the CTA
    static constexpr int NV = BK / RPP;              // four-column loads per thread per stage
    static_assert(NV * RPP == BK, "stage rows must split evenly over the passes");
    const T *X, *cot, *colscale;
    T tsign;
    int N, twoP, j0, c0, kbeg, kend;
    Vec4<T> xr[NV];
    T wpr = T(0), wmr = T(0);

    __device__ __forceinline__ void fetch(int m0)
    {
        const int cc = (threadIdx.x % VPR) * 4, r0 = threadIdx.x / VPR, col = c0 + cc;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const int m = m0 + r0 + q * RPP;
            if (m < kend && col < N) {
                const T s = colscale[m];
                const Vec4<T> x = ld4(X + (size_t)m * N + col);
                xr[q] = {s * x.x, s * x.y, s * x.z, s * x.w};
            } else {
                xr[q] = {T(0), T(0), T(0), T(0)};
            }
        }
        if (threadIdx.x < WIN) {
            int ip = (j0 + m0 + (int)threadIdx.x) % twoP;
            int im = (j0 - m0 - BK + 1 + (int)threadIdx.x) % twoP;
            if (im < 0) im += twoP;
            wpr = cot[ip];
            wmr = cot[im];
        }
    }

    __device__ __forceinline__ void run(DtTiles<T, BN, BK> &sm, T (&acc)[TM][TN])
    {
        const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
        for (int m0 = kbeg; m0 < kend; m0 += BK) {
            {
                const int cc = (threadIdx.x % VPR) * 4, r0 = threadIdx.x / VPR;
#pragma unroll
                for (int q = 0; q < NV; ++q) st4(&sm.Xs[r0 + q * RPP][cc], xr[q]);
            }
            if (threadIdx.x < WIN) {
                sm.Wp[threadIdx.x] = wpr;
                sm.Wm[threadIdx.x] = wmr;
            }
            __syncthreads();
            if (m0 + BK < kend) fetch(m0 + BK);      // next stage in flight while this one computes
            // D_t tile, stored [kk][jj]: K(j0+jj, m0+kk) = Wp[jj+kk] + tsign Wm[jj-kk+BK-1]
            for (int e = threadIdx.x; e < BK * BM; e += DT_THREADS) {
                const int kk = e / BM, jj = e % BM;
                sm.Ks[kk][jj] = sm.Wp[jj + kk] + tsign * sm.Wm[jj - kk + BK - 1];
            }
            __syncthreads();
#pragma unroll 8
            for (int kk = 0; kk < BK; ++kk) {
                T a[TM], b[TN];
#pragma unroll
                for (int i = 0; i < TM; ++i) a[i] = sm.Ks[kk][ty * TM + i];
#pragma unroll
                for (int l = 0; l < TN; ++l) b[l] = sm.Xs[kk][tx * TN + l];
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int l = 0; l < TN; ++l) acc[i][l] += a[i] * b[l];
            }
            __syncthreads();
        }
    }
};

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
// tiles: room for the TMA tiles of U and D_t U (2 warps rows of W words each,
// 128-byte aligned) after the transform buffers
template <typename T>
static size_t rows_smem(int N, int bufs, int warps = ROWS_WARPS, int tiles_w = 0)
{
    const size_t base = (size_t)(N / 2 + warps * bufs * N) * sizeof(cpx<T>);
    return tiles_w ? base + 128 + (size_t)2 * 2 * warps * tiles_w * sizeof(T) : base;
}

// Sets a kernel's dynamic shared-memory limit to the largest size requested so
// far, once per size increase (per device: kernels run on the device current at
// the call).  Done for every size, not only above 48 KB: static shared memory
// counts against the same default limit.
template <typename K>
static cudaError_t set_smem(K kern, size_t bytes)
{
    static thread_local std::map<std::pair<int, const void *>, size_t> done;   // (device, kernel) -> bytes
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
    size_t &have = done[std::make_pair(dev, (const void *)kern)];
    if (bytes <= have) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}

// Calls f(std::integral_constant<int, N>) for the supported section lengths.
template <typename F>
static cudaError_t dispatch_n(int n, F &&f)
{
    switch (n) {
    case 8: return f(std::integral_constant<int, 8>{});
    case 16: return f(std::integral_constant<int, 16>{});
    case 32: return f(std::integral_constant<int, 32>{});
    case 64: return f(std::integral_constant<int, 64>{});
    case 128: return f(std::integral_constant<int, 128>{});
    case 256: return f(std::integral_constant<int, 256>{});
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ks
