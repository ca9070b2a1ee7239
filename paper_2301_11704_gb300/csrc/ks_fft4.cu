// ks_fft4.cu -- the FFT form of the s-contraction for transforms longer than one
// CTA's shared memory holds (Ashtari & Schneider, arXiv 2301.11704, eq.
// rational_diff_matrix, Sec. V.C.1; the convolution identity is stated beside
// the single-CTA form in ks_kernels.cu):
//
//   y = IFFT_F( FFT_F(c_F) / F * FFT_F(z) )[0..P],   F = F1 F2 (powers of two <= 256)
//
// with the index maps n = F2 n1 + n2 and k = k1 + F1 k2, so that
//   FFT:  Z[k1 + F1 k2] = sum_n2 W_F2^(n2 k2) W_F^(n2 k1) sum_n1 W_F1^(n1 k1) z[F2 n1 + n2]
//   IFFT: x[F2 n1 + n2] = sum_k1 W_F1^(-n1 k1) W_F^(-n2 k1) sum_k2 W_F2^(-n2 k2) X[k1 + F1 k2]
// (W_L = e^(-2 pi i / L)).  Three passes per Fourier mode (the mode's two real
// columns packed as one complex sequence), one warp per line transform, the
// line held in registers (k1 and k2 stay in the transforms' scrambled order,
// the spectrum and the twiddles are tabulated in it):
//   pass 1 (per n2): z from the columns, FFT over n1, times W_F^(n2 k1), stored
//          transposed as S[k1][n2] (staged through shared memory);
//   pass 2 (per k1): FFT over n2, times the kernel spectrum (kept in the same
//          order: no transposes), IFFT over k2, times W_F^(-n2 k1);
//   pass 3 (per n2): IFFT over k1 -> y at j = F2 n1 + n2 <= P, and the epilogue
//          of the single-CTA form (store D_t u; or G, the semi-implicit
//          increment and the FP64 |G|^2 with its last-CTA sum).
#include <cmath>

#include "ks_device.cuh"

namespace ks {

namespace {

constexpr int F4W = F4_THREADS / 32;   // lines per CTA

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, size_t smem, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(F4_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args...);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename T>
struct V2of;
template <> struct V2of<float> { using type = float2; };
template <> struct V2of<double> { using type = double2; };

// Shared memory of a pass: the line transform's twiddles, two buffers per warp,
// and a staging tile of F4W lines for the transposed accesses.
template <typename T, int L, int LS>
struct F4Smem {
    static constexpr size_t TW = L / 2, BUF = (size_t)2 * F4W * L, STAGE = (size_t)F4W * (LS + 1);
    static constexpr size_t BYTES = (TW + BUF + STAGE) * sizeof(cpx<T>);
};

// ---- line transforms in registers.  A line of L = 32 R points is held by one
// warp, R values per lane: v[a] at lane l is x[l + 32 a].  The forward transform
// is an R-point DFT within each lane, the twiddles W_L^(a l), and a 32-point
// decimation-in-frequency transform across the lanes by shuffles; it leaves
// X[a + R brev5(l)] in v[a] at lane l.  The inverse takes that layout back to
// natural order (decimation in time across the lanes, the conjugate twiddles,
// the inverse R-point DFT).  Neither scales.  The passes keep the scrambled
// order: an index k of a transformed axis is stored at the position
// (k mod R) * 32 + brev5(k / R), so lane l's register a always maps to
// position a * 32 + l and no pass permutes data.

__device__ __forceinline__ int brev5(int x) { return (int)(__brev((unsigned)x) >> 27); }

template <int R>
__host__ __device__ constexpr int brev_r(int i)
{
    int r = 0;
    for (int b = 1; b < R; b <<= 1, i >>= 1) r = (r << 1) | (i & 1);
    return r;
}

template <typename T>
__device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> cconj(cpx<T> a) { return {a.x, -a.y}; }
template <typename T>
__device__ __forceinline__ cpx<T> cshfl(cpx<T> a, int m)
{
    return {__shfl_xor_sync(0xffffffffu, a.x, m), __shfl_xor_sync(0xffffffffu, a.y, m)};
}

// v * W_8^e (forward, e^(-2 pi i e / 8)) or v * W_8^(-e) (inverse), e < 4; e is a
// constant once the caller's loops are unrolled
template <typename T>
__device__ __forceinline__ cpx<T> mul_w8(cpx<T> v, int e, bool inv)
{
    const T h = T(0.70710678118654752440);
    if (e == 0) return v;
    if (e == 2) return inv ? cpx<T>{-v.y, v.x} : cpx<T>{v.y, -v.x};
    if (e == 1) return inv ? cpx<T>{h * (v.x - v.y), h * (v.x + v.y)} : cpx<T>{h * (v.x + v.y), h * (v.y - v.x)};
    return inv ? cpx<T>{-h * (v.x + v.y), h * (v.x - v.y)} : cpx<T>{h * (v.y - v.x), -h * (v.x + v.y)};
}

// R-point DFT (R <= 8) within a lane, natural order in and out (radix 2, in time)
template <typename T, int R>
__device__ __forceinline__ void reg_dft(cpx<T> (&v)[R], bool inv)
{
    cpx<T> t[R];
#pragma unroll
    for (int i = 0; i < R; ++i) t[brev_r<R>(i)] = v[i];
#pragma unroll
    for (int h = 1; h < R; h <<= 1) {
#pragma unroll
        for (int i = 0; i < R; i += 2 * h) {
#pragma unroll
            for (int j = 0; j < h; ++j) {
                const cpx<T> u = t[i + j], x = mul_w8(t[i + j + h], j * (4 / h), inv);
                t[i + j] = cadd(u, x);
                t[i + j + h] = csub(u, x);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = t[i];
}

// twl[a * 32 + l] = W_L^(a l) (a < R), w32[s] = W_32^s (s < 16)
template <typename T, int R>
__device__ __forceinline__ void reg_fft_fwd(cpx<T> (&v)[R], const cpx<T> *twl, const cpx<T> *w32, int lane)
{
    reg_dft<T, R>(v, false);
#pragma unroll
    for (int a = 1; a < R; ++a) v[a] = cmul(v[a], twl[a * 32 + lane]);
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        const bool up = (lane & m) != 0;
        const cpx<T> w = w32[up ? (lane & (m - 1)) * (16 / m) : 0];   // W_2m^(pos - m) on the upper lanes
#pragma unroll
        for (int a = 0; a < R; ++a) {
            const cpx<T> p = cshfl(v[a], m);
            const cpx<T> d = up ? csub(p, v[a]) : cadd(v[a], p);
            v[a] = (m > 1) ? cmul(d, w) : d;
        }
    }
}

template <typename T, int R>
__device__ __forceinline__ void reg_fft_inv(cpx<T> (&v)[R], const cpx<T> *twl, const cpx<T> *w32, int lane)
{
#pragma unroll
    for (int m = 1; m <= 16; m <<= 1) {
        const bool up = (lane & m) != 0;
        const cpx<T> w = cconj(w32[up ? (lane & (m - 1)) * (16 / m) : 0]);
#pragma unroll
        for (int a = 0; a < R; ++a) {
            const cpx<T> b = (m > 1) ? cmul(v[a], w) : v[a];
            const cpx<T> p = cshfl(b, m);
            v[a] = up ? csub(p, b) : cadd(b, p);
        }
    }
#pragma unroll
    for (int a = 1; a < R; ++a) v[a] = cmul(v[a], cconj(twl[a * 32 + lane]));
    reg_dft<T, R>(v, true);
}

// the line twiddles of a length-L transform from the plain table W_F^k
template <typename T, int L>
__device__ __forceinline__ void load_line_twiddles(cpx<T> *twl, cpx<T> *w32, const cpx<T> *ftw, int F)
{
    for (int t = threadIdx.x; t < L; t += F4_THREADS) twl[t] = ftw[(size_t)((t >> 5) * (t & 31)) * (F / L)];
    for (int t = threadIdx.x; t < 16; t += F4_THREADS) w32[t] = ftw[(size_t)t * (F / 32)];
}

// staging tile row length: conflict-free column access by F4W lines (8-byte
// elements: a pad of two; 16-byte elements: one)
template <typename T, int L>
struct F4Stage {
    static constexpr int LS = L + (sizeof(T) == 4 ? 2 : 1);
    static constexpr size_t BYTES = (size_t)(L + 16 + F4W * LS) * sizeof(cpx<T>);
};

}  // namespace

// ---- pass 1: lines over n1 (length F1), one per n2
template <typename T, int F1, int F2>
__global__ void __launch_bounds__(F4_THREADS) k_f4_p1(CurveDev c, int mode, int discrete, int gate)
{
    using V2 = typename V2of<T>::type;
    constexpr int R = F1 / 32, LS = F4Stage<T, F1>::LS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T> *twl = (cpx<T> *)smem_raw, *w32 = twl + F1, *stage = w32 + 16;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, jm = blockIdx.y;
    const int n2 = blockIdx.x * F4W + warp, F = F1 * F2;
    const cpx<T> *ftw = (const cpx<T> *)c.ftw;
    load_line_twiddles<T, F1>(twl, w32, ftw, F);
    pdl_wait();
    if (gate && !c.sc->active) return;

    const int P = c.P, N = c.nx;
    const T *X = (const T *)(mode == GM_STORE ? c.U : c.R);
    const T *colscale = (const T *)(discrete ? c.sw : c.tau);
    const T s = discrete ? T(-1) : T(1);
    const int ca = 2 * jm, cb = 2 * jm + 1;
    const bool oka = col_allowed(ca, c.sym), okb = col_allowed(cb, c.sym) && jm != 0;
    // z[F2 n1 + n2]: the symmetric extension of the scaled columns (as in the single-CTA form)
    cpx<T> v[R];
#pragma unroll
    for (int a = 0; a < R; ++a) {
        const int k = F2 * (lane + 32 * a) + n2;
        int m = -1;
        T f = T(1);
        if (k == 0) { m = 0; f = T(1) + s; }
        else if (k < P) { m = k; f = s; }
        else if (k == P) { m = P; f = T(1) + s; }
        else if (k < 2 * P) { m = 2 * P - k; }
        v[a] = {0, 0};
        if (m >= 0 && f != T(0)) {
            const T cs = f * colscale[m];
            const V2 xv = *reinterpret_cast<const V2 *>(X + (size_t)m * N + ca);
            v[a].x = oka ? cs * xv.x : T(0);
            v[a].y = okb ? cs * xv.y : T(0);
        }
    }
    __syncthreads();   // twiddles
    reg_fft_fwd<T, R>(v, twl, w32, lane);
    // times W_F^(n2 k1) (table in the scrambled order of k1), into the staging tile
    const cpx<T> *t1 = ftw + F + (size_t)n2 * F1;
#pragma unroll
    for (int a = 0; a < R; ++a) stage[warp * LS + a * 32 + lane] = cmul(v[a], t1[a * 32 + lane]);
    __syncthreads();
    // S[jm][k1][n2] (k1 in the scrambled order): F4W consecutive n2 per k1
    cpx<T> *S = (cpx<T> *)c.f4s + (size_t)jm * F;
    for (int e = threadIdx.x; e < F4W * F1; e += F4_THREADS) {
        const int r = e / F4W, w = e % F4W;
        S[(size_t)r * F2 + blockIdx.x * F4W + w] = stage[w * LS + r];
    }
}

// ---- pass 2: lines over n2 (length F2), one per k1: FFT, spectrum, IFFT
template <typename T, int F1, int F2>
__global__ void __launch_bounds__(F4_THREADS) k_f4_p2(CurveDev c, int gate)
{
    constexpr int R = F2 / 32;
    __shared__ cpx<T> twl[F2], w32[16];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, jm = blockIdx.y, F = F1 * F2;
    const int r = blockIdx.x * F4W + warp;   // position of k1 in the scrambled order
    const cpx<T> *ftw = (const cpx<T> *)c.ftw, *chat = (const cpx<T> *)c.chat + (size_t)r * F2;
    const cpx<T> *t2 = ftw + 2 * (size_t)F + (size_t)r * F2;
    load_line_twiddles<T, F2>(twl, w32, ftw, F);
    pdl_wait();
    if (gate && !c.sc->active) return;

    cpx<T> *S = (cpx<T> *)c.f4s + (size_t)jm * F + (size_t)r * F2;
    cpx<T> v[R];
#pragma unroll
    for (int a = 0; a < R; ++a) v[a] = S[lane + 32 * a];
    __syncthreads();   // twiddles
    reg_fft_fwd<T, R>(v, twl, w32, lane);
#pragma unroll
    for (int a = 0; a < R; ++a) v[a] = cmul(v[a], chat[a * 32 + lane]);   // spectrum in the same order
    reg_fft_inv<T, R>(v, twl, w32, lane);
#pragma unroll
    for (int a = 0; a < R; ++a) S[lane + 32 * a] = cmul(v[a], cconj(t2[lane + 32 * a]));   // W_F^(-n2 k1)
}

// ---- pass 3: lines over k1 (length F1), one per n2: IFFT and the epilogue
template <typename T, int F1, int F2>
__global__ void __launch_bounds__(F4_THREADS) k_f4_p3(CurveDev c, int mode, int discrete, int gate)
{
    using V2 = typename V2of<T>::type;
    constexpr int R = F1 / 32, LS = F4Stage<T, F1>::LS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T> *twl = (cpx<T> *)smem_raw, *w32 = twl + F1, *stage = w32 + 16;
    __shared__ double wsum[F4W];
    __shared__ double red[F4_THREADS];
    __shared__ int am_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, jm = blockIdx.y;
    const int n2 = blockIdx.x * F4W + warp, F = F1 * F2;
    load_line_twiddles<T, F1>(twl, w32, (const cpx<T> *)c.ftw, F);
    DevScalars *sc = c.sc;
    pdl_wait();
    if (gate && !sc->active) return;
    const double lam_d = sc->lambda, dtau_d = sc->dtau;

    // S[jm][k1][n2] for this CTA's F4W values of n2 -> staging tile [line][k1]
    const cpx<T> *S = (const cpx<T> *)c.f4s + (size_t)jm * F;
    for (int e = threadIdx.x; e < F4W * F1; e += F4_THREADS) {
        const int r = e / F4W, w = e % F4W;
        stage[w * LS + r] = S[(size_t)r * F2 + blockIdx.x * F4W + w];
    }
    __syncthreads();
    cpx<T> v[R];
#pragma unroll
    for (int a = 0; a < R; ++a) v[a] = stage[warp * LS + a * 32 + lane];
    reg_fft_inv<T, R>(v, twl, w32, lane);

    // epilogue over the sections j = F2 n1 + n2 <= P of the two columns (n1 = lane + 32 a)
    const int ns = c.ns, N = c.nx, P = c.P;
    const int ca = 2 * jm, cb = 2 * jm + 1;
    const bool oka = col_allowed(ca, c.sym), okb = col_allowed(cb, c.sym) && jm != 0;
    const T *rowscale = (const T *)(discrete ? c.twr : c.sig);
    T *Dout = (T *)c.D, *U = (T *)c.U, *G = (T *)c.G;
    const T *Ah = (const T *)c.A;
    const T pr = ((const T *)c.prec_imex)[jm];
    const T lam = (T)lam_d, dtau = (T)dtau_d;
    const double cw = (jm == 0) ? 1.0 : 2.0;
    double partsum = 0.0;
#pragma unroll
    for (int a = 0; a < R; ++a) {
        const int j = F2 * (lane + 32 * a) + n2;
        if (j >= ns) continue;
        const T rs = rowscale[j];
        const cpx<T> yv = {rs * v[a].x, rs * v[a].y};
        const size_t o = (size_t)j * N + ca;
        if (mode == GM_STORE) {
            *reinterpret_cast<V2 *>(Dout + o) = V2{oka ? yv.x : T(0), okb ? yv.y : T(0)};
            continue;
        }
        const bool interior = (j > 0 && j < P);
        T ga = 0, gb = 0;
        if (interior) {
            const V2 av = *reinterpret_cast<const V2 *>(Ah + o);
            if (oka) ga = -(av.x + (discrete ? -lam * yv.x : lam * yv.x));
            if (okb) gb = -(av.y + (discrete ? -lam * yv.y : lam * yv.y));
            partsum += c.w[j] * cw * ((double)ga * (double)ga + (double)gb * (double)gb);
        }
        if (mode == GM_UPDATE) {
            if (interior) {
                const V2 uv = *reinterpret_cast<const V2 *>(U + o);
                *reinterpret_cast<V2 *>(U + o) = V2{uv.x + dtau * pr * ga, uv.y + dtau * pr * gb};
            }
        } else {
            *reinterpret_cast<V2 *>(G + o) = V2{ga, gb};
        }
    }
    if (mode == GM_STORE) return;

    // ---- FP64 |G|^2: per-CTA partial, last CTA of the grid sums them in a fixed order
    partsum = warp_sum(partsum);
    if (lane == 0) wsum[warp] = partsum;
    __syncthreads();
    const int bid = jm * gridDim.x + blockIdx.x, nb = gridDim.x * gridDim.y;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < F4W; ++w) t += wsum[w];
        c.tile[bid] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(&sc->cnt_gemm, 1u);
        am_last = (prev == (unsigned)nb - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double t = 0.0;
    for (int b = threadIdx.x; b < nb; b += F4_THREADS) t += __ldcg(c.tile + b);
    t = block_sum<F4_THREADS>(t, red);
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

// ---- set-up: the twiddles W_F^k (storage type) and the kernel spectrum
// FFT(c_F)/F in the [k1][k2] order of the passes, by the forward half of the same
// decomposition in FP64: c_F[t] = cot(pi t / 2P) for 0 <= t <= P, c_F[F - t] =
// cot(pi (2P - t) / 2P) for 0 < t < 2P, 0 elsewhere (cot 0 = 0).  FP64 tables
// W_F^p and the intermediate S64[k1][n2] live in the scratch buffer (32 F bytes;
// it holds at least 8 F bytes per mode and N/2 >= 4 modes).
__device__ __forceinline__ double cot_kernel(int n, int F, int P)
{
    int u = -1;
    if (n <= P) u = n;
    else if (n > F - 2 * P) u = 2 * P - (F - n);
    if (u <= 0) return 0.0;
    double sn, cs;
    sincospi((double)u / (double)(2 * P), &sn, &cs);
    return cs / sn;
}

__global__ void k_f4_twiddles(CurveDev c)
{
    const int F = c.F;
    double2 *w64 = (double2 *)c.f4s;   // e^{-2 pi i p / F} as (cos, -sin)
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < F; p += gridDim.x * blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)p / (double)F, &sn, &cs);
        w64[p] = make_double2(cs, -sn);
    }
}

// pass A (per n2): FFT over n1 of c_F[F2 n1 + n2], times W_F^(n2 k1) -> S64[k1][n2]
template <int F1, int F2>
__global__ void __launch_bounds__(F4_THREADS) k_f4_specA(CurveDev c)
{
    using Sm = F4Smem<double, F1, F1>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<double> *tw = (cpx<double> *)smem_raw, *buf = tw + Sm::TW, *stage = buf + Sm::BUF;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, F = F1 * F2;
    const int n2 = blockIdx.x * F4W + warp;
    const cpx<double> *w64 = (const cpx<double> *)c.f4s;
    cpx<double> *S = (cpx<double> *)c.f4s + F;
    for (int t = threadIdx.x; t < F1 / 2; t += F4_THREADS) tw[t] = w64[t * F2];
    cpx<double> *x = buf + (size_t)warp * 2 * F1, *y = x + F1;
    for (int n1 = lane; n1 < F1; n1 += 32) x[n1] = {cot_kernel(F2 * n1 + n2, F, c.P), 0.0};
    __syncthreads();
    cpx<double> *Y = warp_fft<double, F1>(x, y, tw, false, lane);
    for (int k1 = lane; k1 < F1; k1 += 32) stage[(size_t)warp * (F1 + 1) + k1] = cmul(Y[k1], w64[n2 * k1]);
    __syncthreads();
    for (int e = threadIdx.x; e < F4W * F1; e += F4_THREADS) {
        const int k1 = e / F4W, w = e % F4W;
        S[(size_t)k1 * F2 + blockIdx.x * F4W + w] = stage[(size_t)w * (F1 + 1) + k1];
    }
}

// pass B (per k1): FFT over n2 -> spectrum / F in the storage type, both indices
// in the scrambled order of the passes; the plain twiddle table W_F^p
template <typename T, int F1, int F2>
__global__ void __launch_bounds__(F4_THREADS) k_f4_specB(CurveDev c)
{
    using Sm = F4Smem<double, F2, F2>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<double> *tw = (cpx<double> *)smem_raw, *buf = tw + Sm::TW;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, F = F1 * F2;
    const int k1 = blockIdx.x * F4W + warp;
    const cpx<double> *w64 = (const cpx<double> *)c.f4s;
    const cpx<double> *S = (const cpx<double> *)c.f4s + F + (size_t)k1 * F2;
    for (int t = threadIdx.x; t < F2 / 2; t += F4_THREADS) tw[t] = w64[t * F1];
    cpx<double> *x = buf + (size_t)warp * 2 * F2, *y = x + F2;
    for (int n2 = lane; n2 < F2; n2 += 32) x[n2] = S[n2];
    __syncthreads();
    cpx<double> *Z = warp_fft<double, F2>(x, y, tw, false, lane);
    constexpr int R1 = F1 / 32, R2 = F2 / 32;
    cpx<T> *chat = (cpx<T> *)c.chat + (size_t)((k1 % R1) * 32 + brev5(k1 / R1)) * F2, *ftw = (cpx<T> *)c.ftw;
    for (int k2 = lane; k2 < F2; k2 += 32)
        chat[(k2 % R2) * 32 + brev5(k2 / R2)] = {(T)(Z[k2].x / F), (T)(Z[k2].y / F)};
    for (int p = k1 * F2 + lane; p < (k1 + 1) * F2; p += 32) ftw[p] = {(T)w64[p].x, (T)w64[p].y};
}

// the step twiddles W_F^(n2 k1) with k1 at its scrambled position r (k1 = r / 32 +
// R1 brev5(r mod 32)), once as [n2][r] for pass 1 and once as [r][n2] for pass 2
template <typename T, int F1, int F2>
__global__ void k_f4_steptw(CurveDev c)
{
    constexpr int R1 = F1 / 32, F = F1 * F2;
    const cpx<double> *w64 = (const cpx<double> *)c.f4s;
    cpx<T> *t1 = (cpx<T> *)c.ftw + F, *t2 = t1 + F;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < F; p += gridDim.x * blockDim.x) {
        int n2 = p / F1, r = p % F1;
        cpx<double> w = w64[n2 * ((r >> 5) + R1 * brev5(r & 31))];
        t1[p] = {(T)w.x, (T)w.y};
        r = p / F2;
        n2 = p % F2;
        w = w64[n2 * ((r >> 5) + R1 * brev5(r & 31))];
        t2[p] = {(T)w.x, (T)w.y};
    }
}

// ---- launchers
template <typename T, int F1, int F2>
static cudaError_t f4_run(const CurveDev &c, int mode, int discrete, int gate, cudaStream_t st)
{
    const int nm = c.nx / 2;
    const size_t sm1 = F4Stage<T, F1>::BYTES;
    cudaError_t e;
    if ((e = set_smem(k_f4_p1<T, F1, F2>, sm1)) != cudaSuccess) return e;
    if ((e = set_smem(k_f4_p3<T, F1, F2>, sm1)) != cudaSuccess) return e;
    if ((e = launch_pdl(k_f4_p1<T, F1, F2>, dim3(F2 / F4W, nm), sm1, st, c, mode, discrete, gate)) != cudaSuccess)
        return e;
    if ((e = launch_pdl(k_f4_p2<T, F1, F2>, dim3(F1 / F4W, nm), 0, st, c, gate)) != cudaSuccess) return e;
    return launch_pdl(k_f4_p3<T, F1, F2>, dim3(F2 / F4W, nm), sm1, st, c, mode, discrete, gate);
}

template <typename T>
static cudaError_t f4_dispatch(const CurveDev &c, int mode, int discrete, int gate, cudaStream_t st)
{
    if (c.F1 == 64 && c.F2 == 64) return f4_run<T, 64, 64>(c, mode, discrete, gate, st);
    if (c.F1 == 128 && c.F2 == 64) return f4_run<T, 128, 64>(c, mode, discrete, gate, st);
    if (c.F1 == 128 && c.F2 == 128) return f4_run<T, 128, 128>(c, mode, discrete, gate, st);
    if (c.F1 == 256 && c.F2 == 128) return f4_run<T, 256, 128>(c, mode, discrete, gate, st);
    if (c.F1 == 256 && c.F2 == 256) return f4_run<T, 256, 256>(c, mode, discrete, gate, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_f4(const CurveDev &c, int mode, int discrete, int gate, cudaStream_t st)
{
    return c.prec ? f4_dispatch<float>(c, mode, discrete, gate, st) : f4_dispatch<double>(c, mode, discrete, gate, st);
}

template <typename T, int F1, int F2>
static cudaError_t setup_run(const CurveDev &c, cudaStream_t st)
{
    const size_t smA = F4Smem<double, F1, F1>::BYTES, smB = F4Smem<double, F2, F2>::BYTES;
    cudaError_t e;
    if ((e = set_smem(k_f4_specA<F1, F2>, smA)) != cudaSuccess) return e;
    if ((e = set_smem(k_f4_specB<T, F1, F2>, smB)) != cudaSuccess) return e;
    k_f4_twiddles<<<(c.F + 255) / 256, 256, 0, st>>>(c);
    k_f4_specA<F1, F2><<<F2 / F4W, F4_THREADS, smA, st>>>(c);
    k_f4_specB<T, F1, F2><<<F1 / F4W, F4_THREADS, smB, st>>>(c);
    k_f4_steptw<T, F1, F2><<<(c.F + 255) / 256, 256, 0, st>>>(c);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t setup_dispatch(const CurveDev &c, cudaStream_t st)
{
    if (c.F1 == 64 && c.F2 == 64) return setup_run<T, 64, 64>(c, st);
    if (c.F1 == 128 && c.F2 == 64) return setup_run<T, 128, 64>(c, st);
    if (c.F1 == 128 && c.F2 == 128) return setup_run<T, 128, 128>(c, st);
    if (c.F1 == 256 && c.F2 == 128) return setup_run<T, 256, 128>(c, st);
    if (c.F1 == 256 && c.F2 == 256) return setup_run<T, 256, 256>(c, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_setup_f4(const CurveDev &c, cudaStream_t st)
{
    return c.prec ? setup_dispatch<float>(c, st) : setup_dispatch<double>(c, st);
}

}  // namespace ks
