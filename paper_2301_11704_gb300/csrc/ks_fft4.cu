// ks_fft4.cu -- the four-step FFT form of the s-contraction (Ashtari & Schneider,
// arXiv 2301.11704, eq. rational_diff_matrix, Sec. V.C.1; the convolution
// identity is stated beside the single-CTA form in ks_kernels.cu):
//
//   y = IFFT_F( FFT_F(c_F) / F * FFT_F(z) )[0..P],   F = F1 F2 (powers of two, 32 <= F1, F2 <= 256)
//
// with the index maps n = F2 n1 + n2 and k = k1 + F1 k2, so that
//   FFT:  Z[k1 + F1 k2] = sum_n2 W_F2^(n2 k2) W_F^(n2 k1) sum_n1 W_F1^(n1 k1) z[F2 n1 + n2]
//   IFFT: x[F2 n1 + n2] = sum_k1 W_F1^(-n1 k1) W_F^(-n2 k1) sum_k2 W_F2^(-n2 k2) X[k1 + F1 k2]
// (W_L = e^(-2 pi i / L)).  Three passes per Fourier mode (the mode's two real
// columns packed as one complex sequence), one warp per line transform, the
// line held in registers (k1 and k2 stay in the transforms' scrambled order,
// the spectrum and the twiddles are tabulated in it):
//   pass 1 (per n2): z from the columns, FFT over n1, times W_F^(n2 k1), stored
//          transposed as S[k1][n2];
//   pass 2 (per k1): FFT over n2, times the kernel spectrum (kept in the same
//          order: no transposes), IFFT over k2, times W_F^(-n2 k1);
//   pass 3 (per n2): IFFT over k1 -> y at j = F2 n1 + n2 <= P, and the epilogue
//          of the single-CTA form (store D_t u; or G, the semi-implicit
//          increment and the FP64 |G|^2 with its last-CTA sum).
// Three variants of where S lives: a global scratch between three launches
// (k_f4_p1/p2/p3, single curves, F >= 4096); the distributed shared memory of a
// cluster of CTAs per mode group, in one launch that can also apply the step's
// second contraction (k_f4c); one CTA's shared memory per (curve, mode) for
// batched curves (k_f4b, F from 1024 to 8192).  Their set-up computes the
// kernel spectrum by the forward half of the same decomposition in FP64.
#include <cmath>

#include <type_traits>

#include <cooperative_groups.h>

#include "ks_device.cuh"

namespace ks {

namespace {

constexpr int F4W = F4_THREADS / 32;   // lines per CTA
static_assert(F4_THREADS / F4W == 32, "passes 1 and 3 map a CTA's threads to F4W lines x 32 positions");

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

// The cross-lane stages come in two forms.  FP32 (latency-bound): each lane
// fetches its partner's value and computes its half of the butterfly (the lower
// lanes multiply by 1).  FP64 (bound by GB300's FP64 rate): on the register pair
// (a, a + 1) lanes l and l ^ m first swap one value each, so that the lower lane
// holds both inputs of register a's butterfly and the upper lane both of register
// a + 1's; each lane does a whole butterfly and a second swap restores the
// layout: the same shuffles, half the arithmetic.
template <typename T>
__device__ __forceinline__ void lane_swap(cpx<T> &v0, cpx<T> &v1, bool up, int m)
{
    const cpx<T> r = cshfl(up ? v0 : v1, m);
    if (up) v0 = r;
    else v1 = r;
}

// twl[a * 32 + l] = W_L^(a l) (a < R), w32[s] = W_32^s (s < 16)
template <typename T, int R>
__device__ __forceinline__ void reg_fft_fwd(cpx<T> (&v)[R], const cpx<T> *twl, const cpx<T> *w32, int lane)
{
    static_assert(R == 1 || R % 2 == 0, "one value per lane or register pairs");
    reg_dft<T, R>(v, false);
#pragma unroll
    for (int a = 1; a < R; ++a) v[a] = cmul(v[a], twl[a * 32 + lane]);
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        const bool up = (lane & m) != 0;
        if constexpr (sizeof(T) == 8 && R % 2 == 0) {
            const cpx<T> w = w32[(lane & (m - 1)) * (16 / m)];   // W_2m^(position within the half)
#pragma unroll
            for (int a = 0; a < R; a += 2) {
                lane_swap(v[a], v[a + 1], up, m);
                const cpx<T> x = v[a], y = v[a + 1];
                v[a] = cadd(x, y);
                v[a + 1] = (m > 1) ? cmul(csub(x, y), w) : csub(x, y);
                lane_swap(v[a], v[a + 1], up, m);
            }
        } else {
            const cpx<T> w = w32[up ? (lane & (m - 1)) * (16 / m) : 0];   // 1 on the lower lanes
#pragma unroll
            for (int a = 0; a < R; ++a) {
                const cpx<T> p = cshfl(v[a], m);
                const cpx<T> d = up ? csub(p, v[a]) : cadd(v[a], p);
                v[a] = (m > 1) ? cmul(d, w) : d;
            }
        }
    }
}

template <typename T, int R>
__device__ __forceinline__ void reg_fft_inv(cpx<T> (&v)[R], const cpx<T> *twl, const cpx<T> *w32, int lane)
{
    static_assert(R == 1 || R % 2 == 0, "one value per lane or register pairs");
#pragma unroll
    for (int m = 1; m <= 16; m <<= 1) {
        const bool up = (lane & m) != 0;
        if constexpr (sizeof(T) == 8 && R % 2 == 0) {
            const cpx<T> w = cconj(w32[(lane & (m - 1)) * (16 / m)]);
#pragma unroll
            for (int a = 0; a < R; a += 2) {
                lane_swap(v[a], v[a + 1], up, m);
                const cpx<T> x = v[a], y = (m > 1) ? cmul(v[a + 1], w) : v[a + 1];
                v[a] = cadd(x, y);
                v[a + 1] = csub(x, y);
                lane_swap(v[a], v[a + 1], up, m);
            }
        } else {
            const cpx<T> w = cconj(w32[up ? (lane & (m - 1)) * (16 / m) : 0]);
#pragma unroll
            for (int a = 0; a < R; ++a) {
                const cpx<T> b = (m > 1) ? cmul(v[a], w) : v[a];
                const cpx<T> p = cshfl(b, m);
                v[a] = up ? csub(p, b) : cadd(b, p);
            }
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

// Passes 1 and 3 work on MPC modes at once, so that a section row is read and
// written in whole 32-byte sectors (its columns 2 jm0 .. 2 jm0 + 2 MPC - 1), with
// F4W lines each: a tile [mode][line][position] in shared memory holds their
// values between the row accesses, the line transforms and the scratch.  Row
// length LS pads the line so that the column accesses (F4W lines, one or two
// positions) fall in distinct banks: 8-byte elements pad two, 16-byte one.
// In sine storage (HS) a CTA takes a 16-byte half sector: rows there are half as
// long, and half sectors keep as many CTAs on the rows as full storage has.
template <typename T, bool HS = false>
struct F4Sector {
    static constexpr int MPC = (HS ? 16 : 32) / (2 * (int)sizeof(T));   // 4 (FP32) or 2 (FP64); halved in HS
    static constexpr int NV = 2 * MPC;                                  // values of a row sector
};

template <typename T, int L, bool HS = false>
struct F4Stage {
    static constexpr int LS = L + (sizeof(T) == 4 ? 2 : 1);
    static constexpr int TS = F4W * LS;   // tile stride of a mode
    static constexpr size_t BYTES = (size_t)(L + 16 + F4Sector<T, HS>::MPC * TS) * sizeof(cpx<T>);
};

__device__ __forceinline__ void ld_sector(const float *p, float (&x)[8])
{
    const float4 a = reinterpret_cast<const float4 *>(p)[0], b = reinterpret_cast<const float4 *>(p)[1];
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
}
__device__ __forceinline__ void ld_sector(const double *p, double (&x)[4])
{
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
}
__device__ __forceinline__ void st_sector(float *p, const float (&x)[8])
{
    reinterpret_cast<float4 *>(p)[0] = make_float4(x[0], x[1], x[2], x[3]);
    reinterpret_cast<float4 *>(p)[1] = make_float4(x[4], x[5], x[6], x[7]);
}
__device__ __forceinline__ void st_sector(double *p, const double (&x)[4])
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(x[0], x[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(x[2], x[3]);
}
// half sectors (16 bytes)
__device__ __forceinline__ void ld_sector(const float *p, float (&x)[4])
{
    const float4 a = *reinterpret_cast<const float4 *>(p);
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
}
__device__ __forceinline__ void ld_sector(const double *p, double (&x)[2])
{
    const double2 a = *reinterpret_cast<const double2 *>(p);
    x[0] = a.x; x[1] = a.y;
}
__device__ __forceinline__ void st_sector(float *p, const float (&x)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
}
__device__ __forceinline__ void st_sector(double *p, const double (&x)[2])
{
    *reinterpret_cast<double2 *>(p) = make_double2(x[0], x[1]);
}

// the columns 2 jm0 + i of a row sector that the subspace keeps (in full storage
// column 1, the imaginary part of the mean, never; in sine storage column 0)
__device__ __forceinline__ bool sector_col_ok(int jm0, int i, int sym, int hs = 0)
{
    return col_live(2 * jm0 + i, sym, hs);
}

}  // namespace

// ---- pass 1: lines over n1 (length F1), one per (n2, mode)
template <typename T, int F1, int F2, bool HS = false>
__global__ void __launch_bounds__(F4_THREADS) k_f4_p1(CurveDev c, int mode, int discrete, int gate)
{
    using Sec = F4Sector<T, HS>;
    using St = F4Stage<T, F1, HS>;
    constexpr int R = F1 / 32, LS = St::LS, TS = St::TS, MPC = Sec::MPC, NV = Sec::NV;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T> *twl = (cpx<T> *)smem_raw, *w32 = twl + F1, *tile = w32 + 16;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n2_0 = blockIdx.y * F4W, jm0 = blockIdx.x * MPC, F = F1 * F2;
    const cpx<T> *ftw = (const cpx<T> *)c.ftw;
    load_line_twiddles<T, F1>(twl, w32, ftw, F);
    pdl_wait();
    if (gate && !c.sc->active) return;

    constexpr int hs = HS ? 1 : 0;
    const int P = c.P, N = c.W;   // N: the stored columns
    const T *X = (const T *)(mode == GM_STORE ? c.U : c.R);
    const T *colscale = (const T *)(discrete ? c.sw : c.tau);
    const T s = discrete ? T(-1) : T(1);
    // odd sections in full storage (real parts zero): the imaginary columns of
    // modes 2q and 2q + 1 of the block as one complex sequence q, so MPC / 2
    // sequences per block (sine storage holds only those columns: no pairing)
    const bool paired = !HS && (c.sym & 1);
    const int nq = paired ? MPC / 2 : MPC;
    // z[F2 n1 + n2] of the MPC modes (the symmetric extension of the scaled
    // columns, as in the single-CTA form): thread -> line n2_0 + tn, n1 = t / F4W + 32 i.
    // Rows are fetched two at a time, both loads issued before either is used.
    const int tn = threadIdx.x % F4W;
#pragma unroll
    for (int i0 = 0; i0 < R; i0 += 2) {
        T x[2][NV], cs[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = F2 * (threadIdx.x / F4W + 32 * (i0 + h)) + n2_0 + tn;
            int m = -1;
            T f = T(1);
            if (c.f4h) {   // Toeplitz-Hankel form: the column itself, z[k] = x_k for k <= P
                if (k <= P) m = k;
            }
            else if (k == 0) { m = 0; f = T(1) + s; }
            else if (k < P) { m = k; f = s; }
            else if (k == P) { m = P; f = T(1) + s; }
            else if (k < 2 * P) { m = 2 * P - k; }
            cs[h] = T(0);
#pragma unroll
            for (int q = 0; q < NV; ++q) x[h][q] = T(0);
            if (m >= 0 && f != T(0)) {
                cs[h] = f * colscale[m];
                ld_sector(X + (size_t)m * N + 2 * jm0, x[h]);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int n1 = threadIdx.x / F4W + 32 * (i0 + h);
            if (paired) {
#pragma unroll
                for (int q = 0; q < MPC / 2; ++q)
                    tile[q * TS + tn * LS + n1] = {sector_col_ok(jm0, 4 * q + 1, c.sym) ? cs[h] * x[h][4 * q + 1] : T(0),
                                                   sector_col_ok(jm0, 4 * q + 3, c.sym) ? cs[h] * x[h][4 * q + 3] : T(0)};
            } else {
#pragma unroll
                for (int q = 0; q < MPC; ++q)
                    tile[q * TS + tn * LS + n1] = {sector_col_ok(jm0, 2 * q, c.sym, hs) ? cs[h] * x[h][2 * q] : T(0),
                                                   sector_col_ok(jm0, 2 * q + 1, c.sym, hs) ? cs[h] * x[h][2 * q + 1] : T(0)};
            }
        }
    }
    // the step twiddles W_F^(n2 k1) of this warp's line (scrambled order of k1)
    const cpx<T> *t1 = ftw + F + (size_t)(n2_0 + warp) * F1;
    cpx<T> tw1[R];
#pragma unroll
    for (int a = 0; a < R; ++a) tw1[a] = t1[a * 32 + lane];
    __syncthreads();
    for (int q = 0; q < nq; ++q) {
        cpx<T> *line = tile + q * TS + warp * LS;
        cpx<T> v[R];
#pragma unroll
        for (int a = 0; a < R; ++a) v[a] = line[lane + 32 * a];
        __syncwarp();
        reg_fft_fwd<T, R>(v, twl, w32, lane);
#pragma unroll
        for (int a = 0; a < R; ++a) line[a * 32 + lane] = cmul(v[a], tw1[a]);
    }
    __syncthreads();
    // S[jm][k1][n2] (k1 in the scrambled order): F4W consecutive n2 per (sequence, k1);
    // the sequences of a paired block are numbered jm0 / 2 + q
    cpx<T> *S = (cpx<T> *)c.f4s;
    const int sq0 = paired ? jm0 / 2 : jm0;
    for (int e = threadIdx.x; e < nq * F1 * F4W; e += F4_THREADS) {
        const int w = e % F4W, r = (e / F4W) % F1, q = e / (F4W * F1);
        S[((size_t)(sq0 + q) * F1 + r) * F2 + n2_0 + w] = tile[q * TS + w * LS + r];
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

// ---- pass 2 of the Toeplitz-Hankel form (c.f4h): D_t = sigma (H + s T) with
// H_jm = cot[(j + m) mod 2P], T_jm = cot[(j - m) mod 2P], applied to the column
// z (z_m, m <= P) as
//   y = IFFT(s T^ Z + H^ Z(-k)),   T^ = FFT(cot at lags [-P, P]) / F,
//                                  H^ = FFT(cot at lags [0, 2P]) / F,
// where Z(-k) = FFT of z reversed: index -k of the same transform.  With
// k = k1 + F1 k2, -k is row F1 - k1 at k2' = F2 - 1 - k2 (k1 > 0) or row 0 at
// (F2 - k2) mod F2 (k1 = 0).  A warp takes rows k1 and F1 - k1 together (rows 0
// and F1/2 alone): FFT over n2 of both, the products, IFFT, W_F^(-n2 k1).  In
// the transforms' scrambled order (k2 = a + R brev5(l) in register a of lane l)
// the partner of (a, l) is (R - 1 - a, 31 - l): a register reversal and a
// shuffle across 31 lanes; in row 0, (R - a, 31 - l) for a > 0 and lane
// brev5(32 - brev5(l)) for a = 0.
// Three CTAs per SM (a register cap of 85): 5% faster passes than the
// compiler's own choice (95 registers, two CTAs) at F = 32768 (measured).
template <typename T, int F1, int F2>
__global__ void __launch_bounds__(F4_THREADS, 3) k_f4h_p2(CurveDev c, int discrete, int gate)
{
    constexpr int R = F2 / 32, R1 = F1 / 32, NIT = F1 / 2 + 1;
    static_assert(R >= 2, "lines of at least 64 points");
    __shared__ cpx<T> twl[F2], w32[16];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, jm = blockIdx.y, F = F1 * F2;
    const int it = blockIdx.x * F4W + warp;
    const bool valid = it < NIT, pair = it > 0 && it < F1 / 2;
    const int ka = it, kb = F1 - it;
    const int ra = valid ? (ka % R1) * 32 + brev5(ka / R1) : 0, rb = pair ? (kb % R1) * 32 + brev5(kb / R1) : 0;
    const cpx<T> *ftw = (const cpx<T> *)c.ftw, *chat = (const cpx<T> *)c.chat;
    load_line_twiddles<T, F2>(twl, w32, ftw, F);
    // the spectra (set-up tables) before the programmatic wait; in FP64 those of
    // the second row only where they are used (register pressure)
    constexpr bool early_b = sizeof(T) == 4;
    cpx<T> ta[R], ha[R], tb[R], hb[R];
    auto load_spec = [&](int r, cpx<T> (&t)[R], cpx<T> (&h)[R]) {
#pragma unroll
        for (int a = 0; a < R; ++a) {
            t[a] = chat[(size_t)r * F2 + a * 32 + lane];
            h[a] = chat[F + (size_t)r * F2 + a * 32 + lane];
        }
    };
    if (valid) load_spec(ra, ta, ha);
    if (early_b && pair) load_spec(rb, tb, hb);
    pdl_wait();
    if (gate && !c.sc->active) return;
    const T sg = discrete ? T(-1) : T(1);
    cpx<T> *Sa = (cpx<T> *)c.f4s + (size_t)jm * F + (size_t)ra * F2, *Sb = (cpx<T> *)c.f4s + (size_t)jm * F + (size_t)rb * F2;
    cpx<T> va[R], vb[R];
    if (valid) {
#pragma unroll
        for (int a = 0; a < R; ++a) {
            va[a] = Sa[lane + 32 * a];
            if (pair) vb[a] = Sb[lane + 32 * a];
        }
    }
    __syncthreads();   // twiddles
    if (!valid) return;
    reg_fft_fwd<T, R>(va, twl, w32, lane);
    if (pair) reg_fft_fwd<T, R>(vb, twl, w32, lane);
    cpx<T> pa[R], pb[R];   // Z(-k) at each position of rows a and b
    if (pair) {
#pragma unroll
        for (int a = 0; a < R; ++a) {
            pa[a] = cshfl(vb[R - 1 - a], 31);
            pb[a] = cshfl(va[R - 1 - a], 31);
        }
    } else if (ka == F1 / 2) {
#pragma unroll
        for (int a = 0; a < R; ++a) pa[a] = cshfl(va[R - 1 - a], 31);
    } else {   // row 0
        const int src = brev5((32 - brev5(lane)) & 31);
        pa[0] = {__shfl_sync(0xffffffffu, va[0].x, src), __shfl_sync(0xffffffffu, va[0].y, src)};
#pragma unroll
        for (int a = 1; a < R; ++a) pa[a] = cshfl(va[R - a], 31);
    }
    const cpx<T> *t2a = ftw + 2 * (size_t)F + (size_t)ra * F2, *t2b = ftw + 2 * (size_t)F + (size_t)rb * F2;
#pragma unroll
    for (int a = 0; a < R; ++a) {
        const cpx<T> y = cmul(ta[a], va[a]);
        va[a] = cadd(cpx<T>{sg * y.x, sg * y.y}, cmul(ha[a], pa[a]));
    }
    reg_fft_inv<T, R>(va, twl, w32, lane);
#pragma unroll
    for (int a = 0; a < R; ++a) Sa[lane + 32 * a] = cmul(va[a], cconj(t2a[lane + 32 * a]));
    if (!pair) return;
    if (!early_b) load_spec(rb, tb, hb);
#pragma unroll
    for (int a = 0; a < R; ++a) {
        const cpx<T> y = cmul(tb[a], vb[a]);
        vb[a] = cadd(cpx<T>{sg * y.x, sg * y.y}, cmul(hb[a], pb[a]));
    }
    reg_fft_inv<T, R>(vb, twl, w32, lane);
#pragma unroll
    for (int a = 0; a < R; ++a) Sb[lane + 32 * a] = cmul(vb[a], cconj(t2b[lane + 32 * a]));
}

// ---- pass 3: lines over k1 (length F1), one per (n2, mode): IFFT and the epilogue
template <typename T, int F1, int F2, bool HS = false>
__global__ void __launch_bounds__(F4_THREADS) k_f4_p3(CurveDev c, int mode, int discrete, int gate)
{
    // GM_UPDATE_F: the update, then pass 1 of D_t u of the updated columns
    const bool chain = mode == GM_UPDATE_F;
    if (chain) mode = GM_UPDATE;
    using Sec = F4Sector<T, HS>;
    using St = F4Stage<T, F1, HS>;
    constexpr int R = F1 / 32, LS = St::LS, TS = St::TS, MPC = Sec::MPC, NV = Sec::NV;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T> *twl = (cpx<T> *)smem_raw, *w32 = twl + F1, *tile = w32 + 16;
    __shared__ double wsum[F4W];
    __shared__ double red[F4_THREADS];
    __shared__ int am_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n2_0 = blockIdx.y * F4W, jm0 = blockIdx.x * MPC, F = F1 * F2;
    load_line_twiddles<T, F1>(twl, w32, (const cpx<T> *)c.ftw, F);
    DevScalars *sc = c.sc;
    pdl_wait();
    if (gate && !sc->active) return;
    const double lam_d = sc->lambda, dtau_d = sc->dtau;

    // S[jm][k1][n2] of this CTA's lines and sequences -> tile (odd sections in full
    // storage: the block's modes in pairs, as pass 1 wrote them)
    const bool paired = !HS && (c.sym & 1);
    const int nq = paired ? MPC / 2 : MPC, sq0 = paired ? jm0 / 2 : jm0;
    const cpx<T> *S = (const cpx<T> *)c.f4s;
    for (int e = threadIdx.x; e < nq * F1 * F4W; e += F4_THREADS) {
        const int w = e % F4W, r = (e / F4W) % F1, q = e / (F4W * F1);
        tile[q * TS + w * LS + r] = S[((size_t)(sq0 + q) * F1 + r) * F2 + n2_0 + w];
    }
    __syncthreads();
    for (int q = 0; q < nq; ++q) {
        cpx<T> *line = tile + q * TS + warp * LS;
        cpx<T> v[R];
#pragma unroll
        for (int a = 0; a < R; ++a) v[a] = line[a * 32 + lane];
        __syncwarp();
        reg_fft_inv<T, R>(v, twl, w32, lane);
#pragma unroll
        for (int a = 0; a < R; ++a) line[lane + 32 * a] = v[a];
    }
    __syncthreads();

    // epilogue over the sections j = F2 n1 + n2 < N_s: thread -> line n2_0 + tn,
    // n1 = t / F4W + 32 i; the MPC modes' columns of row j as one sector.  Two rows
    // at a time, all their loads issued before the arithmetic.
    constexpr int hs = HS ? 1 : 0;
    const int ns = c.ns, N = c.W, P = c.P, sym = c.sym;   // N: the stored columns
    const T *rowscale = (const T *)(discrete ? c.twr : c.sig);
    T *Dout = (T *)c.D, *U = (T *)c.U, *G = (T *)c.G;
    const T *Ah = (const T *)c.A;
    // the IMEX factors of the sector's columns: full storage, mode jm0 + q / 2 of
    // column q; sine storage, mode 2 jm0 + q
    const T *prec = (const T *)c.prec_imex + (HS ? 2 * jm0 : jm0);
    const T lam = (T)lam_d, dtau = (T)dtau_d;
    const int tn = threadIdx.x % F4W;
    double partsum = 0.0;
#pragma unroll
    for (int i0 = 0; i0 < R; i0 += 2) {
        int jv[2];
        T rsv[2], av[2][NV], uv[2][NV];
        double wv[2] = {0.0, 0.0};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = F2 * (threadIdx.x / F4W + 32 * (i0 + h)) + n2_0 + tn;
            jv[h] = j;
            rsv[h] = rowscale[j < ns ? j : 0];
            if (mode != GM_STORE && j > 0 && j < P) {
                const size_t o = (size_t)j * N + 2 * jm0;
                ld_sector(Ah + o, av[h]);
                if (mode == GM_UPDATE) ld_sector(U + o, uv[h]);
                wv[h] = c.w[j];
            } else if (chain && (j == 0 || j == P)) {
                ld_sector(U + (size_t)j * N + 2 * jm0, uv[h]);   // the end rows, for the chained pass 1
            }
        }
        if (jv[0] >= ns) break;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = jv[h], n1 = threadIdx.x / F4W + 32 * (i0 + h);
            if (j >= ns) break;
            T y[NV];
            if (paired) {
#pragma unroll
                for (int q = 0; q < MPC / 2; ++q) {
                    const cpx<T> t = tile[q * TS + tn * LS + n1];
                    y[4 * q] = T(0);
                    y[4 * q + 1] = sector_col_ok(jm0, 4 * q + 1, sym) ? rsv[h] * t.x : T(0);
                    y[4 * q + 2] = T(0);
                    y[4 * q + 3] = sector_col_ok(jm0, 4 * q + 3, sym) ? rsv[h] * t.y : T(0);
                }
            } else {
#pragma unroll
                for (int q = 0; q < MPC; ++q) {
                    const cpx<T> t = tile[q * TS + tn * LS + n1];
                    y[2 * q] = sector_col_ok(jm0, 2 * q, sym, hs) ? rsv[h] * t.x : T(0);
                    y[2 * q + 1] = sector_col_ok(jm0, 2 * q + 1, sym, hs) ? rsv[h] * t.y : T(0);
                }
            }
            const size_t o = (size_t)j * N + 2 * jm0;
            if (mode == GM_STORE) {
                st_sector(Dout + o, y);
                continue;
            }
            T g[NV];
            if (j > 0 && j < P) {
                T gg = T(0);   // this row's sum over the sector in the storage type, one FP64 term per row
#pragma unroll
                for (int q = 0; q < NV; ++q) {
                    g[q] = sector_col_ok(jm0, q, sym, hs) ? -(av[h][q] + (discrete ? -lam * y[q] : lam * y[q])) : T(0);
                    gg += (((HS ? 2 * jm0 + q : jm0 + q / 2) == 0) ? T(1) : T(2)) * g[q] * g[q];
                }
                partsum += wv[h] * (double)gg;
                if (mode == GM_UPDATE) {
#pragma unroll
                    for (int q = 0; q < NV; ++q) uv[h][q] += dtau * prec[HS ? q : q / 2] * g[q];
                    st_sector(U + o, uv[h]);
                }
            } else {
#pragma unroll
                for (int q = 0; q < NV; ++q) g[q] = T(0);
            }
            if (mode == GM_GRAD) st_sector(G + o, g);
            if (chain) {   // z_j = tau_j u_j of the updated column, at the position the epilogue just read
                const T cs = ((const T *)c.tau)[j];
                if (paired) {
#pragma unroll
                    for (int q = 0; q < MPC / 2; ++q)
                        tile[q * TS + tn * LS + n1] = {sector_col_ok(jm0, 4 * q + 1, sym) ? cs * uv[h][4 * q + 1] : T(0),
                                                       sector_col_ok(jm0, 4 * q + 3, sym) ? cs * uv[h][4 * q + 3] : T(0)};
                } else {
#pragma unroll
                    for (int q = 0; q < MPC; ++q)
                        tile[q * TS + tn * LS + n1] = {sector_col_ok(jm0, 2 * q, sym, hs) ? cs * uv[h][2 * q] : T(0),
                                                       sector_col_ok(jm0, 2 * q + 1, sym, hs) ? cs * uv[h][2 * q + 1] : T(0)};
                }
            }
        }
    }
    if (chain) {
        // pass 1 of D_t u (Toeplitz-Hankel form: z_k = tau_k u_k for k <= P, zero above):
        // the rows past the curve, then FFT over n1, step twiddles, into the scratch
        // locations this CTA read (no other CTA reads them)
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int n1 = threadIdx.x / F4W + 32 * i;
            if (F2 * n1 + n2_0 + tn >= ns)
                for (int q = 0; q < nq; ++q) tile[q * TS + tn * LS + n1] = {T(0), T(0)};
        }
        const cpx<T> *t1 = (const cpx<T> *)c.ftw + F + (size_t)(n2_0 + warp) * F1;
        cpx<T> tw1[R];
#pragma unroll
        for (int a = 0; a < R; ++a) tw1[a] = t1[a * 32 + lane];
        __syncthreads();
        for (int q = 0; q < nq; ++q) {
            cpx<T> *line = tile + q * TS + warp * LS;
            cpx<T> v[R];
#pragma unroll
            for (int a = 0; a < R; ++a) v[a] = line[lane + 32 * a];
            __syncwarp();
            reg_fft_fwd<T, R>(v, twl, w32, lane);
#pragma unroll
            for (int a = 0; a < R; ++a) line[a * 32 + lane] = cmul(v[a], tw1[a]);
        }
        __syncthreads();
        cpx<T> *So = (cpx<T> *)c.f4s;
        for (int e = threadIdx.x; e < nq * F1 * F4W; e += F4_THREADS) {
            const int w = e % F4W, r = (e / F4W) % F1, q = e / (F4W * F1);
            So[((size_t)(sq0 + q) * F1 + r) * F2 + n2_0 + w] = tile[q * TS + w * LS + r];
        }
    }
    if (mode == GM_STORE) return;

    // ---- FP64 |G|^2: per-CTA partial, last CTA of the grid sums them in a fixed order
    partsum = warp_sum(partsum);
    if (lane == 0) wsum[warp] = partsum;
    __syncthreads();
    const int bid = blockIdx.y * gridDim.x + blockIdx.x, nb = gridDim.x * gridDim.y;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < F4W; ++w) t += wsum[w];
        c.tile[bid] = t;
    }
    if (!last_cta_arrive(&sc->cnt_gemm, (unsigned)nb, am_last)) return;
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

// ---- the clustered form: the three passes of MPC modes in one launch, by a
// cluster of CS CTAs that holds the modes' whole intermediate array in
// distributed shared memory.  CTA `rank` owns the scrambled rows r of k1 in
// [rank F1/CS, (rank + 1) F1/CS) (all n2) and the lines n2 in [rank F2/CS, ...):
//   pass 1: FFT over n1 of its lines into a local tile [mode][line][r], then each
//           row's run of its lines copied to the row's owner in 16-byte chunks;
//   pass 2: FFT, spectrum, IFFT over n2 of its own rows, in place;
//   pass 3: its lines' runs copied back from the rows' owners into the tile,
//           IFFT over k1, epilogue.
// Remote shared memory is only moved in contiguous 16-byte chunks (scattered
// 8-byte remote accesses cost several cycles each, measured).  Cluster
// barriers order the passes (release / acquire) and keep every CTA resident
// until its rows have been read; they are hardware barriers of one cluster,
// whose CTAs run together.
__device__ __forceinline__ void cluster_arrive_relaxed() { asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

template <typename T, int NV>
struct RowVec;   // NV values of a section row: 8 or 16 bytes
template <> struct RowVec<float, 2> {
    static __device__ __forceinline__ void ld(const float *p, float (&x)[2]) { const float2 v = *reinterpret_cast<const float2 *>(p); x[0] = v.x; x[1] = v.y; }
    static __device__ __forceinline__ void ldcg(const float *p, float (&x)[2]) { const float2 v = __ldcg(reinterpret_cast<const float2 *>(p)); x[0] = v.x; x[1] = v.y; }
    static __device__ __forceinline__ void st(float *p, const float (&x)[2]) { *reinterpret_cast<float2 *>(p) = make_float2(x[0], x[1]); }
};
template <> struct RowVec<float, 4> {
    static __device__ __forceinline__ void ld(const float *p, float (&x)[4]) { const float4 v = *reinterpret_cast<const float4 *>(p); x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w; }
    static __device__ __forceinline__ void ldcg(const float *p, float (&x)[4]) { const float4 v = __ldcg(reinterpret_cast<const float4 *>(p)); x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w; }
    static __device__ __forceinline__ void st(float *p, const float (&x)[4]) { *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]); }
};
template <> struct RowVec<double, 2> {
    static __device__ __forceinline__ void ld(const double *p, double (&x)[2]) { const double2 v = *reinterpret_cast<const double2 *>(p); x[0] = v.x; x[1] = v.y; }
    static __device__ __forceinline__ void ldcg(const double *p, double (&x)[2]) { const double2 v = __ldcg(reinterpret_cast<const double2 *>(p)); x[0] = v.x; x[1] = v.y; }
    static __device__ __forceinline__ void st(double *p, const double (&x)[2]) { *reinterpret_cast<double2 *>(p) = make_double2(x[0], x[1]); }
};

// one 16-byte chunk of complex values (two FP32 or one FP64)
__device__ __forceinline__ void st_chunk(cpx<float> *p, const cpx<float> (&v)[2])
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
}
__device__ __forceinline__ void st_chunk(cpx<double> *p, const cpx<double> (&v)[1])
{
    *reinterpret_cast<double2 *>(p) = make_double2(v[0].x, v[0].y);
}
__device__ __forceinline__ void ld_chunk(const cpx<float> *p, cpx<float> (&v)[2])
{
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = {t.x, t.y};
    v[1] = {t.z, t.w};
}
__device__ __forceinline__ void ld_chunk(const cpx<double> *p, cpx<double> (&v)[1])
{
    const double2 t = *reinterpret_cast<const double2 *>(p);
    v[0] = {t.x, t.y};
}

// Shared memory of the clustered form: line twiddles, the rows this CTA owns
// B[mode][row][F2] and the tile of its lines L[mode][line][F1 + pad].
template <typename T, int F1, int F2, int MPC>
struct F4C {
    static constexpr int CV = 16 / (int)sizeof(cpx<T>);          // complex values per 16-byte chunk
    static constexpr int LT = F1 + (sizeof(T) == 4 ? 2 : 1);    // tile row: conflict-free column access
    static size_t bytes(int cs)
    {
        return ((size_t)F1 + F2 + 16 + (size_t)MPC * (F1 / cs) * F2 + (size_t)MPC * (F2 / cs) * LT) * sizeof(cpx<T>);
    }
};

template <typename T, int F1, int F2, int MPC, bool STEP>
__global__ void __launch_bounds__(F4_THREADS) k_f4c(CurveDev c, int mode, int discrete, int gate)
{
    // STEP: the fused descent step (mode GM_STEP, two contractions); otherwise one
    // contraction (GM_STORE / GM_UPDATE / GM_GRAD)
    constexpr int NCT = STEP ? 2 : 1;
    namespace cg = cooperative_groups;
    using Cfg = F4C<T, F1, F2, MPC>;
    constexpr int R1 = F1 / 32, R2 = F2 / 32, NV = 2 * MPC, CV = Cfg::CV, LT = Cfg::LT;
    using RV = RowVec<T, NV>;
    cg::cluster_group cluster = cg::this_cluster();
    const int CS = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
    const int RPC = F1 / CS, LPC = F2 / CS, CPS = LPC / CV;   // rows, lines, chunks of a row's run
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T> *tw1 = (cpx<T> *)smem_raw, *tw2 = tw1 + F1, *w32 = tw2 + F2;
    cpx<T> *B = w32 + 16, *Lt = B + (size_t)MPC * RPC * F2;
    __shared__ double wsum[F4W];
    __shared__ double red[F4_THREADS];
    __shared__ int am_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, jm0 = blockIdx.y * MPC, F = F1 * F2;
    const int P = c.P, N = c.W, ns = c.ns, sym = c.sym, hs = c.hs;   // N: the stored columns
    unsigned live = 0;   // bit q: column 2 jm0 + q of the sector is one the subspace keeps
#pragma unroll
    for (int q = 0; q < NV; ++q) live |= sector_col_ok(jm0, q, sym, hs) ? 1u << q : 0u;
    const cpx<T> *ftw = (const cpx<T> *)c.ftw;
    // the contraction being applied: GM_STEP runs the update (adjoint mode
    // `discrete`), then D_t u of the updated state (cmode, cdisc switch between them)
    int cmode = STEP ? GM_UPDATE : mode, cdisc = discrete;
    const T *X = (const T *)(cmode == GM_STORE ? c.U : c.R);
    const T *colscale = (const T *)(cdisc ? c.sw : c.tau);
    const T *rowscale = (const T *)(cdisc ? c.twr : c.sig);
    T *Dout = (T *)c.D, *U = (T *)c.U, *G = (T *)c.G;
    const T *Ah = (const T *)c.A;
    T s = cdisc ? T(-1) : T(1);

    // Inputs of one item of each pass.  The set-up tables of every warp's first
    // item are loaded before the programmatic wait, its field values right after
    // it, so that their latency overlaps the predecessor's tail and the passes.
    // pass 1, line n2: source rows m (-1: zero), scale, step twiddles; the rows' values
    auto p1_tables = [&](int n2, int (&m)[R1], T (&cs)[R1], cpx<T> (&t1)[R1]) {
#pragma unroll
        for (int a = 0; a < R1; ++a) {
            const int k = F2 * (lane + 32 * a) + n2;
            int mm = -1;
            T f = T(1);
            if (k == 0) { mm = 0; f = T(1) + s; }
            else if (k < P) { mm = k; f = s; }
            else if (k == P) { mm = P; f = T(1) + s; }
            else if (k < 2 * P) { mm = 2 * P - k; }
            if (f == T(0)) mm = -1;
            m[a] = mm;
            cs[a] = mm >= 0 ? f * colscale[mm] : T(0);
            t1[a] = ftw[F + (size_t)n2 * F1 + 32 * a + lane];
        }
    };
    auto p1_rows = [&](const int (&m)[R1], T (&x)[R1][NV]) {
#pragma unroll
        for (int a = 0; a < R1; ++a) {
#pragma unroll
            for (int q = 0; q < NV; ++q) x[a][q] = T(0);
            if (m[a] >= 0) RV::ldcg(X + (size_t)m[a] * N + 2 * jm0, x[a]);
        }
    };
    // pass 2, row r: kernel spectrum and step twiddles
    auto p2_tables = [&](int r, cpx<T> (&chv)[R2], cpx<T> (&t2v)[R2]) {
        const cpx<T> *chp = (const cpx<T> *)c.chat + (size_t)r * F2, *t2 = ftw + 2 * (size_t)F + (size_t)r * F2;
#pragma unroll
        for (int a = 0; a < R2; ++a) {
            chv[a] = chp[32 * a + lane];
            t2v[a] = t2[lane + 32 * a];
        }
    };
    // pass 3, line n2, rows a0 and a0 + 1: row scale and quadrature weight; A and u
    auto p3_tables = [&](int n2, int a0, int (&jv)[2], T (&rsv)[2], double (&wv)[2]) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = F2 * (lane + 32 * (a0 + h)) + n2;
            jv[h] = j;
            rsv[h] = rowscale[j < ns ? j : 0];
            wv[h] = (j > 0 && j < P) ? c.w[j] : 0.0;
        }
    };
    auto p3_rows = [&](const int (&jv)[2], T (&av)[2][NV], T (&uv)[2][NV]) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = jv[h];
            if (cmode != GM_STORE && j > 0 && j < P) {
                const size_t o = (size_t)j * N + 2 * jm0;
                RV::ld(Ah + o, av[h]);
                if (cmode == GM_UPDATE) RV::ld(U + o, uv[h]);
            }
        }
    };

    load_line_twiddles<T, F2>(tw2, w32, ftw, F);
    for (int t = threadIdx.x; t < F1; t += F4_THREADS) tw1[t] = ftw[(size_t)((t >> 5) * (t & 31)) * (F / F1)];
    int m1f[R1];
    T cs1f[R1];
    cpx<T> t1f[R1], ch2f[R2], t22f[R2];
    int j3f[2];
    T rs3f[2];
    double w3f[2];
    if (warp < LPC) {
        p1_tables(rank * LPC + warp, m1f, cs1f, t1f);
        p3_tables(rank * LPC + warp, 0, j3f, rs3f, w3f);
    }
    if (warp < MPC * RPC) p2_tables(rank * RPC + warp % RPC, ch2f, t22f);
    DevScalars *sc = c.sc;
    pdl_wait();
    if (gate && !sc->active) return;   // the whole cluster leaves together
    cluster_arrive_relaxed();          // every CTA of the cluster has started (before the first copy)
    T x1f[R1][NV], a3f[2][NV], u3f[2][NV];
    if (warp < LPC) {
        p1_rows(m1f, x1f);
        p3_rows(j3f, a3f, u3f);
    }
    const double lam_d = sc->lambda, dtau_d = sc->dtau;
    const T *prec = (const T *)c.prec_imex + (hs ? 2 * jm0 : jm0);   // the IMEX factors of the sector
    const T lam = (T)lam_d, dtau = (T)dtau_d;
    double partsum = 0.0;
    __syncthreads();   // twiddles

    for (int ct = 0; ct < NCT; ++ct) {
    const bool pf = (ct == 0);   // the prefetched first items belong to the first contraction
    if (ct == 1) {
        cmode = GM_STORE;
        cdisc = 0;
        X = (const T *)c.U;
        colscale = (const T *)c.tau;
        rowscale = (const T *)c.sig;
        s = T(1);
    }

    // ---- pass 1: lines n2 of this CTA, MPC modes each, into the tile
    for (int li = warp; li < LPC; li += F4W) {
        const int n2 = rank * LPC + li;
        int m[R1];
        T x[R1][NV], cs[R1];
        cpx<T> t1[R1];
        if (pf && li == warp) {
#pragma unroll
            for (int a = 0; a < R1; ++a) {
                cs[a] = cs1f[a];
                t1[a] = t1f[a];
#pragma unroll
                for (int q = 0; q < NV; ++q) x[a][q] = x1f[a][q];
            }
        } else {
            p1_tables(n2, m, cs, t1);
            p1_rows(m, x);
        }
#pragma unroll
        for (int q = 0; q < MPC; ++q) {
            cpx<T> v[R1];
#pragma unroll
            for (int a = 0; a < R1; ++a)
                v[a] = {((live >> (2 * q)) & 1u) ? cs[a] * x[a][2 * q] : T(0),
                        ((live >> (2 * q + 1)) & 1u) ? cs[a] * x[a][2 * q + 1] : T(0)};
            reg_fft_fwd<T, R1>(v, tw1, w32, lane);
            cpx<T> *lt = Lt + ((size_t)q * LPC + li) * LT;
#pragma unroll
            for (int a = 0; a < R1; ++a) lt[32 * a + lane] = cmul(v[a], t1[a]);
        }
    }
    __syncthreads();
    if (pf) cluster_wait();   // every CTA has started
    // each row r's run of this CTA's lines -> the row's owner, columns [rank LPC, rank LPC + LPC)
    for (int e = threadIdx.x; e < MPC * F1 * CPS; e += F4_THREADS) {
        const int ch = e % CPS, r = (e / CPS) % F1, q = e / (CPS * F1), owner = r / RPC;
        cpx<T> vals[CV];
#pragma unroll
        for (int i = 0; i < CV; ++i) vals[i] = Lt[((size_t)q * LPC + ch * CV + i) * LT + r];
        cpx<T> *dst = cluster.map_shared_rank(B, owner) + ((size_t)q * RPC + (r - owner * RPC)) * F2 + rank * LPC + ch * CV;
        st_chunk(dst, vals);
    }
    cluster_arrive();
    cluster_wait();

    // ---- pass 2: this CTA's rows, in place
    for (int rl = warp; rl < MPC * RPC; rl += F4W) {
        cpx<T> *row = B + (size_t)rl * F2;
        cpx<T> v[R2], chv[R2], t2v[R2];
        if (pf && rl == warp) {
#pragma unroll
            for (int a = 0; a < R2; ++a) {
                chv[a] = ch2f[a];
                t2v[a] = t22f[a];
            }
        } else {
            p2_tables(rank * RPC + rl % RPC, chv, t2v);
        }
#pragma unroll
        for (int a = 0; a < R2; ++a) v[a] = row[lane + 32 * a];
        reg_fft_fwd<T, R2>(v, tw2, w32, lane);
#pragma unroll
        for (int a = 0; a < R2; ++a) v[a] = cmul(v[a], chv[a]);
        reg_fft_inv<T, R2>(v, tw2, w32, lane);
#pragma unroll
        for (int a = 0; a < R2; ++a) row[lane + 32 * a] = cmul(v[a], cconj(t2v[a]));
    }
    cluster_arrive();
    cluster_wait();

    // ---- pass 3: this CTA's lines copied back into the tile, IFFT over k1, epilogue
    for (int e = threadIdx.x; e < MPC * F1 * CPS; e += F4_THREADS) {
        const int ch = e % CPS, r = (e / CPS) % F1, q = e / (CPS * F1), owner = r / RPC;
        const cpx<T> *src = cluster.map_shared_rank(B, owner) + ((size_t)q * RPC + (r - owner * RPC)) * F2 + rank * LPC + ch * CV;
        cpx<T> vals[CV];
        ld_chunk(src, vals);
#pragma unroll
        for (int i = 0; i < CV; ++i) Lt[((size_t)q * LPC + ch * CV + i) * LT + r] = vals[i];
    }
    // The last contraction: this CTA's rows may be freed once every CTA has
    // copied its runs (the copies have completed: their values are in the tile),
    // so no release is needed.  Before a second contraction the barrier comes
    // after the epilogue instead (release / acquire of the updated state, and the
    // rows are free to be pushed into again).
    const bool last = (ct + 1 == NCT);
    if (last) cluster_arrive_relaxed();
    __syncthreads();

    // epilogue on the sections j = F2 n1 + n2 < N_s (n1 = lane + 32 a; rows two
    // at a time, their loads issued first)
    for (int li = warp; li < LPC; li += F4W) {
        const int n2 = rank * LPC + li;
        cpx<T> y[MPC][R1];
#pragma unroll
        for (int q = 0; q < MPC; ++q) {
            const cpx<T> *lt = Lt + ((size_t)q * LPC + li) * LT;
#pragma unroll
            for (int a = 0; a < R1; ++a) y[q][a] = lt[32 * a + lane];
            reg_fft_inv<T, R1>(y[q], tw1, w32, lane);
        }
#pragma unroll
        for (int a0 = 0; a0 < R1; a0 += 2) {
            int jv[2];
            T rsv[2], av[2][NV], uv[2][NV];
            double wv[2];
            if (pf && li == warp && a0 == 0) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    jv[h] = j3f[h];
                    rsv[h] = rs3f[h];
                    wv[h] = w3f[h];
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        av[h][q] = a3f[h][q];
                        uv[h][q] = u3f[h][q];
                    }
                }
            } else {
                p3_tables(n2, a0, jv, rsv, wv);
                p3_rows(jv, av, uv);
            }
            if (jv[0] >= ns) break;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = jv[h];
                if (j >= ns) continue;
                T yv[NV];
#pragma unroll
                for (int q = 0; q < MPC; ++q) {
                    yv[2 * q] = ((live >> (2 * q)) & 1u) ? rsv[h] * y[q][a0 + h].x : T(0);
                    yv[2 * q + 1] = ((live >> (2 * q + 1)) & 1u) ? rsv[h] * y[q][a0 + h].y : T(0);
                }
                const size_t o = (size_t)j * N + 2 * jm0;
                if (cmode == GM_STORE) {
                    RV::st(Dout + o, yv);
                    continue;
                }
                T g[NV];
                if (j > 0 && j < P) {
                    T gg = T(0);   // the row's sum over the sector in the storage type, one FP64 term per row
#pragma unroll
                    for (int q = 0; q < NV; ++q) {
                        g[q] = ((live >> q) & 1u) ? -(av[h][q] + (cdisc ? -lam * yv[q] : lam * yv[q])) : T(0);
                        gg += (((hs ? 2 * jm0 + q : jm0 + q / 2) == 0) ? T(1) : T(2)) * g[q] * g[q];
                    }
                    partsum += wv[h] * (double)gg;
                    if (cmode == GM_UPDATE) {
#pragma unroll
                        for (int q = 0; q < NV; ++q) uv[h][q] += dtau * prec[hs ? q : q / 2] * g[q];
                        RV::st(U + o, uv[h]);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < NV; ++q) g[q] = T(0);
                }
                if (cmode == GM_GRAD) RV::st(G + o, g);
            }
        }
    }
    if (!last) cluster_arrive();
    cluster_wait();
    }   // contractions
    if (mode == GM_STORE) return;

    // ---- FP64 |G|^2: per-CTA partial, last CTA of the grid sums them in a fixed order
    partsum = warp_sum(partsum);
    if (lane == 0) wsum[warp] = partsum;
    __syncthreads();
    const int bid = blockIdx.y * gridDim.x + blockIdx.x, nb = gridDim.x * gridDim.y;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < F4W; ++w) t += wsum[w];
        c.tile[bid] = t;
    }
    if (!last_cta_arrive(&sc->cnt_gemm, (unsigned)nb, am_last)) return;
    double t = 0.0;
    for (int b = threadIdx.x; b < nb; b += F4_THREADS) t += __ldcg(c.tile + b);
    t = block_sum<F4_THREADS>(t, red);
    if (threadIdx.x == 0) {
        sc->G2 = c.L * t;
        if (STEP || mode == GM_UPDATE) {
            sc->step += 1;
            sc->tau += sc->dtau;
            sc->lambda = sc->lambda_next;
        }
        sc->cnt_gemm = 0;
    }
}

// ---- the one-CTA-per-mode form (batched curves): one CTA holds a mode's whole
// F1 x F2 array in shared memory, rows r of k1 (scrambled) by columns n2, with a
// row stride F2 + 1 so that the column accesses of a warp (32 consecutive rows)
// fall in distinct banks; the three passes of the four-step form with the same
// register line transforms and tables, separated by CTA barriers; the epilogue
// and the per-curve last-CTA FP64 |G|^2 of the one-CTA FFT form.
template <typename T, int F1, int F2>
struct F4B {
    static constexpr int BS = F2 + 1;
    static constexpr size_t BYTES = ((size_t)F1 + F2 + 16 + (size_t)F1 * BS) * sizeof(cpx<T>);
};

template <typename T, int F1, int F2>
__device__ __forceinline__ void f4b_body(const CurveDev &c, int mode, int discrete, int gate, int jm, int nmodes)
{
    using V2 = typename V2of<T>::type;
    constexpr int R1 = F1 / 32, R2 = F2 / 32, BS = F4B<T, F1, F2>::BS, F = F1 * F2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<T> *tw1 = (cpx<T> *)smem_raw, *tw2 = tw1 + F1, *w32 = tw2 + F2, *B = w32 + 16;
    __shared__ double red[F4_THREADS];
    __shared__ int am_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const cpx<T> *ftw = (const cpx<T> *)c.ftw, *chat = (const cpx<T> *)c.chat;
    load_line_twiddles<T, F2>(tw2, w32, ftw, F);
    for (int t = threadIdx.x; t < F1; t += F4_THREADS) tw1[t] = ftw[(size_t)((t >> 5) * (t & 31)) * (F / F1)];
    DevScalars *sc = c.sc;
    pdl_wait();
    if (gate && !sc->active) return;
    // GM_STEP: the update, then D_t u of the updated column in the same CTA (its
    // pass 1 fed from the update's registers: the same (line, position) layout)
    const bool step = mode == GM_STEP && c.f4h;
    if (step) mode = GM_UPDATE;
    const double lam_d = sc->lambda, dtau_d = sc->dtau;
    const int P = c.P, N = c.W, ns = c.ns;   // N: the stored columns
    const T *X = (const T *)(mode == GM_STORE ? c.U : c.R);
    const T *colscale = (const T *)(discrete ? c.sw : c.tau);
    const T s = discrete ? T(-1) : T(1);
    const int ca = 2 * jm, cb = 2 * jm + 1;
    const bool oka = col_live(ca, c.sym, c.hs), okb = col_live(cb, c.sym, c.hs);   // a column pair
    __syncthreads();   // twiddles

    // pass 1: lines n2, FFT over n1, times W_F^(n2 k1), into column n2 of B.  A
    // line's column values are loaded during the previous line's transform (the
    // rows and scales first, then every load of the line at once).
    auto load_line = [&](int n2, V2 (&xv)[R1], T (&cs)[R1]) {
#pragma unroll
        for (int a = 0; a < R1; ++a) {
            const int k = F2 * (lane + 32 * a) + n2;
            int m = -1;
            T f = T(1);
            if (c.f4h) {   // Toeplitz-Hankel form: the column itself
                if (k <= P) m = k;
            }
            else if (k == 0) { m = 0; f = T(1) + s; }
            else if (k < P) { m = k; f = s; }
            else if (k == P) { m = P; f = T(1) + s; }
            else if (k < 2 * P) { m = 2 * P - k; }
            if (f == T(0)) m = -1;
            const int mm = m >= 0 ? m : 0;
            cs[a] = m >= 0 ? f * colscale[mm] : T(0);
            const V2 x = *reinterpret_cast<const V2 *>(X + (size_t)mm * N + ca);
            xv[a] = m >= 0 ? x : V2{T(0), T(0)};
        }
    };
    V2 xv[R1];
    T cs[R1];
    if (warp < F2) load_line(warp, xv, cs);
    for (int n2 = warp; n2 < F2; n2 += F4W) {
        V2 nxv[R1];
        T ncs[R1];
        if (n2 + F4W < F2) load_line(n2 + F4W, nxv, ncs);
        cpx<T> t1[R1];
#pragma unroll
        for (int a = 0; a < R1; ++a) t1[a] = ftw[F + (size_t)n2 * F1 + 32 * a + lane];
        cpx<T> v[R1];
#pragma unroll
        for (int a = 0; a < R1; ++a) v[a] = {oka ? cs[a] * xv[a].x : T(0), okb ? cs[a] * xv[a].y : T(0)};
        reg_fft_fwd<T, R1>(v, tw1, w32, lane);
#pragma unroll
        for (int a = 0; a < R1; ++a) B[(32 * a + lane) * BS + n2] = cmul(v[a], t1[a]);
#pragma unroll
        for (int a = 0; a < R1; ++a) {
            xv[a] = nxv[a];
            cs[a] = ncs[a];
        }
    }
    __syncthreads();

    // pass 2 (sign sg of the Toeplitz part: -1 for the discrete adjoint's transpose)
    auto pass2 = [&](T sg) {
        if (c.f4h) {   // rows k1 and F1 - k1 together (0 and F1/2 alone), as in k_f4h_p2
            for (int it = warp; it <= F1 / 2; it += F4W) {
                const bool pair = it > 0 && it < F1 / 2;
                const int ka = it, kb = F1 - it;
                const int ra = (ka % R1) * 32 + brev5(ka / R1), rb = pair ? (kb % R1) * 32 + brev5(kb / R1) : 0;
                cpx<T> *rowa = B + (size_t)ra * BS, *rowb = B + (size_t)rb * BS;
                cpx<T> va[R2], vb[R2], pa[R2], pb[R2];
#pragma unroll
                for (int a = 0; a < R2; ++a) {
                    va[a] = rowa[lane + 32 * a];
                    if (pair) vb[a] = rowb[lane + 32 * a];
                }
                reg_fft_fwd<T, R2>(va, tw2, w32, lane);
                if (pair) reg_fft_fwd<T, R2>(vb, tw2, w32, lane);
                if (pair) {
#pragma unroll
                    for (int a = 0; a < R2; ++a) {
                        pa[a] = cshfl(vb[R2 - 1 - a], 31);
                        pb[a] = cshfl(va[R2 - 1 - a], 31);
                    }
                } else if (ka == F1 / 2) {
#pragma unroll
                    for (int a = 0; a < R2; ++a) pa[a] = cshfl(va[R2 - 1 - a], 31);
                } else {   // row 0
                    const int src = brev5((32 - brev5(lane)) & 31);
                    pa[0] = {__shfl_sync(0xffffffffu, va[0].x, src), __shfl_sync(0xffffffffu, va[0].y, src)};
#pragma unroll
                    for (int a = 1; a < R2; ++a) pa[a] = cshfl(va[R2 - a], 31);
                }
                // Y = s T^ Z + H^ Z(-k), IFFT, W_F^(-n2 k1), back into the row
                auto finish = [&](int r, cpx<T> *row, cpx<T> (&v)[R2], const cpx<T> (&pp)[R2]) {
                    const cpx<T> *ct = chat + (size_t)r * F2, *chh = chat + F + (size_t)r * F2;
                    const cpx<T> *t2 = ftw + 2 * (size_t)F + (size_t)r * F2;
#pragma unroll
                    for (int a = 0; a < R2; ++a) {
                        const cpx<T> y = cmul(ct[32 * a + lane], v[a]);
                        v[a] = cadd(cpx<T>{sg * y.x, sg * y.y}, cmul(chh[32 * a + lane], pp[a]));
                    }
                    reg_fft_inv<T, R2>(v, tw2, w32, lane);
#pragma unroll
                    for (int a = 0; a < R2; ++a) row[lane + 32 * a] = cmul(v[a], cconj(t2[lane + 32 * a]));
                };
                finish(ra, rowa, va, pa);
                if (pair) finish(rb, rowb, vb, pb);
            }
        }
        // rows r: FFT over n2, kernel spectrum, IFFT, times W_F^(-n2 k1), in place
        for (int r = warp; r < F1 && !c.f4h; r += F4W) {
            cpx<T> *row = B + (size_t)r * BS;
            const cpx<T> *ch = chat + (size_t)r * F2, *t2 = ftw + 2 * (size_t)F + (size_t)r * F2;
            cpx<T> v[R2], chv[R2], t2v[R2];
#pragma unroll
            for (int a = 0; a < R2; ++a) {
                chv[a] = ch[32 * a + lane];
                t2v[a] = t2[lane + 32 * a];
                v[a] = row[lane + 32 * a];
            }
            reg_fft_fwd<T, R2>(v, tw2, w32, lane);
#pragma unroll
            for (int a = 0; a < R2; ++a) v[a] = cmul(v[a], chv[a]);
            reg_fft_inv<T, R2>(v, tw2, w32, lane);
#pragma unroll
            for (int a = 0; a < R2; ++a) row[lane + 32 * a] = cmul(v[a], cconj(t2v[a]));
        }
    };
    pass2(s);
    __syncthreads();

    // pass 3: lines n2, IFFT over k1, epilogue on the sections j = F2 n1 + n2 < N_s;
    // `chain`: then pass 1 of D_t u of the line's updated sections into column n2
    T *Dout = (T *)c.D, *U = (T *)c.U, *G = (T *)c.G;
    const T *Ah = (const T *)c.A;
    const T pra = ((const T *)c.prec_imex)[col_mode(ca, c.hs)], prb = ((const T *)c.prec_imex)[col_mode(cb, c.hs)];
    const T lam = (T)lam_d, dtau = (T)dtau_d;
    const double cw = col_weight(cb, c.hs);   // column a's weight where it is live
    const T *tauc = (const T *)c.tau;
    auto pass3 = [&](int md, bool disc, bool chain) -> double {
        const T *rowscale = (const T *)(disc ? c.twr : c.sig);
        double partsum = 0.0;
        for (int n2 = warp; n2 < F2; n2 += F4W) {
            cpx<T> v[R1];
#pragma unroll
            for (int a = 0; a < R1; ++a) v[a] = B[(32 * a + lane) * BS + n2];
            // the epilogue operands of this line's sections, issued before the transform
            T rs[R1];
            double wj[R1];
            V2 av[R1], uv[R1];
#pragma unroll
            for (int a = 0; a < R1; ++a) {
                const int j = F2 * (lane + 32 * a) + n2;
                rs[a] = rowscale[j < ns ? j : 0];
                wj[a] = 0.0;
                uv[a] = V2{T(0), T(0)};
                if (md != GM_STORE && j > 0 && j < P) {
                    wj[a] = c.w[j];
                    av[a] = *reinterpret_cast<const V2 *>(Ah + (size_t)j * N + ca);
                    if (md == GM_UPDATE) uv[a] = *reinterpret_cast<const V2 *>(U + (size_t)j * N + ca);
                } else if (chain && (j == 0 || j == P)) {
                    uv[a] = *reinterpret_cast<const V2 *>(U + (size_t)j * N + ca);   // end rows, for the chained pass 1
                }
            }
            reg_fft_inv<T, R1>(v, tw1, w32, lane);
#pragma unroll
            for (int a = 0; a < R1; ++a) {
                const int j = F2 * (lane + 32 * a) + n2;
                if (j >= ns) break;
                const cpx<T> yv = {rs[a] * v[a].x, rs[a] * v[a].y};
                const size_t o = (size_t)j * N + ca;
                if (md == GM_STORE) {
                    *reinterpret_cast<V2 *>(Dout + o) = V2{oka ? yv.x : T(0), okb ? yv.y : T(0)};
                    continue;
                }
                const bool interior = (j > 0 && j < P);
                T ga = 0, gb = 0;
                if (interior) {
                    if (oka) ga = -(av[a].x + (disc ? -lam * yv.x : lam * yv.x));
                    if (okb) gb = -(av[a].y + (disc ? -lam * yv.y : lam * yv.y));
                    partsum += wj[a] * cw * (double)(ga * ga + gb * gb);
                }
                if (md == GM_UPDATE) {
                    if (interior) {
                        uv[a] = V2{uv[a].x + dtau * pra * ga, uv[a].y + dtau * prb * gb};
                        *reinterpret_cast<V2 *>(U + o) = uv[a];
                    }
                } else {
                    *reinterpret_cast<V2 *>(G + o) = V2{ga, gb};
                }
            }
            if (chain) {   // z_j = tau_j u_j (j <= P), zero above: FFT over n1, W_F^(n2 k1), into column n2
                cpx<T> z[R1];
#pragma unroll
                for (int a = 0; a < R1; ++a) {
                    const int j = F2 * (lane + 32 * a) + n2;
                    const T cs = j < ns ? tauc[j] : T(0);
                    z[a] = {oka ? cs * uv[a].x : T(0), okb ? cs * uv[a].y : T(0)};
                }
                reg_fft_fwd<T, R1>(z, tw1, w32, lane);
#pragma unroll
                for (int a = 0; a < R1; ++a) B[(32 * a + lane) * BS + n2] = cmul(z[a], ftw[F + (size_t)n2 * F1 + 32 * a + lane]);
            }
        }
        return partsum;
    };
    double partsum = pass3(mode, discrete != 0, step);
    if (step) {   // D_t u of the updated column: passes 2 and 3 of the published operator
        __syncthreads();
        pass2(T(1));
        __syncthreads();
        pass3(GM_STORE, false, false);
    }
    if (mode == GM_STORE) return;

    // ---- FP64 |G|^2 of the curve: per-mode partial, the curve's last CTA sums them
    partsum = block_sum<F4_THREADS>(partsum, red);
    if (threadIdx.x == 0) c.tile[jm] = partsum;
    if (!last_cta_arrive(&sc->cnt_gemm, (unsigned)nmodes, am_last)) return;
    double tt = 0.0;
    for (int b2 = threadIdx.x; b2 < nmodes; b2 += F4_THREADS) tt += __ldcg(c.tile + b2);
    tt = block_sum<F4_THREADS>(tt, red);
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

template <typename T, int F1, int F2>
__global__ void __launch_bounds__(F4_THREADS) k_f4b(CurveDev c, int mode, int discrete, int gate)
{
    f4b_body<T, F1, F2>(c, mode, discrete, gate, blockIdx.x, gridDim.x);
}

// Four CTAs per SM: the register cap this sets (64) measured 9% faster on the
// 256-curve batch step than the compiler's own choice (up to 105 registers).
template <typename T, int F1, int F2>
__global__ void __launch_bounds__(F4_THREADS, 4) k_f4b_batch(const CurveDev *cv, const int2 *items, int mode,
                                                          int discrete, int gate)
{
    const int2 it = items[blockIdx.x];
    const CurveDev &c = cv[it.x];
    f4b_body<T, F1, F2>(c, mode, discrete, gate, it.y, c.W / 2);
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

// the Toeplitz-Hankel form's two sequences (kind 1: cot at lags [-P, P], lag l
// at n = l mod F; kind 2: cot at lags [0, 2P]); kind 0 the extended one above
__device__ __forceinline__ double th_kernel(int n, int F, int P, int kind)
{
    if (kind == 0) return cot_kernel(n, F, P);
    int u = -1;
    if (kind == 1) {
        if (n <= P) u = n;
        else if (n >= F - P) u = n - F + 2 * P;
    } else if (n <= 2 * P) {
        u = n == 2 * P ? 0 : n;
    }
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
__global__ void __launch_bounds__(F4_THREADS) k_f4_specA(CurveDev c, int kind)
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
    for (int n1 = lane; n1 < F1; n1 += 32) x[n1] = {th_kernel(F2 * n1 + n2, F, c.P, kind), 0.0};
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
__global__ void __launch_bounds__(F4_THREADS) k_f4_specB(CurveDev c, int half)
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
    cpx<T> *chat = (cpx<T> *)c.chat + (size_t)half * F + (size_t)((k1 % R1) * 32 + brev5(k1 / R1)) * F2;
    cpx<T> *ftw = (cpx<T> *)c.ftw;
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
template <typename T, int F1, int F2, bool HS>
static cudaError_t f4_run(const CurveDev &c, int mode, int discrete, int gate, cudaStream_t st, cudaEvent_t *pass_ev)
{
    const int nm = c.W / 2;   // column pairs
    const size_t sm1 = F4Stage<T, F1, HS>::BYTES;
    const int nmb = c.W / 2 / F4Sector<T, HS>::MPC;
    cudaError_t e;
    if ((e = set_smem(k_f4_p1<T, F1, F2, HS>, sm1)) != cudaSuccess) return e;
    if ((e = set_smem(k_f4_p3<T, F1, F2, HS>, sm1)) != cudaSuccess) return e;
    // GM_STORE_P23: pass 1 ran inside the preceding update's pass 3
    if (mode == GM_STORE_P23) mode = GM_STORE;
    else if ((e = launch_pdl(k_f4_p1<T, F1, F2, HS>, dim3(nmb, F2 / F4W), sm1, st, c,
                             mode == GM_UPDATE_F ? GM_UPDATE : mode, discrete, gate)) != cudaSuccess)
        return e;
    if (pass_ev && (e = cudaEventRecord(pass_ev[0], st)) != cudaSuccess) return e;
    // pass 2 per sequence: the column pairs, or for odd sections in full storage
    // the modes' imaginary columns in pairs
    const int nseq = ((c.sym & 1) && !c.hs) ? nm / 2 : nm;
    if (c.f4h) e = launch_pdl(k_f4h_p2<T, F1, F2>, dim3((F1 / 2 + 1 + F4W - 1) / F4W, nseq), 0, st, c, discrete, gate);
    else e = launch_pdl(k_f4_p2<T, F1, F2>, dim3(F1 / F4W, nseq), 0, st, c, gate);
    if (e != cudaSuccess) return e;
    if (pass_ev && (e = cudaEventRecord(pass_ev[1], st)) != cudaSuccess) return e;
    return launch_pdl(k_f4_p3<T, F1, F2, HS>, dim3(nmb, F2 / F4W), sm1, st, c, mode, discrete, gate);
}

template <typename T, bool HS>
static cudaError_t f4_dispatch_hs(const CurveDev &c, int mode, int discrete, int gate, cudaStream_t st,
                                  cudaEvent_t *pass_ev)
{
    if (c.F1 == 64 && c.F2 == 64) return f4_run<T, 64, 64, HS>(c, mode, discrete, gate, st, pass_ev);
    if (c.F1 == 128 && c.F2 == 64) return f4_run<T, 128, 64, HS>(c, mode, discrete, gate, st, pass_ev);
    if (c.F1 == 128 && c.F2 == 128) return f4_run<T, 128, 128, HS>(c, mode, discrete, gate, st, pass_ev);
    if (c.F1 == 256 && c.F2 == 128) return f4_run<T, 256, 128, HS>(c, mode, discrete, gate, st, pass_ev);
    if (c.F1 == 256 && c.F2 == 256) return f4_run<T, 256, 256, HS>(c, mode, discrete, gate, st, pass_ev);
    return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t f4_dispatch(const CurveDev &c, int mode, int discrete, int gate, cudaStream_t st,
                               cudaEvent_t *pass_ev)
{
    return c.hs ? f4_dispatch_hs<T, true>(c, mode, discrete, gate, st, pass_ev)
                : f4_dispatch_hs<T, false>(c, mode, discrete, gate, st, pass_ev);
}

template <typename T, int F1, int F2, int MPC, bool STEP>
static cudaError_t f4c_run(const CurveDev &c, int mode, int discrete, int gate, cudaStream_t st)
{
    const size_t sm = F4C<T, F1, F2, MPC>::bytes(c.f4c);
    cudaError_t e = set_smem(k_f4c<T, F1, F2, MPC, STEP>, sm);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c.f4c, c.W / 2 / MPC);
    cfg.blockDim = dim3(F4_THREADS);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = c.f4c;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    e = cudaLaunchKernelEx(&cfg, k_f4c<T, F1, F2, MPC, STEP>, c, mode, discrete, gate);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename T, int MPC>
static cudaError_t f4c_dispatch(const CurveDev &c, int mode, int discrete, int gate, cudaStream_t st)
{
    if (mode == GM_STEP) {   // the fused step exists for the sizes of f4c_fused
        if (!f4c_fused(c.prec, c.W, c.F)) return cudaErrorInvalidValue;
        if (c.F1 == 64 && c.F2 == 64) return f4c_run<T, 64, 64, MPC, true>(c, mode, discrete, gate, st);
        if constexpr (sizeof(T) == 4) {
            if (c.F1 == 128 && c.F2 == 64) return f4c_run<T, 128, 64, MPC, true>(c, mode, discrete, gate, st);
            if (c.F1 == 128 && c.F2 == 128) return f4c_run<T, 128, 128, MPC, true>(c, mode, discrete, gate, st);
        }
        return cudaErrorInvalidValue;
    }
    if (c.F1 == 64 && c.F2 == 64) return f4c_run<T, 64, 64, MPC, false>(c, mode, discrete, gate, st);
    if (c.F1 == 128 && c.F2 == 64) return f4c_run<T, 128, 64, MPC, false>(c, mode, discrete, gate, st);
    if (c.F1 == 128 && c.F2 == 128) return f4c_run<T, 128, 128, MPC, false>(c, mode, discrete, gate, st);
    if (c.F1 == 256 && c.F2 == 128) return f4c_run<T, 256, 128, MPC, false>(c, mode, discrete, gate, st);
    if (c.F1 == 256 && c.F2 == 256) return f4c_run<T, 256, 256, MPC, false>(c, mode, discrete, gate, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_f4(const CurveDev &c, int mode, int discrete, int gate, cudaStream_t st, cudaEvent_t *pass_ev)
{
    if (mode == GM_STEP && !c.f4c) return cudaErrorInvalidValue;
    if ((mode == GM_UPDATE_F || mode == GM_STORE_P23) && !f4h_chained(c)) return cudaErrorInvalidValue;
    if (c.f4c) {
        if (!c.prec) return f4c_dispatch<double, 1>(c, mode, discrete, gate, st);
        return f4c_mpc(c.prec, c.W, c.F1, c.F2) == 2 ? f4c_dispatch<float, 2>(c, mode, discrete, gate, st)
                                          : f4c_dispatch<float, 1>(c, mode, discrete, gate, st);
    }
    return c.prec ? f4_dispatch<float>(c, mode, discrete, gate, st, pass_ev)
                  : f4_dispatch<double>(c, mode, discrete, gate, st, pass_ev);
}

// The one-CTA-per-mode form exists for the lengths a batched curve can have
// (from F = 1024 to 4096, and 8192 in FP32), each in the splits F = F1 F2 the
// batch autotuner chooses from.
template <typename T, typename Fn>
static cudaError_t f4b_dispatch(int F1, int F2, Fn &&fn)
{
    using I = std::integral_constant<int, 32>;
    using J = std::integral_constant<int, 64>;
    using K = std::integral_constant<int, 128>;
    if (F1 == 32 && F2 == 32) return fn(I(), I());
    if (F1 == 64 && F2 == 32) return fn(J(), I());
    if (F1 == 32 && F2 == 64) return fn(I(), J());
    if (F1 == 64 && F2 == 64) return fn(J(), J());
    if (F1 == 128 && F2 == 32) return fn(K(), I());
    if (F1 == 32 && F2 == 128) return fn(I(), K());
    if constexpr (sizeof(T) == 4)
        if (F1 == 128 && F2 == 64) return fn(K(), J());
    return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t f4b_run(const CurveDev &c, int mode, int discrete, int gate, cudaStream_t st)
{
    return f4b_dispatch<T>(c.F1, c.F2, [&](auto f1, auto f2) {
        constexpr int F1 = decltype(f1)::value, F2 = decltype(f2)::value;
        const size_t sm = F4B<T, F1, F2>::BYTES;
        cudaError_t e = set_smem(k_f4b<T, F1, F2>, sm);
        if (e != cudaSuccess) return e;
        return launch_pdl(k_f4b<T, F1, F2>, dim3(c.W / 2), sm, st, c, mode, discrete, gate);
    });
}

cudaError_t launch_f4b(const CurveDev &c, int mode, int discrete, int gate, cudaStream_t st)
{
    return c.prec ? f4b_run<float>(c, mode, discrete, gate, st) : f4b_run<double>(c, mode, discrete, gate, st);
}

template <typename T>
static cudaError_t f4b_batch_run(int F1, int F2, const CurveDev *cv, const int2 *items, int nitems, int mode,
                                 int discrete, int gate, cudaStream_t st)
{
    return f4b_dispatch<T>(F1, F2, [&](auto f1, auto f2) {
        constexpr int G1 = decltype(f1)::value, G2 = decltype(f2)::value;
        const size_t sm = F4B<T, G1, G2>::BYTES;
        cudaError_t e = set_smem(k_f4b_batch<T, G1, G2>, sm);
        if (e != cudaSuccess) return e;
        return launch_pdl(k_f4b_batch<T, G1, G2>, dim3(nitems), sm, st, cv, items, mode, discrete, gate);
    });
}

cudaError_t launch_f4b_batch(int prec, int F1, int F2, const CurveDev *cv, const int2 *items, int nitems, int mode,
                             int discrete, int gate, cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    return prec ? f4b_batch_run<float>(F1, F2, cv, items, nitems, mode, discrete, gate, st)
                : f4b_batch_run<double>(F1, F2, cv, items, nitems, mode, discrete, gate, st);
}

template <typename T, int F1, int F2>
static cudaError_t setup_run(const CurveDev &c, cudaStream_t st)
{
    const size_t smA = F4Smem<double, F1, F1>::BYTES, smB = F4Smem<double, F2, F2>::BYTES;
    cudaError_t e;
    if ((e = set_smem(k_f4_specA<F1, F2>, smA)) != cudaSuccess) return e;
    if ((e = set_smem(k_f4_specB<T, F1, F2>, smB)) != cudaSuccess) return e;
    k_f4_twiddles<<<(c.F + 255) / 256, 256, 0, st>>>(c);
    // one spectrum (the extended sequence), or the Toeplitz then the Hankel one
    for (int half = 0; half < (c.f4h ? 2 : 1); ++half) {
        k_f4_specA<F1, F2><<<F2 / F4W, F4_THREADS, smA, st>>>(c, c.f4h ? 1 + half : 0);
        k_f4_specB<T, F1, F2><<<F1 / F4W, F4_THREADS, smB, st>>>(c, half);
    }
    k_f4_steptw<T, F1, F2><<<(c.F + 255) / 256, 256, 0, st>>>(c);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t setup_dispatch(const CurveDev &c, cudaStream_t st)
{
    if (c.F1 == 32 && c.F2 == 32) return setup_run<T, 32, 32>(c, st);
    if (c.F1 == 64 && c.F2 == 32) return setup_run<T, 64, 32>(c, st);
    if (c.F1 == 32 && c.F2 == 64) return setup_run<T, 32, 64>(c, st);
    if (c.F1 == 64 && c.F2 == 64) return setup_run<T, 64, 64>(c, st);
    if (c.F1 == 128 && c.F2 == 32) return setup_run<T, 128, 32>(c, st);
    if (c.F1 == 32 && c.F2 == 128) return setup_run<T, 32, 128>(c, st);
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
