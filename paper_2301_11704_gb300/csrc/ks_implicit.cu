// ks_implicit.cu -- full-linear-implicit stepping of the descent (Sec. V.C.3).
//
// Semi-implicit forward Euler with every term of G that is linear in u taken
// at the new level.  On the interior rows that part is (lambda^2 D~^2 - a_j^2) u
// for spatial mode j, where D~ is the interior block (rows and columns 1..M) of
// the matrix of eq. rational_diff_matrix.  In increment form a step is
//     (I (1 + dtau a_j^2) - dtau lambda^2 D~^2) delta_j = dtau G_j,   u += delta.
//
// D~ anticommutes with the reflection s -> -s (interior index i <-> M-1-i: the
// theta grid is symmetric about pi/2 and d/ds changes sign under it), so D~^2
// commutes with it and is block diagonal in the orthonormal bases
//     E_a = (e_a + e_{M-1-a}) / sqrt2  (a < M/2),   E_{M/2} = e_{(M-1)/2}  (M odd),
//     O_a = (e_a - e_{M-1-a}) / sqrt2  (a < M/2),
// with blocks B_e = D_eo D_oe (ceil(M/2) square) and B_o = D_oe D_eo (floor(M/2)).
// Each block has real, simple, non-positive eigenvalues (the two blocks share
// them, which is why D~^2 as a whole has them in pairs).  With B_p = V_p diag(mu)
// V_p^-1 the step is, for every column of G at once (all modes, re and im),
//     delta = Q_p V_p diag(dtau / (1 + dtau (a_j^2 - lambda^2 mu))) V_p^-1 Q_p^T G.
//
// Set-up, once per curve and in FP64: the blocks D_eo, D_oe from the closed form
// of D~'s entries, B_e and B_o by products, their eigendecompositions by
// cuSOLVER's nonsymmetric eigensolver (the library is opened at run time), V^-1
// by an LU solve, then V and V^-1 rounded to the storage type.
// Per step (gated like the contractions): two tiled products per block on the
// CUDA cores, the first folding G into the bases on load and scaling by the
// implicit factor, the second unfolding into U's update, plus the step's
// bookkeeping in its last CTA.  The products are HBM/L2 bound at the curve
// sizes of interest (2 (ceil(M/2)^2 + floor(M/2)^2) matrix words per step).
#include "ks_internal.h"
#include "ks_device.cuh"

#include <cusolverDn.h>   // types and constants only; the functions are looked up at run time
#include <dlfcn.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

namespace ks {

size_t implicit_bytes(int ns, int prec)
{
    const size_t ne = (size_t)(ns - 1) / 2, no = (size_t)(ns - 2) / 2, b = prec ? 4 : 8;
    return 2 * (ne * ne + no * no) * b + (ne + no) * 8;
}

// ---------------------------------------------------------------------------
// Set-up
// ---------------------------------------------------------------------------

// Interior D~[i][k] = D_t[i+1][k+1].  With the product-to-sum identity
// cos(m k pi/P) sin(k j pi/P) = [sin(k (j+m) pi/P) + sin(k (j-m) pi/P)] / 2, the
// sum of eq. rational_diff_matrix becomes two sums T(q) = sum_{k=1}^{M} k sin(k q pi/P)
// (its k = 0 and k = P terms vanish; c-bar is 1 on interior columns), and
// sum_{k=1}^{P-1} k sin(k x) at x = q pi/P sums to -(P/2) (-1)^q cot(x/2) for
// q != 0 (mod 2P), 0 otherwise, so
//     D_t[j][m] = sin^2(j pi/P) / (S P) * (T(j + m) + T(j - m)).
__device__ __forceinline__ double imp_T(long q, int P)
{
    long r = q % (2L * P);
    if (r < 0) r += 2L * P;
    if (r == 0) return 0.0;
    double sn, cs;
    sincospi((double)r / (2.0 * P), &sn, &cs);
    return -(0.5 * P) * ((r & 1) ? -1.0 : 1.0) * cs / sn;
}

__device__ __forceinline__ double imp_d(int i, int k, int P, double S)
{
    const int j = i + 1, m = k + 1;
    const double sj = sinpi((double)j / P);
    return sj * sj / (S * P) * (imp_T(j + m, P) + imp_T(j - m, P));
}

// D_oe [no][ne] and D_eo [ne][no], row-major, FP64.
__global__ void k_imp_blocks(int M, double S, double *Doe, double *Deo)
{
    const int P = M + 1, h = M / 2, ne = M - h, no = h;
    const double r2 = 0.70710678118654752440;
    const long n1 = (long)no * ne;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < 2 * n1; e += (long)gridDim.x * blockDim.x) {
        if (e < n1) {   // D_oe[a][b] = O_a^T D~ E_b
            const int a = (int)(e / ne), b = (int)(e % ne), ab = M - 1 - a, bb = M - 1 - b;
            Doe[e] = (b < h) ? 0.5 * (imp_d(a, b, P, S) + imp_d(a, bb, P, S) - imp_d(ab, b, P, S) - imp_d(ab, bb, P, S))
                             : r2 * (imp_d(a, h, P, S) - imp_d(ab, h, P, S));
        } else {        // D_eo[a][b] = E_a^T D~ O_b
            const long f = e - n1;
            const int a = (int)(f / no), b = (int)(f % no), ab = M - 1 - a, bb = M - 1 - b;
            Deo[f] = (a < h) ? 0.5 * (imp_d(a, b, P, S) - imp_d(a, bb, P, S) + imp_d(ab, b, P, S) - imp_d(ab, bb, P, S))
                             : r2 * (imp_d(h, b, P, S) - imp_d(h, bb, P, S));
        }
    }
}

// C (m x n, column-major, ldc = m) = A (m x k, row-major) B (k x n, row-major), FP64.
__global__ void k_imp_gemm64(int m, int n, int k, const double *A, const double *B, double *C)
{
    __shared__ double As[16][17], Bs[16][17];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
    double acc = 0.0;
    for (int k0 = 0; k0 < k; k0 += 16) {
        As[ty][tx] = (row < m && k0 + tx < k) ? A[(size_t)row * k + k0 + tx] : 0.0;
        Bs[ty][tx] = (k0 + ty < k && col < n) ? B[(size_t)(k0 + ty) * n + col] : 0.0;
        __syncthreads();
#pragma unroll
        for (int t = 0; t < 16; ++t) acc += As[ty][t] * Bs[t][tx];
        __syncthreads();
    }
    if (row < m && col < n) C[(size_t)col * m + row] = acc;
}

__global__ void k_imp_identity(int n, double *X)
{
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)n * n; e += (long)gridDim.x * blockDim.x)
        X[e] = (e % n == e / n) ? 1.0 : 0.0;
}

// Row-major storage-type copy of a column-major n x n FP64 matrix.
template <typename T>
__global__ void k_imp_store(int n, const double *Xcm, T *out)
{
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)n * n; e += (long)gridDim.x * blockDim.x) {
        const long r = e / n, c = e % n;
        out[e] = (T)Xcm[c * n + r];
    }
}

// cuSOLVER, opened on first use.
struct Solver {
    bool ok = false;
    char why[256] = {0};
    cusolverStatus_t (*create)(cusolverDnHandle_t *);
    cusolverStatus_t (*destroy)(cusolverDnHandle_t);
    cusolverStatus_t (*set_stream)(cusolverDnHandle_t, cudaStream_t);
    cusolverStatus_t (*create_params)(cusolverDnParams_t *);
    cusolverStatus_t (*destroy_params)(cusolverDnParams_t);
    cusolverStatus_t (*geev_size)(cusolverDnHandle_t, cusolverDnParams_t, cusolverEigMode_t, cusolverEigMode_t, int64_t,
                                  cudaDataType, const void *, int64_t, cudaDataType, const void *, cudaDataType,
                                  const void *, int64_t, cudaDataType, const void *, int64_t, cudaDataType, size_t *,
                                  size_t *);
    cusolverStatus_t (*geev)(cusolverDnHandle_t, cusolverDnParams_t, cusolverEigMode_t, cusolverEigMode_t, int64_t,
                             cudaDataType, void *, int64_t, cudaDataType, void *, cudaDataType, void *, int64_t,
                             cudaDataType, void *, int64_t, cudaDataType, void *, size_t, void *, size_t, int *);
    cusolverStatus_t (*getrf_size)(cusolverDnHandle_t, cusolverDnParams_t, int64_t, int64_t, cudaDataType, const void *,
                                   int64_t, cudaDataType, size_t *, size_t *);
    cusolverStatus_t (*getrf)(cusolverDnHandle_t, cusolverDnParams_t, int64_t, int64_t, cudaDataType, void *, int64_t,
                              int64_t *, cudaDataType, void *, size_t, void *, size_t, int *);
    cusolverStatus_t (*getrs)(cusolverDnHandle_t, cusolverDnParams_t, cublasOperation_t, int64_t, int64_t, cudaDataType,
                              const void *, int64_t, const int64_t *, cudaDataType, void *, int64_t, int *);
};

static const Solver &solver()
{
    static Solver s;
    static std::once_flag once;
    std::call_once(once, [] {
        const char *names[] = {"libcusolver.so.12", "libcusolver.so", "/usr/local/cuda/lib64/libcusolver.so.12"};
        void *h = nullptr;
        for (const char *n : names)
            if ((h = dlopen(n, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
        if (!h) {
            snprintf(s.why, sizeof(s.why), "cuSOLVER not found (%s)", dlerror());
            return;
        }
        bool all = true;
        auto get = [&](auto &fn, const char *name) {
            fn = reinterpret_cast<std::remove_reference_t<decltype(fn)>>(dlsym(h, name));
            if (!fn) {
                all = false;
                snprintf(s.why, sizeof(s.why), "cuSOLVER lacks %s", name);
            }
        };
        get(s.create, "cusolverDnCreate");
        get(s.destroy, "cusolverDnDestroy");
        get(s.set_stream, "cusolverDnSetStream");
        get(s.create_params, "cusolverDnCreateParams");
        get(s.destroy_params, "cusolverDnDestroyParams");
        get(s.geev_size, "cusolverDnXgeev_bufferSize");
        get(s.geev, "cusolverDnXgeev");
        get(s.getrf_size, "cusolverDnXgetrf_bufferSize");
        get(s.getrf, "cusolverDnXgetrf");
        get(s.getrs, "cusolverDnXgetrs");
        s.ok = all;
    });
    return s;
}

// Device buffers of the set-up (stream-ordered, so set-ups on several streams
// do not synchronise the device), released on every path out.
struct DevBufs {
    cudaStream_t st;
    std::vector<void *> p;
    explicit DevBufs(cudaStream_t s) : st(s) {}
    ~DevBufs()
    {
        for (void *q : p) cudaFreeAsync(q, st);
    }
    template <typename T>
    T *get(size_t count)
    {
        void *q = nullptr;
        if (cudaMallocAsync(&q, count * sizeof(T) + 16, st) != cudaSuccess) return nullptr;
        p.push_back(q);
        return (T *)q;
    }
};

struct SolverHandle {
    const Solver &s;
    cusolverDnHandle_t h = nullptr;
    cusolverDnParams_t prm = nullptr;
    explicit SolverHandle(const Solver &sv) : s(sv) {}
    ~SolverHandle()
    {
        if (prm) s.destroy_params(prm);
        if (h) s.destroy(h);
    }
};

// Eigendecomposition of the n x n column-major FP64 block B (destroyed):
// eigenvalues into mu_dev, V and V^-1 (storage type, row-major) into v_out, vi_out.
template <typename T>
static ks_status eig_block(SolverHandle &sh, cudaStream_t st, int n, double *B, double *mu_dev, T *v_out, T *vi_out)
{
    if (n == 0) return KS_OK;
    const Solver &s = sh.s;
    DevBufs mem(st);
    double *VR = mem.get<double>((size_t)n * n), *W = mem.get<double>(2 * (size_t)n);
    double *X = mem.get<double>((size_t)n * n);
    int64_t *piv = mem.get<int64_t>(n);
    int *info = mem.get<int>(1);
    if (!VR || !W || !X || !piv || !info) return report_error(KS_ECUDA, "implicit set-up: device memory for n = %d", n);
    size_t wd = 0, wh = 0;
    if (s.geev_size(sh.h, sh.prm, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR, n, CUDA_R_64F, B, n, CUDA_C_64F,
                    W, CUDA_R_64F, nullptr, n, CUDA_R_64F, VR, n, CUDA_R_64F, &wd, &wh) != CUSOLVER_STATUS_SUCCESS)
        return report_error(KS_ECUDA, "implicit set-up: eigensolver work size");
    char *wdev = mem.get<char>(wd + 1);
    std::vector<char> whost(wh + 1);
    if (!wdev) return report_error(KS_ECUDA, "implicit set-up: eigensolver work memory");
    if (s.geev(sh.h, sh.prm, CUSOLVER_EIG_MODE_NOVECTOR, CUSOLVER_EIG_MODE_VECTOR, n, CUDA_R_64F, B, n, CUDA_C_64F, W,
               CUDA_R_64F, nullptr, n, CUDA_R_64F, VR, n, CUDA_R_64F, wdev, wd, whost.data(), wh, info) !=
        CUSOLVER_STATUS_SUCCESS)
        return report_error(KS_ECUDA, "implicit set-up: eigensolver failed");
    int hinfo = 0;
    std::vector<double> w(2 * (size_t)n);
    if (cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(w.data(), W, w.size() * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return report_error(KS_ECUDA, "implicit set-up: reading the eigenvalues");
    if (hinfo != 0) return report_error(KS_ECUDA, "implicit set-up: eigensolver info %d", hinfo);
    double scale = 0.0;
    for (int i = 0; i < n; ++i) scale = std::fmax(scale, std::fabs(w[2 * i]));
    std::vector<double> mu(n);
    for (int i = 0; i < n; ++i) {
        if (std::fabs(w[2 * i + 1]) > 1e-9 * scale || w[2 * i] > 1e-9 * scale)
            return report_error(KS_EINVAL, "implicit set-up: eigenvalue %g%+gi of D_t^2 is not real and <= 0", w[2 * i],
                                w[2 * i + 1]);
        mu[i] = std::fmin(w[2 * i], 0.0);
    }
    if (cudaMemcpyAsync(mu_dev, mu.data(), n * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return report_error(KS_ECUDA, "implicit set-up: storing the eigenvalues");
    // V^-1: LU of a copy of V (into B, free after the eigensolver), solve against I
    if (cudaMemcpyAsync(B, VR, (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return report_error(KS_ECUDA, "implicit set-up: copy");
    size_t ld = 0, lh = 0;
    if (s.getrf_size(sh.h, sh.prm, n, n, CUDA_R_64F, B, n, CUDA_R_64F, &ld, &lh) != CUSOLVER_STATUS_SUCCESS)
        return report_error(KS_ECUDA, "implicit set-up: LU work size");
    char *ldev = mem.get<char>(ld + 1);
    std::vector<char> lhost(lh + 1);
    if (!ldev) return report_error(KS_ECUDA, "implicit set-up: LU work memory");
    k_imp_identity<<<256, 256, 0, st>>>(n, X);
    if (s.getrf(sh.h, sh.prm, n, n, CUDA_R_64F, B, n, piv, CUDA_R_64F, ldev, ld, lhost.data(), lh, info) !=
            CUSOLVER_STATUS_SUCCESS ||
        s.getrs(sh.h, sh.prm, CUBLAS_OP_N, n, n, CUDA_R_64F, B, n, piv, CUDA_R_64F, X, n, info) !=
            CUSOLVER_STATUS_SUCCESS)
        return report_error(KS_ECUDA, "implicit set-up: inverse of the eigenvectors");
    if (cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return report_error(KS_ECUDA, "implicit set-up: LU status");
    if (hinfo != 0) return report_error(KS_EINVAL, "implicit set-up: eigenvector matrix is singular (info %d)", hinfo);
    k_imp_store<T><<<512, 256, 0, st>>>(n, VR, v_out);
    k_imp_store<T><<<512, 256, 0, st>>>(n, X, vi_out);
    if (cudaStreamSynchronize(st) != cudaSuccess) return report_error(KS_ECUDA, "implicit set-up: storing the bases");
    return KS_OK;
}

template <typename T>
static ks_status setup_implicit_t(const CurveDev &c, cudaStream_t st)
{
    const Solver &s = solver();
    if (!s.ok) return report_error(KS_ECUDA, "implicit stepping needs cuSOLVER: %s", s.why);
    const int M = c.ns - 2, ne = c.ine, no = c.ino;
    DevBufs mem(st);
    double *Doe = mem.get<double>((size_t)no * ne + 1), *Deo = mem.get<double>((size_t)ne * no + 1);
    double *B = mem.get<double>((size_t)ne * ne + 1);
    if (!Doe || !Deo || !B) return report_error(KS_ECUDA, "implicit set-up: device memory");
    SolverHandle sh(s);
    if (s.create(&sh.h) != CUSOLVER_STATUS_SUCCESS || s.create_params(&sh.prm) != CUSOLVER_STATUS_SUCCESS ||
        s.set_stream(sh.h, st) != CUSOLVER_STATUS_SUCCESS)
        return report_error(KS_ECUDA, "implicit set-up: cuSOLVER handle");
    k_imp_blocks<<<1024, 256, 0, st>>>(M, c.S, Doe, Deo);
    T *V = (T *)c.iv, *Vi = (T *)c.ivi;
    // even block B_e = D_eo D_oe
    k_imp_gemm64<<<dim3((ne + 15) / 16, (ne + 15) / 16), 256, 0, st>>>(ne, ne, no, Deo, Doe, B);
    if (cudaGetLastError() != cudaSuccess) return report_error(KS_ECUDA, "implicit set-up: block products");
    ks_status r = eig_block<T>(sh, st, ne, B, c.imu, V, Vi);
    if (r != KS_OK) return r;
    // odd block B_o = D_oe D_eo
    if (no > 0) {
        k_imp_gemm64<<<dim3((no + 15) / 16, (no + 15) / 16), 256, 0, st>>>(no, no, ne, Doe, Deo, B);
        if (cudaGetLastError() != cudaSuccess) return report_error(KS_ECUDA, "implicit set-up: block products");
        r = eig_block<T>(sh, st, no, B, c.imu + ne, V + (size_t)ne * ne, Vi + (size_t)ne * ne);
    }
    if (r == KS_OK && c.ivtc && launch_setup_implicit_tc(c, st) != cudaSuccess)
        r = report_error(KS_ECUDA, "implicit set-up: tensor-core operands");
    if (r == KS_OK && cudaStreamSynchronize(st) != cudaSuccess) r = report_error(KS_ECUDA, "implicit set-up");
    return r;
}

ks_status setup_implicit(const CurveDev &c, cudaStream_t st)
{
    if (!c.impl) return KS_OK;
    return c.prec ? setup_implicit_t<float>(c, st) : setup_implicit_t<double>(c, st);
}

// ---------------------------------------------------------------------------
// Per step
// ---------------------------------------------------------------------------
// Up to four launches, all gated like the contractions:
//   k_imp_fwd:    partial products over K chunks ("splits", so that the grid
//                 fills the GPU) of V_p^-1 (Q_p^T G), folding G into the
//                 bases on load, each partial scaled by the implicit factor
//                 dtau / (1 + dtau (a_j^2 - lambda^2 mu)) (linear, so the sum
//                 of the scaled partials is the scaled sum);
//   k_imp_sum:    Y_p = the sum of those partials in split order (when split);
//   k_imp_back:   partial products of V_p with Y_p;
//   k_imp_finish: the sum of the back partials in split order, unfolded into
//                 U's update, and the step's bookkeeping in the last CTA.
// The products are register-tiled on the CUDA cores: 128 x 64 outputs per CTA,
// 8 x 4 per thread, K in steps of 16 through shared memory.
constexpr int IM_BM = 128, IM_BN = 64, IM_BK = 16, IM_THREADS = 256, IM_TM = 8, IM_TN = 4;

template <typename T>
struct ImSmem {
    __align__(16) T As[IM_BK][IM_BM];
    __align__(16) T Bs[IM_BK][IM_BN];
};

// acc[i][l] += sum_{k in [kb, ke)} A[r0 + 8 ty + i][k] B(k, c0 + 4 tx + l);
// A row-major (nrows x lda), B(k, col) from `loadb` (called for k < ke, col < ncols).
template <typename T, typename LoadB>
__device__ __forceinline__ void im_tile(ImSmem<T> &sm, const T *A, int nrows, int lda, int r0, int kb, int ke, int c0,
                                        int ncols, LoadB loadb, T (&acc)[IM_TM][IM_TN])
{
    constexpr int AL = IM_BM * IM_BK / IM_THREADS, BL = IM_BK * IM_BN / IM_THREADS;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int ar = tid >> 1, ak = (tid & 1) * AL;   // A: a row and 8 consecutive k per thread
    T ra[AL], rb[BL];
    auto fetch = [&](int k0) {
        const bool rok = r0 + ar < nrows;
        const T *arow = A + (size_t)(r0 + ar) * lda;
#pragma unroll
        for (int q = 0; q < AL; ++q) {
            const int k = k0 + ak + q;
            ra[q] = (rok && k < ke) ? arow[k] : T(0);
        }
#pragma unroll
        for (int q = 0; q < BL; ++q) {
            const int e = tid + q * IM_THREADS, k = k0 + e / IM_BN, col = c0 + e % IM_BN;
            rb[q] = (k < ke && col < ncols) ? loadb(k, col) : T(0);
        }
    };
    if (kb >= ke) return;
    fetch(kb);
    for (int k0 = kb; k0 < ke; k0 += IM_BK) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < AL; ++q) sm.As[ak + q][ar] = ra[q];
#pragma unroll
        for (int q = 0; q < BL; ++q) {
            const int e = tid + q * IM_THREADS;
            sm.Bs[e / IM_BN][e % IM_BN] = rb[q];
        }
        __syncthreads();
        if (k0 + IM_BK < ke) fetch(k0 + IM_BK);
#pragma unroll
        for (int kk = 0; kk < IM_BK; ++kk) {
            T a[IM_TM], b[IM_TN];
#pragma unroll
            for (int i = 0; i < IM_TM; ++i) a[i] = sm.As[kk][IM_TM * ty + i];
#pragma unroll
            for (int l = 0; l < IM_TN; ++l) b[l] = sm.Bs[kk][IM_TN * tx + l];
#pragma unroll
            for (int i = 0; i < IM_TM; ++i)
#pragma unroll
                for (int l = 0; l < IM_TN; ++l) acc[i][l] += a[i] * b[l];
        }
    }
}

// The K chunk of split s of a length-n contraction over `splits` chunks.
__device__ __forceinline__ void im_chunk(int n, int splits, int s, int &kb, int &ke)
{
    int kc = (n + splits - 1) / splits;
    kc = (kc + IM_BK - 1) / IM_BK * IM_BK;
    kb = min(n, s * kc);
    ke = min(n, kb + kc);
}

// Pf[s] rows [0, ne) even, [ne, M) odd: the scaled partial of split s.
// Block (bx, by, bz): column tile, row tile, parity * splits + split.
template <typename T>
__device__ __forceinline__ void imp_fwd_body(ImSmem<T> &sm, const CurveDev &c, int bx, int by, int bz, int splits)
{
    DevScalars *sc = c.sc;
    const int p = bz / splits, sp = bz % splits;
    const int M = c.ns - 2, h = M / 2, N = c.nx, ne = c.ine, np = p ? c.ino : ne;
    const int r0 = by * IM_BM, c0 = bx * IM_BN;
    if (r0 >= np) return;
    int kb, ke;
    im_chunk(np, splits, sp, kb, ke);
    const T *G = (const T *)c.G;
    const T r2 = T(0.70710678118654752440);
    const T *A = (const T *)c.ivi + (p ? (size_t)ne * ne : 0);
    T acc[IM_TM][IM_TN];
#pragma unroll
    for (int i = 0; i < IM_TM; ++i)
#pragma unroll
        for (int l = 0; l < IM_TN; ++l) acc[i][l] = T(0);
    if (p == 0)
        im_tile<T>(sm, A, np, np, r0, kb, ke, c0, N, [&](int k, int col) -> T {
            return k < h ? r2 * (G[(size_t)(1 + k) * N + col] + G[(size_t)(M - k) * N + col]) : G[(size_t)(1 + h) * N + col];
        }, acc);
    else
        im_tile<T>(sm, A, np, np, r0, kb, ke, c0, N, [&](int k, int col) -> T {
            return r2 * (G[(size_t)(1 + k) * N + col] - G[(size_t)(M - k) * N + col]);
        }, acc);
    const T lam = (T)sc->lambda, dtau = (T)sc->dtau, tl = T(2.0 * M_PI / c.L);
    const double *mu = c.imu + (p ? ne : 0);
    T *out = (T *)c.isc + (size_t)sp * M * N + (p ? (size_t)ne * N : 0);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int i = 0; i < IM_TM; ++i) {
        const int r = r0 + IM_TM * ty + i;
        if (r >= np) continue;
        const T lm = lam * lam * (T)mu[r];
#pragma unroll
        for (int l = 0; l < IM_TN; ++l) {
            const int col = c0 + IM_TN * tx + l;
            if (col >= N) continue;
            const T kw = tl * (T)(col >> 1), a = kw * kw * kw * kw - kw * kw;
            out[(size_t)r * N + col] = dtau / (T(1) + dtau * (a * a - lm)) * acc[i][l];
        }
    }
}

// Pb[s] (after the c.isplits forward partials) rows [0, ne) even, [ne, M) odd:
// partial of split s of V_p Y_p.
template <typename T>
__device__ __forceinline__ void imp_back_body(ImSmem<T> &sm, const CurveDev &c, int bx, int by, int bz, int splits_f,
                                              int splits)
{
    const int p = bz / splits, sp = bz % splits;
    const int M = c.ns - 2, N = c.nx, ne = c.ine, np = p ? c.ino : ne;
    const int r0 = by * IM_BM, c0 = bx * IM_BN;
    if (r0 >= np) return;
    int kb, ke;
    im_chunk(np, splits, sp, kb, ke);
    const size_t off = p ? (size_t)ne * N : 0, stride = (size_t)M * N;
    const T *Pf = (const T *)c.isc;
    const T *A = (const T *)c.iv + (p ? (size_t)ne * ne : 0);
    T acc[IM_TM][IM_TN];
#pragma unroll
    for (int i = 0; i < IM_TM; ++i)
#pragma unroll
        for (int l = 0; l < IM_TN; ++l) acc[i][l] = T(0);
    im_tile<T>(sm, A, np, np, r0, kb, ke, c0, N, [&](int k, int col) -> T {
        const T *y = Pf + off + (size_t)k * N + col;
        T t = y[0];
        for (int q = 1; q < splits_f; ++q) t += y[q * stride];
        return t;
    }, acc);
    T *out = (T *)c.isc + (size_t)(c.isplits + sp) * stride + off;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int i = 0; i < IM_TM; ++i) {
        const int r = r0 + IM_TM * ty + i;
        if (r >= np) continue;
#pragma unroll
        for (int l = 0; l < IM_TN; ++l) {
            const int col = c0 + IM_TN * tx + l;
            if (col < N) out[(size_t)r * N + col] = acc[i][l];
        }
    }
}

// U += Q (delta_e, delta_o), delta_p the split sums of the back partials; the
// step's bookkeeping in the last of the curve's nbx finishing CTAs.
template <typename T>
__device__ __forceinline__ void imp_finish_body(const CurveDev &c, int bx, int nbx, int splits, int &am_last)
{
    DevScalars *sc = c.sc;
    const int M = c.ns - 2, h = M / 2, N = c.nx, ne = c.ine;
    const size_t stride = (size_t)M * N;
    const T *Pb = (const T *)c.isc + (size_t)c.isplits * stride;
    T *U = (T *)c.U;
    const T r2 = T(0.70710678118654752440);
    const long total = (long)ne * N;
    for (long e = bx * (long)IM_THREADS + threadIdx.x; e < total; e += (long)nbx * IM_THREADS) {
        const int a = (int)(e / N), col = (int)(e % N);
        if (!col_allowed(col, c.sym)) continue;
        T de = T(0), dd = T(0);
        for (int q = 0; q < splits; ++q) {
            de += Pb[q * stride + (size_t)a * N + col];
            if (a < h) dd += Pb[q * stride + (size_t)(ne + a) * N + col];
        }
        if (a < h) {
            U[(size_t)(1 + a) * N + col] += r2 * (de + dd);
            U[(size_t)(M - a) * N + col] += r2 * (de - dd);
        } else {
            U[(size_t)(1 + h) * N + col] += de;
        }
    }
    if (!last_cta_arrive(&sc->cnt_gemm, (unsigned)nbx, am_last)) return;
    if (threadIdx.x == 0) {
        sc->step += 1;
        sc->tau += sc->dtau;
        sc->lambda = sc->lambda_next;
        sc->cnt_gemm = 0;
    }
}

// Y = the split sum of the forward partials, in split order, into split 0's slot
// (the back product then reads one value per element instead of `splits`).
template <typename T>
__global__ void __launch_bounds__(IM_THREADS) k_imp_sum(CurveDev c, int splits, int gate)
{
    pdl_wait();
    if (gate && !c.sc->active) return;
    const size_t stride = (size_t)(c.ns - 2) * c.nx;
    T *Pf = (T *)c.isc;
    for (size_t e = blockIdx.x * (size_t)IM_THREADS + threadIdx.x; e < stride; e += (size_t)gridDim.x * IM_THREADS) {
        T t = Pf[e];
        for (int q = 1; q < splits; ++q) t += Pf[q * stride + e];
        Pf[e] = t;
    }
}

template <typename T>
__global__ void __launch_bounds__(IM_THREADS) k_imp_fwd(CurveDev c, int splits, int gate)
{
    __shared__ ImSmem<T> sm;
    pdl_wait();
    if (gate && !c.sc->active) return;
    imp_fwd_body<T>(sm, c, blockIdx.x, blockIdx.y, blockIdx.z, splits);
}

template <typename T>
__global__ void __launch_bounds__(IM_THREADS) k_imp_back(CurveDev c, int splits, int gate)
{
    __shared__ ImSmem<T> sm;
    pdl_wait();
    if (gate && !c.sc->active) return;
    imp_back_body<T>(sm, c, blockIdx.x, blockIdx.y, blockIdx.z, 1, splits);   // forward partials summed
}

template <typename T>
__global__ void __launch_bounds__(IM_THREADS) k_imp_finish(CurveDev c, int splits, int gate)
{
    __shared__ int am_last;
    pdl_wait();
    if (gate && !c.sc->active) return;
    imp_finish_body<T>(c, blockIdx.x, gridDim.x, splits, am_last);
}

// Batched curves (one K chunk each): items (curve, bx, by, parity) of the two
// products, (curve, bx, nbx, 0) of the finishing pass.
template <typename T>
__global__ void __launch_bounds__(IM_THREADS) k_imp_fwd_batch(const CurveDev *cv, const int4 *items)
{
    __shared__ ImSmem<T> sm;
    pdl_wait();
    const int4 it = items[blockIdx.x];
    const CurveDev &c = cv[it.x];
    if (!c.sc->active) return;
    imp_fwd_body<T>(sm, c, it.y, it.z, it.w, 1);
}

template <typename T>
__global__ void __launch_bounds__(IM_THREADS) k_imp_back_batch(const CurveDev *cv, const int4 *items)
{
    __shared__ ImSmem<T> sm;
    pdl_wait();
    const int4 it = items[blockIdx.x];
    const CurveDev &c = cv[it.x];
    if (!c.sc->active) return;
    imp_back_body<T>(sm, c, it.y, it.z, it.w, 1, 1);
}

template <typename T>
__global__ void __launch_bounds__(IM_THREADS) k_imp_finish_batch(const CurveDev *cv, const int4 *items)
{
    __shared__ int am_last;
    pdl_wait();
    const int4 it = items[blockIdx.x];
    const CurveDev &c = cv[it.x];
    if (!c.sc->active) return;
    imp_finish_body<T>(c, it.y, it.z, 1, am_last);
}

template <typename K, typename... Args>
static cudaError_t imp_launch(K kern, dim3 grid, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(IM_THREADS);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args...);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// K splits that bring the product's grid to about two CTAs per SM.
static int imp_splits(const CurveDev &c)
{
    const int tiles = ((c.nx + IM_BN - 1) / IM_BN) * ((c.ine + IM_BM - 1) / IM_BM) * 2;
    int s = (2 * 152 + tiles - 1) / tiles;
    const int smax = std::max(1, c.ino / (4 * IM_BK));   // chunks of at least 64
    return std::max(1, std::min(std::min(s, c.isplits), smax));
}

size_t implicit_scratch_bytes(int ns, int nx, int prec, int splits)
{
    return 2 * (size_t)splits * (size_t)(ns - 2) * nx * (prec ? 4 : 8);
}

void implicit_batch_items(const CurveDev &c, int curve, std::vector<int4> &prod, std::vector<int4> &fin)
{
    const int gx = (c.nx + IM_BN - 1) / IM_BN, gy = (c.ine + IM_BM - 1) / IM_BM;
    for (int p = 0; p < 2; ++p)
        for (int by = 0; by < gy; ++by) {
            if (by * IM_BM >= (p ? c.ino : c.ine)) continue;
            for (int bx = 0; bx < gx; ++bx) prod.push_back(make_int4(curve, bx, by, p));
        }
    const long total = (long)c.ine * c.nx;
    const int nbx = (int)std::min<long>(8, (total + IM_THREADS - 1) / IM_THREADS);
    for (int bx = 0; bx < nbx; ++bx) fin.push_back(make_int4(curve, bx, nbx, 0));
}

// The tensor-core products (FP32 storage, N >= 32): K split so that the grid of
// 128-row tiles of both parities holds about two CTAs per SM.
static cudaError_t implicit_tc_run(const CurveDev &c, int gate, cudaStream_t st)
{
    const int tiles = ((c.ine + 127) / 128) * 2, nk = (c.ino + 31) / 32;
    const int sp = std::max(1, std::min(std::min((2 * 152 + tiles - 1) / tiles, c.isplits), std::max(1, nk / 2)));
    cudaError_t e = launch_implicit_tc(c, sp, gate, st, 0);
    const long total = (long)c.ine * c.nx;
    if (e == cudaSuccess && sp > 1)
        e = imp_launch(k_imp_sum<float>, dim3((int)std::min<long>(4 * 152, (2 * total + IM_THREADS - 1) / IM_THREADS)), st,
                       c, sp, gate);
    if (e == cudaSuccess) e = launch_implicit_tc(c, sp, gate, st, 1);
    if (e != cudaSuccess) return e;
    const int gf = (int)std::min<long>(4 * 152, (total + IM_THREADS - 1) / IM_THREADS);
    return imp_launch(k_imp_finish<float>, dim3(gf), st, c, sp, gate);
}

template <typename T>
static cudaError_t implicit_t(const CurveDev &c, int gate, cudaStream_t st)
{
    if (sizeof(T) == 4 && c.ivtc) return implicit_tc_run(c, gate, st);
    const int sp = imp_splits(c);
    const int gx = (c.nx + IM_BN - 1) / IM_BN, gy = (c.ine + IM_BM - 1) / IM_BM;
    cudaError_t e = imp_launch(k_imp_fwd<T>, dim3(gx, gy, 2 * sp), st, c, sp, gate);
    const long total = (long)c.ine * c.nx;
    if (e == cudaSuccess && sp > 1)
        e = imp_launch(k_imp_sum<T>, dim3((int)std::min<long>(4 * 152, (2 * total + IM_THREADS - 1) / IM_THREADS)), st,
                       c, sp, gate);
    if (e == cudaSuccess) e = imp_launch(k_imp_back<T>, dim3(gx, gy, 2 * sp), st, c, sp, gate);
    if (e != cudaSuccess) return e;
    const int gf = (int)std::min<long>(4 * 152, (total + IM_THREADS - 1) / IM_THREADS);
    return imp_launch(k_imp_finish<T>, dim3(gf), st, c, sp, gate);
}

cudaError_t launch_implicit_update(const CurveDev &c, int gate, cudaStream_t st)
{
    if (!c.impl) return cudaErrorInvalidValue;
    return c.prec ? implicit_t<float>(c, gate, st) : implicit_t<double>(c, gate, st);
}

cudaError_t launch_implicit_batch(int prec, const CurveDev *cv, const int4 *prod, int nprod, const int4 *fin, int nfin,
                                  cudaStream_t st)
{
    if (nprod <= 0) return cudaSuccess;
    cudaError_t e;
    if (prec) {
        e = imp_launch(k_imp_fwd_batch<float>, dim3(nprod), st, cv, prod);
        if (e == cudaSuccess) e = imp_launch(k_imp_back_batch<float>, dim3(nprod), st, cv, prod);
        if (e == cudaSuccess) e = imp_launch(k_imp_finish_batch<float>, dim3(nfin), st, cv, fin);
    } else {
        e = imp_launch(k_imp_fwd_batch<double>, dim3(nprod), st, cv, prod);
        if (e == cudaSuccess) e = imp_launch(k_imp_back_batch<double>, dim3(nprod), st, cv, prod);
        if (e == cudaSuccess) e = imp_launch(k_imp_finish_batch<double>, dim3(nfin), st, cv, fin);
    }
    return e;
}

}  // namespace ks
