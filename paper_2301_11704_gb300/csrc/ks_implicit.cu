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

// Device buffers of the set-up, released on every path out.
struct DevBufs {
    std::vector<void *> p;
    ~DevBufs()
    {
        for (void *q : p) cudaFree(q);
    }
    template <typename T>
    T *get(size_t count)
    {
        void *q = nullptr;
        if (cudaMalloc(&q, count * sizeof(T) + 16) != cudaSuccess) return nullptr;
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
    DevBufs mem;
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
    DevBufs mem;
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
constexpr int IM_BM = 64, IM_BK = 16, IM_THREADS = 256;

template <typename T, int BN>
struct ImSmem {
    T As[IM_BM][IM_BK + 1];
    __align__(16) T Bs[IM_BK][BN];
};

// acc[i][l] += sum_k A[r0 + 4 ty + i][k] * B(k, c0 + TN tx + l) for k < kdim;
// A row-major with nrows rows and kdim columns, B(k, col) from `loadb`.
template <typename T, int BN, typename LoadB>
__device__ __forceinline__ void im_product(ImSmem<T, BN> &sm, const T *A, int nrows, int kdim, int r0, int c0, int ncols,
                                           LoadB loadb, T (&acc)[4][BN / 16])
{
    constexpr int TN = BN / 16, AL = IM_BM * IM_BK / IM_THREADS, BL = IM_BK * BN / IM_THREADS;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    T ra[AL], rb[BL];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int q = 0; q < AL; ++q) {
            const int e = tid + q * IM_THREADS, r = e / IM_BK, k = k0 + e % IM_BK;
            ra[q] = (r0 + r < nrows && k < kdim) ? A[(size_t)(r0 + r) * kdim + k] : T(0);
        }
#pragma unroll
        for (int q = 0; q < BL; ++q) {
            const int e = tid + q * IM_THREADS, k = k0 + e / BN, col = c0 + e % BN;
            rb[q] = (k < kdim && col < ncols) ? loadb(k, col) : T(0);
        }
    };
    fetch(0);
    for (int k0 = 0; k0 < kdim; k0 += IM_BK) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < AL; ++q) {
            const int e = tid + q * IM_THREADS;
            sm.As[e / IM_BK][e % IM_BK] = ra[q];
        }
#pragma unroll
        for (int q = 0; q < BL; ++q) {
            const int e = tid + q * IM_THREADS;
            sm.Bs[e / BN][e % BN] = rb[q];
        }
        __syncthreads();
        if (k0 + IM_BK < kdim) fetch(k0 + IM_BK);
#pragma unroll
        for (int kk = 0; kk < IM_BK; ++kk) {
            T a[4], b[TN];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = sm.As[4 * ty + i][kk];
#pragma unroll
            for (int l = 0; l < TN; ++l) b[l] = sm.Bs[kk][TN * tx + l];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int l = 0; l < TN; ++l) acc[i][l] += a[i] * b[l];
        }
    }
}

// Y_p = diag(dtau / (1 + dtau (a_j^2 - lambda^2 mu_p))) V_p^-1 Q_p^T G into the
// D_t u buffer (free between the update contraction and the next D_t u): rows
// [0, ne) even, [ne, M) odd.  blockIdx.z = parity.
template <typename T, int BN>
__global__ void __launch_bounds__(IM_THREADS) k_imp_fwd(CurveDev c, int gate)
{
    __shared__ ImSmem<T, BN> sm;
    pdl_wait();
    DevScalars *sc = c.sc;
    if (gate && !sc->active) return;
    const int p = blockIdx.z, M = c.ns - 2, h = M / 2, N = c.nx, ne = c.ine;
    const int np = p ? c.ino : ne;
    const int r0 = blockIdx.y * IM_BM, c0 = blockIdx.x * BN;
    if (r0 >= np) return;
    const T *G = (const T *)c.G;
    const T r2 = T(0.70710678118654752440);
    const T *A = (const T *)c.ivi + (p ? (size_t)ne * ne : 0);
    constexpr int TN = BN / 16;
    T acc[4][TN];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int l = 0; l < TN; ++l) acc[i][l] = T(0);
    if (p == 0)
        im_product<T, BN>(sm, A, np, np, r0, c0, N, [&](int k, int col) -> T {
            return k < h ? r2 * (G[(size_t)(1 + k) * N + col] + G[(size_t)(M - k) * N + col]) : G[(size_t)(1 + h) * N + col];
        }, acc);
    else
        im_product<T, BN>(sm, A, np, np, r0, c0, N, [&](int k, int col) -> T {
            return r2 * (G[(size_t)(1 + k) * N + col] - G[(size_t)(M - k) * N + col]);
        }, acc);
    const double lam = sc->lambda, dtau = sc->dtau;
    const double *mu = c.imu + (p ? ne : 0);
    T *Y = (T *)c.D + (p ? (size_t)ne * N : 0);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + 4 * ty + i;
        if (r >= np) continue;
        const double lm = lam * lam * mu[r];
#pragma unroll
        for (int l = 0; l < TN; ++l) {
            const int col = c0 + TN * tx + l;
            if (col >= N) continue;
            const double kw = 2.0 * M_PI * (double)(col >> 1) / c.L, a = kw * kw * kw * kw - kw * kw;
            Y[(size_t)r * N + col] = (T)(dtau / (1.0 + dtau * (a * a - lm)) * (double)acc[i][l]);
        }
    }
}

// U += Q (V_e Y_e, V_o Y_o), then the step's bookkeeping in the last CTA.
template <typename T, int BN>
__global__ void __launch_bounds__(IM_THREADS) k_imp_back(CurveDev c, int gate)
{
    __shared__ ImSmem<T, BN> sm;
    __shared__ int am_last;
    pdl_wait();
    DevScalars *sc = c.sc;
    if (gate && !sc->active) return;
    const int M = c.ns - 2, h = M / 2, N = c.nx, ne = c.ine, no = c.ino;
    const int r0 = blockIdx.y * IM_BM, c0 = blockIdx.x * BN;
    const T *Y = (const T *)c.D;
    const T *V = (const T *)c.iv;
    constexpr int TN = BN / 16;
    T ae[4][TN], ao[4][TN];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int l = 0; l < TN; ++l) ae[i][l] = ao[i][l] = T(0);
    im_product<T, BN>(sm, V, ne, ne, r0, c0, N, [&](int k, int col) -> T { return Y[(size_t)k * N + col]; }, ae);
    if (no > 0)
        im_product<T, BN>(sm, V + (size_t)ne * ne, no, no, r0, c0, N,
                          [&](int k, int col) -> T { return Y[(size_t)(ne + k) * N + col]; }, ao);
    T *U = (T *)c.U;
    const T r2 = T(0.70710678118654752440);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int a = r0 + 4 * ty + i;
        if (a >= ne) continue;
#pragma unroll
        for (int l = 0; l < TN; ++l) {
            const int col = c0 + TN * tx + l;
            if (col >= N || !col_allowed(col, c.sym)) continue;
            if (a < h) {
                U[(size_t)(1 + a) * N + col] += r2 * (ae[i][l] + ao[i][l]);
                U[(size_t)(M - a) * N + col] += r2 * (ae[i][l] - ao[i][l]);
            } else {
                U[(size_t)(1 + h) * N + col] += ae[i][l];
            }
        }
    }
    const unsigned nb = gridDim.x * gridDim.y;
    if (!last_cta_arrive(&sc->cnt_gemm, nb, am_last)) return;
    if (threadIdx.x == 0) {
        sc->step += 1;
        sc->tau += sc->dtau;
        sc->lambda = sc->lambda_next;
        sc->cnt_gemm = 0;
    }
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

template <typename T, int BN>
static cudaError_t implicit_t(const CurveDev &c, int gate, cudaStream_t st)
{
    const int gx = (c.nx + BN - 1) / BN, gy = (c.ine + IM_BM - 1) / IM_BM;
    cudaError_t e = imp_launch(k_imp_fwd<T, BN>, dim3(gx, gy, 2), st, c, gate);
    if (e != cudaSuccess) return e;
    return imp_launch(k_imp_back<T, BN>, dim3(gx, gy), st, c, gate);
}

cudaError_t launch_implicit_update(const CurveDev &c, int gate, cudaStream_t st)
{
    if (!c.impl) return cudaErrorInvalidValue;
    // narrow column tiles where the grid would not fill the GPU
    const bool narrow = c.nx <= 32 || (c.nx / 64) * ((c.ine + IM_BM - 1) / IM_BM) < 2 * 152;
    if (c.prec) return narrow ? implicit_t<float, 32>(c, gate, st) : implicit_t<float, 64>(c, gate, st);
    return narrow ? implicit_t<double, 32>(c, gate, st) : implicit_t<double, 64>(c, gate, st);
}

}  // namespace ks
