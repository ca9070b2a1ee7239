// ks_step.cu -- many descent steps of one curve (dense form of the
// s-contraction) in one persistent cooperative launch (Ashtari & Schneider,
// arXiv 2301.11704, Sec. V.C).
//
// A step is the same arithmetic as the three step kernels of ks_kernels.cu
// (rows_body; the staged contraction with D_t; the fused gradient / update
// epilogue; D_t u of the new state), with grid-wide barriers in place of
// kernel boundaries:
//
//   gate      a curve that is done or at its step limit stops here
//   rows      units of 2 PS_WARPS sections: r^, A^, per-unit FP64 row sums
//   barrier   every CTA reduces the units' sums in the same order (J^2, J_arc,
//             dJ^2/dl) and takes the same convergence decision; CTA 0 records
//             them; a converged curve stops here
//   D r       units (tile, split): partial contraction of W^-1 D_t^T W r^ (or
//             D_t r^) into part[split]
//   barrier
//   update    element-parallel: sum of the splits in split order, G = -(A^ + e),
//             u += dtau G / (1 + dtau a_j^2), per-CTA FP64 |G|^2
//   barrier
//   D u       CTA 0 reduces |G|^2 and advances step, tau and lambda; all units:
//             partial contraction of D_t u into part[split]
//   barrier
//   store     element-parallel: D = sum of the splits
//   barrier
//
// The split partials are summed in the same order as the cluster reduction of
// k_dt, so u and D_t u match the multi-kernel step bit for bit.
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "ks_device.cuh"

namespace ks {

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Barrier over all CTAs of a cooperative launch (all co-resident).  Arrivals
// count up monotonically in sc->bar (every launch of a curve has the same grid
// size, so a launch starts at a multiple of it); thread 0 of each CTA releases
// the CTA's writes, arrives, and polls with acquire loads until every CTA has
// arrived.  The poll gives up after about a second of clock cycles, or as soon
// as another CTA has given up, recording the failure in sc->err: the launch then
// ends and its results are invalid.
struct GridBarrier {
    unsigned long long *count;
    int *err;
    unsigned long long target;
    unsigned nb;

    __device__ __forceinline__ void init(DevScalars *sc)
    {
        count = &sc->bar;
        err = &sc->err;
        nb = gridDim.x;
        target = ld_acquire(count) / nb * nb;
    }

    __device__ __forceinline__ bool sync()
    {
        __shared__ int ok_s;
        __syncthreads();
        if (threadIdx.x == 0) {
            int ok = 1;
            target += nb;
            __threadfence();
            atomicAdd(count, 1ull);
            const long long t0 = clock64();
            while (ld_acquire(count) < target) {
                if (*(volatile int *)err) {
                    ok = 0;
                    break;
                }
                if (clock64() - t0 > (1ll << 31)) {
                    atomicExch(err, 2);
                    ok = 0;
                    break;
                }
            }
            __threadfence();
            ok_s = ok;
        }
        __syncthreads();
        return ok_s != 0;
    }
};

// Partial contraction of unit u = (tile_c, tile_r, split) into part[split]:
// X = r^ with the adjoint's scaling (update) or u with D_t's (store).
template <typename T, int BN>
__device__ __forceinline__ void dt_partial(const CurveDev &c, int mode, int discrete, int u, DtTiles<T, BN> &sm)
{
    constexpr int TM = DtContract<T, BN>::TM, TN = DtContract<T, BN>::TN;
    const int tc = u % c.tiles_c, tr = (u / c.tiles_c) % c.tiles_r, ks = u / (c.tiles_c * c.tiles_r);
    const int ns = c.ns, N = c.nx;
    DtContract<T, BN> k;
    k.X = (const T *)(mode == GM_STORE ? c.U : c.R);
    k.cot = (const T *)c.cot;
    k.colscale = (const T *)(discrete ? c.sw : c.tau);
    k.tsign = discrete ? T(-1) : T(1);
    k.N = N;
    k.twoP = 2 * c.P;
    k.j0 = tr * DT_BM;
    k.c0 = tc * BN;
    k.kbeg = ks * c.kchunk;
    k.kend = min(ns, k.kbeg + c.kchunk);
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int l = 0; l < TN; ++l) acc[i][l] = T(0);
    if (k.kbeg < k.kend) k.fetch(k.kbeg);
    k.run(sm, acc);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T *part = (T *)c.part + (size_t)ks * ns * N;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int j = k.j0 + ty * TM + i;
#pragma unroll
        for (int l = 0; l < TN; ++l) {
            const int col = k.c0 + tx * TN + l;
            if (j < ns && col < N) part[(size_t)j * N + col] = acc[i][l];
        }
    }
}

// Epilogue over the elements of the grid-stride range of this thread: y =
// rowscale_j * (sum of the splits in split order), then D = y (store) or
// G = -(A^ + e) and the semi-implicit increment of u (update; the same
// expressions as k_dt).  Returns this thread's FP64 share of sum_m w_m |G_m|^2.
template <typename T, int N>
__device__ __forceinline__ double dt_finish(const CurveDev &c, int mode, int discrete, double lam_d, double dtau_d)
{
    const int ns = c.ns, P = c.P, nsplit = c.ksplit;
    const size_t total = (size_t)ns * N;
    const T *part = (const T *)c.part;
    const T *rowscale = (const T *)(discrete ? c.twr : c.sig);
    const T *Ah = (const T *)c.A, *pr = (const T *)c.prec_imex;
    T *U = (T *)c.U, *Dout = (T *)c.D;
    const T lam = (T)lam_d, dtau = (T)dtau_d;
    double partsum = 0.0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / N), col = (int)(e % N);
        T t = T(0);
        for (int q = 0; q < nsplit; ++q) t += part[(size_t)q * total + e];
        const T y = rowscale[j] * t;
        if (mode == GM_STORE) {
            Dout[e] = y;
            continue;
        }
        if (j > 0 && j < P) {
            T g = 0;
            if (col != 1 && col_allowed(col, c.sym)) {
                const T ev = discrete ? -lam * y : lam * y;
                g = -(Ah[e] + ev);
                const double cw = (col < 2) ? 1.0 : 2.0;
                partsum += c.w[j] * cw * (double)g * (double)g;
            }
            U[e] = U[e] + dtau * pr[col >> 1] * g;
        }
    }
    return partsum;
}

template <typename T, int N, int BN>
__global__ void __launch_bounds__(PS_THREADS) k_step(CurveDev c, int discrete, long long nsteps)
{
    __shared__ DtTiles<T, BN> sm;
    __shared__ double red[PS_THREADS];
    __shared__ int gate_s;
    DevScalars *sc = c.sc;
    GridBarrier gb;
    gb.init(sc);
    const int nru = (c.ns + 2 * PS_WARPS - 1) / (2 * PS_WARPS);
    const int ndt = c.tiles_c * c.tiles_r * c.ksplit;
    for (long long it = 0; it < nsteps; ++it) {
        // gate of the step (the same values in every CTA): done, or at the step limit
        if (threadIdx.x == 0) {
            const int done = *(volatile int *)&sc->done;
            const long long step = *(volatile long long *)&sc->step, limit = *(volatile long long *)&sc->limit;
            gate_s = !(done || step >= limit);
            if (!gate_s && blockIdx.x == 0) sc->active = 0;
        }
        __syncthreads();
        if (!gate_s) break;
        for (int u = blockIdx.x; u < nru; u += gridDim.x) {
            rows_body<T, N, PS_WARPS>(c, ROWS_STEP, u, nru, false);
            __syncthreads();
        }
        if (!gb.sync()) return;
        // every CTA reduces the units' partial sums in the same fixed order and
        // takes the same convergence decision; CTA 0 records the scalars
        if (!rows_finish<PS_THREADS>(c, ROWS_STEP, nru, blockIdx.x == 0)) break;
        const double lam = *(volatile double *)&sc->lambda, dtau = *(volatile double *)&sc->dtau;

        for (int u = blockIdx.x; u < ndt; u += gridDim.x) dt_partial<T, BN>(c, GM_UPDATE, discrete, u, sm);
        if (!gb.sync()) return;
        double ps = dt_finish<T, N>(c, GM_UPDATE, discrete, lam, dtau);
        ps = block_sum<PS_THREADS>(ps, red);
        if (threadIdx.x == 0) c.gpart[blockIdx.x] = ps;
        if (!gb.sync()) return;

        if (blockIdx.x == 0) {
            double t = 0.0;
            for (int b = threadIdx.x; b < (int)gridDim.x; b += PS_THREADS) t += __ldcg(c.gpart + b);
            t = block_sum<PS_THREADS>(t, red);
            if (threadIdx.x == 0) {
                sc->G2 = c.L * t;
                sc->step += 1;
                sc->tau += sc->dtau;
                sc->lambda = sc->lambda_next;
            }
        }
        for (int u = blockIdx.x; u < ndt; u += gridDim.x) dt_partial<T, BN>(c, GM_STORE, 0, u, sm);
        if (!gb.sync()) return;
        dt_finish<T, N>(c, GM_STORE, 0, 0.0, 0.0);
        if (!gb.sync()) return;
    }
}

// Grid of the cooperative launch: every CTA co-resident (occupancy x SMs), at
// most PS_MAX_CTAS.  Cached per (device, kernel).
template <typename K>
static cudaError_t persistent_grid(K kern, size_t smem, int *grid)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void *>, int> cache;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    auto key = std::make_pair(dev, (const void *)kern);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *grid = it->second;
        return cudaSuccess;
    }
    int coop = 0, nsm = 0, per_sm = 0;
    if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev)) != cudaSuccess) return e;
    if (!coop) return cudaErrorNotSupported;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PS_THREADS, smem)) != cudaSuccess) return e;
    const int g = std::min(per_sm * nsm, PS_MAX_CTAS);
    if (g < 1) return cudaErrorInvalidConfiguration;
    cache[key] = g;
    *grid = g;
    return cudaSuccess;
}

template <typename T>
static cudaError_t step_t(const CurveDev &c, int discrete, long long nsteps, cudaStream_t st)
{
    return dispatch_n(c.nx, [&](auto nn) {
        constexpr int NN = decltype(nn)::value;
        constexpr int BN = NN >= 64 ? 64 : 32;
        if (c.bn != BN || !c.part || !c.gpart) return cudaErrorInvalidValue;
        auto kern = k_step<T, NN, BN>;
        const size_t sm = rows_smem<T>(NN, 3, PS_WARPS);
        cudaError_t e = set_smem(kern, sm);
        if (e != cudaSuccess) return e;
        int grid = 0;
        if ((e = persistent_grid(kern, sm, &grid)) != cudaSuccess) return e;
        CurveDev cc = c;
        void *args[] = {(void *)&cc, (void *)&discrete, (void *)&nsteps};
        e = cudaLaunchCooperativeKernel((const void *)kern, dim3(grid), dim3(PS_THREADS), args, sm, st);
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    });
}

cudaError_t launch_step_persistent(const CurveDev &c, int discrete, long long nsteps, cudaStream_t st)
{
    if (nsteps <= 0) return cudaSuccess;
    return c.prec ? step_t<float>(c, discrete, nsteps, st) : step_t<double>(c, discrete, nsteps, st);
}

}  // namespace ks
