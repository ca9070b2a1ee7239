// ks_tc.cu -- the dense s-contraction with D_t on the tensor cores (tcgen05,
// FP32 storage).  Ashtari & Schneider, arXiv 2301.11704, eq.
// rational_diff_matrix, Sec. V.C.1.
//
//   Y[j][col] = rowscale_j * sum_m (cot[(j+m) mod 2P] + tsign cot[(j-m) mod 2P]) colscale_m X[m][col]
//
// CTA (tile_c, tile_r, split) computes a TC_M x BN output tile over the sections
// of its split, in stages of TC_KC sections: every thread builds part of the
// stage's D_t block (from two contiguous windows of the cot table) and of the
// scaled X block, each split into three TF32 parts x = x0 + x1 + x2 (x0 = x
// rounded to TF32, x1 the rounded remainder, x2 the rest; 33 bits represent every
// FP32 value exactly), in the K-major no-swizzle layout of the MMA operands; one
// thread then issues, per 8 sections, the six products a0b2 + a1b1 + a2b0 +
// a0b1 + a1b0 + a0b0 (the dropped cross terms are below 2^-33 of the product)
// with FP32 accumulation in tensor memory (tcgen05.mma kind::tf32, M = 128) and
// commits them to the stage's mbarrier.  Two stage buffers and two accumulators:
// the next stage is built while the current one is multiplied, and each stage's
// accumulator is read back (tcgen05.ld) and added, in stage order, to FP32
// registers once its products are done -- the tensor cores' accumulation (not
// rounded to nearest) then spans 32 sections only, however long the split.  The
// splits of a tile (one thread-block cluster) are summed in split order through
// distributed shared memory, and the epilogue is that of k_dt (store D_t u; or
// G, the semi-implicit increment and |G|^2).
//
// Operand layout (per stage, per part): core matrices of 8 rows x 16 bytes (4
// TF32 values along K), rows at 16 B, the K-adjacent core matrices 128 B apart
// (leading byte offset), the row-adjacent groups TC_KC * 32 B apart (stride
// byte offset); one 8-section MMA step advances the operand start by 256 B.
#include <cooperative_groups.h>

#include "ks_device.cuh"
#include "ks_tcgen05.cuh"

namespace ks {

namespace tc {

__device__ __forceinline__ float tf32(float x)
{
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// x = x0 + x1 + x2 exactly, each part a TF32 value (x0 = x rounded to TF32, x1 the
// remainder rounded to TF32, x2 what is left: at most 2 significant bits).
__device__ __forceinline__ void split3(float x, float &x0, float &x1, float &x2)
{
    x0 = tf32(x);
    const float r = x - x0;
    x1 = tf32(r);
    x2 = tf32(r - x1);
}

}  // namespace tc

template <int BN>
struct TcCfg {
    static constexpr int MMA_N = BN < 16 ? 16 : BN;           // MMA N (a multiple of 16 for M = 128)
    static constexpr int TMEM_COLS = 2 * MMA_N < 32 ? 32 : 2 * MMA_N;   // two accumulators
    static constexpr int HALF = MMA_N / 2 < 16 ? 16 : MMA_N / 2;   // columns read back per thread
    static constexpr int SBO = TC_KC * 32;                     // bytes between row groups of 8
    static constexpr int A_BYTES = TC_M * TC_KC * 4;           // one part of one stage
    static constexpr int B_BYTES = MMA_N * TC_KC * 4;
    static constexpr int XV = TC_KC * (MMA_N / 4);             // four-column X loads per stage
    static constexpr int NXV = (XV + TC_THREADS - 1) / TC_THREADS;
    static constexpr int PT_LD = MMA_N + 1;                    // padded row of the partial tile
    static constexpr int PARTS = 3;                            // TF32 parts of each operand
    static constexpr size_t SMEM = (size_t)2 * PARTS * (A_BYTES + B_BYTES);
    static_assert((size_t)TC_M * PT_LD * 4 <= (size_t)2 * PARTS * A_BYTES, "partial tile fits the operand space");
};

template <int BN>
__global__ void __launch_bounds__(TC_THREADS) k_dt_tc(CurveDev c, int mode, int discrete, int gate)
{
    namespace cg = cooperative_groups;
    using Cfg = TcCfg<BN>;
    constexpr int WIN = TC_M + TC_KC - 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *Abase = smem_raw;                                   // [stage][part] A blocks
    unsigned char *Bbase = smem_raw + 2 * Cfg::PARTS * Cfg::A_BYTES;   // [stage][part] B blocks
    float *Pt = (float *)smem_raw;                                     // partial tile, after the MMAs
    __shared__ float Wp[WIN + 1], Wm[WIN + 1];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ unsigned tmem_slot;
    __shared__ double red[TC_THREADS];
    __shared__ int am_last;
    DevScalars *sc = c.sc;
    pdl_wait();
    const int g_active = sc->active;
    const double lam_d = sc->lambda, dtau_d = sc->dtau;
    const long long wb = wait_bound(*sc);
    if (gate && !g_active) return;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile_c = blockIdx.x, tile_r = blockIdx.y, ks = blockIdx.z;
    const int tiles_c = gridDim.x, tiles_r = gridDim.y, nsplit = gridDim.z;
    const int ns = c.ns, N = c.nx, P = c.P, twoP = 2 * P;
    const int j0 = tile_r * TC_M, c0 = tile_c * BN;
    const int kbeg = ks * c.tc_kchunk, kend = min(ns, kbeg + c.tc_kchunk);
    const int nst = (kend - kbeg + TC_KC - 1) / TC_KC;
    const float *X = (const float *)(mode == GM_STORE ? c.U : c.R);
    const float *cot = (const float *)c.cot;
    const float *colscale = (const float *)(discrete ? c.sw : c.tau);
    const float *rowscale = (const float *)(discrete ? c.twr : c.sig);
    const float tsign = discrete ? -1.f : 1.f;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::su32(&tmem_slot)),
                     "r"(Cfg::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::su32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::su32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }

    // ---- register-staged operands of one stage: cot windows and scaled X values
    float wpr = 0.f, wmr = 0.f;
    Vec4<float> xr[Cfg::NXV];
    auto fetch = [&](int m0) {
        if (tid < WIN) {
            int ip = (j0 + m0 + tid) % twoP;
            int im = (j0 - m0 - TC_KC + 1 + tid) % twoP;
            if (im < 0) im += twoP;
            wpr = cot[ip];
            wmr = cot[im];
        }
#pragma unroll
        for (int q = 0; q < Cfg::NXV; ++q) {
            const int e = tid + q * TC_THREADS;
            const int k = e / (Cfg::MMA_N / 4), col = c0 + 4 * (e % (Cfg::MMA_N / 4)), m = m0 + k;
            if (e < Cfg::XV && m < kend && col < N) {
                const float s = colscale[m];
                const Vec4<float> x = ld4(X + (size_t)m * N + col);
                xr[q] = {s * x.x, s * x.y, s * x.z, s * x.w};
            } else {
                xr[q] = {0.f, 0.f, 0.f, 0.f};
            }
        }
    };
    if (nst > 0) fetch(kbeg);

    // ---- epilogue bookkeeping: this CTA finishes the row band [r0, r1) of the tile
    const int rows_per = (TC_M + nsplit - 1) / nsplit;
    const int r0 = min(TC_M, ks * rows_per), r1 = min(TC_M, r0 + rows_per);
    const int band = (r1 - r0) * BN;

    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const unsigned tmem = tmem_slot;
    constexpr unsigned IDESC = tc::idesc_tf32(TC_M, Cfg::MMA_N);

    // this thread's accumulator row (TMEM lane) and columns: warp w reads lanes
    // 32 (w % 4) .. + 31, the column half w / 4
    const int quarter = warp & 3, half = warp >> 2;
    const int row = 32 * quarter + lane, cb0 = half * Cfg::HALF;
    const bool reads = cb0 < Cfg::MMA_N;
    float racc[Cfg::HALF];
#pragma unroll
    for (int i = 0; i < Cfg::HALF; ++i) racc[i] = 0.f;
    auto add_stage = [&](int buf) {   // adds accumulator buf (a finished stage) to the registers
        if (!reads) return;
#pragma unroll
        for (int cb = 0; cb < Cfg::HALF; cb += 16) {
            float v[16];
            tc::ld16(tmem + ((unsigned)(32 * quarter) << 16) + buf * Cfg::MMA_N + cb0 + cb, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) racc[cb + i] += v[i];
        }
    };

    bool ok = true;
    for (int s = 0; s < nst; ++s) {
        const int buf = s & 1;
        if (s >= 2) {   // stage s-2 has been multiplied: its operands and accumulator are free
            if (!tc::bar_wait(&mbar[buf], ((s - 2) >> 1) & 1, ok ? wb : -1)) {
                ok = false;
                tc::bar_wait(&mbar[buf], ((s - 2) >> 1) & 1);   // its products still read this stage
            }
            tc::fence_after();
            add_stage(buf);
        }
        if (tid < WIN) {
            Wp[tid] = wpr;
            Wm[tid] = wmr;
        }
        Vec4<float> xs[Cfg::NXV];
#pragma unroll
        for (int q = 0; q < Cfg::NXV; ++q) xs[q] = xr[q];
        __syncthreads();
        if (s + 1 < nst) fetch(kbeg + (s + 1) * TC_KC);   // next stage in flight

        unsigned char *A0 = Abase + (size_t)(Cfg::PARTS * buf) * Cfg::A_BYTES, *A1 = A0 + Cfg::A_BYTES,
                      *A2 = A1 + Cfg::A_BYTES;
        unsigned char *B0 = Bbase + (size_t)(Cfg::PARTS * buf) * Cfg::B_BYTES, *B1 = B0 + Cfg::B_BYTES,
                      *B2 = B1 + Cfg::B_BYTES;
        // D_t block, K[r][k] = Wp[r + k] + tsign Wm[r - k + TC_KC - 1]; a warp writes 512 contiguous bytes
#pragma unroll
        for (int q = 0; q < TC_M * TC_KC / 4 / TC_THREADS; ++q) {
            const int e = tid + q * TC_THREADS;
            const int r8 = e & 7, k4 = (e >> 3) & (TC_KC / 4 - 1), g = e / (2 * TC_KC);
            const int r = g * 8 + r8, k = 4 * k4;
            float p0[4], p1[4], p2[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) tc::split3(Wp[r + k + i] + tsign * Wm[r - k - i + TC_KC - 1], p0[i], p1[i], p2[i]);
            const int off = g * Cfg::SBO + k4 * 128 + r8 * 16;
            *reinterpret_cast<float4 *>(A0 + off) = make_float4(p0[0], p0[1], p0[2], p0[3]);
            *reinterpret_cast<float4 *>(A1 + off) = make_float4(p1[0], p1[1], p1[2], p1[3]);
            *reinterpret_cast<float4 *>(A2 + off) = make_float4(p2[0], p2[1], p2[2], p2[3]);
        }
        // scaled X block, transposed into the K-major layout
#pragma unroll
        for (int q = 0; q < Cfg::NXV; ++q) {
            const int e = tid + q * TC_THREADS;
            if (e < Cfg::XV) {
                const int k = e / (Cfg::MMA_N / 4), n = 4 * (e % (Cfg::MMA_N / 4));
                const float v[4] = {xs[q].x, xs[q].y, xs[q].z, xs[q].w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int nn = n + i;
                    const int off = (nn >> 3) * Cfg::SBO + (k >> 2) * 128 + (nn & 7) * 16 + (k & 3) * 4;
                    float q0, q1, q2;
                    tc::split3(v[i], q0, q1, q2);
                    *reinterpret_cast<float *>(B0 + off) = q0;
                    *reinterpret_cast<float *>(B1 + off) = q1;
                    *reinterpret_cast<float *>(B2 + off) = q2;
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0) {
#pragma unroll
            for (int s8 = 0; s8 < TC_KC / 8; ++s8) {
                const unsigned long long a0 = tc::sdesc(A0 + 256 * s8, 128, Cfg::SBO);
                const unsigned long long a1 = tc::sdesc(A1 + 256 * s8, 128, Cfg::SBO);
                const unsigned long long a2 = tc::sdesc(A2 + 256 * s8, 128, Cfg::SBO);
                const unsigned long long b0 = tc::sdesc(B0 + 256 * s8, 128, Cfg::SBO);
                const unsigned long long b1 = tc::sdesc(B1 + 256 * s8, 128, Cfg::SBO);
                const unsigned long long b2 = tc::sdesc(B2 + 256 * s8, 128, Cfg::SBO);
                const unsigned d = tmem + buf * Cfg::MMA_N;
                tc::mma_tf32(d, a0, b2, IDESC, s8 > 0 ? 1 : 0);
                tc::mma_tf32(d, a1, b1, IDESC, 1);
                tc::mma_tf32(d, a2, b0, IDESC, 1);
                tc::mma_tf32(d, a0, b1, IDESC, 1);
                tc::mma_tf32(d, a1, b0, IDESC, 1);
                tc::mma_tf32(d, a0, b0, IDESC, 1);
            }
            tc::commit(&mbar[buf]);
        }
    }
    // the last two stages (a commit tracks every earlier MMA of the issuing thread)
    for (int s = nst >= 2 ? nst - 2 : 0; s < nst; ++s) {
        if (!tc::bar_wait(&mbar[s & 1], (s >> 1) & 1, ok ? wb : -1)) {
            ok = false;
            tc::bar_wait(&mbar[s & 1], (s >> 1) & 1);
        }
        tc::fence_after();
        add_stage(s & 1);
    }
    if (!ok && tid == 0) atomicExch(&sc->err, 3);

    // ---- the tile's sums -> partial tile in shared memory (operand space is free now)
    if (reads) {
#pragma unroll
        for (int i = 0; i < Cfg::HALF; ++i) Pt[row * Cfg::PT_LD + cb0 + i] = racc[i];
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::TMEM_COLS) : "memory");

    // ---- the band's sums over the splits (in split order), then the epilogue
    cg::cluster_group cluster = cg::this_cluster();
    if (nsplit > 1) cluster.sync();
    float *U = (float *)c.U, *G = (float *)c.G, *Dout = (float *)c.D;
    const float *Ah = (const float *)c.A, *pr = (const float *)c.prec_imex;
    const float lam = (float)lam_d, dtau = (float)dtau_d;
    double partsum = 0.0;
    for (int e = tid; e < band; e += TC_THREADS) {
        const int rr = r0 + e / BN, cc = e % BN;
        const int j = j0 + rr, col = c0 + cc;
        float t = 0.f;
        if (nsplit > 1) {
            for (int q = 0; q < nsplit; ++q) t += cluster.map_shared_rank(Pt, q)[rr * Cfg::PT_LD + cc];
        } else {
            t = Pt[rr * Cfg::PT_LD + cc];
        }
        if (j >= ns || col >= N) continue;
        const size_t o = (size_t)j * N + col;
        const float y = rowscale[j] * t;
        if (mode == GM_STORE) {
            Dout[o] = y;
            continue;
        }
        const bool interior = (j > 0 && j < P);
        float g = 0.f;
        if (interior && col != 1 && col_allowed(col, c.sym)) {
            const float ev = discrete ? -lam * y : lam * y;
            g = -(Ah[o] + ev);
            const double cw = (col < 2) ? 1.0 : 2.0;
            partsum += c.w[j] * cw * (double)g * (double)g;
        }
        if (mode == GM_UPDATE) {
            if (interior) U[o] = U[o] + dtau * pr[col >> 1] * g;
        } else {
            G[o] = g;
        }
    }
    if (nsplit > 1) cluster.sync();   // no CTA leaves while its partial tile may still be read
    if (mode == GM_STORE) return;

    // ---- FP64 |G|^2: per-CTA partial, last CTA of the grid sums them in a fixed order
    partsum = block_sum<TC_THREADS>(partsum, red);
    const int bid = (ks * tiles_r + tile_r) * tiles_c + tile_c, nb = tiles_c * tiles_r * nsplit;
    if (tid == 0) c.tile[bid] = partsum;
    if (!last_cta_arrive(&sc->cnt_gemm, (unsigned)nb, am_last)) return;
    double t = 0.0;
    for (int b = tid; b < nb; b += TC_THREADS) t += __ldcg(c.tile + b);
    t = block_sum<TC_THREADS>(t, red);
    if (tid == 0) {
        sc->G2 = c.L * t;
        if (mode == GM_UPDATE) {
            sc->step += 1;
            sc->tau += sc->dtau;
            sc->lambda = sc->lambda_next;
        }
        sc->cnt_gemm = 0;
    }
}

template <int BN>
static cudaError_t launch_tc_t(const CurveDev &c, int mode, int discrete, int gate, cudaStream_t st)
{
    const size_t sm = TcCfg<BN>::SMEM;
    cudaError_t e = set_smem(k_dt_tc<BN>, sm);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c.tc_tiles_c, c.tc_tiles_r, c.tc_ksplit);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = 1;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = c.tc_ksplit;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    e = cudaLaunchKernelEx(&cfg, k_dt_tc<BN>, c, mode, discrete, gate);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_dt_tc(const CurveDev &c, int mode, int discrete, int gate, cudaStream_t st)
{
    switch (c.tc_bn) {
    case 64: return launch_tc_t<64>(c, mode, discrete, gate, st);
    case 32: return launch_tc_t<32>(c, mode, discrete, gate, st);
    case 16: return launch_tc_t<16>(c, mode, discrete, gate, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ks
