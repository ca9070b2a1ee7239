// ks_implicit_tc.cu -- the two products of the full-linear-implicit increment
// (Sec. V.C.3; see ks_implicit.cu) on the fifth-generation tensor cores, for
// FP32 storage and N >= 32 (the MMA's N = N_x).
//
// Product of one parity p and one K range ("split"):
//   C[128 x N] = A[128 x K] B[K x N],
// A = 128 rows of V_p^-1 (forward) or V_p (back), B = the folded G (forward) or
// Y_p (back).  Both operands are split into two BF16 parts (x = x0 + x1, x1 the
// BF16 rounding of what x0 left; exact differences in FP32) and the three part
// products a0 b1 + a1 b0 + a0 b0 are accumulated in FP32 in tensor memory
// (about 2^-17 relative per product, the BF16X2 precision): the increment is a
// preconditioner applied to dtau G, whose fixed points do not depend on it.
// A is split once at set-up into the K-major operand layout, one contiguous
// block per (row tile, K chunk) that one bulk copy (TMA engine) brings in; B is
// split on the fly by the CTA's threads.  K is taken in chunks of 32 through two
// stages; thread 0 issues the copies and the products (tcgen05.mma, M = 128,
// N = N_x, K = 16, kind::f16) and commits each chunk to the mbarrier that frees
// its stage.  Every wait is bounded; a wait that gives up sets the curve's error
// word, no further copy or product is issued, and the copies and products in
// flight are waited for before TMEM is freed.  The epilogue (the implicit factor
// for the forward product) writes the split partials that k_imp_sum and
// k_imp_finish of ks_implicit.cu then take.
#include <cuda_bf16.h>

#include "ks_device.cuh"
#include "ks_internal.h"
#include "ks_tcgen05.cuh"

namespace ks {

namespace {

constexpr int IT_M = 128;        // rows per CTA: MMA M, TMEM lanes
constexpr int IT_KC = 32;        // K per chunk
constexpr int IT_THREADS = 256;  // B-operand producers; in the epilogue two per row (one per column half)
constexpr int IT_NP = 2;         // BF16 parts per operand
constexpr int IT_SBO = (IT_KC / 8) * 128;

template <int N>
struct ItCfg {
    static constexpr int A_PART = IT_M * IT_KC * 2;
    static constexpr int B_PART = N * IT_KC * 2;
    static constexpr int A_STAGE = IT_NP * A_PART;
    static constexpr int B_STAGE = IT_NP * B_PART;
    static constexpr size_t SMEM = 2 * (size_t)(A_STAGE + B_STAGE);
    static constexpr unsigned TMEM_COLS = N;   // N in {32, 64, 128, 256}
};

__device__ __forceinline__ int it_kmaj(int row, int k)
{
    return (row >> 3) * IT_SBO + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// 8 consecutive K values of one operand row, as two BF16 parts, 16 bytes each.
__device__ __forceinline__ void it_put8(unsigned char *stage, int part_bytes, int row, int k0, const float (&x)[8])
{
    unsigned w0[4], w1[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(x[2 * i] - hf.x, x[2 * i + 1] - hf.y);
        w0[i] = *reinterpret_cast<const unsigned *>(&h);
        w1[i] = *reinterpret_cast<const unsigned *>(&l);
    }
    *reinterpret_cast<uint4 *>(stage + it_kmaj(row, k0)) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
    *reinterpret_cast<uint4 *>(stage + part_bytes + it_kmaj(row, k0)) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
}

// Row tiles and K chunks of a parity block of n rows (padded with zeros).
__host__ __device__ inline int it_tiles(int n) { return (n + IT_M - 1) / IT_M; }
__host__ __device__ inline int it_chunks(int n) { return (n + IT_KC - 1) / IT_KC; }
__host__ __device__ inline size_t it_block_bytes(int n)
{
    return (size_t)it_tiles(n) * it_chunks(n) * IT_NP * (IT_M * IT_KC * 2);
}

}  // namespace

size_t implicit_tc_bytes(int ns)
{
    const int ne = (ns - 1) / 2, no = (ns - 2) / 2;
    return 2 * (it_block_bytes(ne) + it_block_bytes(no));
}

// Set-up: V^-1 and V of both parities (FP32, row-major, in c.ivi / c.iv) into
// the operand layout: [matrix][parity] blocks of [row tile][K chunk][part][kmaj].
__global__ void k_imp_tc_split(CurveDev c)
{
    const int ne = c.ine, no = c.ino;
    const size_t be = it_block_bytes(ne), bo = it_block_bytes(no);
    for (int mat = 0; mat < 2; ++mat)
        for (int p = 0; p < 2; ++p) {
            const int n = p ? no : ne;
            const float *X = (const float *)(mat == 0 ? c.ivi : c.iv) + (p ? (size_t)ne * ne : 0);
            unsigned char *dst = (unsigned char *)c.ivtc + (size_t)mat * (be + bo) + (p ? be : 0);
            const int nt = it_tiles(n), nk = it_chunks(n);
            // one unit: a (tile, chunk, row, k-block of 8)
            const long units = (long)nt * nk * IT_M * (IT_KC / 8);
            for (long u = blockIdx.x * (long)blockDim.x + threadIdx.x; u < units; u += (long)gridDim.x * blockDim.x) {
                const int kb = (int)(u % (IT_KC / 8));
                long v = u / (IT_KC / 8);
                const int r = (int)(v % IT_M);
                v /= IT_M;
                const int kc = (int)(v % nk), rt = (int)(v / nk);
                const int row = rt * IT_M + r, k0 = kc * IT_KC + 8 * kb;
                float x[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) x[i] = (row < n && k0 + i < n) ? X[(size_t)row * n + k0 + i] : 0.f;
                unsigned char *chunk = dst + ((size_t)rt * nk + kc) * IT_NP * (IT_M * IT_KC * 2);
                it_put8(chunk, IT_M * IT_KC * 2, r, 8 * kb, x);
            }
        }
}

// FWD: Pf[split] rows of parity p = phi (V_p^-1 Q_p^T G); else Pb[split] rows of
// parity p = V_p Y_p (Y = Pf[0] after the split sum).  Block (row tile, parity, split).
template <int N, bool FWD>
__global__ void __launch_bounds__(IT_THREADS, 1) k_imp_tc(CurveDev c, int splits, int gate)
{
    using Cfg = ItCfg<N>;
    extern __shared__ __align__(1024) unsigned char smem_t[];
    unsigned char *As = smem_t, *Bs = smem_t + 2 * Cfg::A_STAGE;
    __shared__ __align__(8) unsigned long long a_full[2], b_full[2], mma_done[2];
    __shared__ unsigned tmem_slot;
    __shared__ int sbad;
    pdl_wait();
    DevScalars *sc = c.sc;
    if (gate && !sc->active) return;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int rt = blockIdx.x, p = blockIdx.y, sp = blockIdx.z;
    const int M = c.ns - 2, h = M / 2, ne = c.ine, np = p ? c.ino : ne;
    if (rt * IT_M >= np) return;
    const int nk = it_chunks(np);
    int kc = (nk + splits - 1) / splits;
    const int q0 = min(nk, sp * kc), q1 = min(nk, q0 + kc);
    const long long wb = wait_bound(*sc);
    const size_t be = it_block_bytes(ne), bo = it_block_bytes(c.ino);
    const unsigned char *Ablk = (const unsigned char *)c.ivtc + (FWD ? 0 : (be + bo)) + (p ? be : 0) +
                                (size_t)rt * nk * Cfg::A_STAGE;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::su32(&tmem_slot)),
                     "r"(Cfg::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            tc::bar_init(&a_full[i], 1);
            tc::bar_init(&b_full[i], IT_THREADS);
            tc::bar_init(&mma_done[i], 1);
        }
        sbad = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const unsigned tmem = tmem_slot;
    volatile int *vbad = &sbad;
    auto fail = [&]() {
        if (!*vbad) {
            *vbad = 1;
            atomicExch(&sc->err, 5);
        }
    };

    const int Nn = c.nx;
    const float *G = (const float *)c.G;
    const float *Y = (const float *)c.isc + (p ? (size_t)ne * Nn : 0);
    const float r2 = 0.70710678118654752440f;
    // B chunk q: units (col, k-block of 8) of 8 values, UPT per thread.  `fetch`
    // issues every load of a chunk at once (rows and predicates computed first,
    // no branch between the loads), one chunk ahead of `produce`, which folds,
    // splits and writes the operand stage.
    constexpr int UNITS = N * (IT_KC / 8), UPT = (UNITS + IT_THREADS - 1) / IT_THREADS;
    const float *Bsrc = FWD ? G : Y;
    auto fetch = [&](int q, float (&xa)[UPT][8], float (&xb)[UPT][8]) {
#pragma unroll
        for (int j = 0; j < UPT; ++j) {
            const int u = tid + j * IT_THREADS, col = u % N, kb = u / N, k0 = q * IT_KC + 8 * kb;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int k = k0 + e;
                const bool v = u < UNITS && k < np;
                const int ra = FWD ? 1 + k : k;
                const int rb = (p == 0 && k >= h) ? ra : M - k;   // the mirror row (odd M: the middle alone)
                xa[j][e] = v ? Bsrc[(size_t)ra * Nn + col] : 0.f;
                xb[j][e] = (FWD && v) ? G[(size_t)rb * Nn + col] : 0.f;
            }
        }
    };
    auto produce = [&](int q, unsigned char *bst, const float (&xa)[UPT][8], const float (&xb)[UPT][8]) {
#pragma unroll
        for (int j = 0; j < UPT; ++j) {
            const int u = tid + j * IT_THREADS, col = u % N, kb = u / N, k0 = q * IT_KC + 8 * kb;
            if (u >= UNITS) continue;
            float x[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                if (!FWD) x[e] = xa[j][e];
                else if (p == 0) x[e] = (k0 + e < h) ? r2 * (xa[j][e] + xb[j][e]) : xa[j][e];
                else x[e] = r2 * (xa[j][e] - xb[j][e]);
            }
            it_put8(bst, Cfg::B_PART, col, 8 * kb, x);
        }
    };
    float ca[UPT][8], cb[UPT][8];
    if (q1 > q0) fetch(q0, ca, cb);
    constexpr unsigned IDESC = tc::idesc_bf16(IT_M, N);
    int copied = 0, landed = 0;   // thread 0: chunks whose A copy was issued / waited for
    if (tid == 0 && q1 > q0) {     // the first chunk's A block; each later one a chunk ahead
        tc::bulk_g2s(As, Ablk + (size_t)q0 * Cfg::A_STAGE, (unsigned)Cfg::A_STAGE, &a_full[0]);
        copied = 1;
    }
    for (int q = q0; q < q1; ++q) {
        const int i = q - q0, st = i & 1;
        // the B stage of chunk i - 2 is free once its products are done
        if (i >= 2 && !*vbad && !tc::bar_wait(&mma_done[st], ((i - 2) >> 1) & 1, wb)) fail();
        // A of chunk i + 1 into the stage chunk i - 1 used, once its products are done
        if (tid == 0 && !*vbad && q + 1 < q1 && copied == i + 1) {
            if (i >= 1 && !tc::bar_wait(&mma_done[st ^ 1], ((i - 1) >> 1) & 1, wb)) {
                fail();
            } else {
                tc::bulk_g2s(As + (st ^ 1) * Cfg::A_STAGE, Ablk + (size_t)(q + 1) * Cfg::A_STAGE,
                             (unsigned)Cfg::A_STAGE, &a_full[st ^ 1]);
                copied = i + 2;
            }
        }
        // B chunk: the next chunk's loads in flight while this one is written
        unsigned char *bst = Bs + st * Cfg::B_STAGE;
        float na[UPT][8], nb[UPT][8];
        if (q + 1 < q1) fetch(q + 1, na, nb);
        produce(q, bst, ca, cb);
#pragma unroll
        for (int j = 0; j < UPT; ++j)
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                ca[j][e] = na[j][e];
                cb[j][e] = nb[j][e];
            }
        tc::fence_async_smem();
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::su32(&b_full[st])) : "memory");
        if (tid == 0) {
            bool ok = !*vbad && copied >= i + 1;
            if (ok && !tc::bar_wait(&a_full[st], (i >> 1) & 1, wb)) ok = false;
            if (ok) landed = i + 1;
            if (ok && !tc::bar_wait(&b_full[st], (i >> 1) & 1, wb)) ok = false;
            if (ok) {
                tc::fence_after();
                const unsigned char *a0 = As + st * Cfg::A_STAGE, *b0 = bst;
#pragma unroll
                for (int s = 0; s < IT_KC / 16; ++s) {
                    // part pairs, smallest first: (0,1) (1,0) (0,0)
                    constexpr int pa[3] = {0, 1, 0}, pb[3] = {1, 0, 0};
#pragma unroll
                    for (int t = 0; t < 3; ++t) {
                        const unsigned long long ad = tc::sdesc(a0 + pa[t] * Cfg::A_PART + 256 * s, 128, IT_SBO);
                        const unsigned long long bd = tc::sdesc(b0 + pb[t] * Cfg::B_PART + 256 * s, 128, IT_SBO);
                        tc::mma_f16(tmem, ad, bd, IDESC, (i > 0 || s > 0 || t > 0) ? 1 : 0);
                    }
                }
            } else {
                fail();
            }
            tc::commit(&mma_done[st]);   // also when nothing was issued: keeps the phases in step
        }
    }
    // the last chunk's products (and, after a failed wait, every copy in flight)
    const int nq = q1 - q0;
    if (nq > 0) {
        const int il = nq - 1;
        if (!tc::bar_wait(&mma_done[il & 1], (il >> 1) & 1, wb)) {
            fail();
            tc::bar_wait(&mma_done[il & 1], (il >> 1) & 1);
        }
    }
    if (tid == 0)   // copies issued but not waited for (only after a wait gave up)
        for (int i = landed; i < copied; ++i) tc::bar_wait(&a_full[i & 1], (i >> 1) & 1);
    tc::fence_after();

    // epilogue: this thread's row of the accumulator (TMEM lane 32 (warp % 4) +
    // lane), half of the N columns (warp / 4), in steps of 16
    const int lrow = 32 * (warp & 3) + (tid & 31), half = warp >> 2;
    const int r = rt * IT_M + lrow;
    const bool ok = !*vbad && r < np;   // an empty K range (nq = 0) writes zeros
    const size_t stride = (size_t)M * Nn;
    float *out = (float *)c.isc + (size_t)(FWD ? sp : c.isplits + sp) * stride + (p ? (size_t)ne * Nn : 0) +
                 (size_t)r * Nn;
    const float lam = (float)sc->lambda, dtau = (float)sc->dtau, tl = (float)(2.0 * M_PI / c.L);
    const float lm = FWD && ok ? lam * lam * (float)c.imu[(p ? ne : 0) + r] : 0.f;
#pragma unroll 1
    for (int c0 = half * (N / 2); c0 < (half + 1) * (N / 2); c0 += 16) {
        float v[16];
        tc::ld16(tmem + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)c0, v);
        if (!ok) continue;
        float y[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int col = c0 + e;
            y[e] = nq > 0 ? v[e] : 0.f;
            if (FWD) {
                const float kw = tl * (float)(col >> 1), a = kw * kw * kw * kw - kw * kw;
                y[e] *= dtau / (1.f + dtau * (a * a - lm));
            }
        }
#pragma unroll
        for (int e = 0; e < 16; e += 4)
            *reinterpret_cast<float4 *>(out + c0 + e) = make_float4(y[e], y[e + 1], y[e + 2], y[e + 3]);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::TMEM_COLS) : "memory");
}

cudaError_t launch_setup_implicit_tc(const CurveDev &c, cudaStream_t st)
{
    if (!c.ivtc) return cudaSuccess;
    k_imp_tc_split<<<1024, 256, 0, st>>>(c);
    return cudaGetLastError();
}

template <int N>
static cudaError_t imp_tc_pair(const CurveDev &c, int splits, int gate, cudaStream_t st, int which)
{
    using Cfg = ItCfg<N>;
    auto kern = which == 0 ? k_imp_tc<N, true> : k_imp_tc<N, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(it_tiles(c.ine), 2, splits);
    cfg.blockDim = dim3(IT_THREADS);
    cfg.dynamicSmemBytes = Cfg::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, c, splits, gate);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// which = 0: the forward product, 1: the back product.
cudaError_t launch_implicit_tc(const CurveDev &c, int splits, int gate, cudaStream_t st, int which)
{
    switch (c.nx) {
    case 32: return imp_tc_pair<32>(c, splits, gate, st, which);
    case 64: return imp_tc_pair<64>(c, splits, gate, st, which);
    case 128: return imp_tc_pair<128>(c, splits, gate, st, which);
    case 256: return imp_tc_pair<256>(c, splits, gate, st, which);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ks
