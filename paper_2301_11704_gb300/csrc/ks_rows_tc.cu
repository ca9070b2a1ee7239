// ks_rows_tc.cu -- the row phase of one evaluation (Ashtari & Schneider, arXiv
// 2301.11704: eq. KSE, eq. KSE_residual, eq. KSE_G, the pseudo-spectral products
// of Sec. V.C.1) with the Fourier transforms of the sections as dense products
// on the fifth-generation tensor cores (tcgen05), operands split into BF16 parts.
//
// A section of N modes is N real words (N/2 complex coefficients interleaved,
// Im of mode 0 and the Nyquist mode held at zero).  Its one forward or backward
// DFT (Sec. V.C.1) is a product with a fixed N x N real matrix:
//   inverse  u[n]  = sum_i uh[i] C[i][n],  C[2j][n] = c_j cos(2 pi j n / N),
//                                          C[2j+1][n] = -c_j sin(2 pi j n / N),
//                                          c_0 = 1, c_j = 2, C[1][.] = 0;
//   forward  wh[i] = sum_n w[n] E[n][i],   E[n][2j] = cos(2 pi j n / N) / N,
//                                          E[n][2j+1] = -sin(2 pi j n / N) / N, E[.][1] = 0.
// A CTA takes 128 sections (one TMEM lane each, two threads: one per half of every
// K-chunk of 32) through four products
// [128 x N] x [N x N] with FP32 accumulators in tensor memory:
//   G1  u   = uh C               -> accumulator T0
//   G2  wh  = (u u) E            -> T1; then per section f^ = -(1/2) i k wh - a_j uh,
//                                   r^ = f^ - l d^ (0 on the end rows), the row sums
//                                   of the cost, r^ written out
//   G3  r_x = (i k r^) C         -> T1
//       y   = u r_x              -> T0 (over u)
//   G4  p^  = y E                -> T1; then A^ = p^ - a_j r^ = (Df)^T r (eq. KSE_G)
// Split BF16: an FP32 operand x is written as x0 + x1 (+ x2), each part the BF16
// rounding of what the earlier parts left (x - x0 and x - x0 - x1 are exact in
// FP32); the DFT matrices are split the same way from FP64 values at set-up.  A
// product keeps the part products a0 b0 + a0 b1 + a1 b0 (two parts: about 2^-17
// relative, the BF16X2 precision) or also a0 b2 + a1 b1 + a2 b0 (three parts:
// about 2^-24, BF16X3), issued smallest first.
//
// Pipeline: K is taken in chunks of 32; the four products form one stream of
// 4 N/32 chunks.  Thread 0 copies each chunk of the DFT matrix (all its parts,
// laid out at set-up in the operand order, one bulk copy) into one of three
// B stages on an mbarrier one chunk ahead; every thread writes its section's
// split operand chunk into one of two A stages; thread 0 issues the chunk's
// tcgen05.mma (M = 128, N = N, K = 16, kind::f16) and commits them to the
// chunk's mbarrier, which frees both stages.  Every wait is bounded: a wait that
// gives up sets the curve's error word, no further copy or product is issued,
// the copies in flight are waited for (again bounded) and TMEM is freed.
//
// Operand layout (K-major, no swizzle): core matrices of 8 rows x 16 bytes (8
// BF16 along K), rows 16 B apart, K-adjacent core matrices 128 B apart (LBO),
// row groups 512 B apart (SBO); one MMA (K = 16) spans two core matrices.
#include <cuda_bf16.h>

#include "ks_device.cuh"
#include "ks_tcgen05.cuh"

namespace ks {

namespace {

constexpr int XT_M = 128;          // sections per CTA: MMA M, TMEM lanes
constexpr int XT_PROD = 256;       // operand and epilogue threads: two per section, one per half of each chunk
constexpr int XT_THREADS = XT_PROD + 32;   // and one warp that issues the bulk copies and the products
constexpr int XT_KC = 32;          // K per pipeline chunk
constexpr int XT_HV = XT_KC / 2;   // values of a chunk per thread
constexpr int XT_PARTS = 3;        // parts stored per DFT-matrix chunk
constexpr int XT_ASTAGES = 2, XT_BSTAGES = 3;
constexpr int XT_SBO = (XT_KC / 8) * 128;

template <int N, int NP>
struct XtCfg {
    static constexpr int NCH = N / XT_KC;                 // chunks per product
    static constexpr int QTOT = 4 * NCH;                  // chunks of the four products
    static constexpr int A_PART = XT_M * XT_KC * 2;       // bytes of one part of an A chunk
    static constexpr int B_PART = N * XT_KC * 2;          // bytes of one part of a B chunk
    static constexpr int A_STAGE = NP * A_PART;
    static constexpr int B_STAGE = NP * B_PART;
    static constexpr size_t SMEM = (size_t)XT_ASTAGES * A_STAGE + (size_t)XT_BSTAGES * B_STAGE;
    static constexpr unsigned TMEM_COLS = 2 * N;          // T0 and T1
    static_assert(SMEM <= 227 * 1024, "pipeline stages fit the shared memory");
};

// byte offset of element (row, k) of a K-major chunk (k < XT_KC)
__device__ __forceinline__ int kmaj_off(int row, int k)
{
    return (row >> 3) * XT_SBO + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Writes this thread's half of a row of a chunk (XT_HV FP32 values: the K-blocks
// 2 h and 2 h + 1 of 8 values each) as NP BF16 parts.
template <int NP>
__device__ __forceinline__ void put_split(unsigned char *stage, int A_PART, int row, int h, const float (&v)[XT_HV])
{
#pragma unroll
    for (int kb = 0; kb < XT_HV / 8; ++kb) {
        float x[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = v[8 * kb + i];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            unsigned w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const __nv_bfloat162 b = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
                w[i] = *reinterpret_cast<const unsigned *>(&b);
                if (p + 1 < NP) {   // what this part left
                    const float2 f = __bfloat1622float2(b);
                    x[2 * i] -= f.x;
                    x[2 * i + 1] -= f.y;
                }
            }
            *reinterpret_cast<uint4 *>(stage + p * A_PART + kmaj_off(row, 8 * (2 * h + kb))) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

__device__ __forceinline__ void ld_half(const float *p, float (&v)[XT_HV])
{
#pragma unroll
    for (int i = 0; i < XT_HV / 4; ++i) {
        const float4 q = reinterpret_cast<const float4 *>(p)[i];
        v[4 * i] = q.x;
        v[4 * i + 1] = q.y;
        v[4 * i + 2] = q.z;
        v[4 * i + 3] = q.w;
    }
}

__device__ __forceinline__ void st_half(float *p, const float (&v)[XT_HV])
{
#pragma unroll
    for (int i = 0; i < XT_HV / 4; ++i)
        reinterpret_cast<float4 *>(p)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}

// XT_HV accumulator columns of this thread's lane, in two steps: tld_issue starts
// the load (warp-collective: the warp reconverges first), tld_wait waits for every
// load this thread started and ties the registers to that wait, so that no read
// of them is scheduled before it.
__device__ __forceinline__ void tld_issue(unsigned taddr, unsigned (&r)[XT_HV])
{
    __syncwarp();
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
}

__device__ __forceinline__ void tld_wait(unsigned (&r)[XT_HV])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
}

__device__ __forceinline__ void tld_wait(unsigned (&r)[XT_HV], unsigned (&r2)[XT_HV])
{
    tld_wait(r);
    asm volatile("" : "+r"(r2[0]), "+r"(r2[1]), "+r"(r2[2]), "+r"(r2[3]), "+r"(r2[4]), "+r"(r2[5]), "+r"(r2[6]),
                 "+r"(r2[7]), "+r"(r2[8]), "+r"(r2[9]), "+r"(r2[10]), "+r"(r2[11]), "+r"(r2[12]), "+r"(r2[13]),
                 "+r"(r2[14]), "+r"(r2[15]));
}


__device__ __forceinline__ void tst(unsigned taddr, const float (&v)[XT_HV])
{
    __syncwarp();
    tc::st16(taddr, v);
}

template <int N, int NP>
__global__ void __launch_bounds__(XT_THREADS, 1) k_rows_tc(CurveDev c, int mode, StepArm arm)
{
    using Cfg = XtCfg<N, NP>;
    constexpr int H = N / 2, NW = XT_THREADS / 32;
    extern __shared__ __align__(1024) unsigned char smem_x[];
    unsigned char *As = smem_x;                                        // [2][NP][A_PART]
    unsigned char *Bs = smem_x + XT_ASTAGES * Cfg::A_STAGE;           // [3][NP][B_PART]
    // full_b: a DFT-matrix chunk has landed; a_full: an operand chunk is written
    // (XT_PROD arrivals); mma_done: the products of a chunk are complete (commit)
    __shared__ __align__(8) unsigned long long full_b[XT_BSTAGES], mma_done[XT_BSTAGES], a_full[XT_ASTAGES];
    __shared__ unsigned tmem_slot;
    __shared__ int sbad;   // a bounded wait gave up: no more copies or products are issued
    __shared__ float tk[H], ta[H];
    __shared__ float hsum[XT_M][5];
    __shared__ double wpart[NW][5];
    __shared__ int am_last;
    DevScalars *sc = c.sc;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool issuer = warp == XT_PROD / 32;
    // producers: section row r (TMEM lane 32 (warp % 4) + lane), column half h of every chunk
    const int r = 32 * (warp & 3) + lane, h = (warp >> 2) & 1, co = h * XT_HV;
    const int blk = blockIdx.x, nblk = gridDim.x;
    const int ns = c.ns, P = c.P;
    const int m = blk * XT_M + r;
    const bool has = !issuer && m < ns, in = has && m > 0 && m < P;
    const float *U = (const float *)c.U, *D = (const float *)c.D;
    float *R = (float *)c.R, *A = (float *)c.A;
    const unsigned char *xdft = (const unsigned char *)c.xdft;

    // tables written at set-up (before the programmatic wait)
    for (int j = tid; j < H; j += XT_THREADS) {
        tk[j] = ((const float *)c.kj)[j];
        ta[j] = ((const float *)c.aj)[j];
    }
    const double wm = has ? c.w[m] : 0.0;
    pdl_wait();
    const int g_done = arm.on ? 0 : sc->done;
    const long long g_step = sc->step, g_limit = arm.on ? g_step + arm.nsteps : sc->limit;
    const double lamd = sc->lambda;
    const long long wb = wait_bound(*sc);
    if (arm.on && blk == 0 && tid == 0) {
        sc->limit = g_limit;
        sc->tol = arm.tol;
        sc->done = 0;
        sc->status = 0;
    }
    if (mode == ROWS_STEP && (g_done || g_step >= g_limit)) {
        if (blk == 0 && tid == 0) sc->active = 0;
        return;
    }

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::su32(&tmem_slot)),
                     "r"(Cfg::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < XT_BSTAGES; ++i) {
            tc::bar_init(&full_b[i], 1);
            tc::bar_init(&mma_done[i], 1);
        }
        for (int i = 0; i < XT_ASTAGES; ++i) tc::bar_init(&a_full[i], XT_PROD);
        sbad = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const unsigned tmem = tmem_slot;
    volatile int *vbad = &sbad;
    float s[5] = {0.f, 0.f, 0.f, 0.f, 0.f};   // row sums |r|^2, |d|^2, <d,r>, |u|^2, |f|^2 (Parseval weights)

    if (issuer) {
        // ---- the chunk stream: product q / NCH (C, E, C, E), K-chunk q % NCH.  One
        // thread: bulk copy of each DFT-matrix chunk two ahead, the products of each
        // chunk once its operand chunk and matrix chunk are in, a commit per chunk.
        if (lane == 0) {
            constexpr unsigned IDESC = tc::idesc_bf16(XT_M, N);
            auto issue_b = [&](int q) {
                const int X = (q / Cfg::NCH) & 1, cch = q % Cfg::NCH, sb = q % XT_BSTAGES;
                tc::bulk_g2s(Bs + sb * Cfg::B_STAGE, xdft + (size_t)((X * Cfg::NCH + cch) * XT_PARTS) * Cfg::B_PART,
                             (unsigned)Cfg::B_STAGE, &full_b[sb]);
            };
            bool ok = true;
            int issued_b = 1, waited_b = -1;
            issue_b(0);
            issue_b(1);
            for (int q = 0; q < Cfg::QTOT; ++q) {
                const int g = q / Cfg::NCH, cch = q % Cfg::NCH, sa = q & 1, sb = q % XT_BSTAGES;
                ok = ok && !*vbad;
                if (ok && !tc::bar_wait(&a_full[sa], (q >> 1) & 1, wb)) ok = false;
                if (ok && !tc::bar_wait(&full_b[sb], (q / XT_BSTAGES) & 1, wb)) ok = false;
                if (ok) {
                    waited_b = q;
                    tc::fence_after();
                    const unsigned dcol = tmem + (g == 0 ? 0u : (unsigned)N);
                    const unsigned char *a0 = As + sa * Cfg::A_STAGE, *b0 = Bs + sb * Cfg::B_STAGE;
#pragma unroll
                    for (int s = 0; s < XT_KC / 16; ++s) {
                        // part pairs, smallest first: (0,2) (1,1) (2,0) (0,1) (1,0) (0,0)
                        constexpr int npair = NP == 3 ? 6 : 3;
                        constexpr int pa3[6] = {0, 1, 2, 0, 1, 0}, pb3[6] = {2, 1, 0, 1, 0, 0};
                        constexpr int pa2[3] = {0, 1, 0}, pb2[3] = {1, 0, 0};
#pragma unroll
                        for (int t = 0; t < npair; ++t) {
                            const int pa = NP == 3 ? pa3[t] : pa2[t], pb = NP == 3 ? pb3[t] : pb2[t];
                            const unsigned long long ad = tc::sdesc(a0 + pa * Cfg::A_PART + 256 * s, 128, XT_SBO);
                            const unsigned long long bd = tc::sdesc(b0 + pb * Cfg::B_PART + 256 * s, 128, XT_SBO);
                            tc::mma_f16(dcol, ad, bd, IDESC, (cch > 0 || s > 0 || t > 0) ? 1 : 0);
                        }
                    }
                } else if (!*vbad) {
                    *vbad = 1;
                    atomicExch(&sc->err, 4);
                }
                tc::commit(&mma_done[sb]);   // also when nothing was issued: keeps the phases in step
                // matrix chunk q + 2 into the stage of chunk q - 1, once its products are done
                if (ok && q + 2 < Cfg::QTOT) {
                    if (q >= 1 && !tc::bar_wait(&mma_done[(q - 1) % XT_BSTAGES], ((q - 1) / XT_BSTAGES) & 1, wb)) {
                        ok = false;
                        *vbad = 1;
                        atomicExch(&sc->err, 4);
                    } else {
                        issue_b(q + 2);
                        issued_b = q + 2;
                    }
                }
            }
            // copies that may still be landing (after a wait gave up), and the last products
            for (int qq = waited_b + 1; qq <= issued_b; ++qq) tc::bar_wait(&full_b[qq % XT_BSTAGES], (qq / XT_BSTAGES) & 1);
            tc::bar_wait(&mma_done[(Cfg::QTOT - 1) % XT_BSTAGES], ((Cfg::QTOT - 1) / XT_BSTAGES) & 1);
        }
        __syncwarp();
    } else {
        // ---- producers: operand chunks, and the pointwise work between the products
        const unsigned lane_base = tmem + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)co;
        const float lam = (float)lamd;
        const size_t ro = (size_t)(has ? m : 0) * N + co;
        const float *Urow = U + ro, *Drow = D + ro;
        float *Rrow = R + ro, *Arow = A + ro;
        auto fail = [&]() {
            if (!*vbad) {
                *vbad = 1;
                atomicExch(&sc->err, 4);
            }
        };

        // one product.  `fetch(cch, buf)` starts loading what chunk cch of this
        // thread's half row needs, one chunk ahead; `ready(buf)` completes it;
        // `produce(cch, buf, v)` turns it into operand values.
        // Chunks are taken in pairs with two buffers (b0 for even chunks, b1 for odd
        // ones): a buffer whose TMEM load is in flight is never read or copied
        // before `ready` has waited for it.
        int q = 0;
        auto product = [&](auto &&fetch, auto &&ready, auto &&produce) {
            auto chunk = [&](int cch, unsigned (&b)[XT_HV]) {
                const int sa = q & 1;
                // the operand stage of chunk q - 2 is free once its products are done
                if (q >= 2 && !*vbad && !tc::bar_wait(&mma_done[(q - 2) % XT_BSTAGES], ((q - 2) / XT_BSTAGES) & 1, wb))
                    fail();
                float v[XT_HV];
                produce(cch, b, v);
                if (!has) {
#pragma unroll
                    for (int i = 0; i < XT_HV; ++i) v[i] = 0.f;
                }
                put_split<NP>(As + sa * Cfg::A_STAGE, Cfg::A_PART, r, h, v);
                tc::fence_async_smem();   // the generic writes, before the products read them
                tc::fence_before();       // and this thread's TMEM reads, before later products write
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::su32(&a_full[sa])) : "memory");
                ++q;
            };
            static_assert(Cfg::NCH % 2 == 0, "chunks are taken in pairs");
            unsigned b0[XT_HV], b1[XT_HV];
            fetch(0, b0);
#pragma unroll 1
            for (int cch = 0; cch < Cfg::NCH; cch += 2) {
                ready(b0);
                fetch(cch + 1, b1);
                chunk(cch, b0);
                ready(b1);
                if (cch + 2 < Cfg::NCH) fetch(cch + 2, b0);
                chunk(cch + 1, b1);
            }
            // the product is complete once its last chunk's mbarrier has fired
            const int ql = q - 1;
            if (!*vbad && !tc::bar_wait(&mma_done[ql % XT_BSTAGES], (ql / XT_BSTAGES) & 1, wb)) fail();
            tc::fence_after();
        };
        auto fetch_row = [&](const float *row) {
            return [row, has = has](int cch, unsigned (&b)[XT_HV]) {
                float t[XT_HV];
                if (has) ld_half(row + cch * XT_KC, t);
                else {
#pragma unroll
                    for (int i = 0; i < XT_HV; ++i) t[i] = 0.f;
                }
#pragma unroll
                for (int i = 0; i < XT_HV; ++i) b[i] = __float_as_uint(t[i]);
            };
        };
        auto no_wait = [](unsigned (&)[XT_HV]) {};
        auto fetch_t0 = [&](int cch, unsigned (&b)[XT_HV]) { tld_issue(lane_base + cch * XT_KC, b); };
        auto wait_t = [](unsigned (&b)[XT_HV]) { tld_wait(b); };
        // first mode of this thread's half of chunk cch
        auto mode0 = [&](int cch) { return cch * (XT_KC / 2) + h * (XT_HV / 2); };

        // ---- G1: u = uh C
        product(fetch_row(Urow), no_wait, [&](int cch, const unsigned (&b)[XT_HV], float (&v)[XT_HV]) {
#pragma unroll
            for (int i = 0; i < XT_HV; ++i) v[i] = __uint_as_float(b[i]);
            if (cch == 0 && h == 0) v[1] = 0.f;
        });
        // ---- G2: wh = (u u) E
        product(fetch_t0, wait_t, [&](int, const unsigned (&b)[XT_HV], float (&v)[XT_HV]) {
#pragma unroll
            for (int i = 0; i < XT_HV; ++i) {
                const float x = __uint_as_float(b[i]);
                v[i] = x * x;
            }
        });
        // ---- f^, r^ = f^ - l d^, row sums; r^ out (the next chunk's u^, d^ and
        // accumulator columns in flight)
        {
            auto fu = fetch_row(Urow), fd = fetch_row(Drow);
            auto step = [&](int cch, const unsigned (&u)[XT_HV], const unsigned (&d)[XT_HV], const unsigned (&wr)[XT_HV]) {
                float rv[XT_HV];
                const int j0 = mode0(cch);
#pragma unroll
                for (int i = 0; i < XT_HV / 2; ++i) {
                    const int j = j0 + i;
                    const float k = tk[j], a = ta[j], hk = 0.5f * k;
                    const float wre = __uint_as_float(wr[2 * i]), wim = __uint_as_float(wr[2 * i + 1]);
                    const float ur = __uint_as_float(u[2 * i]), ui = j == 0 ? 0.f : __uint_as_float(u[2 * i + 1]);
                    const float dr = __uint_as_float(d[2 * i]), di = j == 0 ? 0.f : __uint_as_float(d[2 * i + 1]);
                    const float fr = hk * wim - a * ur, fi = j == 0 ? 0.f : -hk * wre - a * ui;
                    cpx<float> rr = {0.f, 0.f};
                    if (in) rr = project(cpx<float>{fr - lam * dr, fi - lam * di}, j, c.sym);
                    if (j == 0) rr.y = 0.f;
                    rv[2 * i] = rr.x;
                    rv[2 * i + 1] = rr.y;
                    const float cw = j == 0 ? 1.f : 2.f;
                    s[0] += cw * (rr.x * rr.x + rr.y * rr.y);
                    s[1] += cw * (dr * dr + di * di);
                    s[2] += cw * (dr * rr.x + di * rr.y);
                    s[3] += cw * (ur * ur + ui * ui);
                    s[4] += cw * (fr * fr + fi * fi);
                }
                if (has) st_half(Rrow + cch * XT_KC, rv);
            };
            unsigned u0[XT_HV], d0[XT_HV], w0[XT_HV], u1[XT_HV], d1[XT_HV], w1[XT_HV];
            fu(0, u0);
            fd(0, d0);
            tld_issue(lane_base + N, w0);
#pragma unroll 1
            for (int cch = 0; cch < Cfg::NCH; cch += 2) {
                tld_wait(w0);
                fu(cch + 1, u1);
                fd(cch + 1, d1);
                tld_issue(lane_base + N + (cch + 1) * XT_KC, w1);
                step(cch, u0, d0, w0);
                tld_wait(w1);
                if (cch + 2 < Cfg::NCH) {
                    fu(cch + 2, u0);
                    fd(cch + 2, d0);
                    tld_issue(lane_base + N + (cch + 2) * XT_KC, w0);
                }
                step(cch + 1, u1, d1, w1);
            }
        }
        if (h == 1) {
#pragma unroll
            for (int k = 0; k < 5; ++k) hsum[r][k] = s[k];
        }
        // ---- G3: r_x = (i k r^) C   (r^ as just written by this thread)
        product(fetch_row(Rrow), no_wait, [&](int cch, const unsigned (&rb)[XT_HV], float (&v)[XT_HV]) {
            const int j0 = mode0(cch);
#pragma unroll
            for (int i = 0; i < XT_HV / 2; ++i) {
                const float k = tk[j0 + i];
                v[2 * i] = -k * __uint_as_float(rb[2 * i + 1]);
                v[2 * i + 1] = k * __uint_as_float(rb[2 * i]);
            }
        });
        // ---- y = u r_x into T0 (the next chunk's columns in flight)
        {
            auto step = [&](int cch, const unsigned (&ua)[XT_HV], const unsigned (&xa)[XT_HV]) {
                float y[XT_HV];
#pragma unroll
                for (int i = 0; i < XT_HV; ++i) y[i] = __uint_as_float(ua[i]) * __uint_as_float(xa[i]);
                tst(lane_base + cch * XT_KC, y);
            };
            unsigned u0[XT_HV], x0[XT_HV], u1[XT_HV], x1[XT_HV];
            tld_issue(lane_base, u0);
            tld_issue(lane_base + N, x0);
#pragma unroll 1
            for (int cch = 0; cch < Cfg::NCH; cch += 2) {
                tld_wait(u0, x0);
                tld_issue(lane_base + (cch + 1) * XT_KC, u1);
                tld_issue(lane_base + N + (cch + 1) * XT_KC, x1);
                step(cch, u0, x0);
                tld_wait(u1, x1);
                if (cch + 2 < Cfg::NCH) {
                    tld_issue(lane_base + (cch + 2) * XT_KC, u0);
                    tld_issue(lane_base + N + (cch + 2) * XT_KC, x0);
                }
                step(cch + 1, u1, x1);
            }
            tc::wait_st();
        }
        // ---- G4: p^ = y E
        product(fetch_t0, wait_t, [&](int, const unsigned (&b)[XT_HV], float (&v)[XT_HV]) {
#pragma unroll
            for (int i = 0; i < XT_HV; ++i) v[i] = __uint_as_float(b[i]);
        });
        // ---- A^ = p^ - a_j r^ (the next chunk's r^ and columns in flight)
        {
            auto fr = fetch_row(Rrow);
            auto step = [&](int cch, const unsigned (&rb)[XT_HV], const unsigned (&pr)[XT_HV]) {
                float ph[XT_HV];
                const int j0 = mode0(cch);
#pragma unroll
                for (int i = 0; i < XT_HV / 2; ++i) {
                    const int j = j0 + i;
                    const float a = ta[j];
                    cpx<float> av = project(cpx<float>{__uint_as_float(pr[2 * i]) - a * __uint_as_float(rb[2 * i]),
                                                       __uint_as_float(pr[2 * i + 1]) - a * __uint_as_float(rb[2 * i + 1])},
                                            j, c.sym);
                    if (j == 0) av.y = 0.f;
                    ph[2 * i] = av.x;
                    ph[2 * i + 1] = av.y;
                }
                if (has) st_half(Arow + cch * XT_KC, ph);
            };
            unsigned r0[XT_HV], p0[XT_HV], r1[XT_HV], p1[XT_HV];
            fr(0, r0);
            tld_issue(lane_base + N, p0);
#pragma unroll 1
            for (int cch = 0; cch < Cfg::NCH; cch += 2) {
                tld_wait(p0);
                fr(cch + 1, r1);
                tld_issue(lane_base + N + (cch + 1) * XT_KC, p1);
                step(cch, r0, p0);
                tld_wait(p1);
                if (cch + 2 < Cfg::NCH) {
                    fr(cch + 2, r0);
                    tld_issue(lane_base + N + (cch + 2) * XT_KC, p0);
                }
                step(cch + 1, r1, p1);
            }
        }
        tc::fence_before();
    }

    // ---- every product is done and every TMEM access complete: free TMEM
    __syncthreads();
    tc::fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::TMEM_COLS) : "memory");

    // ---- per-section FP64 terms (|q_m|^2 = L sum_j c_j |q^_j|^2; the two halves'
    // sums added lower half first), CTA partials
    double t[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (has && h == 0) {
        float st[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) st[k] = s[k] + hsum[r][k];
        const double L = c.L, nr = L * st[0], nd = L * st[1], ndr = L * st[2];
        const double al = fabs(lamd), sd = sqrt(nd);
        if (in) {
            t[0] = wm * nr;
            t[1] = wm * sqrt(nr) * al * sd;
            t[2] = wm * al * sd;
            t[3] = wm * ndr;
            t[4] = wm * lamd * lamd * nd;
        }
        double *rs = c.rowsc + (size_t)m * 4;
        rs[0] = in ? nr : L * st[3];
        rs[1] = nd;
        rs[2] = ndr;
        rs[3] = L * st[4];
    }
    {
        const double ws = warp_sum5(t, lane);
        const int v = (lane >> 2) & 7;
        if ((lane & 3) == 0 && v < 5) wpart[warp][v] = ws;
    }
    __syncthreads();
    if (tid < 5) {
        double tt = 0.0;
#pragma unroll
        for (int w = 0; w < NW; ++w) tt += wpart[w][tid];
        c.bpart[(size_t)blk * 5 + tid] = tt;
    }
    // ---- last CTA: the FP64 reduction over the CTAs' partial sums
    if (!last_cta_arrive(&sc->cnt_rows, (unsigned)nblk, am_last)) return;
    rows_finish<XT_THREADS>(c, mode, nblk, true, arm);
}

// Set-up: the DFT matrices C (inverse) and E (forward, with 1/N) split into three
// BF16 parts from FP64 values (trig of exact integer angles j n mod N), stored
// per (matrix, K-chunk, part) in the K-major operand layout of one B chunk.
template <int N>
__global__ void k_setup_xdft(CurveDev c)
{
    constexpr int NCH = N / XT_KC, B_PART = N * XT_KC * 2;
    unsigned char *out = (unsigned char *)c.xdft;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * N * N; e += gridDim.x * blockDim.x) {
        const int X = e / (N * N), nout = (e / N) % N, kin = e % N;
        const int i = X == 0 ? kin : nout, n = X == 0 ? nout : kin;   // spectral word, grid point
        const int j = i >> 1;
        double v = 0.0;
        if (i != 1) {
            double s, co;
            sincospi(2.0 * (double)((j * n) % N) / (double)N, &s, &co);
            const double t = (i & 1) ? -s : co;
            v = X == 0 ? (j ? 2.0 : 1.0) * t : t / (double)N;
        }
        const int cch = kin / XT_KC, k = kin % XT_KC;
        const int off = (nout >> 3) * XT_SBO + (k >> 3) * 128 + (nout & 7) * 16 + (k & 7) * 2;
        double rem = v;
#pragma unroll
        for (int p = 0; p < XT_PARTS; ++p) {
            const __nv_bfloat16 h = __float2bfloat16_rn((float)rem);
            rem -= (double)__bfloat162float(h);
            *reinterpret_cast<__nv_bfloat16 *>(out + (size_t)((X * NCH + cch) * XT_PARTS + p) * B_PART + off) = h;
        }
    }
}

template <int N, int NP>
cudaError_t rows_tc_run(const CurveDev &c, int mode, cudaStream_t st, StepArm arm)
{
    using Cfg = XtCfg<N, NP>;
    cudaError_t e = set_smem(k_rows_tc<N, NP>, Cfg::SMEM);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((c.ns + XT_M - 1) / XT_M);
    cfg.blockDim = dim3(XT_THREADS);
    cfg.dynamicSmemBytes = Cfg::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_rows_tc<N, NP>, c, mode, arm);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace

size_t xdft_bytes(int nx) { return (size_t)2 * XT_PARTS * nx * nx * 2; }

cudaError_t launch_setup_xdft(const CurveDev &c, cudaStream_t st)
{
    const int total = 2 * c.nx * c.nx, grid = (total + 255) / 256;
    switch (c.nx) {
    case 64: k_setup_xdft<64><<<grid, 256, 0, st>>>(c); break;
    case 128: k_setup_xdft<128><<<grid, 256, 0, st>>>(c); break;
    case 256: k_setup_xdft<256><<<grid, 256, 0, st>>>(c); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_rows_tc(const CurveDev &c, int mode, cudaStream_t st, StepArm arm)
{
    const bool three = c.xtc == 3;
    switch (c.nx) {
    case 64: return three ? rows_tc_run<64, 3>(c, mode, st, arm) : rows_tc_run<64, 2>(c, mode, st, arm);
    case 128: return three ? rows_tc_run<128, 3>(c, mode, st, arm) : rows_tc_run<128, 2>(c, mode, st, arm);
    case 256: return three ? rows_tc_run<256, 3>(c, mode, st, arm) : rows_tc_run<256, 2>(c, mode, st, arm);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ks
