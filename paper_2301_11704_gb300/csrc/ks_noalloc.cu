// ks_noalloc.cu -- ks_cost_noalloc: the cost of a curve computed without any
// device allocation, for callers that cannot allocate device memory.
//
// Who needs this: a host program that embeds this library but owns every
// device allocation itself and hands over only input and output buffers; a
// time-critical loop in which cudaMalloc (with its implicit synchronisation and
// unbounded latency) is not acceptable; a process whose device memory is fully
// reserved up front.  Such a caller cannot provide the workspace that
// ks_curve_create needs, so this entry point keeps its scratch in one
// statically sized device array that the CUDA runtime sets up when the
// library's module is loaded on a device.
//
// The scratch array (KS_NOALLOC_SCRATCH_BYTES) is held on every device that
// loads this library until the process exits.  All calls share it and it keeps
// the last call's contents: each call rewrites everything it reads (tables,
// spectral fields, and the reduction scalars and arrival counters, which are
// cleared before use), and calls that overlap on the GPU -- on two streams, or
// from two threads -- race on it and give wrong results.
#include <cmath>

#include "../../include/ksconn.h"
#include "ks_internal.h"

static __device__ __align__(256) unsigned char g_noalloc_scratch[KS_NOALLOC_SCRATCH_BYTES];

namespace {

// J^2 and J_arc of the evaluation, or NaN in both when a bounded device-side
// wait of one of its kernels gave up (sc->err set): the launch's results are
// then invalid, and the caller sees it in the outputs instead of a wrong cost.
__global__ void k_export_cost(const ks::DevScalars *sc, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const bool bad = sc->err != 0;
        out[0] = bad ? __longlong_as_double(0x7ff8000000000000ll) : sc->J2;
        out[1] = bad ? __longlong_as_double(0x7ff8000000000000ll) : sc->Jarc;
    }
}

ks_status na_fail(ks_status s, const char *what, cudaError_t e)
{
    return ks::report_error(s, "ks_cost_noalloc: %s: %s", what, cudaGetErrorString(e));
}

}  // namespace

extern "C" ks_status ks_cost_noalloc(const ks_params *p, const void *u_dev, double *out_dev, void *stream)
{
    if (!p || !u_dev || !out_dev)
        return ks::report_error(KS_EINVAL, "ks_cost_noalloc: p, u_dev and out_dev are required");
    ks_status s = ks::check_params(p);
    if (s != KS_OK) return s;
    const ks::Layout lay = ks::curve_layout(p, 0);
    if (lay.total > (size_t)KS_NOALLOC_SCRATCH_BYTES)
        return ks::report_error(KS_ENOMEM,
                                "ks_cost_noalloc: a %d x %d curve needs %zu bytes of scratch; the built-in array holds %zu",
                                p->ns, p->nx, lay.total, (size_t)KS_NOALLOC_SCRATCH_BYTES);
    // Device address of the scratch array, looked up on every call with the
    // caller's device current.  In host code the array's name is only a host-side
    // stand-in; the address belongs to the module loaded in the current context,
    // and a cached one would go stale once that context is reset and the module
    // loaded again (the lookup is cheap once the module is loaded).
    void *base = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
    if (e != cudaSuccess) return na_fail(KS_ECUDA, "cudaGetSymbolAddress", e);
    if (!base) return ks::report_error(KS_ECUDA, "ks_cost_noalloc: cudaGetSymbolAddress returned a null address");

    const ks::CurveDev d = ks::bind_layout(p, lay, base);

    cudaStream_t st = (cudaStream_t)stream;
    // tables, then the scalars and arrival counters (cleared: they must start at zero)
    if ((e = ks::launch_setup(d, p->dtau, st)) != cudaSuccess) return na_fail(KS_ECUDA, "set-up kernel", e);
    if ((e = ks::launch_scalars_init(d, p->lambda, 0, p->dtau, 0.0, p->conv, st)) != cudaSuccess)
        return na_fail(KS_ECUDA, "scalar reset", e);
    // u (storage type, physical) -> FP64 scratch -> spectral state
    if ((e = ks::launch_widen(d, u_dev, st)) != cudaSuccess) return na_fail(KS_ECUDA, "widen", e);
    if ((e = ks::launch_row_fwd_x(d, d.U, 0, st)) != cudaSuccess) return na_fail(KS_ECUDA, "forward transform", e);
    // D_t u, then the row phase with the FP64 cost reduction
    if ((e = ks::launch_dt(d, ks::GM_STORE, 0, 0, st)) != cudaSuccess) return na_fail(KS_ECUDA, "D_t u", e);
    if ((e = ks::launch_rows(d, ks::ROWS_EVAL, st)) != cudaSuccess) return na_fail(KS_ECUDA, "row phase", e);
    k_export_cost<<<1, 32, 0, st>>>(d.sc, out_dev);
    if ((e = cudaGetLastError()) != cudaSuccess) return na_fail(KS_ECUDA, "export", e);
    return KS_OK;
}
