// ks_capi.cu -- the C ABI declared in include/ksconn.h: argument checks,
// workspace layout, and the order of kernel launches for each entry point.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ksconn.h"
#include "ks_internal.h"

struct ks_curve {
    ks_params p;
    ks::Layout lay;
    ks::CurveDev d;
    cudaStream_t st;
    int device;
    // profiling: events[EV_PER_ENTRY * entry + 2 * phase] / [.. + 1] bracket one
    // phase; [.. + 6], [.. + 7] (update) and [.. + 8], [.. + 9] (D_t u) mark the
    // ends of the first two passes of the three-launch four-step form; an entry
    // is a kernel-per-phase step (prof_steps = 0) or a persistent launch of
    // prof_steps steps (phase 0 only)
    std::vector<cudaEvent_t> events;
    std::vector<int64_t> prof_steps;
    int prof_cap = 0;      // entries that fit in `events`
    int prof_used = 0;     // entries recorded so far
    // CUDA graph of GRAPH_STEPS descent steps, captured once on a private stream
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t gstream = nullptr;
    int gdiscrete = -1;
    // tensor maps of U and D_t U for the FFT row phase's tile loads (d.rowmaps)
    ks::RowMaps rmaps{};
    // pinned host copy of the scalars at the start of a descend call (read back
    // with the final ones, one synchronisation per call)
    ks::DevScalars *h0 = nullptr;
};

static const int GRAPH_STEPS = 16;
static const int EV_PER_ENTRY = 12;

static thread_local char g_err[512];

static ks_status fail(ks_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

#define KS_CUDA(call)                                                                           \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return fail(KS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

namespace {

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

ks_status validate(const ks_params *p)
{
    if (!p) return fail(KS_EINVAL, "params is NULL");
    if (!(p->L > 0) || !std::isfinite(p->L)) return fail(KS_EINVAL, "L must be finite and > 0 (got %g)", p->L);
    if (!is_pow2(p->nx) || p->nx < 8 || p->nx > 256)
        return fail(KS_EINVAL, "nx must be a power of two in [8, 256] (got %d)", p->nx);
    if (p->ns < 3 || p->ns > 65536) return fail(KS_EINVAL, "ns must be in [3, 65536] (got %d)", p->ns);
    if (!(p->S > 0) || !std::isfinite(p->S)) return fail(KS_EINVAL, "S must be finite and > 0 (got %g)", p->S);
    if (!std::isfinite(p->s0)) return fail(KS_EINVAL, "s0 must be finite");
    if (!std::isfinite(p->lambda)) return fail(KS_EINVAL, "lambda must be finite");
    if (!(p->dtau > 0) || !std::isfinite(p->dtau)) return fail(KS_EINVAL, "dtau must be finite and > 0 (got %g)", p->dtau);
    if (!(p->dtau_lambda >= 0) || !std::isfinite(p->dtau_lambda)) return fail(KS_EINVAL, "dtau_lambda must be finite and >= 0");
    if (p->lambda_free != 0 && p->lambda_free != 1) return fail(KS_EINVAL, "lambda_free must be 0 or 1");
    if (p->precision < KS_FP64 || p->precision > KS_BF16X3)
        return fail(KS_EINVAL, "precision must be KS_FP64, KS_FP32, KS_BF16X2 or KS_BF16X3");
    if (ks::xtc_of(p->precision) && p->nx != 64 && p->nx != 128 && p->nx != 256)
        return fail(KS_EINVAL, "split-BF16 x-transforms need nx in {64, 128, 256} (got %d)", p->nx);
    if (p->adjoint != KS_ADJ_PAPER && p->adjoint != KS_ADJ_DISCRETE) return fail(KS_EINVAL, "adjoint must be KS_ADJ_PAPER or KS_ADJ_DISCRETE");
    if (p->conv < KS_CONV_JARC || p->conv > KS_CONV_JREL) return fail(KS_EINVAL, "conv must be a ks_conv value");
    if (p->check_ends != 0 && p->check_ends != 1) return fail(KS_EINVAL, "check_ends must be 0 or 1");
    if (p->symmetry < 0 || p->symmetry > 7) return fail(KS_EINVAL, "symmetry must be in [0, 7]");
    if (p->symmetry & KS_SYM_SINE) {
        if (!(p->symmetry & KS_SYM_ODD)) return fail(KS_EINVAL, "sine storage (symmetry bit 2) needs odd sections (bit 0)");
        if (p->nx < 16) return fail(KS_EINVAL, "sine storage needs nx >= 16 (got %d)", p->nx);
        if (p->precision != KS_FP64 && p->precision != KS_FP32)
            return fail(KS_EINVAL, "sine storage needs precision KS_FP64 or KS_FP32 (the FFT row phase)");
        if (p->s_transform == 3) return fail(KS_EINVAL, "sine storage takes s_transform 0, 1, 2, 4 or 5");
        if (p->launch != 0 || p->scheme != KS_SCHEME_IMEX)
            return fail(KS_EINVAL, "sine storage needs launch = 0 and scheme KS_SCHEME_IMEX");
    }
    if (p->s_transform < 0 || p->s_transform > 5) return fail(KS_EINVAL, "s_transform must be in [0, 5]");
    if ((p->s_transform == 4 || p->s_transform == 5) && ks::fft4_size(p->ns, ks::storage32(p->precision), 1) == 0)
        return fail(KS_EINVAL, "s_transform = four-step FFT needs %d <= 3 (N_s - 1) <= %d (rounded up to a power of two)",
                    ks::F4_FMIN / 2 + 1, ks::F4_FMAX);
    if (p->s_transform == 5) {
        int F1 = 0, F2 = 0;
        ks::f4_split(ks::fft4_size(p->ns, ks::storage32(p->precision), 1), F1, F2);
        if (!ks::f4c_fits(ks::storage32(p->precision), F1, F2))
            return fail(KS_EINVAL, "s_transform = clustered four-step FFT holds F <= 32768 in FP64 (N_s <= 10923)");
    }
    if (p->s_transform == 3 && !ks::storage32(p->precision))
        return fail(KS_EINVAL, "s_transform = tensor cores needs FP32 storage");
    if (p->launch < 0 || p->launch > 1) return fail(KS_EINVAL, "launch must be 0 or 1");
    if (p->scheme != KS_SCHEME_IMEX && p->scheme != KS_SCHEME_IMPLICIT)
        return fail(KS_EINVAL, "scheme must be KS_SCHEME_IMEX or KS_SCHEME_IMPLICIT");
    if (p->scheme == KS_SCHEME_IMPLICIT && (p->launch != 0 || p->ns < 4 || p->ns > 16384))
        return fail(KS_EINVAL, "implicit stepping needs launch = 0 and 4 <= N_s <= 16384");
    if (p->s_transform == 2 && ks::fft_size(p->ns, ks::storage32(p->precision)) == 0 &&
        ks::fft4_size(p->ns, ks::storage32(p->precision)) == 0)
        return fail(KS_EINVAL, "s_transform = FFT supports N_s <= %d", ks::F4_FMAX / 3 + 1);
    return KS_OK;
}

ks::CurveDev make_dev(const ks_params *p, const ks::Layout &l, void *ws) { return ks::bind_layout(p, l, ws); }

ks_status check_handle(ks_curve *c)
{
    if (!c) return fail(KS_EINVAL, "curve handle is NULL");
    return KS_OK;
}

// D_t u of the current state (kept in the workspace for the next evaluation).
ks_status refresh_dt_u(ks_curve *c)
{
    KS_CUDA(ks::launch_dt(c->d, ks::GM_STORE, 0, 0, c->st));
    return KS_OK;
}

ks_status read_scalars(ks_curve *c, ks::DevScalars *h)
{
    KS_CUDA(cudaMemcpyAsync(h, c->d.sc, sizeof(*h), cudaMemcpyDeviceToHost, c->st));
    KS_CUDA(cudaStreamSynchronize(c->st));
    if (h->err) return fail(KS_ETIMEOUT, "a device-side copy did not complete in time; re-initialise the curve");
    return KS_OK;
}

// The clustered four-step form applies the update and D_t u of the updated state
// in one launch (GM_STEP) at the sizes of f4c_fused; every other form in two.
static bool fused_step(const ks_curve *c)
{
    return c->d.f4c != 0 && !c->d.impl && ks::f4c_fused(c->d.prec, c->d.W, c->d.F);
}

// The update of one step: the update contraction (G and |G|^2), and for the
// implicit scheme the two products of its increment.
// D_t u of the updated state in a step: its first pass already ran inside the
// update when the form chains them.
static int store_mode(const ks_curve *c) { return ks::f4h_chained(c->d) ? ks::GM_STORE_P23 : ks::GM_STORE; }

// impl_ev (may be null): two events bracketing the implicit products.
static ks_status launch_update(ks_curve *c, int discrete, cudaStream_t st, cudaEvent_t *pass_ev,
                               cudaEvent_t *impl_ev = nullptr)
{
    if (!c->d.impl) {
        const int um = fused_step(c) ? ks::GM_STEP : (ks::f4h_chained(c->d) ? ks::GM_UPDATE_F : ks::GM_UPDATE);
        KS_CUDA(ks::launch_dt(c->d, um, discrete, 1, st, pass_ev));
        return KS_OK;
    }
    KS_CUDA(ks::launch_dt(c->d, ks::GM_GRAD, discrete, 1, st, pass_ev));
    if (impl_ev) KS_CUDA(cudaEventRecord(impl_ev[0], st));
    KS_CUDA(ks::launch_implicit_update(c->d, 1, st));
    if (impl_ev) KS_CUDA(cudaEventRecord(impl_ev[1], st));
    return KS_OK;
}
// The three-launch four-step form, whose passes are timed one by one.
static bool three_pass(const ks_curve *c) { return c->d.f4 && !c->d.f4c && !c->d.f4b; }

ks_status launch_step(ks_curve *c, int discrete, cudaStream_t st)
{
    KS_CUDA(ks::launch_rows(c->d, ks::ROWS_STEP, st));
    ks_status s = launch_update(c, discrete, st, nullptr);
    if (s != KS_OK) return s;
    if (!fused_step(c)) KS_CUDA(ks::launch_dt(c->d, store_mode(c), 0, 1, st));
    return KS_OK;
}

// Captures GRAPH_STEPS steps into an executable graph (once per curve and
// adjoint mode).  Every kernel reads its gates from the device scalars, so the
// same graph serves any step count and stops cleanly at convergence.
ks_status ensure_graph(ks_curve *c, int discrete)
{
    if (c->gexec && c->gdiscrete == discrete) return KS_OK;
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    if (!c->gstream) KS_CUDA(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
    KS_CUDA(cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
    ks_status s = KS_OK;
    for (int i = 0; i < GRAPH_STEPS && s == KS_OK; ++i) s = launch_step(c, discrete, c->gstream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->gstream, &graph);
    if (s != KS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess) return fail(KS_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        c->gexec = nullptr;
        return fail(KS_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    c->gdiscrete = discrete;
    return KS_OK;
}

// Steps per launch of the persistent kernel (a converged curve leaves early).
static const int64_t PERSISTENT_STEPS = 1024;

ks_status enqueue_steps(ks_curve *c, int64_t nsteps, double tol)
{
    const int discrete = c->p.adjoint == KS_ADJ_DISCRETE;
    const bool persistent = c->p.launch == 1 && c->d.part;
    const bool graph = !persistent && c->prof_used >= c->prof_cap && nsteps >= GRAPH_STEPS;
    // the kernel-per-phase loop arms the step limit in its first row phase; the
    // persistent kernel and the graph replay read it as set by k_set_limit
    if (persistent || graph || nsteps <= 0) KS_CUDA(ks::launch_set_limit(c->d, (long long)nsteps, tol, c->st));
    if (persistent) {
        for (int64_t done = 0; done < nsteps; done += PERSISTENT_STEPS) {
            const int64_t n = std::min(PERSISTENT_STEPS, nsteps - done);
            const bool prof = c->prof_used < c->prof_cap;
            cudaEvent_t *ev = prof ? &c->events[(size_t)EV_PER_ENTRY * c->prof_used] : nullptr;
            if (prof) KS_CUDA(cudaEventRecord(ev[0], c->st));
            KS_CUDA(ks::launch_step_persistent(c->d, discrete, (long long)n, c->st));
            if (prof) {
                KS_CUDA(cudaEventRecord(ev[1], c->st));
                c->prof_steps[c->prof_used] = n;
                c->prof_used++;
            }
        }
        return KS_OK;
    }
    if (graph) {
        ks_status s = ensure_graph(c, discrete);
        if (s != KS_OK) return s;
        for (int64_t g = 0; g < nsteps / GRAPH_STEPS; ++g) KS_CUDA(cudaGraphLaunch(c->gexec, c->st));
        for (int64_t r = 0; r < nsteps % GRAPH_STEPS; ++r) {
            s = launch_step(c, discrete, c->st);
            if (s != KS_OK) return s;
        }
        return KS_OK;
    }
    for (int64_t s = 0; s < nsteps; ++s) {
        const bool prof = c->prof_used < c->prof_cap;
        cudaEvent_t *ev = prof ? &c->events[(size_t)EV_PER_ENTRY * c->prof_used] : nullptr;
        cudaEvent_t *pass_u = (prof && three_pass(c)) ? ev + 6 : nullptr, *pass_d = pass_u ? ev + 8 : nullptr;
        if (prof) KS_CUDA(cudaEventRecord(ev[0], c->st));
        const ks::StepArm arm = {(long long)nsteps, tol, s == 0 ? 1 : 0};
        KS_CUDA(ks::launch_rows(c->d, ks::ROWS_STEP, c->st, arm));
        if (prof) KS_CUDA(cudaEventRecord(ev[1], c->st));
        if (prof) KS_CUDA(cudaEventRecord(ev[2], c->st));
        ks_status us = launch_update(c, discrete, c->st, pass_u, (prof && c->d.impl) ? ev + 10 : nullptr);
        if (us != KS_OK) return us;
        if (prof) KS_CUDA(cudaEventRecord(ev[3], c->st));
        if (prof) KS_CUDA(cudaEventRecord(ev[4], c->st));
        if (!fused_step(c)) KS_CUDA(ks::launch_dt(c->d, store_mode(c), 0, 1, c->st, pass_d));
        if (prof) {
            KS_CUDA(cudaEventRecord(ev[5], c->st));
            c->prof_steps[c->prof_used] = 0;
            c->prof_used++;
        }
    }
    return KS_OK;
}

void release_events(ks_curve *c)
{
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    c->events.clear();
    c->prof_steps.clear();
    c->prof_cap = 0;
    c->prof_used = 0;
}

}  // namespace

namespace ks {
// Helpers for other translation units of the library: the same parameter rules
// and the same thread-local message as the entry points of this file.
ks_status check_params(const ks_params *p) { return validate(p); }

ks_status report_error(ks_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}
}  // namespace ks

extern "C" {

const char *ks_last_error(void) { return g_err; }

int32_t ks_version(void) { return (1 << 16) | 0; }

size_t ks_curve_workspace_bytes(const ks_params *p)
{
    if (validate(p) != KS_OK) return 0;
    return ks::curve_layout(p, p->launch == 1).total;
}

int32_t ks_curve_fft_length(const ks_params *p)
{
    if (validate(p) != KS_OK) return -1;
    return ks::curve_layout(p, 0).F;
}

int32_t ks_curve_s_form(const ks_params *p)
{
    if (validate(p) != KS_OK) return -1;
    const ks::Layout l = ks::curve_layout(p, 0);
    if (l.f4) return l.f4c ? 5 : 4;
    if (l.F) return 2;
    return l.tc ? 3 : 1;
}

ks_status ks_curve_create(const ks_params *p, const double *u_plus_host, const double *u_minus_host,
                          const void *u_init_dev, void *workspace_dev, size_t workspace_bytes, void *stream,
                          ks_curve **out)
{
    g_err[0] = 0;
    ks_status s = validate(p);
    if (s != KS_OK) return s;
    if (!out) return fail(KS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!u_plus_host || !u_minus_host) return fail(KS_EINVAL, "u_plus_host and u_minus_host are required");
    if (!workspace_dev) return fail(KS_EINVAL, "workspace_dev is NULL");
    if (((uintptr_t)workspace_dev) & 255) return fail(KS_EINVAL, "workspace_dev must be 256-byte aligned");
    for (int n = 0; n < p->nx; ++n)
        if (!std::isfinite(u_plus_host[n]) || !std::isfinite(u_minus_host[n]))
            return fail(KS_EINVAL, "u_plus/u_minus contain non-finite values");
    ks::Layout lay = ks::curve_layout(p, p->launch == 1);
    if (workspace_bytes < lay.total)
        return fail(KS_ENOMEM, "workspace has %zu bytes, %zu needed", workspace_bytes, lay.total);

    ks_curve *c = new (std::nothrow) ks_curve();
    if (!c) return fail(KS_ENOMEM, "host allocation of the handle failed");
    c->p = *p;
    c->lay = lay;
    c->d = make_dev(p, lay, workspace_dev);
    c->st = (cudaStream_t)stream;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return fail(KS_ECUDA, "cudaGetDevice failed");
    }
    ks_status r = KS_OK;
    do {
        if (cudaMallocHost((void **)&c->h0, sizeof(ks::DevScalars)) != cudaSuccess) {
            c->h0 = nullptr;
            r = fail(KS_ENOMEM, "pinned host allocation of the scalars failed");
            break;
        }
        if (!c->d.xtc && p->ns >= ks::ROWS_TMA_MIN_NS) {
            const cudaError_t e = ks::make_row_maps(c->d, &c->rmaps);
            if (e != cudaSuccess) {
                r = fail(KS_ECUDA, "encoding the row phase's tensor maps failed: %s", cudaGetErrorString(e));
                break;
            }
            c->d.rowmaps = &c->rmaps;
        }
        const size_t nb = (size_t)p->nx * sizeof(double);
        if (cudaMemcpyAsync(c->d.ends, u_plus_host, nb, cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
            cudaMemcpyAsync(c->d.ends + p->nx, u_minus_host, nb, cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
            cudaMemsetAsync(c->d.pert, 0, (size_t)(p->nx + ks::MAX_PERT + ks::MAX_PERT * p->nx) * 8, c->st) != cudaSuccess) {
            r = fail(KS_ECUDA, "copy of the end sections failed: %s", cudaGetErrorString(cudaGetLastError()));
            break;
        }
        cudaError_t e = ks::launch_setup(c->d, p->dtau, c->st);
        if (e == cudaSuccess)
            e = ks::launch_scalars_init(c->d, p->lambda, p->lambda_free, p->dtau, p->dtau_lambda, p->conv, c->st);
        if (e == cudaSuccess) {
            if (u_init_dev) {
                e = ks::launch_widen(c->d, u_init_dev, c->st);
                if (e == cudaSuccess) e = ks::launch_set_ends(c->d, c->st);
            } else {
                e = ks::launch_trial(c->d, 0.0, 0, 0, c->st);
            }
        }
        if (e == cudaSuccess) e = ks::launch_row_fwd_x(c->d, c->d.U, 0, c->st);
        if (e == cudaSuccess) e = ks::launch_dt(c->d, ks::GM_STORE, 0, 0, c->st);
        if (e == cudaSuccess && p->check_ends) e = ks::launch_rows(c->d, ks::ROWS_EVAL, c->st);
        if (e != cudaSuccess) {
            r = fail(KS_ECUDA, "set-up kernels failed: %s", cudaGetErrorString(e));
            break;
        }
        if ((r = ks::setup_implicit(c->d, c->st)) != KS_OK) break;
        ks::DevScalars h;
        r = read_scalars(c, &h);
        if (r != KS_OK) break;
        if (p->check_ends) {
            double fp = std::sqrt(h.f2_plus), fm = std::sqrt(h.f2_minus);
            double up = std::sqrt(h.u2_plus), um = std::sqrt(h.u2_minus);
            if (fp > 1e-8 * (1.0 + up) || fm > 1e-8 * (1.0 + um)) {
                r = fail(KS_ENOTEQUILIBRIUM, "end sections are not equilibria: |f(u_+)| = %.3e, |f(u_-)| = %.3e", fp, fm);
                break;
            }
        }
    } while (0);
    if (r != KS_OK) {
        ks_curve_destroy(c);
        return r;
    }
    *out = c;
    return KS_OK;
}

ks_status ks_curve_set_stream(ks_curve *c, void *stream)
{
    ks_status s = check_handle(c);
    if (s != KS_OK) return s;
    c->st = (cudaStream_t)stream;
    return KS_OK;
}

ks_status ks_curve_init_trial(ks_curve *c, double a, const double *v_host, int32_t npert, const double *amps_host,
                              const double *vp_host)
{
    ks_status s = check_handle(c);
    if (s != KS_OK) return s;
    if (npert < 0 || npert > ks::MAX_PERT) return fail(KS_EINVAL, "npert must be in [0, %d]", ks::MAX_PERT);
    if (npert > 0 && (!amps_host || !vp_host)) return fail(KS_EINVAL, "amps_host and vp_host are required when npert > 0");
    if (a != 0.0 && !v_host) return fail(KS_EINVAL, "v_host is required when a != 0");
    if (!std::isfinite(a)) return fail(KS_EINVAL, "a must be finite");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(KS_ECUDA, "cannot select the curve's device");
    const int N = c->p.nx;
    if (v_host) KS_CUDA(cudaMemcpyAsync(c->d.pert, v_host, N * 8, cudaMemcpyHostToDevice, c->st));
    if (npert > 0) {
        KS_CUDA(cudaMemcpyAsync(c->d.pert + N, amps_host, npert * 8, cudaMemcpyHostToDevice, c->st));
        KS_CUDA(cudaMemcpyAsync(c->d.pert + N + ks::MAX_PERT, vp_host, (size_t)npert * N * 8, cudaMemcpyHostToDevice, c->st));
    }
    KS_CUDA(ks::launch_trial(c->d, a, v_host != nullptr && a != 0.0, npert, c->st));
    KS_CUDA(ks::launch_row_fwd_x(c->d, c->d.U, 0, c->st));
    s = refresh_dt_u(c);
    if (s != KS_OK) return s;
    KS_CUDA(ks::launch_scalars_init(c->d, c->p.lambda, c->p.lambda_free, c->p.dtau, c->p.dtau_lambda, c->p.conv, c->st));
    KS_CUDA(cudaStreamSynchronize(c->st));
    return KS_OK;
}

ks_status ks_curve_residual(ks_curve *c, void *r_dev)
{
    ks_status s = check_handle(c);
    if (s != KS_OK) return s;
    if (!r_dev) return fail(KS_EINVAL, "r_dev is NULL");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(KS_ECUDA, "cannot select the curve's device");
    KS_CUDA(ks::launch_rows(c->d, ks::ROWS_EVAL, c->st));
    KS_CUDA(ks::launch_row_inv(c->d, c->d.R, r_dev, 0, c->st));
    return KS_OK;
}

ks_status ks_curve_cost(ks_curve *c, double *J2, double *J_arc)
{
    ks_status s = check_handle(c);
    if (s != KS_OK) return s;
    DeviceGuard g(c->device);
    if (!g.ok) return fail(KS_ECUDA, "cannot select the curve's device");
    KS_CUDA(ks::launch_rows(c->d, ks::ROWS_EVAL, c->st));
    ks::DevScalars h;
    s = read_scalars(c, &h);
    if (s != KS_OK) return s;
    if (J2) *J2 = h.J2;
    if (J_arc) *J_arc = h.Jarc;
    return KS_OK;
}

ks_status ks_curve_gradient(ks_curve *c, int32_t euclidean, void *g_dev, double *dJ2_dlambda)
{
    ks_status s = check_handle(c);
    if (s != KS_OK) return s;
    if (!g_dev) return fail(KS_EINVAL, "g_dev is NULL");
    if (euclidean != 0 && euclidean != 1) return fail(KS_EINVAL, "euclidean must be 0 or 1");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(KS_ECUDA, "cannot select the curve's device");
    const int discrete = euclidean ? 1 : (c->p.adjoint == KS_ADJ_DISCRETE);
    KS_CUDA(ks::launch_rows(c->d, ks::ROWS_EVAL, c->st));
    KS_CUDA(ks::launch_dt(c->d, ks::GM_GRAD, discrete, 0, c->st));
    KS_CUDA(ks::launch_row_inv(c->d, c->d.G, g_dev, euclidean ? 1 : 0, c->st));
    if (dJ2_dlambda) {
        ks::DevScalars h;
        s = read_scalars(c, &h);
        if (s != KS_OK) return s;
        *dJ2_dlambda = h.dJdl;
    }
    return KS_OK;
}

ks_status ks_curve_descend_async(ks_curve *c, int64_t nsteps, double tol)
{
    ks_status s = check_handle(c);
    if (s != KS_OK) return s;
    if (nsteps < 0) return fail(KS_EINVAL, "nsteps must be >= 0");
    if (!std::isfinite(tol)) return fail(KS_EINVAL, "tol must be finite");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(KS_ECUDA, "cannot select the curve's device");
    return enqueue_steps(c, nsteps, tol);
}

ks_status ks_curve_descend(ks_curve *c, int64_t nsteps, double tol, int64_t *steps_done, double *J, double *J_arc)
{
    ks_status s = check_handle(c);
    if (s != KS_OK) return s;
    if (nsteps < 0) return fail(KS_EINVAL, "nsteps must be >= 0");
    if (!std::isfinite(tol)) return fail(KS_EINVAL, "tol must be finite");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(KS_ECUDA, "cannot select the curve's device");
    // the step count at the start, copied before the steps and read after them
    KS_CUDA(cudaMemcpyAsync(c->h0, c->d.sc, sizeof(ks::DevScalars), cudaMemcpyDeviceToHost, c->st));
    s = enqueue_steps(c, nsteps, tol);
    if (s != KS_OK) return s;
    KS_CUDA(ks::launch_rows(c->d, ks::ROWS_EVAL, c->st));
    ks::DevScalars h;
    s = read_scalars(c, &h);
    if (s != KS_OK) return s;
    const ks::DevScalars h0 = *c->h0;
    if (steps_done) *steps_done = h.step - h0.step;
    if (J) *J = std::sqrt(h.J2);
    if (J_arc) *J_arc = h.Jarc;
    if (h.status == KS_ENONFINITE || !std::isfinite(h.J2))
        return fail(KS_ENONFINITE, "the cost became non-finite after %lld steps", (long long)(h.step - h0.step));
    if (tol > 0 && !h.done) return fail(KS_ENOTCONV, "tolerance %.3e not reached in %lld steps", tol, (long long)nsteps);
    return KS_OK;
}

ks_status ks_curve_scalars(ks_curve *c, ks_scalars *out)
{
    ks_status s = check_handle(c);
    if (s != KS_OK) return s;
    if (!out) return fail(KS_EINVAL, "out is NULL");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(KS_ECUDA, "cannot select the curve's device");
    ks::DevScalars h;
    s = read_scalars(c, &h);
    if (s != KS_OK) return s;
    out->J = std::sqrt(h.J2);
    out->J_arc = h.Jarc;
    out->dJ2_dlambda = h.dJdl;
    out->G_norm = std::sqrt(h.G2);
    out->Dnorm = h.Dnorm;
    out->lambda = h.lambda;
    out->tau = h.tau;
    out->step = h.step;
    out->converged = h.done && h.status == 0;
    out->status = h.status;
    return KS_OK;
}

ks_status ks_curve_get_state(ks_curve *c, void *u_dev, double *lambda, double *tau)
{
    ks_status s = check_handle(c);
    if (s != KS_OK) return s;
    DeviceGuard g(c->device);
    if (!g.ok) return fail(KS_ECUDA, "cannot select the curve's device");
    if (u_dev) KS_CUDA(ks::launch_row_inv(c->d, c->d.U, u_dev, 0, c->st));
    if (lambda || tau) {
        ks::DevScalars h;
        s = read_scalars(c, &h);
        if (s != KS_OK) return s;
        if (lambda) *lambda = h.lambda;
        if (tau) *tau = h.tau;
    }
    return KS_OK;
}

ks_status ks_curve_set_state(ks_curve *c, const void *u_dev, double lambda, double tau)
{
    ks_status s = check_handle(c);
    if (s != KS_OK) return s;
    if (!u_dev) return fail(KS_EINVAL, "u_dev is NULL");
    if (!std::isfinite(lambda) || !std::isfinite(tau)) return fail(KS_EINVAL, "lambda and tau must be finite");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(KS_ECUDA, "cannot select the curve's device");
    // the forward transform straight from the input, in FP64 or, for FP32
    // storage, double-float (the linear term of f multiplies each coefficient by
    // a_j ~ k_j^4: a coefficient must keep its own relative precision, not that
    // of the largest one, which an FP32 transform would give it)
    KS_CUDA(ks::launch_row_fwd(c->d, u_dev, c->d.U, c->st));
    s = refresh_dt_u(c);
    if (s != KS_OK) return s;
    KS_CUDA(ks::launch_set_lambda_tau(c->d, lambda, tau, c->st));
    return KS_OK;
}

ks_status ks_curve_profile(ks_curve *c, int32_t max_steps)
{
    ks_status s = check_handle(c);
    if (s != KS_OK) return s;
    if (max_steps < 0 || max_steps > (1 << 20)) return fail(KS_EINVAL, "max_steps must be in [0, 2^20]");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(KS_ECUDA, "cannot select the curve's device");
    KS_CUDA(cudaStreamSynchronize(c->st));
    release_events(c);
    c->events.resize((size_t)EV_PER_ENTRY * max_steps);
    for (size_t i = 0; i < c->events.size(); ++i) {
        if (cudaEventCreate(&c->events[i]) != cudaSuccess) {
            c->events.resize(i);
            release_events(c);
            return fail(KS_ECUDA, "cudaEventCreate failed");
        }
    }
    c->prof_steps.assign((size_t)max_steps, 0);
    c->prof_cap = max_steps;
    return KS_OK;
}

ks_status ks_curve_profile_read(ks_curve *c, ks_profile *out)
{
    ks_status s = check_handle(c);
    if (s != KS_OK) return s;
    if (!out) return fail(KS_EINVAL, "out is NULL");
    DeviceGuard g(c->device);
    if (!g.ok) return fail(KS_ECUDA, "cannot select the curve's device");
    KS_CUDA(cudaStreamSynchronize(c->st));
    *out = ks_profile{};
    for (int st = 0; st < c->prof_used; ++st) {
        if (c->prof_steps[st] > 0) {
            float ms = 0.f;
            KS_CUDA(cudaEventElapsedTime(&ms, c->events[(size_t)EV_PER_ENTRY * st], c->events[(size_t)EV_PER_ENTRY * st + 1]));
            out->step_ms += ms;
            out->step_launches += 1;
            out->step_steps += c->prof_steps[st];
            continue;
        }
        const cudaEvent_t *ev = &c->events[(size_t)EV_PER_ENTRY * st];
        for (int ph = 0; ph < 3; ++ph) {
            if (ph == 2 && fused_step(c)) continue;   // D_t u ran inside the update launch
            float ms = 0.f;
            KS_CUDA(cudaEventElapsedTime(&ms, ev[2 * ph], ev[2 * ph + 1]));
            out->ms[ph] += ms;
            out->launches[ph] += 1;
        }
        if (c->d.impl) {
            float ms = 0.f;
            KS_CUDA(cudaEventElapsedTime(&ms, ev[10], ev[11]));
            out->impl_ms += ms;
            out->impl_launches += 1;
        }
        if (three_pass(c)) {
            for (int ph = 0; ph < 2; ++ph) {
                // pass boundaries: phase start, end of pass 1, end of pass 2, phase end
                // (for the update of the implicit scheme: the start of its products)
                const cudaEvent_t b[4] = {ev[2 + 2 * ph], ev[6 + 2 * ph], ev[7 + 2 * ph],
                                          (ph == 0 && c->d.impl) ? ev[10] : ev[3 + 2 * ph]};
                for (int q = 0; q < 3; ++q) {
                    float ms = 0.f;
                    KS_CUDA(cudaEventElapsedTime(&ms, b[q], b[q + 1]));
                    out->pass_ms[ph][q] += ms;
                    out->pass_launches[ph][q] += 1;
                }
            }
        }
    }
    return KS_OK;
}

ks_status ks_curve_debug_wait_limit(ks_curve *c, int64_t cycles)
{
    ks_status s = check_handle(c);
    if (s != KS_OK) return s;
    DeviceGuard g(c->device);
    if (!g.ok) return fail(KS_ECUDA, "cannot select the curve's device");
    KS_CUDA(ks::launch_set_wait_cycles(c->d, (long long)cycles, c->st));
    return KS_OK;
}

ks_status ks_curve_destroy(ks_curve *c)
{
    if (!c) return KS_OK;
    {
        DeviceGuard g(c->device);
        release_events(c);
        if (c->gexec) cudaGraphExecDestroy(c->gexec);
        if (c->gstream) cudaStreamDestroy(c->gstream);
        if (c->h0) cudaFreeHost(c->h0);
    }
    delete c;
    return KS_OK;
}

}  // extern "C"
