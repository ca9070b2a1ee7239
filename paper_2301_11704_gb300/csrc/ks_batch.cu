// ks_batch.cu -- many independent curves (uneven N_s, N and L) descending
// together: every phase of a step is one launch over the work items (curve,
// block) of all curves, captured once into a CUDA graph and replayed.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ksconn.h"
#include "ks_internal.h"

namespace {

const int BATCH_GRAPH_STEPS = 16;

struct Group {
    int key;              // N (rows), tile width (dense s-phase) or F (FFT s-phase)
    size_t off;           // offset of the item list in the item area
    int count;
    int sub = 0;          // FFT s-phase: F1 of the split F = F1 (F / F1)
};

}  // namespace

struct ks_batch {
    int nb = 0;
    int prec = 0;
    int discrete = 0;
    cudaStream_t st = nullptr;
    int device = 0;
    std::vector<ks_params> p;
    std::vector<size_t> off;            // per-curve workspace offsets
    std::vector<ks::CurveDev> cv;       // host copy of the device curve array
    ks::CurveDev *cv_dev = nullptr;
    unsigned char *items_dev = nullptr; // item area
    size_t items_cap = 0;
    std::vector<Group> rows, dts;
    std::vector<Group> ffts;            // (curve, mode) items of the FFT-form curves, one group per F
    int impl = 0;                       // full-linear-implicit stepping
    Group imp_prod{}, imp_fin{};        // its items: the two products, the finishing pass
    int tile_pref = 0;                  // 0: per-curve default, 32 or 64: forced (autotuner)
    int row_warps = ks::ROWS_WARPS;     // warps per row-phase CTA (two sections each): 4 or 8 (autotuner)
    float tuned_ms = 0.f;               // the autotuner's time of a step with its choice
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t gstream = nullptr;
};

namespace {

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// Bytes of the batch header: curve array and the largest item lists.
void header_sizes(int nb, const ks_params *p, size_t *cv_bytes, size_t *items_bytes)
{
    size_t rows = 0, tiles = 0, modes = 0, imp = 0;
    for (int i = 0; i < nb; ++i) {
        rows += (p[i].ns + ks::ROWS_PER_CTA - 1) / ks::ROWS_PER_CTA;
        tiles += (size_t)((p[i].ns + ks::DT_BM - 1) / ks::DT_BM) * ((p[i].nx + 31) / 32);
        modes += p[i].nx / 2;
        if (p[i].scheme == KS_SCHEME_IMPLICIT)   // the increment's products (<= 2 per tile) and finishing pass (<= 8)
            imp += 2 * (size_t)((p[i].nx + 63) / 64) * ((p[i].ns - 1) / 2 / 128 + 1) + 8;
    }
    *cv_bytes = al256((size_t)nb * sizeof(ks::CurveDev));
    *items_bytes = al256(rows * sizeof(int2)) + al256(tiles * sizeof(int4)) + al256(modes * sizeof(int2)) +
                   al256(imp * sizeof(int4));
}

ks_status validate_batch(int nb, const ks_params *p)
{
    if (nb <= 0 || nb > 65536) return ks::report_error(KS_EINVAL, "batch size must be in [1, 65536]");
    if (!p) return ks::report_error(KS_EINVAL, "params is NULL");
    for (int i = 0; i < nb; ++i) {
        ks_status s = ks::check_params(&p[i]);
        if (s != KS_OK) return s;
        if (p[i].precision != p[0].precision)
            return ks::report_error(KS_EINVAL, "all curves of a batch must have the same precision");
        if (ks::xtc_of(p[i].precision))
            return ks::report_error(KS_EINVAL, "batches run the FFT row phase: precision must be KS_FP64 or KS_FP32");
        if (p[i].adjoint != p[0].adjoint)
            return ks::report_error(KS_EINVAL, "all curves of a batch must have the same adjoint mode");
        if (p[i].scheme != p[0].scheme)
            return ks::report_error(KS_EINVAL, "all curves of a batch must have the same scheme");
    }
    return KS_OK;
}

// (Re)builds the curve array and the work-item lists for the current tile choice.
ks_status build_items(ks_batch *b)
{
    std::map<int, std::vector<int2>> rows;
    std::map<int, std::vector<int4>> dts;
    std::map<std::pair<int, int>, std::vector<int2>> fft;   // by (F, F1): each group launched with its own shared memory
    for (int i = 0; i < b->nb; ++i) {
        ks::CurveDev &c = b->cv[i];
        const int rs = 2 * b->row_warps;
        c.row_blocks = (c.ns + rs - 1) / rs;
        for (int k = 0; k < c.row_blocks; ++k) rows[c.nx].push_back(make_int2(i, k));
        if (c.F > 0) {
            for (int jm = 0; jm < c.W / 2; ++jm) fft[std::make_pair(c.F, c.f4b ? c.F1 : 0)].push_back(make_int2(i, jm));
            continue;
        }
        // the contraction's columns: W (N_x, or N_x / 2 in sine storage)
        const int bn = b->tile_pref ? (c.W < 64 ? 32 : b->tile_pref) : (c.W >= 64 ? 64 : 32);
        c.bn = bn;
        c.tiles_c = (c.W + bn - 1) / bn;
        for (int tr = 0; tr < c.tiles_r; ++tr)
            for (int tc = 0; tc < c.tiles_c; ++tc) dts[bn].push_back(make_int4(i, tc, tr, 0));
    }
    size_t cvb, itb;
    header_sizes(b->nb, b->p.data(), &cvb, &itb);
    std::vector<unsigned char> host(itb, 0);
    size_t o = 0;
    b->rows.clear();
    b->dts.clear();
    for (auto &kv : rows) {
        b->rows.push_back({kv.first, o, (int)kv.second.size()});
        memcpy(host.data() + o, kv.second.data(), kv.second.size() * sizeof(int2));
        o += kv.second.size() * sizeof(int2);
    }
    o = al256(o);
    for (auto &kv : dts) {
        b->dts.push_back({kv.first, o, (int)kv.second.size()});
        memcpy(host.data() + o, kv.second.data(), kv.second.size() * sizeof(int4));
        o += kv.second.size() * sizeof(int4);
    }
    o = al256(o);
    b->ffts.clear();
    for (auto it = fft.rbegin(); it != fft.rend(); ++it) {   // largest F (longest CTAs) first
        b->ffts.push_back({it->first.first, o, (int)it->second.size(), it->first.second});
        memcpy(host.data() + o, it->second.data(), it->second.size() * sizeof(int2));
        o += it->second.size() * sizeof(int2);
    }
    if (b->impl) {
        std::vector<int4> prod, fin;
        for (int i = 0; i < b->nb; ++i) ks::implicit_batch_items(b->cv[i], i, prod, fin);
        o = al256(o);
        b->imp_prod = {0, o, (int)prod.size()};
        if (o + (prod.size() + fin.size()) * sizeof(int4) <= itb) {
            memcpy(host.data() + o, prod.data(), prod.size() * sizeof(int4));
            o += prod.size() * sizeof(int4);
            b->imp_fin = {0, o, (int)fin.size()};
            memcpy(host.data() + o, fin.data(), fin.size() * sizeof(int4));
            o += fin.size() * sizeof(int4);
        } else {
            o = itb + 1;
        }
    }
    if (o > itb) return ks::report_error(KS_ENOMEM, "batch item lists exceed their reserved space");
    cudaError_t e = cudaMemcpyAsync(b->items_dev, host.data(), o, cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->cv_dev, b->cv.data(), b->nb * sizeof(ks::CurveDev), cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);   // host vectors die at return
    if (e != cudaSuccess) return ks::report_error(KS_ECUDA, "batch item upload: %s", cudaGetErrorString(e));
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    return KS_OK;
}

// The FFT items of one transform length: the one-CTA FFT form, or from F = 1024
// on its four-step variant (register line transforms).
static cudaError_t launch_fft_group(const ks_batch *b, const Group &g, int mode, int discrete, cudaStream_t st)
{
    const int2 *items = (const int2 *)(b->items_dev + g.off);
    if (g.sub > 0)
        return ks::launch_f4b_batch(b->prec, g.sub, g.key / g.sub, b->cv_dev, items, g.count, mode, discrete, 1, st);
    return ks::launch_sconv_batch(b->prec, g.key, b->cv_dev, items, g.count, mode, discrete, 1, st);
}

ks_status launch_step(ks_batch *b, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    for (const Group &g : b->rows)
        if (e == cudaSuccess)
            e = ks::launch_rows_batch(b->prec, g.key, b->row_warps, b->cv_dev, (const int2 *)(b->items_dev + g.off), g.count,
                                      ks::ROWS_STEP, st);
    // the update contraction; for the implicit scheme it writes G, whose increment follows
    const int um = b->impl ? ks::GM_GRAD : ks::GM_UPDATE;
    for (const Group &g : b->dts)
        if (e == cudaSuccess)
            e = ks::launch_dt_batch(b->prec, g.key, b->cv_dev, (const int4 *)(b->items_dev + g.off), g.count,
                                    um, b->discrete, 1, st);
    // the batched four-step groups run the update and D_t u of the updated columns
    // in one launch (GM_STEP) unless the implicit increment comes between them
    const bool chain = !b->impl;
    for (const Group &g : b->ffts)
        if (e == cudaSuccess) e = launch_fft_group(b, g, (chain && g.sub > 0) ? ks::GM_STEP : um, b->discrete, st);
    if (b->impl && e == cudaSuccess)
        e = ks::launch_implicit_batch(b->prec, b->cv_dev, (const int4 *)(b->items_dev + b->imp_prod.off),
                                      b->imp_prod.count, (const int4 *)(b->items_dev + b->imp_fin.off),
                                      b->imp_fin.count, st);
    for (const Group &g : b->dts)
        if (e == cudaSuccess)
            e = ks::launch_dt_batch(b->prec, g.key, b->cv_dev, (const int4 *)(b->items_dev + g.off), g.count,
                                    ks::GM_STORE, 0, 1, st);
    for (const Group &g : b->ffts)
        if (e == cudaSuccess && !(chain && g.sub > 0)) e = launch_fft_group(b, g, ks::GM_STORE, 0, st);
    if (e != cudaSuccess) return ks::report_error(KS_ECUDA, "batched step launch: %s", cudaGetErrorString(e));
    return KS_OK;
}

ks_status ensure_graph(ks_batch *b)
{
    if (b->gexec) return KS_OK;
    cudaError_t e = cudaSuccess;
    if (!b->gstream) e = cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return ks::report_error(KS_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    ks_status s = KS_OK;
    for (int i = 0; i < BATCH_GRAPH_STEPS && s == KS_OK; ++i) s = launch_step(b, b->gstream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->gstream, &graph);
    if (s != KS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e != cudaSuccess) return ks::report_error(KS_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        b->gexec = nullptr;
        return ks::report_error(KS_ECUDA, "graph instantiation: %s", cudaGetErrorString(e));
    }
    return KS_OK;
}

ks_status enqueue(ks_batch *b, int64_t nsteps, double tol)
{
    cudaError_t e = ks::launch_set_limit_batch(b->cv_dev, b->nb, (long long)nsteps, tol, b->st);
    if (e != cudaSuccess) return ks::report_error(KS_ECUDA, "set limit: %s", cudaGetErrorString(e));
    int64_t full = nsteps / BATCH_GRAPH_STEPS, rest = nsteps % BATCH_GRAPH_STEPS;
    if (full > 0) {
        ks_status s = ensure_graph(b);
        if (s != KS_OK) return s;
        for (int64_t g = 0; g < full; ++g) {
            e = cudaGraphLaunch(b->gexec, b->st);
            if (e != cudaSuccess) return ks::report_error(KS_ECUDA, "graph launch: %s", cudaGetErrorString(e));
        }
    }
    for (int64_t r = 0; r < rest; ++r) {
        ks_status s = launch_step(b, b->st);
        if (s != KS_OK) return s;
    }
    return KS_OK;
}

ks_status read_all(ks_batch *b, std::vector<ks::DevScalars> &h)
{
    h.resize(b->nb);
    for (int i = 0; i < b->nb; ++i) {
        cudaError_t e = cudaMemcpyAsync(&h[i], b->cv[i].sc, sizeof(ks::DevScalars), cudaMemcpyDeviceToHost, b->st);
        if (e != cudaSuccess) return ks::report_error(KS_ECUDA, "scalar read: %s", cudaGetErrorString(e));
    }
    cudaError_t e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return ks::report_error(KS_ECUDA, "scalar read: %s", cudaGetErrorString(e));
    for (size_t i = 0; i < h.size(); ++i)
        if (h[i].err)
            return ks::report_error(KS_ETIMEOUT, "curve %zu: a device-side copy did not complete in time", i);
    return KS_OK;
}

ks_status eval_all(ks_batch *b)
{
    cudaError_t e = cudaSuccess;
    for (const Group &g : b->rows)
        if (e == cudaSuccess)
            e = ks::launch_rows_batch(b->prec, g.key, b->row_warps, b->cv_dev, (const int2 *)(b->items_dev + g.off), g.count,
                                      ks::ROWS_EVAL, b->st);
    if (e != cudaSuccess) return ks::report_error(KS_ECUDA, "batched evaluation: %s", cudaGetErrorString(e));
    return KS_OK;
}

// The implicit scheme's set-up of every curve (eigendecompositions), spread
// over host threads with a stream each after the batch stream's set-up work.
ks_status setup_implicit_all(ks_batch *b)
{
    cudaError_t e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return ks::report_error(KS_ECUDA, "batch set-up: %s", cudaGetErrorString(e));
    const int nt = std::max(1, std::min(8, b->nb));
    std::vector<ks_status> st(nt, KS_OK);
    std::vector<std::string> msg(nt);
    std::atomic<int> next{0};
    auto work = [&](int t) {
        if (cudaSetDevice(b->device) != cudaSuccess) {
            st[t] = KS_ECUDA;
            msg[t] = "cannot select the batch's device";
            return;
        }
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            st[t] = KS_ECUDA;
            msg[t] = "stream creation";
            return;
        }
        for (int i = next++; i < b->nb && st[t] == KS_OK; i = next++) {
            st[t] = ks::setup_implicit(b->cv[i], s);
            if (st[t] != KS_OK) msg[t] = "curve " + std::to_string(i) + ": " + ks_last_error();
        }
        cudaStreamDestroy(s);
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(work, t);
    work(0);
    for (auto &x : th) x.join();
    for (int t = 0; t < nt; ++t)
        if (st[t] != KS_OK) return ks::report_error(st[t], "implicit set-up, %s", msg[t].c_str());
    return KS_OK;
}

}  // namespace

extern "C" {

size_t ks_batch_workspace_bytes(int32_t nb, const ks_params *params)
{
    if (validate_batch(nb, params) != KS_OK) return 0;
    size_t cvb, itb;
    header_sizes(nb, params, &cvb, &itb);
    size_t total = cvb + itb;
    for (int i = 0; i < nb; ++i)
        total += ks::make_layout(params[i].ns, params[i].nx, ks::storage32(params[i].precision), 0, 0,
                                 params[i].s_transform, 0, 0, params[i].scheme == KS_SCHEME_IMPLICIT,
                                 (params[i].symmetry & KS_SYM_SINE) ? 1 : 0).total;
    return total;
}

ks_status ks_batch_create(int32_t nb, const ks_params *params, const double *u_plus_host, const double *u_minus_host,
                          void *workspace_dev, size_t workspace_bytes, void *stream, ks_batch **out)
{
    ks_status s = validate_batch(nb, params);
    if (s != KS_OK) return s;
    if (!out || !u_plus_host || !u_minus_host || !workspace_dev)
        return ks::report_error(KS_EINVAL, "out, u_plus_host, u_minus_host and workspace_dev are required");
    *out = nullptr;
    if (((uintptr_t)workspace_dev) & 255) return ks::report_error(KS_EINVAL, "workspace_dev must be 256-byte aligned");
    const size_t need = ks_batch_workspace_bytes(nb, params);
    if (workspace_bytes < need)
        return ks::report_error(KS_ENOMEM, "batch workspace has %zu bytes, %zu needed", workspace_bytes, need);
    ks_batch *b = new (std::nothrow) ks_batch();
    if (!b) return ks::report_error(KS_ENOMEM, "host allocation of the batch handle failed");
    b->nb = nb;
    b->prec = ks::storage32(params[0].precision);
    b->discrete = params[0].adjoint == KS_ADJ_DISCRETE;
    b->impl = params[0].scheme == KS_SCHEME_IMPLICIT;
    b->st = (cudaStream_t)stream;
    cudaGetDevice(&b->device);
    b->p.assign(params, params + nb);
    size_t cvb, itb;
    header_sizes(nb, params, &cvb, &itb);
    unsigned char *base = (unsigned char *)workspace_dev;
    b->cv_dev = (ks::CurveDev *)base;
    b->items_dev = base + cvb;
    b->items_cap = itb;
    size_t o = cvb + itb;
    b->cv.resize(nb);
    size_t xoff = 0;
    for (int i = 0; i < nb; ++i) {
        const ks::Layout l = ks::make_layout(params[i].ns, params[i].nx, b->prec, 0, 0, params[i].s_transform, 0, 0,
                                             params[i].scheme == KS_SCHEME_IMPLICIT,
                                             (params[i].symmetry & KS_SYM_SINE) ? 1 : 0);
        b->off.push_back(o);
        b->cv[i] = ks::bind_layout(&params[i], l, base + o);
        o += l.total;
    }
    s = KS_OK;
    for (int i = 0; i < nb && s == KS_OK; ++i) {
        const ks::CurveDev &c = b->cv[i];
        const size_t nbytes = (size_t)c.nx * sizeof(double);
        cudaError_t e = cudaMemcpyAsync(c.ends, u_plus_host + xoff, nbytes, cudaMemcpyHostToDevice, b->st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c.ends + c.nx, u_minus_host + xoff, nbytes, cudaMemcpyHostToDevice, b->st);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(c.pert, 0, (size_t)(c.nx + ks::MAX_PERT + ks::MAX_PERT * c.nx) * 8, b->st);
        if (e == cudaSuccess) e = ks::launch_setup(c, params[i].dtau, b->st);
        if (e == cudaSuccess)
            e = ks::launch_scalars_init(c, params[i].lambda, params[i].lambda_free, params[i].dtau,
                                        params[i].dtau_lambda, params[i].conv, b->st);
        if (e == cudaSuccess) e = ks::launch_trial(c, 0.0, 0, 0, b->st);
        if (e == cudaSuccess) e = ks::launch_row_fwd_x(c, c.U, 0, b->st);
        if (e == cudaSuccess) e = ks::launch_dt(c, ks::GM_STORE, 0, 0, b->st);
        if (e != cudaSuccess) s = ks::report_error(KS_ECUDA, "batch set-up of curve %d: %s", i, cudaGetErrorString(e));
        xoff += c.nx;
    }
    if (s == KS_OK && b->impl) s = setup_implicit_all(b);
    if (s == KS_OK) s = build_items(b);
    if (s != KS_OK) {
        delete b;
        return s;
    }
    *out = b;
    return KS_OK;
}

ks_status ks_batch_init_trial(ks_batch *b, int32_t npert, const double *amps_host, const double *vp_host)
{
    if (!b) return ks::report_error(KS_EINVAL, "batch handle is NULL");
    if (npert < 0 || npert > ks::MAX_PERT) return ks::report_error(KS_EINVAL, "npert must be in [0, %d]", ks::MAX_PERT);
    if (npert > 0 && (!amps_host || !vp_host)) return ks::report_error(KS_EINVAL, "amps_host and vp_host are required");
    size_t voff = 0;
    for (int i = 0; i < b->nb; ++i) {
        const ks::CurveDev &c = b->cv[i];
        const ks_params &p = b->p[i];
        cudaError_t e = cudaSuccess;
        if (npert > 0) {
            e = cudaMemcpyAsync(c.pert + c.nx, amps_host + (size_t)i * npert, npert * 8, cudaMemcpyHostToDevice, b->st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c.pert + c.nx + ks::MAX_PERT, vp_host + voff, (size_t)npert * c.nx * 8,
                                    cudaMemcpyHostToDevice, b->st);
        }
        if (e == cudaSuccess) e = ks::launch_trial(c, 0.0, 0, npert, b->st);
        if (e == cudaSuccess) e = ks::launch_row_fwd_x(c, c.U, 0, b->st);
        if (e == cudaSuccess) e = ks::launch_dt(c, ks::GM_STORE, 0, 0, b->st);
        if (e == cudaSuccess)
            e = ks::launch_scalars_init(c, p.lambda, p.lambda_free, p.dtau, p.dtau_lambda, p.conv, b->st);
        if (e != cudaSuccess) return ks::report_error(KS_ECUDA, "trial curve %d: %s", i, cudaGetErrorString(e));
        voff += (size_t)npert * c.nx;
    }
    cudaError_t e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return ks::report_error(KS_ECUDA, "trial curves: %s", cudaGetErrorString(e));
    return KS_OK;
}

ks_status ks_batch_descend_async(ks_batch *b, int64_t nsteps, double tol)
{
    if (!b) return ks::report_error(KS_EINVAL, "batch handle is NULL");
    if (nsteps < 0 || !std::isfinite(tol)) return ks::report_error(KS_EINVAL, "nsteps must be >= 0 and tol finite");
    return enqueue(b, nsteps, tol);
}

ks_status ks_batch_descend(ks_batch *b, int64_t nsteps, double tol, int64_t *steps_done, double *J, double *J_arc)
{
    if (!b) return ks::report_error(KS_EINVAL, "batch handle is NULL");
    if (nsteps < 0 || !std::isfinite(tol)) return ks::report_error(KS_EINVAL, "nsteps must be >= 0 and tol finite");
    std::vector<ks::DevScalars> h0, h;
    ks_status s = read_all(b, h0);
    if (s == KS_OK) s = enqueue(b, nsteps, tol);
    if (s == KS_OK) s = eval_all(b);
    if (s == KS_OK) s = read_all(b, h);
    if (s != KS_OK) return s;
    bool nonfinite = false, all_done = true;
    for (int i = 0; i < b->nb; ++i) {
        if (steps_done) steps_done[i] = h[i].step - h0[i].step;
        if (J) J[i] = std::sqrt(h[i].J2);
        if (J_arc) J_arc[i] = h[i].Jarc;
        if (h[i].status == KS_ENONFINITE || !std::isfinite(h[i].J2)) nonfinite = true;
        if (!h[i].done) all_done = false;
    }
    if (nonfinite) return ks::report_error(KS_ENONFINITE, "a curve's cost became non-finite");
    if (tol > 0 && !all_done) return ks::report_error(KS_ENOTCONV, "not every curve reached tolerance %.3e", tol);
    return KS_OK;
}

ks_status ks_batch_scalars(ks_batch *b, ks_scalars *out)
{
    if (!b || !out) return ks::report_error(KS_EINVAL, "batch handle and out are required");
    std::vector<ks::DevScalars> h;
    ks_status s = read_all(b, h);
    if (s != KS_OK) return s;
    for (int i = 0; i < b->nb; ++i) {
        out[i].J = std::sqrt(h[i].J2);
        out[i].J_arc = h[i].Jarc;
        out[i].dJ2_dlambda = h[i].dJdl;
        out[i].G_norm = std::sqrt(h[i].G2);
        out[i].Dnorm = h[i].Dnorm;
        out[i].lambda = h[i].lambda;
        out[i].tau = h[i].tau;
        out[i].step = h[i].step;
        out[i].converged = h[i].done && h[i].status == 0;
        out[i].status = h[i].status;
    }
    return KS_OK;
}

ks_status ks_batch_get_state(ks_batch *b, int32_t i, void *u_dev)
{
    if (!b || !u_dev || i < 0 || i >= b->nb) return ks::report_error(KS_EINVAL, "bad batch handle, index or pointer");
    cudaError_t e = ks::launch_row_inv(b->cv[i], b->cv[i].U, u_dev, 0, b->st);
    if (e != cudaSuccess) return ks::report_error(KS_ECUDA, "get_state: %s", cudaGetErrorString(e));
    return KS_OK;
}

ks_status ks_batch_autotune(ks_batch *b, int32_t steps, int32_t *chosen)
{
    if (!b || steps <= 0) return ks::report_error(KS_EINVAL, "batch handle required and steps > 0");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return ks::report_error(KS_ECUDA, "autotune events");
    }
    // time of `steps` real descent steps of every curve with the current knobs (the
    // trial steps count in each curve's step counter and tau)
    auto time_steps = [&](float *ms) -> ks_status {
        ks_status s = build_items(b);
        if (s == KS_OK) s = enqueue(b, 2, 0.0);   // warm-up (and the graph for these items)
        if (s != KS_OK) return s;
        cudaError_t e = cudaEventRecord(e0, b->st);
        if (e == cudaSuccess) {
            s = enqueue(b, steps, 0.0);
            if (s != KS_OK) return s;
            e = cudaEventRecord(e1, b->st);
        }
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
        if (e != cudaSuccess) return ks::report_error(KS_ECUDA, "autotune timing: %s", cudaGetErrorString(e));
        return KS_OK;
    };
    // the split F = F1 (F / F1) of every four-step curve of length F, with its tables
    auto set_split = [&](int F, int f1) -> ks_status {
        for (int i = 0; i < b->nb; ++i) {
            ks::CurveDev &c = b->cv[i];
            if (!c.f4b || c.F != F || c.F1 == f1) continue;
            c.F1 = f1;
            c.F2 = F / f1;
            cudaError_t e = ks::launch_setup_f4(c, b->st);
            if (e != cudaSuccess) return ks::report_error(KS_ECUDA, "autotune set-up: %s", cudaGetErrorString(e));
        }
        return KS_OK;
    };
    ks_status s = KS_OK;
    float best = 1e30f, ms = 0.f;
    // knob 1: sections per row-phase CTA
    int best_w = b->row_warps;
    for (int w : {ks::ROWS_WARPS, 2 * ks::ROWS_WARPS}) {
        b->row_warps = w;
        if ((s = time_steps(&ms)) != KS_OK) break;
        if (ms < best) { best = ms; best_w = w; }
    }
    b->row_warps = best_w;
    // knob 2: the split of each length of the four-step curves
    std::map<int, int> lens;   // F -> current F1
    for (int i = 0; i < b->nb && s == KS_OK; ++i)
        if (b->cv[i].f4b) lens[b->cv[i].F] = b->cv[i].F1;
    for (auto &kv : lens) {
        if (s != KS_OK) break;
        int F1s[3];
        const int n = ks::f4b_splits(kv.first, b->prec, F1s);
        int best_f1 = kv.second;
        for (int k = 0; k < n && s == KS_OK && n > 1; ++k) {
            if ((s = set_split(kv.first, F1s[k])) != KS_OK) break;
            if ((s = time_steps(&ms)) != KS_OK) break;
            if (ms < best) { best = ms; best_f1 = F1s[k]; }
        }
        if (s == KS_OK) s = set_split(kv.first, best_f1);
    }
    // knob 3: the column tile of dense-form curves with N >= 64
    bool dense = false;
    for (int i = 0; i < b->nb; ++i) dense = dense || (b->cv[i].F == 0 && b->cv[i].W >= 64);
    if (dense && s == KS_OK) {
        int best_t = b->tile_pref;
        for (int t : {64, 32}) {
            b->tile_pref = t;
            if ((s = time_steps(&ms)) != KS_OK) break;
            if (ms < best) { best = ms; best_t = t; }
        }
        b->tile_pref = best_t;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != KS_OK) return s;
    b->tuned_ms = best / (float)steps;
    s = build_items(b);
    if (chosen) *chosen = 2 * b->row_warps;
    return s;
}

ks_status ks_batch_get_tuning(ks_batch *b, ks_batch_tuning *out)
{
    if (!b || !out) return ks::report_error(KS_EINVAL, "batch handle and out are required");
    *out = ks_batch_tuning{};
    out->row_sections = 2 * b->row_warps;
    out->dense_tile = b->tile_pref;
    std::map<int, int> lens;
    for (int i = 0; i < b->nb; ++i)
        if (b->cv[i].f4b) lens[b->cv[i].F] = b->cv[i].F1;
    for (auto &kv : lens) {
        if (out->nlen >= 8) break;
        out->F[out->nlen] = kv.first;
        out->F1[out->nlen] = kv.second;
        out->nlen++;
    }
    out->ms_per_step = b->tuned_ms;
    return KS_OK;
}

ks_status ks_batch_destroy(ks_batch *b)
{
    if (!b) return KS_OK;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->gstream) cudaStreamDestroy(b->gstream);
    delete b;
    return KS_OK;
}

}  // extern "C"
