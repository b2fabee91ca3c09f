// C entry points of the GB300 photon-transport library (declared in include/rt.h):
// context, workspaces, order of calls, CUDA-graph capture of the sub-cycle loop.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "rt_internal.cuh"

namespace rt {

rt_status fail(rt_ctx* c, rt_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

rt_status cuda_fail(rt_ctx* c, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    if (c) c->err = m;
    return e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA;
}

static int64_t g_generation = 0;

rt_status ensure(rt_ctx* c, DevBuf& b, size_t bytes, const char* what) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return RT_OK;
    if (b.p) {
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(c, RT_ERR_OOM, std::string("device allocation failed: ") + what);
    }
    b.bytes = bytes;
    ++g_generation;   // buffers captured in graphs moved
    return RT_OK;
}

static void free_buf(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

static void destroy_prof(std::vector<ProfRec>& v) {
    for (auto& r : v) {
        cudaEventDestroy(r.start);
        cudaEventDestroy(r.stop);
    }
    v.clear();
}

static void drop_graphs(rt_ctx* c) {
    for (auto& kv : c->graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        destroy_prof(kv.second.prof);
    }
    c->graphs.clear();
    c->last_prof = nullptr;
}

// inside a stream capture a plain record only orders the capture; an external record
// becomes an event-record node that fires on every replay
static void record_event(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &st);
    if (st == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else cudaEventRecord(e, s);
}

int prof_begin(rt_ctx* c, cudaStream_t s, int kind) {
    if (!c->profiling || !c->prof_sink) return -1;
    if (c->profiling >= 2) {   // pair passes only, one in every profiling - 1
        if (kind != RT_KERNEL_FLUX) return -1;
        if (c->prof_pairs++ % (c->profiling - 1) != 0) return -1;
    }
    ProfRec r;
    r.kind = kind;
    if (cudaEventCreate(&r.start) != cudaSuccess) return -1;
    if (cudaEventCreate(&r.stop) != cudaSuccess) {
        cudaEventDestroy(r.start);
        return -1;
    }
    record_event(r.start, s);
    c->prof_sink->push_back(r);
    return (int)c->prof_sink->size() - 1;
}

void prof_end(rt_ctx* c, cudaStream_t s, int idx) {
    if (idx < 0 || !c->prof_sink) return;
    record_event((*c->prof_sink)[idx].stop, s);
}

static size_t tsize(const rt_ctx* c) { return c->fp64 ? 8 : 4; }

static rt_status check_ready(rt_ctx* c) {
    if (!c) return RT_ERR_INVALID;
    c->err.clear();
    if (!c->built) return fail(c, RT_ERR_STATE, "rt_neighbours has not been called");
    RT_CUDA(c, cudaSetDevice(c->device));
    return RT_OK;
}

// state buffers used by the transport calls (allocated in rt_neighbours)
static rt_status ensure_state(rt_ctx* c) {
    const int64_t n = c->n;
    const int G = c->cfg.n_groups;
    RT_TRY(ensure(c, c->U_a, (size_t)4 * G * n * tsize(c), "state"));
    RT_TRY(ensure(c, c->U_b, (size_t)4 * G * n * tsize(c), "state"));
    RT_TRY(ensure(c, c->grad_t, (size_t)12 * G * n * tsize(c), "gradients"));
    RT_TRY(ensure(c, c->alpha_s, (size_t)n * tsize(c), "absorption"));
    RT_TRY(ensure(c, c->L_dev, (size_t)std::max<int64_t>(c->n_src, 1) * G * 8, "luminosities"));
    RT_TRY(ensure(c, c->dt_dev, 64, "dt"));
    RT_TRY(ensure(c, c->energy_part, (size_t)G * 512 * 8 + (size_t)G * 8, "energy"));
    if (c->n_src > 0) RT_TRY(ensure(c, c->inj_dense, (size_t)G * n * 8, "injection"));
    // per-pair flux slots of one group chunk (at most 4 groups)
    const int gc = G < kMaxGC ? G : kMaxGC;
    RT_TRY(ensure(c, c->pairbuf, (size_t)std::max<int64_t>(c->n_directed / 2, 1) * 4 * gc * tsize(c), "pair fluxes"));
    if (!c->fp64 && G <= kMaxGC)
        RT_TRY(ensure(c, c->frec, (size_t)(12 + 16 * G + kRowRot) * n * 4, "packed flux rows"));
    return RT_OK;
}

}  // namespace rt

using namespace rt;

extern "C" {

rt_status rt_create(const rt_config* cfg, int64_t n, int64_t n_src, void* cuda_stream, rt_ctx** out) {
    if (!out) return RT_ERR_INVALID;
    *out = nullptr;
    rt_ctx* c = new (std::nothrow) rt_ctx();
    if (!c) return RT_ERR_OOM;
    *out = c;
    if (!cfg) return fail(c, RT_ERR_INVALID, "cfg is NULL");
    c->cfg = *cfg;
    c->n = n;
    c->n_owned = n;
    c->n_src = n_src;
    c->stream = (cudaStream_t)cuda_stream;
    if (n < 2 || n >= ((int64_t)1 << 31)) return fail(c, RT_ERR_INVALID, "n must be in [2, 2^31)");
    if (n_src < 0 || n_src >= ((int64_t)1 << 20)) return fail(c, RT_ERR_INVALID, "n_src must be in [0, 2^20)");
    if (cfg->n_groups < 1 || cfg->n_groups > 64) return fail(c, RT_ERR_INVALID, "n_groups must be in [1, 64]");
    if (!(cfg->c_red > 0.0) || !std::isfinite(cfg->c_red)) return fail(c, RT_ERR_INVALID, "c_red must be > 0");
    if (!(cfg->eta_res > 0.0) || !(cfg->eta_res_star > 0.0)) return fail(c, RT_ERR_INVALID, "eta_res must be > 0");
    for (int a = 0; a < 3; ++a)
        if (!(cfg->box[a] > 0.0) || !std::isfinite(cfg->box[a])) return fail(c, RT_ERR_INVALID, "box must be > 0");
    if (cfg->precision != RT_FP64 && cfg->precision != RT_FP32_MIXED)
        return fail(c, RT_ERR_INVALID, "precision must be RT_FP64 or RT_FP32_MIXED");
    if (cfg->limiter_variant != 0) return fail(c, RT_ERR_INVALID, "limiter_variant must be 0 (minmod)");
    if (cfg->riemann_solver != RT_RIEMANN_GLF && cfg->riemann_solver != RT_RIEMANN_HLL)
        return fail(c, RT_ERR_INVALID, "riemann_solver must be RT_RIEMANN_GLF or RT_RIEMANN_HLL");
    if (cfg->h_tol < 0.0 || cfg->h_tol > 1e-3) return fail(c, RT_ERR_INVALID, "h_tol must be in [0, 1e-3]");
    c->fp64 = cfg->precision == RT_FP64;
    RT_CUDA(c, cudaGetDevice(&c->device));
    RT_CUDA(c, cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device));
    RT_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    RT_TRY(ensure(c, c->flags, 64, "flags"));
    RT_CUDA(c, cudaMemset(c->flags.p, 0, 64));
    RT_TRY(ensure_state(c));
    if (cfg->riemann_solver == RT_RIEMANN_HLL) {
        // the wave-speed table, interleaved (lmax, lmin) per node, in working precision
        const int nodes = RT_WAVE_NF * RT_WAVE_NTH;
        std::vector<double> lmax(nodes), lmin(nodes);
        build_wave_table(lmax.data(), lmin.data());
        RT_TRY(ensure(c, c->wave_t, (size_t)2 * nodes * tsize(c), "wave-speed table"));
        if (c->fp64) {
            std::vector<double> t(2 * nodes);
            for (int k = 0; k < nodes; ++k) t[2 * k] = lmax[k], t[2 * k + 1] = lmin[k];
            RT_CUDA(c, cudaMemcpy(c->wave_t.p, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice));
        } else {
            std::vector<float> t(2 * nodes);
            for (int k = 0; k < nodes; ++k) t[2 * k] = (float)lmax[k], t[2 * k + 1] = (float)lmin[k];
            RT_CUDA(c, cudaMemcpy(c->wave_t.p, t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice));
        }
    }
    return RT_OK;
}

rt_status rt_set_stream(rt_ctx* c, void* s) {
    if (!c) return RT_ERR_INVALID;
    c->stream = (cudaStream_t)s;
    return RT_OK;
}

static rt_status neighbours(rt_ctx* c, const double* x, const double* m, const double* xsrc, double* h_out,
                            const double* h_in, const double* hs_in, const double* oms_in = nullptr,
                            const double* octw_in = nullptr) {
    if (!c) return RT_ERR_INVALID;
    c->err.clear();
    if (!x) return fail(c, RT_ERR_INVALID, "x_dev is NULL");
    if (c->n_src > 0 && !xsrc) return fail(c, RT_ERR_INVALID, "xsrc_dev is NULL with n_src > 0");
    RT_CUDA(c, cudaSetDevice(c->device));
    c->built = false;
    c->has_bins = false;   // bins live in the sorted order and depend on the pair lists
    int64_t gen0 = g_generation;
    int64_t targets0 = c->n_inj_targets;
    rt_status s = build_neighbours(c, x, m, xsrc, h_in, hs_in, oms_in, octw_in);
    if (s != RT_OK) {
        drop_graphs(c);
        return s;
    }
    RT_TRY(ensure_state(c));
    // captured graphs hold buffer addresses, the injection grid size and the pair count (the
    // pair pass's grid and slot bound), which a rebuild can change without moving a buffer
    std::vector<int64_t> shape{c->n_directed, c->n_inj_targets, c->n_inj_entries};
    if (g_generation != gen0 || c->n_inj_targets != targets0 || shape != c->graph_shape) drop_graphs(c);
    c->graph_shape = shape;
    if (h_out) {
        // h in caller order
        RT_TRY(field_out(c, c->h_d.as<double>(), h_out, 1));
    }
    c->built = true;
    return RT_OK;
}

rt_status rt_neighbours(rt_ctx* c, const double* x, const double* m, const double* xsrc, double* h_out) {
    return neighbours(c, x, m, xsrc, h_out, nullptr, nullptr);
}

rt_status rt_neighbours_given_h(rt_ctx* c, const double* x, const double* m, const double* xsrc, const double* h_in,
                                const double* hs_in) {
    if (!c) return RT_ERR_INVALID;
    if (!h_in) return fail(c, RT_ERR_INVALID, "h_dev is NULL");
    if (c->n_src > 0 && !hs_in) return fail(c, RT_ERR_INVALID, "hs_dev is NULL with n_src > 0");
    return neighbours(c, x, m, xsrc, nullptr, h_in, hs_in);
}

rt_status rt_neighbours_given_fields(rt_ctx* c, const double* x, const double* m, const double* xsrc,
                                     const double* h_in, const double* hs_in, const double* omegas_in,
                                     const double* octw_in) {
    if (!c) return RT_ERR_INVALID;
    if (!h_in) return fail(c, RT_ERR_INVALID, "h_dev is NULL");
    if (c->n_src > 0 && (!hs_in || !omegas_in || !octw_in))
        return fail(c, RT_ERR_INVALID, "hs_dev, omegas_dev or octw_dev is NULL with n_src > 0");
    return neighbours(c, x, m, xsrc, nullptr, h_in, hs_in, omegas_in, octw_in);
}

rt_status rt_source_norms(rt_ctx* c, double* omegas_dev, double* octw_dev) {
    RT_TRY(check_ready(c));
    if (c->n_src == 0) return RT_OK;
    if (!omegas_dev || !octw_dev) return fail(c, RT_ERR_INVALID, "NULL omegas_dev or octw_dev");
    RT_CUDA(c, cudaMemcpyAsync(omegas_dev, c->omegas_d.p, (size_t)c->n_src * 8, cudaMemcpyDeviceToDevice, c->stream));
    RT_CUDA(c, cudaMemcpyAsync(octw_dev, c->omegas_d.as<double>() + c->n_src, (size_t)c->n_src * 64,
                               cudaMemcpyDeviceToDevice, c->stream));
    return RT_OK;
}

rt_status rt_source_fields(rt_ctx* c, double* hs_dev) {
    RT_TRY(check_ready(c));
    if (!hs_dev) return fail(c, RT_ERR_INVALID, "hs_dev is NULL");
    if (c->n_src > 0)
        RT_CUDA(c, cudaMemcpyAsync(hs_dev, c->hs_d.p, (size_t)c->n_src * 8, cudaMemcpyDeviceToDevice, c->stream));
    return RT_OK;
}

rt_status rt_set_owned(rt_ctx* c, int64_t n_owned) {
    if (!c) return RT_ERR_INVALID;
    c->err.clear();
    if (n_owned < 0 || n_owned > c->n) return fail(c, RT_ERR_INVALID, "n_owned must be in [0, n]");
    c->n_owned = n_owned;
    return RT_OK;
}

rt_status rt_gradients(rt_ctx* c, const void* U, void* gradU) {
    RT_TRY(check_ready(c));
    if (!U || !gradU) return fail(c, RT_ERR_INVALID, "NULL array");
    const int G = c->cfg.n_groups;
    RT_TRY(state_in(c, U, c->U_a.p, 4 * G, 4 * G, 0));
    RT_TRY(launch_gradient(c, c->stream, c->U_a.p));
    RT_TRY(state_out(c, c->grad_t.p, gradU, 12 * G, 12 * G, 0));
    return RT_OK;
}

rt_status rt_step_bins(rt_ctx* c, void* U, const double* Lsrc, const double* alpha) {
    RT_TRY(check_ready(c));
    if (!U) return fail(c, RT_ERR_INVALID, "U_dev is NULL");
    if (!c->has_bins) return fail(c, RT_ERR_STATE, "rt_set_time_bins has not been called since rt_neighbours");
    const int G = c->cfg.n_groups;
    const bool has_src = Lsrc && c->n_src > 0 && c->n_inj_targets > 0;
    RT_TRY(state_in(c, U, c->U_a.p, 4 * G, 4 * G, 0));
    RT_TRY(set_step_inputs(c, c->dt_min, Lsrc, alpha));
    RT_CUDA(c, cudaMemsetAsync(c->acc_t.p, 0, (size_t)32 * G * c->n, c->stream));   // 32 B per (particle, group)
    for (int s = 0; s < (1 << c->bins_max); ++s)
        RT_TRY(launch_step_bins(c, c->stream, s, c->U_a.p, has_src, alpha != nullptr));
    RT_TRY(state_out(c, c->U_a.p, U, 4 * G, 4 * G, 0));
    return RT_OK;
}

rt_status rt_drift(rt_ctx* c, void* U, const double* v, double dt_drift) {
    RT_TRY(check_ready(c));
    if (!U || !v) return fail(c, RT_ERR_INVALID, "NULL array");
    if (!std::isfinite(dt_drift)) return fail(c, RT_ERR_INVALID, "dt_drift must be finite");
    const int G = c->cfg.n_groups;
    RT_TRY(state_in(c, U, c->U_a.p, 4 * G, 4 * G, 0));
    RT_TRY(launch_gradient(c, c->stream, c->U_a.p));
    RT_TRY(launch_drift(c, c->stream, c->U_a.p, v, dt_drift));
    RT_TRY(state_out(c, c->U_a.p, U, 4 * G, 4 * G, 0));
    return RT_OK;
}

rt_status rt_transport_step(rt_ctx* c, double dt, void* U, const double* Lsrc, const double* alpha) {
    RT_TRY(check_ready(c));
    if (!U) return fail(c, RT_ERR_INVALID, "U_dev is NULL");
    if (!std::isfinite(dt) || dt < 0) return fail(c, RT_ERR_INVALID, "dt must be finite and >= 0");
    const int G = c->cfg.n_groups;
    bool has_src = Lsrc && c->n_src > 0 && c->n_inj_targets > 0;
    RT_TRY(state_in(c, U, c->U_a.p, 4 * G, 4 * G, 0));
    RT_TRY(set_step_inputs(c, dt, Lsrc, alpha));
    if (c->profiling) {
        destroy_prof(c->plain_prof);
        c->prof_sink = &c->plain_prof;
        c->prof_pairs = 0;
    }
    rt_status s = launch_step(c, c->stream, c->U_a.p, c->U_b.p, has_src, alpha != nullptr);
    c->prof_sink = nullptr;
    if (c->profiling) c->last_prof = &c->plain_prof;
    RT_TRY(s);
    RT_TRY(state_out(c, c->U_b.p, U, 4 * G, 4 * G, 0));
    return RT_OK;
}

rt_status rt_transport_step_given_gradients(rt_ctx* c, double dt, void* U, const void* gradU, const double* alpha) {
    RT_TRY(check_ready(c));
    if (!U || !gradU) return fail(c, RT_ERR_INVALID, "U_dev or gradU_dev is NULL");
    if (!std::isfinite(dt) || dt < 0) return fail(c, RT_ERR_INVALID, "dt must be finite and >= 0");
    const int G = c->cfg.n_groups;
    RT_TRY(state_in(c, U, c->U_a.p, 4 * G, 4 * G, 0));
    RT_TRY(state_in(c, gradU, c->grad_t.p, 12 * G, 12 * G, 0));
    RT_TRY(set_step_inputs(c, dt, nullptr, alpha));
    RT_TRY(launch_flux_given(c, c->stream, c->U_a.p, c->U_b.p, alpha != nullptr));
    RT_TRY(state_out(c, c->U_b.p, U, 4 * G, 4 * G, 0));
    return RT_OK;
}

rt_status rt_set_fields(rt_ctx* c, int64_t first, int64_t count, const double* omega, const double* B) {
    RT_TRY(check_ready(c));
    if (first < 0 || count < 0 || first > c->n || count > c->n - first)
        return fail(c, RT_ERR_INVALID, "rt_set_fields: [first, first + count) must lie in [0, N)");
    if (count > 0 && (!omega || !B)) return fail(c, RT_ERR_INVALID, "rt_set_fields: NULL omega or B");
    return set_fields(c, first, count, omega, B);
}

rt_status rt_inject(rt_ctx* c, double dt, void* U, const double* Lsrc) {
    RT_TRY(check_ready(c));
    if (!U) return fail(c, RT_ERR_INVALID, "U_dev is NULL");
    if (!std::isfinite(dt) || dt < 0) return fail(c, RT_ERR_INVALID, "dt must be finite and >= 0");
    if (!Lsrc || c->n_src == 0 || c->n_inj_targets == 0) return RT_OK;
    const int G = c->cfg.n_groups;
    RT_TRY(state_in(c, U, c->U_a.p, 4 * G, 4 * G, 0));
    RT_TRY(set_step_inputs(c, dt, Lsrc, nullptr));
    RT_TRY(launch_inject(c, c->stream, c->U_a.p));
    RT_TRY(state_out(c, c->U_a.p, U, 4 * G, 4 * G, 0));
    return RT_OK;
}

rt_status rt_subcycle(rt_ctx* c, int32_t n_sub, double dt, void* U, const double* Lsrc, const double* alpha) {
    RT_TRY(check_ready(c));
    if (!U) return fail(c, RT_ERR_INVALID, "U_dev is NULL");
    if (n_sub < 0 || n_sub > 100000) return fail(c, RT_ERR_INVALID, "n_sub must be in [0, 100000]");
    if (!std::isfinite(dt) || dt < 0) return fail(c, RT_ERR_INVALID, "dt must be finite and >= 0");
    if (n_sub == 0) return RT_OK;
    const int G = c->cfg.n_groups;
    bool has_src = Lsrc && c->n_src > 0 && c->n_inj_targets > 0;
    bool has_alpha = alpha != nullptr;
    RT_TRY(state_in(c, U, c->U_a.p, 4 * G, 4 * G, 0));
    RT_TRY(set_step_inputs(c, dt, Lsrc, alpha));
    // sub-cycles after the first take their injection from the previous gather
    RT_TRY(set_dense_injection(c, has_src && n_sub > 1));
    GraphKey key{n_sub, has_src ? 1 : 0, has_alpha ? 1 : (c->has_alpha_g ? 2 : 0)};
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
        GraphEntry entry;
        cudaGraph_t graph = nullptr;
        RT_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        void* a = c->U_a.p;
        void* b = c->U_b.p;
        rt_status s = RT_OK;
        int64_t l0 = c->launches;
        c->prof_sink = c->profiling ? &entry.prof : nullptr;
        c->prof_pairs = 0;
        for (int k = 0; k < n_sub && s == RT_OK; ++k) {
            s = launch_step(c, c->cap_stream, a, b, has_src, has_alpha, k == 0, k + 1 < n_sub);
            std::swap(a, b);
        }
        c->prof_sink = nullptr;
        entry.kernels = c->launches - l0;
        c->launches = l0;
        cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
        if (s != RT_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            destroy_prof(entry.prof);
            if (s != RT_OK) return s;
            return cuda_fail(c, e, "cudaStreamEndCapture");
        }
        e = cudaGraphInstantiate(&entry.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            destroy_prof(entry.prof);
            return cuda_fail(c, e, "cudaGraphInstantiate");
        }
        it = c->graphs.emplace(key, entry).first;
    }
    RT_CUDA(c, cudaGraphLaunch(it->second.exec, c->stream));
    c->launches += it->second.kernels;
    if (c->profiling) c->last_prof = &it->second.prof;
    void* fin = (n_sub % 2 == 0) ? c->U_a.p : c->U_b.p;
    RT_TRY(state_out(c, fin, U, 4 * G, 4 * G, 0));
    return RT_OK;
}

rt_status rt_adjoint(rt_ctx* c, int32_t n_sub, double dt, int32_t ckpt_every, const void* U0, const double* Lsrc,
                     const double* alpha, const void* dLdU_final, void* dLdU0, double* dLdLsrc) {
    RT_TRY(check_ready(c));
    if (!U0 || !dLdU_final || !dLdU0) return fail(c, RT_ERR_INVALID, "NULL array");
    if (n_sub < 1 || n_sub > 100000) return fail(c, RT_ERR_INVALID, "n_sub must be in [1, 100000]");
    if (ckpt_every < 1) return fail(c, RT_ERR_INVALID, "ckpt_every must be >= 1");
    if (c->cfg.riemann_solver != RT_RIEMANN_GLF)
        return fail(c, RT_ERR_INVALID, "rt_adjoint differentiates the GLF flux only (riemann_solver = RT_RIEMANN_GLF)");
    if (c->has_alpha_g && !alpha)
        return fail(c, RT_ERR_INVALID, "rt_adjoint differentiates the grey sink only (clear the absorbers)");
    if (!std::isfinite(dt) || dt < 0) return fail(c, RT_ERR_INVALID, "dt must be finite and >= 0");
    const int G = c->cfg.n_groups;
    bool has_src = Lsrc && c->n_src > 0 && c->n_inj_targets > 0;
    RT_TRY(set_step_inputs(c, dt, Lsrc, alpha));
    RT_TRY(ensure(c, c->lam_a, (size_t)4 * G * c->n * tsize(c), "adjoint"));
    RT_TRY(ensure(c, c->lam_b, (size_t)4 * G * c->n * tsize(c), "adjoint"));
    RT_TRY(state_in(c, U0, c->U_a.p, 4 * G, 4 * G, 0));
    RT_TRY(state_in(c, dLdU_final, c->lam_a.p, 4 * G, 4 * G, 0));
    if (dLdLsrc && c->n_src > 0)
        RT_CUDA(c, cudaMemsetAsync(dLdLsrc, 0, (size_t)c->n_src * G * sizeof(double), c->stream));
    RT_TRY(run_adjoint(c, n_sub, ckpt_every, has_src, alpha != nullptr, c->U_a.p, c->lam_a.p, c->lam_b.p,
                       (dLdLsrc && c->n_src > 0) ? dLdLsrc : nullptr));
    RT_TRY(state_out(c, c->lam_b.p, dLdU0, 4 * G, 4 * G, 0));
    return RT_OK;
}

rt_status rt_energy(rt_ctx* c, const void* U, double* E_host) {
    RT_TRY(check_ready(c));
    if (!U || !E_host) return fail(c, RT_ERR_INVALID, "NULL array");
    const int G = c->cfg.n_groups;
    RT_TRY(state_in(c, U, c->U_a.p, 4 * G, 4 * G, 0));
    double* out = c->energy_part.as<double>() + (size_t)G * 512;
    RT_TRY(launch_energy(c, c->stream, c->U_a.p, out));
    RT_CUDA(c, cudaMemcpyAsync(E_host, out, G * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    int timed_out = 0;
    RT_CUDA(c, cudaMemcpyAsync(&timed_out, c->flags.as<int>() + F_TIMEOUT, sizeof(int), cudaMemcpyDeviceToHost,
                               c->stream));
    RT_CUDA(c, cudaStreamSynchronize(c->stream));
    if (timed_out)
        return fail(c, RT_ERR_TIMEOUT, "a device-side wait of the pair kernel ran out since the last rt_neighbours");
    return RT_OK;
}

rt_status rt_particle_fields(rt_ctx* c, double* h, double* omega, double* V, double* B) {
    RT_TRY(check_ready(c));
    if (h) RT_TRY(field_out(c, c->h_d.as<double>(), h, 1));
    if (omega) RT_TRY(field_out(c, c->omega_d.as<double>(), omega, 1));
    if (V) RT_TRY(field_out(c, c->V_d.as<double>(), V, 1));
    if (B) {
        // [6][N] sorted -> [N][3][3] caller order
        static const int map[9] = {0, 3, 4, 3, 1, 5, 4, 5, 2};
        RT_TRY(ensure(c, c->seg, (size_t)6 * c->n * 8, "scratch"));
        RT_TRY(field_out(c, c->B_d.as<double>(), c->seg.as<double>(), 6));
        for (int q = 0; q < 9; ++q)
            RT_CUDA(c, cudaMemcpy2DAsync(B + q, 9 * sizeof(double), c->seg.as<double>() + (size_t)map[q] * c->n,
                                         sizeof(double), sizeof(double), c->n, cudaMemcpyDeviceToDevice, c->stream));
    }
    return RT_OK;
}

}  // extern "C"

namespace rt {
__global__ void k_pairs_export(const int64_t* __restrict__ row_off, const int32_t* __restrict__ cols,
                               const int32_t* __restrict__ perm, const int32_t* __restrict__ inv_perm, int64_t n,
                               const int64_t* __restrict__ out_off, int32_t* out_cols) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t p = inv_perm[i];
    int64_t b = row_off[p], e = row_off[p + 1], o = out_off[i];
    for (int64_t k = b; k < e; ++k) out_cols[o + (k - b)] = perm[cols[k]];
}

__global__ void k_row_counts(const int64_t* __restrict__ row_off, const int32_t* __restrict__ inv_perm, int64_t n,
                             int64_t* cnt) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t p = inv_perm[i];
    cnt[i] = row_off[p + 1] - row_off[p];
}
}  // namespace rt

extern "C" {

rt_status rt_pairs(rt_ctx* c, int64_t* offsets, int32_t* cols) {
    RT_TRY(check_ready(c));
    if (!offsets || !cols) return fail(c, RT_ERR_INVALID, "NULL array");
    const int64_t n = c->n;
    // counts in caller order -> host prefix sum (diagnostic path, not the hot path)
    RT_TRY(ensure(c, c->seg, (size_t)(n + 1) * 8, "scratch"));
    int64_t* cnt = c->seg.as<int64_t>();
    k_row_counts<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->row_off.as<int64_t>(),
                                                                      c->inv_perm.as<int32_t>(), n, cnt);
    ++c->launches;
    std::string err;
    int64_t* h = new (std::nothrow) int64_t[n + 1];
    if (!h) return fail(c, RT_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaMemcpyAsync(h + 1, cnt, n * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        delete[] h;
        return cuda_fail(c, e, "rt_pairs counts");
    }
    h[0] = 0;
    for (int64_t i = 0; i < n; ++i) h[i + 1] += h[i];
    e = cudaMemcpyAsync(offsets, h, (n + 1) * 8, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    delete[] h;
    if (e != cudaSuccess) return cuda_fail(c, e, "rt_pairs offsets");
    k_pairs_export<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
        c->row_off.as<int64_t>(), c->cols.as<int32_t>(), c->perm.as<int32_t>(), c->inv_perm.as<int32_t>(), n, offsets,
        cols);
    ++c->launches;
    RT_CUDA(c, cudaGetLastError());
    return RT_OK;
}

rt_status rt_diagnostics(rt_ctx* c, rt_diag* out) {
    if (!c || !out) return RT_ERR_INVALID;
    c->err.clear();
    unsigned long long cl = 0;
    int timed_out = 0;
    if (c->flags.p) {
        RT_CUDA(c, cudaMemcpyAsync(&cl, c->flags.as<int>() + F_CLAMP, 8, cudaMemcpyDeviceToHost, c->stream));
        RT_CUDA(c, cudaMemcpyAsync(&timed_out, c->flags.as<int>() + F_TIMEOUT, sizeof(int), cudaMemcpyDeviceToHost,
                                   c->stream));
        RT_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    c->diag.clamp_events = (int64_t)cl;
    c->diag.wait_timeouts = timed_out;
    // the float gradient runs one thread per (particle, group) in variants 1 and 2
    const int gc = c->cfg.n_groups < kMaxGC ? c->cfg.n_groups : kMaxGC;
    c->diag.threads_per_particle = (!c->fp64 && c->tune.gradient_variant >= 1) ? gc : 1;
    c->diag.kernel_launches = c->launches;
    *out = c->diag;
    return RT_OK;
}

rt_status rt_set_profiling(rt_ctx* c, int32_t on) {
    if (!c) return RT_ERR_INVALID;
    c->err.clear();
    if (on < 0 || on > 1000) return fail(c, RT_ERR_INVALID, "rt_set_profiling: on must be in [0, 1000]");
    const int v = on;
    if (v != c->profiling) {
        RT_CUDA(c, cudaStreamSynchronize(c->stream));
        drop_graphs(c);
        destroy_prof(c->plain_prof);
        c->profiling = v;
    }
    return RT_OK;
}

rt_status rt_kernel_times(rt_ctx* c, double* ms, int64_t* launches) {
    if (!c || !ms || !launches) return RT_ERR_INVALID;
    c->err.clear();
    for (int k = 0; k < RT_KERNEL_KINDS; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    if (!c->last_prof) return RT_OK;
    RT_CUDA(c, cudaStreamSynchronize(c->stream));
    for (const ProfRec& r : *c->last_prof) {
        float t = 0.f;
        RT_CUDA(c, cudaEventElapsedTime(&t, r.start, r.stop));
        if (r.kind >= 0 && r.kind < RT_KERNEL_KINDS) {
            ms[r.kind] += t;
            launches[r.kind] += 1;
        }
    }
    return RT_OK;
}

rt_status rt_set_tuning(rt_ctx* c, const rt_tuning* t) {
    if (!c) return RT_ERR_INVALID;
    c->err.clear();
    if (!t) return fail(c, RT_ERR_INVALID, "rt_set_tuning: NULL tuning");
    if (t->flux_variant < 0 || t->flux_variant > 2 || t->gather_variant < 0 || t->gather_variant > 1 ||
        t->gradient_variant < 0 || t->gradient_variant > 2)
        return fail(c, RT_ERR_INVALID,
                    "rt_set_tuning: flux_variant and gradient_variant must be 0, 1 or 2, gather_variant 0 or 1");
    rt_tuning v = *t;
    if (v.cell_eighths == 0) v.cell_eighths = c->tune.cell_eighths;
    const int gb = v.gradient_block, hb = v.gather_block, pw = v.pair_warps;
    if (v.cell_eighths < 2 || v.cell_eighths > 16 || !(gb == 0 || gb == 32 || gb == 64 || gb == 128 || gb == 256) ||
        !(hb == 0 || (hb >= 64 && hb <= 512 && hb % 32 == 0)) || !(pw == 0 || pw == 1 || pw == 2 || pw == 4))
        return fail(c, RT_ERR_INVALID,
                    "rt_set_tuning: cell_eighths in [2, 16], gradient_block 0/32/64/128/256, gather_block 0 or a "
                    "multiple of 32 in [64, 512], pair_warps 0/1/2/4");
    if (std::memcmp(&v, &c->tune, sizeof(v)) != 0) {
        RT_CUDA(c, cudaStreamSynchronize(c->stream));
        drop_graphs(c);
        c->tune = v;
    }
    return RT_OK;
}

// candidate k of rt_autotune: flux variant k / 6, gather variant (k / 3) % 2, gradient variant k % 3
static rt_tuning tune_candidate(const rt_tuning& shape, int k) {
    rt_tuning t = shape;
    t.flux_variant = k / 6;
    t.gather_variant = (k / 3) % 2;
    t.gradient_variant = k % 3;
    return t;
}

rt_status rt_autotune(rt_ctx* c, const void* U, double dt, int32_t n_sub, const double* Lsrc, const double* alpha,
                      int32_t repeats, rt_tuning* best, double* ms_out) {
    RT_TRY(check_ready(c));
    if (!U || !best) return fail(c, RT_ERR_INVALID, "rt_autotune: NULL U or best");
    if (n_sub < 1 || n_sub > 1000) return fail(c, RT_ERR_INVALID, "rt_autotune: n_sub must be in [1, 1000]");
    if (repeats < 1 || repeats > 100) return fail(c, RT_ERR_INVALID, "rt_autotune: repeats must be in [1, 100]");
    if (!std::isfinite(dt) || dt < 0) return fail(c, RT_ERR_INVALID, "dt must be finite and >= 0");
    const int G = c->cfg.n_groups;
    const bool has_src = Lsrc && c->n_src > 0 && c->n_inj_targets > 0;
    const bool has_alpha = alpha != nullptr;
    RT_TRY(set_step_inputs(c, dt, Lsrc, alpha));
    const rt_tuning saved = c->tune;
    int best_k = -1;
    double best_ms = 0.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rt_status st = RT_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        st = fail(c, RT_ERR_CUDA, "rt_autotune: cudaEventCreate failed");
    }
    for (int k = 0; k < RT_TUNE_CANDIDATES && st == RT_OK; ++k) {
        c->tune = tune_candidate(saved, k);
        if (c->fp64 && k > 0) {       // the double path has one variant
            if (ms_out) ms_out[k] = ms_out[0];
            continue;
        }
        double kbest = 0.0;
        for (int r = 0; r <= repeats && st == RT_OK; ++r) {   // r = 0 warms up
            st = state_in(c, U, c->U_a.p, 4 * G, 4 * G, 0);
            if (st != RT_OK) break;
            void* a = c->U_a.p;
            void* b = c->U_b.p;
            if (cudaEventRecord(e0, c->stream) != cudaSuccess) st = fail(c, RT_ERR_CUDA, "cudaEventRecord");
            for (int i = 0; i < n_sub && st == RT_OK; ++i) {
                st = launch_step(c, c->stream, a, b, has_src, has_alpha);
                std::swap(a, b);
            }
            if (st != RT_OK) break;
            float t = 0.f;
            if (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
                st = fail(c, RT_ERR_CUDA, "rt_autotune: event timing failed");
                break;
            }
            if (r == 1 || (r > 1 && t < kbest)) kbest = t;
        }
        if (st != RT_OK) break;
        if (ms_out) ms_out[k] = kbest;
        if (best_k < 0 || kbest < best_ms) {
            best_k = k;
            best_ms = kbest;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    c->tune = saved;
    if (st != RT_OK) return st;
    const rt_tuning win = c->fp64 ? saved : tune_candidate(saved, best_k);
    *best = win;
    return rt_set_tuning(c, &win);
}

rt_status rt_wait_selftest(rt_ctx* c, uint64_t budget_cycles) {
    if (!c) return RT_ERR_INVALID;
    c->err.clear();
    if (budget_cycles < 1 || budget_cycles > 4000000000ull)
        return fail(c, RT_ERR_INVALID, "rt_wait_selftest: budget_cycles must be in [1, 4e9]");
    RT_CUDA(c, cudaSetDevice(c->device));
    bool ran_out = false;
    RT_TRY(wait_selftest(c, budget_cycles, &ran_out));
    if (ran_out) return fail(c, RT_ERR_TIMEOUT, "rt_wait_selftest: the bounded wait ran out, as expected");
    return RT_OK;
}

rt_status rt_get_tuning(const rt_ctx* c, rt_tuning* t) {
    if (!c || !t) return RT_ERR_INVALID;
    *t = c->tune;
    return RT_OK;
}

const char* rt_last_error(const rt_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

void rt_destroy(rt_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    destroy_prof(c->plain_prof);
    DevBuf* bufs[] = {&c->keys_in, &c->keys_out, &c->idx_in, &c->perm, &c->inv_perm, &c->cell_start, &c->cub_tmp,
                      &c->xs_d, &c->xq, &c->m_s, &c->h_d, &c->H2f, &c->h_prev, &c->omega_d, &c->V_d, &c->B_d, &c->cond_d, &c->pos_t,
                      &c->geo_t, &c->omega_t, &c->counts, &c->row_off, &c->cols, &c->cols_cap, &c->blk, &c->pkeys, &c->pkeys_alt, &c->n_low,
                      &c->n_up, &c->up_off, &c->low_slot, &c->pair_ends, &c->pairbuf, &c->flags, &c->red_tmp,
                      &c->xsrc_d, &c->hs_d, &c->omegas_d, &c->src_counts, &c->src_off, &c->inj_key,
                      &c->inj_key_out, &c->inj_val, &c->inj_val_out, &c->inj_targets, &c->inj_off, &c->inj_src,
                      &c->inj_coef, &c->src_entry_gas, &c->src_entry_xi, &c->U_a, &c->U_b, &c->grad_t, &c->frec, &c->wave_t, &c->alpha_g_c, &c->alpha_g_s,
                      &c->sigma_d, &c->bins_s, &c->bins_tmp, &c->acc_t, &c->bins_nmin, &c->order_b, &c->order_m,
                      &c->order_q, &c->bin_keys, &c->bin_keys2, &c->bin_vals, &c->bin_cub, &c->bin_hist, &c->alpha_s,
                      &c->L_dev, &c->dt_dev, &c->energy_part, &c->ck, &c->seg, &c->lam_a, &c->lam_b, &c->adj_w,
                      &c->adj_x, &c->adj_ub, &c->adj_gam, &c->adj_lam};
    for (DevBuf* b : bufs) free_buf(*b);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

}  // extern "C"
