// Internal declarations of the GB300 photon-transport library: the context, device
// buffers, and the per-pair device arithmetic shared by the forward and adjoint kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/rt.h"

namespace rt {

// H = kKappa * h for the 3D cubic spline (Dehnen & Aly 2012, Table 1, as used by the thesis).
constexpr double kKappa = 1.825742;
// sigma = 16 / pi, Eq. cubic-spline-kernel in 3D.
constexpr double kSigma = 5.0929581789406507446;   // 16 / pi
// int slots of the context's 64-byte flag buffer (cleared by every rt_neighbours): error
// flags of the build, the clamp counter (64-bit, slots 8-9) and the device-wait time-out flag
enum FlagSlot { F_BADPOS = 0, F_NOCONV = 1, F_GEOM = 2, F_ILL = 3, F_SRC_NOCONV = 4, F_REFINE = 5, F_BADH = 6,
                F_NSLOTS = 8, F_CLAMP = 8,
                F_TIMEOUT = 12, F_SCRATCH = 13, F_ROWMAX = 14, F_SELFTEST = 15 };
constexpr int kMaxGC = 4;                          // groups handled by one pair-kernel launch
// Packed flux rows start with a prefix that repeats their last kRowRot words: a row copy that
// starts at word kRowRot delivers the row, one that starts at word 0 delivers it rotated by
// four 16-byte chunks (the pair pass uses both, see k_flux_tma).
constexpr int kRowRot = 16;

// ------------------------------------------------------------------------------------
// Device buffer that only grows.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

struct GraphKey {
    int n_sub, has_src, has_alpha;   // has_alpha: 0 none, 1 grey, 2 per group
    bool operator<(const GraphKey& o) const {
        return std::tie(n_sub, has_src, has_alpha) < std::tie(o.n_sub, o.has_src, o.has_alpha);
    }
};

// events recorded around one profiled launch
struct ProfRec {
    int kind;
    cudaEvent_t start, stop;
};

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;               // kernel nodes per replay
    std::vector<ProfRec> prof;         // event nodes (profiling on)
};

}  // namespace rt

struct rt_ctx {
    rt_config cfg{};
    int64_t n = 0, n_src = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    int device = 0, sm_count = 0;
    std::string err;
    bool built = false;
    bool fp64 = true;

    // cell list
    int nc[3] = {1, 1, 1};
    double cell[3] = {1, 1, 1};
    int64_t ncells = 0;
    int key_bits = 1;

    // build buffers
    rt::DevBuf keys_in, keys_out, idx_in, perm, inv_perm, cell_start, cell_end, cub_tmp;
    rt::DevBuf xs_d, xq, m_s;
    rt::DevBuf h_d, omega_d, V_d, B_d, cond_d;           // double per particle
    rt::DevBuf H2f;                                     // float (kappa h)^2, pair-search prefilter
    rt::DevBuf h_prev;                                  // h of the last call, caller order (first guess)
    bool has_h_prev = false;
    bool has_hs_prev = false;                           // hs_d holds the sources' h of the last call
    rt::DevBuf pos_t, geo_t, omega_t;                   // working precision per particle (pair kernels)
    rt::DevBuf counts, row_off, cols;                   // symmetric pair lists (CSR), rows ascending
    // rows of row_cap entries that the counting walk of the pair search also fills (0: off);
    // set from the longest row of the last call
    rt::DevBuf cols_cap;
    int64_t row_cap = 0;
    rt::DevBuf blk;                                     // coarse blocks: largest H and reach radius
    rt::DevBuf pkeys, pkeys_alt;                        // (row, col) keys of the sort-based build
    rt::DevBuf n_low, n_up, up_off, low_slot, pair_ends; // lower / upper split, pair slots
    rt::DevBuf pairbuf;                                 // per-pair fluxes of one group chunk
    // sizes that captured graphs bake in besides buffer addresses (pair count, injection
    // targets and entries): a rebuild that changes them drops the graphs
    std::vector<int64_t> graph_shape;
    rt::DevBuf flags;                                   // int32 error flags + counters
    rt::DevBuf red_tmp;                                 // small reduction scratch (double)
    int64_t n_directed = 0;
    int64_t n_owned = 0;                                // rt_energy sums caller indices [0, n_owned)

    // sources / injection
    rt::DevBuf xsrc_d, hs_d, omegas_d, src_counts, src_off, inj_key, inj_key_out, inj_val, inj_val_out;
    rt::DevBuf inj_targets, inj_off, inj_src, inj_coef, src_entry_gas, src_entry_xi;
    int64_t n_inj_entries = 0, n_inj_targets = 0;

    // state records (sorted order, working precision): U [N][4G] (double-buffered), grad U [N][12G]
    rt::DevBuf U_a, U_b, grad_t, alpha_s, L_dev, dt_dev, energy_part;
    rt::DevBuf inj_dense;                               // dt sum coef L per (particle, group), [N][G] double
    bool inj_dense_ready = false;                       // filled by set_step_inputs for this call
    rt::DevBuf frec;                                    // packed float flux-input rows (G <= 4)
    rt::DevBuf wave_t;                                  // HLL wave-speed table, working precision
    // photo-ionisation sink per group (rt_set_absorbers): alpha in caller order [G][N]
    // (double), its sorted working-precision copy [N][G], the cross sections
    rt::DevBuf alpha_g_c, alpha_g_s, sigma_d;
    bool has_alpha_g = false;
    bool step_alpha_g = false;                          // the current call applies it
    // individual time bins (rt_set_time_bins): sorted int8 bins, flux accumulators [N][4G]
    rt::DevBuf bins_s, bins_tmp, acc_t;
    bool has_bins = false;
    int bins_max = 0;
    double dt_min = 0.0;
    // active sets: a particle starts at min-step s iff b <= ctz(s) (all at s = 0), touches a
    // starting partner iff nmin <= ctz(s), a pair interacts iff min(b_k, b_l) <= ctz(s); the
    // particles ordered by b and by nmin and the pair slots by level make every active set a
    // prefix (cum_*[level] = entries with a key <= level)
    rt::DevBuf bins_nmin, order_b, order_m, order_q, bin_keys, bin_keys2, bin_vals, bin_cub, bin_hist;
    std::vector<int64_t> cum_b, cum_m, cum_q;
    CUtensorMap rows_map{};                             // tensor map of frec (tile::gather4)
    const void* rows_map_for = nullptr;
    int64_t rows_map_n = 0;
    // adjoint
    rt::DevBuf ck, seg, lam_a, lam_b, adj_w, adj_x, adj_ub, adj_gam, adj_lam;
    int64_t ck_cap = 0, seg_cap = 0;

    // diagnostics
    rt_diag diag{};
    // launch variants of the float pair kernels (rt_set_tuning); the double path has one
    rt_tuning tune{2, 1, 2, 4, 0, 0, 0};

    std::map<rt::GraphKey, rt::GraphEntry> graphs;

    // tracing
    int profiling = 0;                       // rt_set_profiling's mode
    int64_t prof_pairs = 0;                  // pair-pass launches seen in the current call
    int64_t launches = 0;                    // own kernel launches (see rt_diag)
    std::vector<rt::ProfRec>* prof_sink = nullptr;   // where launch helpers append records
    std::vector<rt::ProfRec> plain_prof;     // records of the last plain step
    const std::vector<rt::ProfRec>* last_prof = nullptr;
};

// ------------------------------------------------------------------------------------
// Host helpers (rt_api.cu)
namespace rt {
rt_status fail(rt_ctx* c, rt_status s, const std::string& msg);
rt_status cuda_fail(rt_ctx* c, cudaError_t e, const char* what);
rt_status ensure(rt_ctx* c, DevBuf& b, size_t bytes, const char* what);
// HLL wave speeds over (f, theta), [RT_WAVE_NF][RT_WAVE_NTH] each (rt_hll.cu)
void build_wave_table(double* lmax, double* lmin);
// record a start event before a profiled launch (returns the index, or -1 when off)
int prof_begin(rt_ctx* c, cudaStream_t s, int kind);
void prof_end(rt_ctx* c, cudaStream_t s, int idx);
}  // namespace rt

#define RT_CUDA(ctx, call)                                         \
    do {                                                           \
        cudaError_t e__ = (call);                                  \
        if (e__ != cudaSuccess) return rt::cuda_fail(ctx, e__, #call); \
    } while (0)

#define RT_TRY(call)                       \
    do {                                   \
        rt_status s__ = (call);            \
        if (s__ != RT_OK) return s__;      \
    } while (0)

// entry points of the kernel files
namespace rt {
// h_in [N] / hs_in [S] (caller order, device): given smoothing lengths (no solve), or NULL;
// with them, oms_in [S] / octw_in [S][8]: the sources' omega_s and octant sums, or NULL
rt_status build_neighbours(rt_ctx* c, const double* x, const double* m, const double* xsrc,
                           const double* h_in = nullptr, const double* hs_in = nullptr,
                           const double* oms_in = nullptr, const double* octw_in = nullptr);
// caller-order component-major arrays <-> sorted records (comps values at record offset off)
rt_status state_in(rt_ctx* c, const void* U_user, void* rec, int comps, int RS, int off);
rt_status state_out(rt_ctx* c, const void* rec, void* U_user, int comps, int RS, int off);
// sorted double per-particle fields [comps][N] -> caller order
rt_status field_out(rt_ctx* c, const double* src_sorted, double* dst_user, int comps);
rt_status set_step_inputs(rt_ctx* c, double dt, const double* Lsrc, const double* alpha);
// fills inj_dense from the inputs of set_step_inputs (when on and there are targets)
rt_status set_dense_injection(rt_ctx* c, bool on);
// rt_wait_selftest's kernel: *ran_out = the bounded wait on a never-completed barrier ran out
rt_status wait_selftest(rt_ctx* c, unsigned long long budget, bool* ran_out);
// one sub-cycle: injection (if inject_first), gradients, pair fluxes, update and sink; with
// inject_after the gather also adds the next sub-cycle's injection (inj_dense), which then
// starts with inject_first = false
rt_status launch_step(rt_ctx* c, cudaStream_t s, void* Uin, void* Uout, bool has_src, bool has_alpha,
                      bool inject_first = true, bool inject_after = false);
rt_status launch_gradient(rt_ctx* c, cudaStream_t s, void* rec);
// the flux stage (pair fluxes, update, sink) with the gradients already in grad_t (sorted)
rt_status launch_flux_given(rt_ctx* c, cudaStream_t s, void* Uin, void* Uout, bool has_alpha);
// omega, V and B of caller particles [first, first + count) given (device, double)
rt_status set_fields(rt_ctx* c, int64_t first, int64_t count, const double* omega, const double* B);
// one min-step `step` of a hydro step with individual time bins (c->bins_s, c->acc_t)
rt_status launch_step_bins(rt_ctx* c, cudaStream_t s, int step, void* U, bool has_src, bool has_alpha);
// rec += grad_t . (v dt) per component (needs launch_gradient on rec first)
rt_status launch_drift(rt_ctx* c, cudaStream_t s, void* rec, const double* v, double dt);
rt_status launch_inject(rt_ctx* c, cudaStream_t s, void* rec);
rt_status launch_energy(rt_ctx* c, cudaStream_t s, const void* rec, double* out_dev);
rt_status run_adjoint(rt_ctx* c, int n_sub, int ckpt_every, bool has_src, bool has_alpha, const void* U0_sorted,
                      const void* lam_final_sorted, void* lam0_sorted, double* dLdL_dev);
}  // namespace rt

// ------------------------------------------------------------------------------------
// Device arithmetic shared by the forward and adjoint pair kernels.
namespace rt {

// Dimensionless cubic-spline shape w(q), q = r / H; W = sigma / H^3 * w(q)
// (Eq. cubic-spline-kernel; q = 0 in the first branch, zero for q >= 1).
template <class T>
__device__ __forceinline__ T spline_w(T q) {
    if (q >= T(1)) return T(0);
    T a = T(1) - q;
    T w = a * a * a;
    if (q <= T(0.5)) {
        T b = T(0.5) - q;
        w -= T(4) * b * b * b;
    }
    return w;
}

// d w / d q
template <class T>
__device__ __forceinline__ T spline_dw(T q) {
    if (q >= T(1)) return T(0);
    T a = T(1) - q;
    T d = T(-3) * a * a;
    if (q <= T(0.5)) {
        T b = T(0.5) - q;
        d += T(12) * b * b;
    }
    return d;
}


}  // namespace rt
