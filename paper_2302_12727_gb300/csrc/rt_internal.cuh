// Internal declarations of the GB300 photon-transport library: the context, device
// buffers, and the per-pair device arithmetic shared by the forward and adjoint kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <tuple>

#include "../../include/rt.h"

namespace rt {

// H = kKappa * h for the 3D cubic spline (Dehnen & Aly 2012, Table 1, as used by the thesis).
constexpr double kKappa = 1.825742;
// sigma = 16 / pi, Eq. cubic-spline-kernel in 3D.
constexpr double kSigma = 5.0929581789406507446;   // 16 / pi
constexpr int kMaxGC = 4;                          // groups handled by one pair-kernel launch

// ------------------------------------------------------------------------------------
// Device buffer that only grows.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

// Per-particle geometry consumed by the pair kernels, cell-sorted order.  For the double
// path positions are doubles; for the float path positions are 32-bit fixed point in units
// of box / 2^32, so that x_j - x_i is an exact integer difference whose wrap-around is the
// periodic minimal image.
template <class T>
struct Geom {
    const void* x;        // double[3][N] (T = double) or uint32[3][N] (T = float)
    const T* invH;        // 1 / H_i
    const T* h;           // h_i
    const T* omega;       // omega_i = 1 / V_i
    const T* Bp;          // [6][N]  V_i^2 sigma / H_i^3 * B_i  (xx, yy, zz, xy, xz, yz)
    T scale[3];           // fixed-point unit per axis (float path)
    double box[3];        // box (double path, minimal image)
    int periodic;
    int64_t n;
};

struct GraphKey {
    int n_sub, has_src, has_alpha;
    bool operator<(const GraphKey& o) const {
        return std::tie(n_sub, has_src, has_alpha) < std::tie(o.n_sub, o.has_src, o.has_alpha);
    }
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
    rt::DevBuf invH_t, h_t, omega_t, Bp_t;              // working precision per particle
    rt::DevBuf counts, row_off, cols;                   // symmetric pair lists (CSR)
    rt::DevBuf flags;                                   // int32 error flags + counters
    rt::DevBuf red_tmp;                                 // small reduction scratch (double)
    int64_t n_directed = 0;

    // sources / injection
    rt::DevBuf xsrc_d, hs_d, omegas_d, src_counts, src_off, inj_key, inj_key_out, inj_val, inj_val_out;
    rt::DevBuf inj_targets, inj_off, inj_src, inj_coef, src_entry_gas, src_entry_xi;
    int64_t n_inj_entries = 0, n_inj_targets = 0;

    // state (sorted order, working precision)
    rt::DevBuf U_a, U_b, grad, alpha_s, L_dev, dt_dev, energy_part;
    // adjoint
    rt::DevBuf ck, seg, lam_a, lam_b, gbar, lbar_part, lbar_acc;
    int64_t ck_cap = 0, seg_cap = 0;

    // diagnostics
    rt_diag diag{};
    int tpp = 1;   // threads per particle for pair kernels

    std::map<rt::GraphKey, cudaGraphExec_t> graphs;
};

// ------------------------------------------------------------------------------------
// Host helpers (rt_api.cu)
namespace rt {
rt_status fail(rt_ctx* c, rt_status s, const std::string& msg);
rt_status cuda_fail(rt_ctx* c, cudaError_t e, const char* what);
rt_status ensure(rt_ctx* c, DevBuf& b, size_t bytes, const char* what);
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
rt_status build_neighbours(rt_ctx* c, const double* x, const double* m, const double* xsrc);
rt_status to_sorted(rt_ctx* c, const void* U_user, void* U_sorted, int comps);
rt_status from_sorted(rt_ctx* c, const void* U_sorted, void* U_user, int comps);
rt_status set_step_inputs(rt_ctx* c, double dt, const double* Lsrc, const double* alpha);
rt_status launch_step(rt_ctx* c, cudaStream_t s, void* Uin, void* Uout, bool has_src, bool has_alpha);
rt_status launch_gradient(rt_ctx* c, cudaStream_t s, const void* U, void* grad);
rt_status launch_energy(rt_ctx* c, cudaStream_t s, const void* U_sorted, double* out_dev);
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

template <class T>
__device__ __forceinline__ T fast_rcp(T x) { return T(1) / x; }

// Minmod of Eq. rt-minmod with sign tests (no product, so nothing underflows).
template <class T>
__device__ __forceinline__ T minmod(T a, T b) {
    bool same = (a > T(0) && b > T(0)) || (a < T(0) && b < T(0));
    if (!same) return T(0);
    return (fabs(a) < fabs(b)) ? a : b;
}

// M1 flux of one group state contracted with A (Eq. eddington-group, flux tensor of
// Eq. rt-meshless): out = (F . A, c^2 E D A) with D A = (1-chi)/2 A + (3chi-1)/2 (n.A) n.
// Written without n = F/|F|: (3chi-1)/2 n n^T = b(u) u / |F|^2 F F^T, u = min(f^2, 1),
// b(u) = (3chi-1)/(2u) = 6 (1 + 1/(4+2s)) / (5+2s), s = sqrt(4-3u), which is finite at u = 0.
template <class T>
__device__ __forceinline__ void m1_dot(T E, T Fx, T Fy, T Fz, T Ax, T Ay, T Az, T c, T& oE, T& oFx, T& oFy,
                                       T& oFz) {
    T FA = Fx * Ax + Fy * Ay + Fz * Az;
    oE = FA;
    if (!(E > T(0))) {
        oFx = oFy = oFz = T(0);
        return;
    }
    T F2 = Fx * Fx + Fy * Fy + Fz * Fz;
    T icE = T(1) / (c * E);
    T icE2 = icE * icE;
    T u = F2 * icE2;
    T sc = icE2;                         // u / |F|^2
    if (u > T(1)) {
        u = T(1);
        sc = T(1) / F2;
    }
    T s = sqrt(T(4) - T(3) * u);
    T den = T(1) / (T(5) + T(2) * s);
    T a_iso = (T(1) + s - T(2) * u) * den;            // (1 - chi) / 2
    T b = T(6) * (T(1) + T(1) / (T(4) + T(2) * s)) * den;
    T cE = c * c * E;
    T t = b * FA * sc;
    oFx = cE * (a_iso * Ax + t * Fx);
    oFy = cE * (a_iso * Ay + t * Fy);
    oFz = cE * (a_iso * Az + t * Fz);
}

}  // namespace rt
