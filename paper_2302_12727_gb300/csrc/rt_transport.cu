// Transport kernels of the FVPM photon-transport step (Ivkovic 2023, Part III,
// "One RT Time Step"): injection, least-squares gradients, the pair flux loop with
// minmod-limited face states, M1 closure and GLF flux, the explicit update, the grey sink
// and the energy diagnostic.
//
// Layout (cell-sorted order): per particle a state record of 4G values (E, Fx, Fy, Fz per
// group), a gradient record of 12G values (d/dx, d/dy, d/dz per component), a position
// record (fixed-point uint4 for the float path, 4 doubles for the double path) and a
// geometry record of 8 values {1/H, h, Bp (6)} with Bp = V^2 sigma / H^3 B so that
// V_i psitilde_j(x_i) = Bp_i d w(q).  A neighbour's data is then a few 16-byte loads.
//
// The gradient kernels run one thread per particle (or per particle and group) over its
// symmetric neighbour list.  The flux of each unordered pair (k < l) is evaluated once, by
// one thread with k as the left state, and stored in the pair's slot (three launch variants:
// direct loads, cp.async staging, or TMA row gathers of packed flux rows that the gradient
// pass writes); a gather kernel lets every particle add the fluxes of its upper pairs and
// subtract those of its lower pairs in a fixed order.  Both particles thus apply the very
// same Phi_kl with opposite signs: the exchange is exactly antisymmetric, and so exactly
// conservative, deterministic, and free of atomics.  With individual time bins the same
// kernels run on the active sets of each min-step (BINS instantiations) and the fluxes are
// weighted by min(dt_k, dt_l) and accumulated until each particle's step ends.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "rt_pair.cuh"

namespace rt {

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Default block sizes of the shuffle gradient and the per-group gather (rt_tuning's
// gradient_block and gather_block choose others at run time).  Rows of different lengths
// make the warps of a block finish at different times, and a block's registers are freed
// only with its last warp: 64-thread gradient blocks run 3% faster than 256-thread ones
// (0.139 against 0.144 ms per launch on the 262,144-particle set); the gather, whose warps
// finish more evenly, keeps 256 (128 is 2% slower there).  The kernels are compiled for the
// largest block of their range, with the register cap the default block had.
constexpr int kGradBlock = 64, kGatherBlock = 256, kGradBlockMax = 256, kGatherBlockMax = 512;

static int grad_block(const rt_ctx* c) {
    if (c->tune.gradient_block > 0) return c->tune.gradient_block;
    return c->tune.gradient_variant == 2 ? kGradBlock : 256;
}
static int gather_block(const rt_ctx* c) { return c->tune.gather_block > 0 ? c->tune.gather_block : kGatherBlock; }
static int pair_warps(const rt_ctx* c) { return c->tune.pair_warps > 0 ? c->tune.pair_warps : 1; }

// ------------------------------------------------------------------------------------
// caller order <-> cell-sorted records
template <class T>
__global__ void k_state_in(const T* __restrict__ src, const int32_t* __restrict__ perm, int64_t n, int comps, int RS,
                           int off, T* __restrict__ rec) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t i = perm[p];
    for (int c = 0; c < comps; ++c) rec[p * RS + off + c] = src[c * n + i];
}

template <class T>
__global__ void k_state_out(const T* __restrict__ rec, const int32_t* __restrict__ inv_perm, int64_t n, int comps,
                            int RS, int off, T* __restrict__ dst) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t p = inv_perm[i];
    for (int c = 0; c < comps; ++c) dst[c * n + i] = rec[p * RS + off + c];
}

// plain SoA gathers (double per-particle fields)
template <class T>
__global__ void k_from_sorted(const T* __restrict__ src, const int32_t* __restrict__ inv_perm, int64_t n, int comps,
                              T* dst) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t p = inv_perm[i];
    for (int c = 0; c < comps; ++c) dst[c * n + i] = src[c * n + p];
}

template <class T>
__global__ void k_alpha_sorted(const double* __restrict__ alpha, const int32_t* __restrict__ perm, int64_t n, T* out) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    out[p] = (T)alpha[perm[p]];
}

// per-group absorption [G][N] (caller order) -> [N][G] sorted, working precision
template <class T>
__global__ void k_alpha_g_sorted(const double* __restrict__ ag, const int32_t* __restrict__ perm, int64_t n, int G,
                                 T* out) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t i = perm[p];
    for (int g = 0; g < G; ++g) out[p * G + g] = (T)ag[(int64_t)g * n + i];
}

__global__ void k_set_scalar(double* dst, double v) { *dst = v; }

// ------------------------------------------------------------------------------------
// a5: injection, one thread per target particle: E_g += dt * sum_e coef_e L[src_e][g]
// (coef = xi / V_target), accumulated in double.
template <class T>
__global__ void k_inject(const int32_t* __restrict__ targets, const int32_t* __restrict__ off,
                         const int32_t* __restrict__ src, const double* __restrict__ coef,
                         const double* __restrict__ L, int G, const double* __restrict__ dt_dev, int64_t n_targets,
                         int RS, T* rec, const int8_t* __restrict__ bins, int s) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_targets) return;
    double dt = *dt_dev;
    int64_t p = targets[t];
    if (bins) {   // time bins: only particles starting a step, for their own step
        const int b = bins[p];
        if (s & ((1 << b) - 1)) return;
        dt = ldexp(dt, b);
    }
    for (int g = 0; g < G; ++g) {
        double acc = 0.0;
        for (int e = off[t]; e < off[t + 1]; ++e) acc += coef[e] * L[(int64_t)src[e] * G + g];
        T* E = rec + p * RS + 4 * g;
        *E = (T)__dadd_rn((double)*E, __dmul_rn(dt, acc));
    }
}

// The same increments dt sum coef L per (particle, group) into inj [N][G] (zeroed before),
// for a gather epilogue to add: E = (T)((double)E + inj) rounds as k_inject does.
__global__ void k_inject_dense(const int32_t* __restrict__ targets, const int32_t* __restrict__ off,
                               const int32_t* __restrict__ src, const double* __restrict__ coef,
                               const double* __restrict__ L, int G, const double* __restrict__ dt_dev,
                               int64_t n_targets, double* __restrict__ inj) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_targets) return;
    const double dt = *dt_dev;
    const int64_t p = targets[t];
    for (int g = 0; g < G; ++g) {
        double acc = 0.0;
        for (int e = off[t]; e < off[t + 1]; ++e) acc += coef[e] * L[(int64_t)src[e] * G + g];
        inj[p * G + g] = __dmul_rn(dt, acc);
    }
}

// the logical words of particle i's packed flux row (after its prefix)
template <class T>
__device__ __forceinline__ T* packed_row(const PairArgs<T>& a, int64_t i) {
    return a.frec + i * (int64_t)(a.RW + kRowRot) + kRowRot;
}

// logical words [w, w + K) of a packed row (w a multiple of 4); those among the last kRowRot
// are written into the prefix too
template <int K, class T>
__device__ __forceinline__ void row_store(const PairArgs<T>& a, T* row, int w, const T* v) {
    vstore<K>(row + w, v);
#pragma unroll
    for (int k = 0; k < K; k += 4)
        if (w + k >= a.RW - kRowRot) vstore<4>(row + (w + k) - a.RW, v + k);
}

// position and geometry words of particle i's packed flux row (never among the last kRowRot)
template <class T>
__device__ __forceinline__ void packed_static(const PairArgs<T>& a, int64_t i, T* row) {
    if constexpr (std::is_same<T, float>::value) {
        *reinterpret_cast<uint4*>(row) = reinterpret_cast<const uint4*>(a.pos)[i];
        float g8[8];
        vload<8>(a.geo + 8 * i, g8);
        vstore<8>(row + 4, g8);
    }
}

// ------------------------------------------------------------------------------------
// a6: least-squares gradient (Eq. gradient) of the groups [g0, g0 + GC):
// grad Q_i = omega_i Bp_i sum_j (Q_j - Q_i) w(r_ij / H_i) d_ij,  d_ij = x_j - x_i
template <class T, int GC, bool BINS = false>
__global__ void __launch_bounds__(128) k_gradient(PairArgs<T> a, const T* __restrict__ rec, T* __restrict__ grad,
                                                  int g0) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if constexpr (BINS) {   // time bins: the particles starting a step (an ordered prefix)
        if (i >= a.count) return;
        i = a.order[i];
    } else {
        if (i >= a.n) return;
    }
    constexpr int NC = 4 * GC;
    const T* tag = nullptr;
    Pos<T> pi = load_pos(tag, a.pos, i);
    const T iH = a.geo[8 * i];
    const int RS = 4 * a.G;
    T ui[NC];
    vload<NC>(rec + i * RS + 4 * g0, ui);
    T acc[NC][3];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c][0] = acc[c][1] = acc[c][2] = T(0);
    const int64_t e0 = a.row_off[i], e1 = a.row_off[i + 1];
    // two neighbours per iteration: both neighbours' loads are in flight together
    for (int64_t e = e0; e < e1; e += 2) {
        const bool two = e + 1 < e1;
        const int j0 = a.cols[e];
        const int j1 = two ? a.cols[e + 1] : j0;
        Pos<T> p0 = load_pos(tag, a.pos, j0);
        Pos<T> p1 = load_pos(tag, a.pos, j1);
        T u0[NC], u1[NC];
        vload<NC>(rec + (int64_t)j0 * RS + 4 * g0, u0);
        vload<NC>(rec + (int64_t)j1 * RS + 4 * g0, u1);
        T dx0, dy0, dz0, dx1, dy1, dz1;
        sep(a.sp, pi, p0, dx0, dy0, dz0);
        sep(a.sp, pi, p1, dx1, dy1, dz1);
        T w0 = spline_w_(sqrt_(dx0 * dx0 + dy0 * dy0 + dz0 * dz0) * iH);
        T w1 = two ? spline_w_(sqrt_(dx1 * dx1 + dy1 * dy1 + dz1 * dz1) * iH) : T(0);
        T wx0 = w0 * dx0, wy0 = w0 * dy0, wz0 = w0 * dz0;
        T wx1 = w1 * dx1, wy1 = w1 * dy1, wz1 = w1 * dz1;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            T dq0 = u0[c] - ui[c];
            T dq1 = u1[c] - ui[c];
            acc[c][0] += dq0 * wx0 + dq1 * wx1;
            acc[c][1] += dq0 * wy0 + dq1 * wy1;
            acc[c][2] += dq0 * wz0 + dq1 * wz1;
        }
    }
    T M[6];
    const T om = a.omega[i];
#pragma unroll
    for (int k = 0; k < 6; ++k) M[k] = om * a.geo[8 * i + 2 + k];
    T out[3 * NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) sym_mv(M, acc[c][0], acc[c][1], acc[c][2], out[3 * c], out[3 * c + 1], out[3 * c + 2]);
    if (a.frec) {
        T* row = packed_row(a, i);
        row_store<3 * NC>(a, row, 12 + 4 * a.G + 12 * g0, out);
        row_store<NC>(a, row, 12 + 4 * g0, ui);
        if (g0 == 0) packed_static(a, i, row);
    } else {
        vstore<3 * NC>(grad + i * 12 * a.G + 12 * g0, out);
    }
}

// Float gradient with one thread per (particle, group): the GC lanes of a particle read the
// same neighbour position and neighbouring 16-byte pieces of the same state record, so a
// warp request touches about 32 / GC records instead of 32.  Same neighbour pairing and
// order of accumulation as k_gradient.
template <int GC>
__global__ void __launch_bounds__(256) k_gradient_g(PairArgs<float> a, const float* __restrict__ rec,
                                                    float* __restrict__ grad, int g0) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i = t / GC;
    if (i >= a.n) return;
    const int g = (int)(t - i * GC);
    const float* tag = nullptr;
    const Pos<float> pi = load_pos(tag, a.pos, i);
    const float iH = a.geo[8 * i];
    const int RS = 4 * a.G;
    const int off = 4 * (g0 + g);
    float ui[4];
    vload<4>(rec + i * RS + off, ui);
    float acc[4][3];
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c][0] = acc[c][1] = acc[c][2] = 0.f;
    const int64_t e0 = a.row_off[i], e1 = a.row_off[i + 1];
    for (int64_t e = e0; e < e1; e += 2) {
        const bool two = e + 1 < e1;
        const int j0 = a.cols[e];
        const int j1 = two ? a.cols[e + 1] : j0;
        Pos<float> p0 = load_pos(tag, a.pos, j0);
        Pos<float> p1 = load_pos(tag, a.pos, j1);
        float u0[4], u1[4];
        vload<4>(rec + (int64_t)j0 * RS + off, u0);
        vload<4>(rec + (int64_t)j1 * RS + off, u1);
        float dx0, dy0, dz0, dx1, dy1, dz1;
        sep(a.sp, pi, p0, dx0, dy0, dz0);
        sep(a.sp, pi, p1, dx1, dy1, dz1);
        float w0 = spline_w_(sqrt_(dx0 * dx0 + dy0 * dy0 + dz0 * dz0) * iH);
        float w1 = two ? spline_w_(sqrt_(dx1 * dx1 + dy1 * dy1 + dz1 * dz1) * iH) : 0.f;
        float wx0 = w0 * dx0, wy0 = w0 * dy0, wz0 = w0 * dz0;
        float wx1 = w1 * dx1, wy1 = w1 * dy1, wz1 = w1 * dz1;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float dq0 = u0[c] - ui[c];
            float dq1 = u1[c] - ui[c];
            acc[c][0] += dq0 * wx0 + dq1 * wx1;
            acc[c][1] += dq0 * wy0 + dq1 * wy1;
            acc[c][2] += dq0 * wz0 + dq1 * wz1;
        }
    }
    float M[6];
    const float om = a.omega[i];
#pragma unroll
    for (int k = 0; k < 6; ++k) M[k] = om * a.geo[8 * i + 2 + k];
    float out[12];
#pragma unroll
    for (int c = 0; c < 4; ++c) sym_mv(M, acc[c][0], acc[c][1], acc[c][2], out[3 * c], out[3 * c + 1], out[3 * c + 2]);
    if (a.frec) {
        float* row = packed_row(a, i);
        row_store<12>(a, row, 12 + 4 * a.G + 12 * (g0 + g), out);
        row_store<4>(a, row, 12 + off, ui);
        if (g0 + g == 0) packed_static(a, i, row);
    } else {
        vstore<12>(grad + i * 12 * a.G + 12 * (g0 + g), out);
    }
}

// Float gradient with the GC lanes of a particle sharing the neighbour geometry: a warp
// holds 32 / GC particles; per block of 2 GC neighbours each lane computes the separation,
// spline weight and w d of two consecutive neighbours and passes them to the particle's
// other lanes with warp shuffles, so the geometry is computed once instead of GC times.
// Neighbours stay paired (e, e + 1) from the row start and the accumulation is the same
// expression in the same order as k_gradient_g, so the result bits are the same.  With four
// groups (eight particles per warp, every lane busy) five blocks per SM (48 registers, a few
// spilled) beat four at 64 registers by 7%; with three groups they lose 2%.
template <int GC>
__global__ void __launch_bounds__(kGradBlockMax, GC == 4 ? 1280 / kGradBlockMax : 0) k_gradient_s(PairArgs<float> a, const float* __restrict__ rec,
                                                    float* __restrict__ grad, int g0) {
    constexpr int P = 32 / GC;                     // particles per warp
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int q = lane / GC, g = lane - (lane / GC) * GC;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t i = warp * P + q;
    const bool act = q < P && i < a.n;             // lanes past P GC and past the last particle idle
    const int64_t ii = act ? i : 0;
    const float* tag = nullptr;
    const Pos<float> pi = load_pos(tag, a.pos, ii);
    const float iH = a.geo[8 * ii];
    const int RS = 4 * a.G;
    const int off = 4 * (g0 + g);
    float ui[4];
    vload<4>(rec + ii * RS + off, ui);
    float acc[4][3];
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c][0] = acc[c][1] = acc[c][2] = 0.f;
    const int64_t e0 = a.row_off[ii], e1 = act ? a.row_off[ii + 1] : e0;
    int nit = (int)((e1 - e0 + 2 * GC - 1) / (2 * GC));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nit = max(nit, __shfl_xor_sync(FULL, nit, o));
    const int base = q * GC;                       // first lane of this particle
    // this lane's pair of neighbours; below four groups their indices load one iteration
    // ahead (at four, the register cap of five blocks per SM leaves no room for them)
    constexpr bool PF = GC < 4;
    int64_t ea = e0 + 2 * g;
    int j0 = 0, j1 = 0;
    if constexpr (PF) {
        j0 = ea < e1 ? a.cols[ea] : 0;
        j1 = ea + 1 < e1 ? a.cols[ea + 1] : j0;
    }
    for (int it = 0; it < nit; ++it) {
        const bool has = ea < e1, two = ea + 1 < e1;
        if constexpr (!PF) {
            j0 = has ? a.cols[ea] : 0;
            j1 = two ? a.cols[ea + 1] : j0;
        }
        const int64_t en = ea + 2 * GC;
        int j0n = 0, j1n = 0;
        if constexpr (PF) {
            j0n = en < e1 ? a.cols[en] : 0;
            j1n = en + 1 < e1 ? a.cols[en + 1] : j0n;
        }
        const Pos<float> p0 = load_pos(tag, a.pos, j0);
        const Pos<float> p1 = load_pos(tag, a.pos, j1);
        float dx0, dy0, dz0, dx1, dy1, dz1;
        sep(a.sp, pi, p0, dx0, dy0, dz0);
        sep(a.sp, pi, p1, dx1, dy1, dz1);
        float w0 = spline_w_(sqrt_(dx0 * dx0 + dy0 * dy0 + dz0 * dz0) * iH);
        float w1 = two ? spline_w_(sqrt_(dx1 * dx1 + dy1 * dy1 + dz1 * dz1) * iH) : 0.f;
        float wx0 = w0 * dx0, wy0 = w0 * dy0, wz0 = w0 * dz0;
        float wx1 = w1 * dx1, wy1 = w1 * dy1, wz1 = w1 * dz1;
        const int hj0 = has ? j0 : -1;
#pragma unroll
        for (int u = 0; u < GC; ++u) {
            const int src = base + u;
            const int J0 = __shfl_sync(FULL, hj0, src), J1 = __shfl_sync(FULL, j1, src);
            const float X0 = __shfl_sync(FULL, wx0, src), Y0 = __shfl_sync(FULL, wy0, src),
                        Z0 = __shfl_sync(FULL, wz0, src);
            const float X1 = __shfl_sync(FULL, wx1, src), Y1 = __shfl_sync(FULL, wy1, src),
                        Z1 = __shfl_sync(FULL, wz1, src);
            if (J0 < 0) continue;
            float u0[4], u1[4];
            vload<4>(rec + (int64_t)J0 * RS + off, u0);
            vload<4>(rec + (int64_t)J1 * RS + off, u1);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float dq0 = u0[c] - ui[c];
                float dq1 = u1[c] - ui[c];
                acc[c][0] += dq0 * X0 + dq1 * X1;
                acc[c][1] += dq0 * Y0 + dq1 * Y1;
                acc[c][2] += dq0 * Z0 + dq1 * Z1;
            }
        }
        ea = en;
        if constexpr (PF) {
            j0 = j0n;
            j1 = j1n;
        }
    }
    if (!act) return;
    float M[6];
    const float om = a.omega[i];
#pragma unroll
    for (int k = 0; k < 6; ++k) M[k] = om * a.geo[8 * i + 2 + k];
    float out[12];
#pragma unroll
    for (int c = 0; c < 4; ++c) sym_mv(M, acc[c][0], acc[c][1], acc[c][2], out[3 * c], out[3 * c + 1], out[3 * c + 2]);
    if (a.frec) {
        float* row = packed_row(a, i);
        row_store<12>(a, row, 12 + 4 * a.G + 12 * (g0 + g), out);
        row_store<4>(a, row, 12 + off, ui);
        if (g0 + g == 0) packed_static(a, i, row);
    } else {
        vstore<12>(grad + i * 12 * a.G + 12 * (g0 + g), out);
    }
}

// ------------------------------------------------------------------------------------
// a7 + a8: pair fluxes, explicit update, grey sink, optional fix-up, groups [g0, g0 + GC).

// Pass 1 of the flux: one thread per unordered pair (k, l), k < l, evaluates Phi_kl once with
// k as the left state and stores it in the pair's slot.
template <class T, int GC, bool HLL, bool BINS = false>
__global__ void __launch_bounds__(128) k_flux(PairArgs<T> a, FluxExtra<T> x, const T* __restrict__ rec,
                                              T* __restrict__ pairbuf, int g0) {
    int64_t slot = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if constexpr (BINS) {   // time bins: the pairs with a starting member (an ordered prefix)
        if (slot >= a.count) return;
        slot = a.order[slot];
    } else {
        if (slot >= a.n_pairs) return;
    }
    constexpr int NC = 4 * GC;
    const T* tag = nullptr;
    const int G = a.G, RS = 4 * G;
    const int2 kl = a.ends[slot];
    const int64_t i = kl.x, j = kl.y;
    T wgt = T(1);
    if constexpr (BINS) wgt = T(1 << min(a.bins[i], a.bins[j]));   // min(dt_k, dt_l) / dt_min
    const Pos<T> pi = load_pos(tag, a.pos, i);
    const Pos<T> pj = load_pos(tag, a.pos, j);
    T gi8[8], gj8[8];
    vload<8>(a.geo + 8 * i, gi8);
    vload<8>(a.geo + 8 * j, gj8);
    T dx, dy, dz;
    sep(a.sp, pi, pj, dx, dy, dz);              // d = x_l - x_k
    // A_kl = (Bp_k w_k + Bp_l w_l) d  (Eq. HopkinsAij)
    T r = sqrt_(dx * dx + dy * dy + dz * dz);
    T si = spline_w_(r * gi8[0]);
    T sj = spline_w_(r * gj8[0]);
    T M[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) M[q] = gi8[2 + q] * si + gj8[2 + q] * sj;
    T Ax, Ay, Az;
    sym_mv(M, dx, dy, dz, Ax, Ay, Az);
    T An = sqrt_(Ax * Ax + Ay * Ay + Az * Az);
    T diss = T(0.5) * x.c * An;
    T ih = rcp_(gi8[1] + gj8[1]);
    T wi = gi8[1] * ih, wj = gj8[1] * ih;
    const T* ri = rec + i * RS;
    const T* rj = rec + j * RS;
    const T* qi = a.grad + i * 12 * G;
    const T* qj = a.grad + j * 12 * G;
    T out[NC];
#pragma unroll
    for (int g = 0; g < GC; ++g) {
        const int gg = g0 + g;
        T ui[4], uj[4], gri[12], grj[12];
        vload<4>(ri + 4 * gg, ui);
        vload<4>(rj + 4 * gg, uj);
        vload<12>(qi + 12 * gg, gri);
        vload<12>(qj + 12 * gg, grj);
        pair_flux<HLL>(ui, uj, gri, grj, dx, dy, dz, wi, wj, Ax, Ay, Az, diss, x.c, x.wave, An, &out[4 * g]);
    }
    if constexpr (BINS) {
#pragma unroll
        for (int c = 0; c < NC; ++c) out[c] *= wgt;
    }
    vstore<NC>(pairbuf + slot * NC, out);
}

// ------------------------------------------------------------------------------------
// Per-particle sum of one group's pair fluxes (E, Fx, Fy, Fz), in a fixed order.  The double
// path adds in double.  The float path keeps the energy row as a compensated float sum:
// Knuth's TwoSum gives the exact rounding error of every addition and a second float
// collects those errors (the cascaded summation of Ogita, Rump and Oishi, "Accurate sum and
// dot product", 2005), so for the ~50 terms of a particle the sum's error stays near
// (50 u)^2 of the sum of magnitudes (u = 2^-24) instead of 50 u; the update then forms the
// energy from the pair in double.  The flux rows add in float.  (A double energy sum costs
// the same gather 2.4 times its time on GB300, whose FP64 rate is 1/64 of FP32; compensated
// flux rows 1.3 times.)  With individual time bins the accumulators stay in memory between
// min-steps: 32 bytes per (particle, group) in both precisions.
template <class T>
struct FluxAcc;

template <>
struct FluxAcc<double> {
    double v[4];
    __device__ __forceinline__ void zero() { v[0] = v[1] = v[2] = v[3] = 0.0; }
    __device__ __forceinline__ void add(const double p[4]) {
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] += p[c];
    }
    __device__ __forceinline__ void sub(const double p[4]) {
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] -= p[c];
    }
    __device__ __forceinline__ double energy() const { return v[0]; }
    __device__ __forceinline__ double flux(int c) const { return v[1 + c]; }
    __device__ __forceinline__ void load(const double* m) { vload<4>(m, v); }
    __device__ __forceinline__ void store(double* m) const { vstore<4>(m, v); }
};

// s + x = t + e exactly (TwoSum, branch-free); e is added to the error sum k
__device__ __forceinline__ void two_sum_into(float& s, float& k, float x) {
    const float t = __fadd_rn(s, x);
    const float z = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(x, z));
    k = __fadd_rn(k, e);
    s = t;
}

template <>
struct FluxAcc<float> {
    float es, ek;    // energy row: sum and error sum
    float f[3];      // flux rows
    __device__ __forceinline__ void zero() { es = ek = f[0] = f[1] = f[2] = 0.f; }
    __device__ __forceinline__ void add(const float p[4]) {
        two_sum_into(es, ek, p[0]);
#pragma unroll
        for (int c = 0; c < 3; ++c) f[c] += p[1 + c];
    }
    __device__ __forceinline__ void sub(const float p[4]) {
        two_sum_into(es, ek, -p[0]);
#pragma unroll
        for (int c = 0; c < 3; ++c) f[c] -= p[1 + c];
    }
    __device__ __forceinline__ double energy() const { return (double)es + (double)ek; }
    __device__ __forceinline__ float flux(int c) const { return f[c]; }
    // record: {es, ek, f0, f1 | f2, unused x 3}
    __device__ __forceinline__ void load(const float* m) {
        const float4 a = *reinterpret_cast<const float4*>(m);
        es = a.x; ek = a.y; f[0] = a.z; f[1] = a.w;
        f[2] = m[4];
    }
    __device__ __forceinline__ void store(float* m) const {
        *reinterpret_cast<float4*>(m) = make_float4(es, ek, f[0], f[1]);
        m[4] = f[2];
    }
};

// words of T per (particle, group) accumulator record in memory (32 bytes)
template <class T>
struct AccRec {
    static constexpr int words = 32 / (int)sizeof(T);
};

// U_g(t + dt) = (U_g - f acc_g) sink for one group (Eq. transport-update-explicit with
// f = dt / V_i, then the forward-Euler sink), the fix-up E >= 0 when on (returns 1 if it
// fired), then the next sub-cycle's injection inj (double, 0 when none).  The float path
// forms the energy from its compensated sum in double and rounds once, before the fix-up
// and the injection, exactly where a plain step stores it.
template <class T>
__device__ __forceinline__ int update_group(T u[4], const FluxAcc<T>& acc, T f, T sink, int clamp, const double* inj) {
    T v0;
    if constexpr (std::is_same<T, float>::value)
        v0 = (float)(((double)u[0] - (double)f * acc.energy()) * (double)sink);
    else
        v0 = (u[0] - f * acc.energy()) * sink;
    int fired = 0;
    if (clamp && v0 < T(0)) {
        v0 = T(0);
        fired = 1;
    }
    if (inj) v0 = (T)__dadd_rn((double)v0, *inj);
    u[0] = v0;
#pragma unroll
    for (int c = 0; c < 3; ++c) u[1 + c] = (u[1 + c] - f * acc.flux(c)) * sink;
    return fired;
}

// Pass 2 with individual time bins: particle i adds to its accumulators the slots of the
// pairs that interacted at min-step s (all of them if i starts a step, else those whose
// partner starts one), in the same order as the uniform gather; at the end of its own step
// ((s + 1) mod 2^b_i = 0) it applies U_i - dt_min / V_i acc_i, the sink over its step
// dt_min 2^b_i and the fix-up, and clears the accumulators.  The states are updated in place
// (this pass runs after the pair pass, and each particle writes only its own record).
template <class T, int GC>
__device__ __forceinline__ void gather_bins(const PairArgs<T>& a, const FluxExtra<T>& x, const T* __restrict__ rec,
                                            const T* __restrict__ pairbuf, T* __restrict__ out, int g0, int64_t i) {
    constexpr int NC = 4 * GC, AW = AccRec<T>::words;
    const int RS = 4 * a.G;
    const int bi = a.bins[i];
    const int mask = (1 << bi) - 1;
    const bool start_i = !(a.s & mask);
    T* accp = x.acc + (i * a.G + g0) * AW;
    FluxAcc<T> acc[GC];
#pragma unroll
    for (int g = 0; g < GC; ++g) acc[g].load(accp + g * AW);
    const int64_t r0 = a.row_off[i], s0 = a.up_off[i], s1 = a.up_off[i + 1];
    const int nl = a.n_low[i];
    for (int64_t sl = s0; sl < s1; ++sl) {
        const int l = a.cols[r0 + nl + (sl - s0)];
        if (!start_i && (a.s & ((1 << a.bins[l]) - 1))) continue;
        T phi[NC];
        vload<NC>(pairbuf + sl * NC, phi);
#pragma unroll
        for (int g = 0; g < GC; ++g) acc[g].add(phi + 4 * g);
    }
    const int32_t* ls = a.low_slot + (r0 - s0);
    for (int e = 0; e < nl; ++e) {
        const int k = a.cols[r0 + e];
        if (!start_i && (a.s & ((1 << a.bins[k]) - 1))) continue;
        T phi[NC];
        vload<NC>(pairbuf + (int64_t)ls[e] * NC, phi);
#pragma unroll
        for (int g = 0; g < GC; ++g) acc[g].sub(phi + 4 * g);
    }
    if ((a.s + 1) & mask) {   // the step of i goes on (the state is updated in place)
#pragma unroll
        for (int g = 0; g < GC; ++g) acc[g].store(accp + g * AW);
        return;
    }
    T ui[NC];
    vload<NC>(rec + i * RS + 4 * g0, ui);
    const T dt = (T)(*x.dt_dev);
    const T dti = (T)ldexp(*x.dt_dev, bi);
    const T f = dt * a.omega[i];
    T sink = T(1);
    if (x.alpha) sink = fmax_(T(1) - x.c * x.alpha[i] * dti, T(0));
    int nclamp = 0;
#pragma unroll
    for (int g = 0; g < GC; ++g) {
        const T sk = x.alpha_g ? fmax_(T(1) - x.c * x.alpha_g[i * a.G + g0 + g] * dti, T(0)) : sink;
        nclamp += update_group<T>(ui + 4 * g, acc[g], f, sk, x.clamp, nullptr);
        acc[g].zero();
        acc[g].store(accp + g * AW);
    }
    vstore<NC>(out + i * RS + 4 * g0, ui);
    if (nclamp) atomicAdd(x.clamp_count, (unsigned long long)nclamp);
}

// particles whose step ends at min-step s without any interaction at s (no starting partner,
// nmin > tz): apply the accumulators, the sink over the step and the fix-up, in place
template <class T, int GC>
__global__ void k_finalize_bins(PairArgs<T> a, FluxExtra<T> x, T* __restrict__ rec, int g0) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= a.count) return;
    const int64_t i = a.order[t];
    if (a.nmin[i] <= a.tz) return;       // finalised by the gather of this min-step
    constexpr int NC = 4 * GC, AW = AccRec<T>::words;
    const int RS = 4 * a.G;
    T* accp = x.acc + (i * a.G + g0) * AW;
    T ui[NC];
    vload<NC>(rec + i * RS + 4 * g0, ui);
    const int bi = a.bins[i];
    const T dt = (T)(*x.dt_dev);
    const T dti = (T)ldexp(*x.dt_dev, bi);
    const T f = dt * a.omega[i];
    T sink = T(1);
    if (x.alpha) sink = fmax_(T(1) - x.c * x.alpha[i] * dti, T(0));
    int nclamp = 0;
#pragma unroll
    for (int g = 0; g < GC; ++g) {
        FluxAcc<T> acc;
        acc.load(accp + g * AW);
        const T sk = x.alpha_g ? fmax_(T(1) - x.c * x.alpha_g[i * a.G + g0 + g] * dti, T(0)) : sink;
        nclamp += update_group<T>(ui + 4 * g, acc, f, sk, x.clamp, nullptr);
        acc.zero();
        acc.store(accp + g * AW);
    }
    vstore<NC>(rec + i * RS + 4 * g0, ui);
    if (nclamp) atomicAdd(x.clamp_count, (unsigned long long)nclamp);
}

// Pass 2: particle i adds the fluxes of its own upper pairs (contiguous slots) and subtracts
// those of its lower pairs (k < i, read from k's slots), in a fixed order; then
// U_i(t + dt) = U_i - dt / V_i sum_l F_il . A_il, the sink and the fix-up.
template <class T, int GC, bool BINS = false>
__global__ void __launch_bounds__(128) k_flux_gather(PairArgs<T> a, FluxExtra<T> x, const T* __restrict__ rec,
                                                     const T* __restrict__ pairbuf, T* __restrict__ out, int g0) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if constexpr (BINS) {   // the particles with a starting partner or themselves starting
        if (i < a.count) gather_bins<T, GC>(a, x, rec, pairbuf, out, g0, a.order[i]);
        return;
    }
    if (i >= a.n) return;
    constexpr int NC = 4 * GC;
    const int RS = 4 * a.G;
    FluxAcc<T> acc[GC];
#pragma unroll
    for (int g = 0; g < GC; ++g) acc[g].zero();
    const int64_t r0 = a.row_off[i], s0 = a.up_off[i], s1 = a.up_off[i + 1];
    for (int64_t sl = s0; sl < s1; ++sl) {
        T phi[NC];
        vload<NC>(pairbuf + sl * NC, phi);
#pragma unroll
        for (int g = 0; g < GC; ++g) acc[g].add(phi + 4 * g);
    }
    const int nl = a.n_low[i];
    const int32_t* ls = a.low_slot + (r0 - s0);
    int e = 0;
    for (; e + 4 <= nl; e += 4) {     // four loads in flight, subtracted in order
        T p[4][NC];
#pragma unroll
        for (int u = 0; u < 4; ++u) vload<NC>(pairbuf + (int64_t)ls[e + u] * NC, p[u]);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int g = 0; g < GC; ++g) acc[g].sub(p[u] + 4 * g);
    }
    for (; e < nl; ++e) {
        T phi[NC];
        vload<NC>(pairbuf + (int64_t)ls[e] * NC, phi);
#pragma unroll
        for (int g = 0; g < GC; ++g) acc[g].sub(phi + 4 * g);
    }
    const T dt = (T)(*x.dt_dev);
    const T f = dt * a.omega[i];
    T sink = T(1);
    if (x.alpha) sink = fmax_(T(1) - x.c * x.alpha[i] * dt, T(0));
    T ui[NC];
    vload<NC>(rec + i * RS + 4 * g0, ui);
    int nclamp = 0;
#pragma unroll
    for (int g = 0; g < GC; ++g) {
        const T sk = x.alpha_g ? fmax_(T(1) - x.c * x.alpha_g[i * a.G + g0 + g] * dt, T(0)) : sink;
        nclamp += update_group<T>(ui + 4 * g, acc[g], f, sk, x.clamp, x.inj ? x.inj + i * a.G + g0 + g : nullptr);
    }
    vstore<NC>(out + i * RS + 4 * g0, ui);
    if (nclamp) atomicAdd(x.clamp_count, (unsigned long long)nclamp);
}

// Float pass 1 with the neighbour records staged through shared memory.  One thread per
// pair slot as in k_flux, but the 32 l-records a warp needs (position, geometry, state and
// gradient of the launched groups) are first copied by the whole warp, one array at a time,
// so that each 16-byte request of the warp covers a few consecutive records instead of 32
// scattered ones; the per-pair loads of the direct kernel saturate the L1 data pipe.  The
// k side needs no staging: consecutive slots mostly share k, so its loads are broadcasts.
// The arithmetic is the same as k_flux's.
template <int GC>
struct Staged {
    static constexpr int RW = 12 + 16 * GC;   // words per staged record: pos 4, geo 8, state 4GC, grad 12GC
    static constexpr int WARPS = 4;
    static constexpr size_t bytes = (size_t)WARPS * 32 * RW * sizeof(float);
};

template <int GC, bool HLL>
__global__ void __launch_bounds__(128) k_flux_staged(PairArgs<float> a, FluxExtra<float> x,
                                                     const float* __restrict__ rec, float* __restrict__ pairbuf,
                                                     int g0) {
    constexpr int NC = 4 * GC, RW = Staged<GC>::RW;
    // RW / 4 is odd for every GC, so the lanes' 16-byte reads of their own records are free
    // of bank conflicts
    __shared__ __align__(16) float st[Staged<GC>::WARPS * 32 * RW];
    const int lane = threadIdx.x & 31;
    float* ws = st + (threadIdx.x >> 5) * 32 * RW;
    const int64_t slot = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool act = slot < a.n_pairs;
    // lanes past the last slot stage particle 0 (always present) and store nothing
    const int2 kl = act ? a.ends[slot] : make_int2(0, 0);
    const int G = a.G, RS = 4 * G;
    const unsigned FULL = 0xffffffffu;
    cp_async16(ws + lane * RW, reinterpret_cast<const uint4*>(a.pos) + kl.y);
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const int t = m * 32 + lane, r = t >> 1, q = t & 1;
        const int64_t l = __shfl_sync(FULL, kl.y, r);
        cp_async16(ws + r * RW + 4 + 4 * q, a.geo + 8 * l + 4 * q);
    }
#pragma unroll
    for (int m = 0; m < GC; ++m) {
        const int t = m * 32 + lane, r = t / GC, q = t - r * GC;
        const int64_t l = __shfl_sync(FULL, kl.y, r);
        cp_async16(ws + r * RW + 12 + 4 * q, rec + l * RS + 4 * g0 + 4 * q);
    }
#pragma unroll
    for (int m = 0; m < 3 * GC; ++m) {
        const int t = m * 32 + lane, r = t / (3 * GC), q = t - r * (3 * GC);
        const int64_t l = __shfl_sync(FULL, kl.y, r);
        cp_async16(ws + r * RW + 12 + 4 * GC + 4 * q, a.grad + l * 12 * G + 12 * g0 + 4 * q);
    }
    const float* tag = nullptr;
    const int64_t i = kl.x;
    const Pos<float> pi = load_pos(tag, a.pos, i);
    float gi8[8], gj8[8];
    vload<8>(a.geo + 8 * i, gi8);
    cp_async_wait_all();
    __syncwarp();
    const float* mine = ws + lane * RW;
    const uint4 pv = *reinterpret_cast<const uint4*>(mine);
    const Pos<float> pj = {pv.x, pv.y, pv.z};
    vload<8>(mine + 4, gj8);
    float dx, dy, dz;
    sep(a.sp, pi, pj, dx, dy, dz);
    float r = sqrt_(dx * dx + dy * dy + dz * dz);
    float si = spline_w_(r * gi8[0]);
    float sj = spline_w_(r * gj8[0]);
    float M[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) M[q] = gi8[2 + q] * si + gj8[2 + q] * sj;
    float Ax, Ay, Az;
    sym_mv(M, dx, dy, dz, Ax, Ay, Az);
    float An = sqrt_(Ax * Ax + Ay * Ay + Az * Az);
    float diss = 0.5f * x.c * An;
    float ih = rcp_(gi8[1] + gj8[1]);
    float wi = gi8[1] * ih, wj = gj8[1] * ih;
    const float* ri = rec + i * RS;
    const float* qi = a.grad + i * 12 * G;
    float out[NC];
#pragma unroll
    for (int g = 0; g < GC; ++g) {
        const int gg = g0 + g;
        float ui[4], uj[4], gri[12], grj[12];
        vload<4>(ri + 4 * gg, ui);
        vload<4>(mine + 12 + 4 * g, uj);
        vload<12>(qi + 12 * gg, gri);
        vload<12>(mine + 12 + 4 * GC + 12 * g, grj);
        pair_flux<HLL>(ui, uj, gri, grj, dx, dy, dz, wi, wj, Ax, Ay, Az, diss, x.c, x.wave, An, &out[4 * g]);
    }
    if (act) vstore<NC>(pairbuf + slot * NC, out);
}

// Float pass 1 with the neighbour rows fetched by the tensor memory accelerator.  The
// gradient pass has packed each particle's flux inputs (position, geometry, state and
// gradient) into one row; each warp gathers the rows of its 32 l-particles into shared
// memory with eight tile::gather4 copies (four rows each).  The copies bypass the
// load/store pipeline whose wavefronts bound the direct kernel; the k side is loaded
// directly (mostly broadcasts).  Same arithmetic as k_flux.  A copy that does not complete
// within the wait budget sets err_flag, and the warp returns without storing.
template <int G>
struct PackedRows {
    static constexpr int RW = 12 + 16 * G;              // words per row
    static constexpr int SLOT = (4 * RW + 31) / 32 * 32; // four rows, padded to 128 bytes
    static constexpr int WF = 8 * SLOT;                 // floats per warp
    static constexpr uint32_t bytes = 32u * RW * 4u;    // bytes gathered per warp
};

// BINS: the pairs of the ordered prefix a.order[0, a.count) (time bins: those with a
// starting member), their fluxes scaled by 2^min(b_k, b_l) as in k_flux.
// One warp per block: each warp's shared rows are freed as soon as it finishes, instead of
// with the last warp of a four-warp block, and the register cap of 27 (24 for four groups)
// resident blocks per SM lets shared memory, not registers, bound the occupancy.  Measured
// against four-warp blocks at 80 registers: 0.169 against 0.180 ms per launch on the
// 262,144-particle set (G = 3), 1.78 against 1.93 ms on the 2,097,152-particle set (G = 4).
// Up to kTmaWarpsMax warps per block (rt_tuning's pair_warps, default 1); the register cap is
// that of 27 (24 at G = 4) one-warp blocks per SM whatever the block size
constexpr int kTmaWarpsMax = 4;
template <int G>
struct TmaMinBlocks {
    static constexpr int value = G >= 4 ? 6 : 7;   // blocks of kTmaWarpsMax warps
};
template <int G, bool HLL, bool BINS = false>
__global__ void __launch_bounds__(kTmaWarpsMax * 32, TmaMinBlocks<G>::value) k_flux_tma(PairArgs<float> a, FluxExtra<float> x,
                                                  float* __restrict__ pairbuf,
                                                  const __grid_constant__ CUtensorMap rows, int* err_flag,
                                                  unsigned long long budget) {
    using R = PackedRows<G>;
    constexpr int NC = 4 * G, RW = R::RW;
    // dynamic: R::WF floats per warp of the block plus 128 bytes, from which the rows start at
    // the first 128-byte boundary (the slots of the row gathers are 128-byte aligned)
    extern __shared__ __align__(128) float sm_dyn[];
    __shared__ __align__(8) uint64_t bar[kTmaWarpsMax];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t sm0 = smem_u32(sm_dyn);
    float* sm = sm_dyn + (((sm0 + 127u) & ~127u) - sm0) / 4u;
    float* ws = sm + wid * R::WF;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool act = t < (BINS ? a.count : a.n_pairs);
    const int64_t slot = BINS ? (act ? (int64_t)a.order[t] : 0) : t;
    // lanes past the last slot gather particle 0 (always present) and store nothing
    const int2 kl = act ? a.ends[slot] : make_int2(0, 0);
    const uint32_t mb = smem_u32(&bar[wid]);
    if (lane == 0) {
        mbar_init(mb, 1);
        mbar_expect_tx(mb, R::bytes);
    }
    __syncwarp();
    const unsigned FULL = 0xffffffffu;
    const int q = lane & 7;
    const int r0 = __shfl_sync(FULL, kl.y, 4 * q), r1 = __shfl_sync(FULL, kl.y, 4 * q + 1);
    const int r2 = __shfl_sync(FULL, kl.y, 4 * q + 2), r3 = __shfl_sync(FULL, kl.y, 4 * q + 3);
    // even slots get the rows as they are (copy from word kRowRot), odd slots rotated by four
    // chunks (copy from word 0 of the prefixed row)
    if (lane < 8) tma_gather4(smem_u32(ws + q * R::SLOT), &rows, (q & 1) ? 0 : kRowRot, r0, r1, r2, r3, mb);
    const int64_t i = kl.x;
    const float* rk = packed_row(a, i);
    const uint4 pkv = *reinterpret_cast<const uint4*>(rk);
    const Pos<float> pi = {pkv.x, pkv.y, pkv.z};
    float gi8[8], gj8[8];
    vload<8>(rk + 4, gi8);
    if (!mbar_wait(mb, 0, budget)) {
        atomicExch(err_flag, 1);
        // let the copies still in flight land before the block exits, however short the
        // caller's budget (a copy lands in microseconds; this wait too is bounded)
        mbar_wait(mb, 0, budget > 2000000000ull ? budget : 2000000000ull);
        return;
    }
    // this lane's row: slot lane / 4, row lane % 4 within it.  A quarter-warp reads the rows
    // of one even and one odd slot; the slots start on the same bank, and the rows of a slot
    // cover four of the eight 16-byte bank groups at any one chunk, so the odd slot's rotation
    // by four chunks sends its lanes to the other four (all but the last four chunks).
    // Logical chunk c is at chunk c (even slot), c + 4 or, for the last four, c + 4 - RW / 4.
    const float* rl = ws + (lane >> 2) * R::SLOT + (lane & 3) * RW;
    const bool odd = (lane >> 2) & 1;
    const float* rlA = rl + (odd ? kRowRot : 0);
    const float* rlB = rl + (odd ? kRowRot - RW : 0);
    constexpr int NCH = RW / 4;
    auto lrow = [&](int c) -> const float* { return (c < NCH - kRowRot / 4 ? rlA : rlB) + 4 * c; };
    const uint4 pv = *reinterpret_cast<const uint4*>(lrow(0));
    const Pos<float> pj = {pv.x, pv.y, pv.z};
    vload<8>(lrow(1), gj8);
    float dx, dy, dz;
    sep(a.sp, pi, pj, dx, dy, dz);
    float r = sqrt_(dx * dx + dy * dy + dz * dz);
    float si = spline_w_(r * gi8[0]);
    float sj = spline_w_(r * gj8[0]);
    float M[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) M[k] = gi8[2 + k] * si + gj8[2 + k] * sj;
    float Ax, Ay, Az;
    sym_mv(M, dx, dy, dz, Ax, Ay, Az);
    float An = sqrt_(Ax * Ax + Ay * Ay + Az * Az);
    float diss = 0.5f * x.c * An;
    float ih = rcp_(gi8[1] + gj8[1]);
    float wi = gi8[1] * ih, wj = gj8[1] * ih;
    float out[NC];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        float ui[4], uj[4], gri[12], grj[12];
        vload<4>(rk + 12 + 4 * g, ui);
        vload<4>(lrow(3 + g), uj);
        vload<12>(rk + 12 + 4 * G + 12 * g, gri);
        vload<4>(lrow(3 + G + 3 * g), grj);
        vload<4>(lrow(4 + G + 3 * g), grj + 4);
        vload<4>(lrow(5 + G + 3 * g), grj + 8);
        pair_flux<HLL>(ui, uj, gri, grj, dx, dy, dz, wi, wj, Ax, Ay, Az, diss, x.c, x.wave, An, &out[4 * g]);
    }
    if constexpr (BINS) {
        const float wgt = (float)(1 << min(a.bins[kl.x], a.bins[kl.y]));   // min(dt_k, dt_l) / dt_min
#pragma unroll
        for (int c = 0; c < NC; ++c) out[c] *= wgt;
    }
    if (act) vstore<NC>(pairbuf + slot * NC, out);
}

// Float pass 2 with one thread per (particle, group): the lanes of one particle read the
// 16-byte pieces of a slot that lie side by side, so a warp request touches about 32 / GC
// slots instead of 32.  Same order of additions and subtractions as k_flux_gather.
template <int GC>
__global__ void __launch_bounds__(kGatherBlockMax) k_flux_gather_g(PairArgs<float> a, FluxExtra<float> x,
                                                       const float* __restrict__ rec,
                                                       const float* __restrict__ pairbuf, float* __restrict__ out,
                                                       int g0) {
    // blocks run from the last particles to the first: the pair pass wrote the slots in
    // ascending order, so the most recent (still L2-resident) slots are read first
    const int64_t t = (gridDim.x - 1 - blockIdx.x) * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i = t / GC;
    if (i >= a.n) return;
    const int g = (int)(t - i * GC);
    constexpr int NC = 4 * GC;
    const int RS = 4 * a.G;
    const float* pb = pairbuf + 4 * g;
    FluxAcc<float> acc;
    acc.zero();
    const int64_t r0 = a.row_off[i], s0 = a.up_off[i], s1 = a.up_off[i + 1];
    // batches of up to eight loads in flight (the last one predicated), added in order
    for (int64_t sl = s0; sl < s1; sl += 8) {
        const int m = s1 - sl < 8 ? (int)(s1 - sl) : 8;
        float p[8][4];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (u < m) vload<4>(pb + (sl + u) * NC, p[u]);
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (u < m) acc.add(p[u]);
    }
    const int nl = a.n_low[i];
    const int32_t* ls = a.low_slot + (r0 - s0);
    for (int e = 0; e < nl; e += 8) {   // up to eight slot indices, then their loads in flight
        const int m = nl - e < 8 ? nl - e : 8;
        int32_t q[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (u < m) q[u] = ls[e + u];
        float p[8][4];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (u < m) vload<4>(pb + (int64_t)q[u] * NC, p[u]);
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (u < m) acc.sub(p[u]);
    }
    const float dt = (float)(*x.dt_dev);
    const float f = dt * a.omega[i];
    float sink = 1.f;
    if (x.alpha) sink = fmax_(1.f - x.c * x.alpha[i] * dt, 0.f);
    if (x.alpha_g) sink = fmax_(1.f - x.c * x.alpha_g[i * a.G + g0 + g] * dt, 0.f);
    float ui[4];
    const int64_t o = i * RS + 4 * (g0 + g);
    vload<4>(rec + o, ui);
    const int nclamp = update_group<float>(ui, acc, f, sink, x.clamp, x.inj ? x.inj + i * a.G + g0 + g : nullptr);
    vstore<4>(out + o, ui);
    if (nclamp) atomicAdd(x.clamp_count, (unsigned long long)nclamp);
}

// ------------------------------------------------------------------------------------
// Drift correction (Sec. "Dealing With Particle Drifts"): U_i += grad U_i . (v_i dt_drift)
// for every component, on the sorted records; v in caller order (SoA doubles).
template <class T>
__global__ void k_drift(T* __restrict__ rec, const T* __restrict__ grad, const double* __restrict__ v,
                        const int32_t* __restrict__ perm, int64_t n, int G, double dt) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t i = perm[p];
    const T dx = (T)(v[i] * dt), dy = (T)(v[n + i] * dt), dz = (T)(v[2 * n + i] * dt);
    T* u = rec + p * 4 * G;
    const T* g = grad + p * 12 * G;
    for (int c = 0; c < 4 * G; ++c) u[c] += g[3 * c] * dx + g[3 * c + 1] * dy + g[3 * c + 2] * dz;
}

rt_status launch_drift(rt_ctx* c, cudaStream_t s, void* rec, const double* v, double dt) {
    unsigned nb = nblk(c->n, 256);
    if (c->fp64)
        k_drift<double><<<nb, 256, 0, s>>>((double*)rec, c->grad_t.as<double>(), v, c->perm.as<int32_t>(), c->n,
                                           c->cfg.n_groups, dt);
    else
        k_drift<float><<<nb, 256, 0, s>>>((float*)rec, c->grad_t.as<float>(), v, c->perm.as<int32_t>(), c->n,
                                          c->cfg.n_groups, dt);
    ++c->launches;
    RT_CUDA(c, cudaGetLastError());
    return RT_OK;
}

// ------------------------------------------------------------------------------------
// a10: energy per group, sum_i V_i E_i,g in double; fixed grid and tree order.
constexpr int kEnergyBlocks = 512;

// Particles of caller index >= owned (the ghost copies of a domain decomposition) are left out.
template <class T>
__global__ void k_energy_part(const T* __restrict__ rec, int RS, const double* __restrict__ V, int64_t n, int G,
                              const int32_t* __restrict__ perm, int64_t owned, double* part) {
    __shared__ double sm[256];
    for (int g = 0; g < G; ++g) {
        double s = 0.0;
        for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
            if (owned >= n || perm[p] < owned) s += V[p] * (double)rec[p * RS + 4 * g];
        sm[threadIdx.x] = s;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[g * gridDim.x + blockIdx.x] = sm[0];
        __syncthreads();
    }
}

__global__ void k_energy_final(const double* __restrict__ part, int nb, int G, double* out) {
    int g = threadIdx.x;
    if (g >= G) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[g * nb + b];
    out[g] = s;
}

// ------------------------------------------------------------------------------------
// the pair kernels use no shared memory: give the whole unified L1 to the cache
template <class T>
static void set_carveouts() {
    static bool done = false;
    if (done) return;
    done = true;
    const void* fs[] = {(const void*)k_gradient<T, 1>, (const void*)k_gradient<T, 2>, (const void*)k_gradient<T, 3>,
                        (const void*)k_gradient<T, 4>, (const void*)k_flux<T, 1, false>,
                        (const void*)k_flux<T, 2, false>, (const void*)k_flux<T, 3, false>,
                        (const void*)k_flux<T, 4, false>, (const void*)k_flux<T, 1, true>,
                        (const void*)k_flux<T, 2, true>, (const void*)k_flux<T, 3, true>,
                        (const void*)k_flux<T, 4, true>,
                        (const void*)k_flux_gather<T, 1>, (const void*)k_flux_gather<T, 2>,
                        (const void*)k_flux_gather<T, 3>, (const void*)k_flux_gather<T, 4>};
    for (const void* f : fs) cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
    (void)cudaGetLastError();
}

template <class T>
static void launch_gradient_t(rt_ctx* c, cudaStream_t s, T* rec, bool packed = false) {
    set_carveouts<T>();
    PairArgs<T> a = pair_args<T>(c);
    if (packed) a.frec = c->frec.as<T>();
    const int G = c->cfg.n_groups;
    unsigned nb = nblk(c->n, 128);
    for (int g0 = 0; g0 < G; g0 += kMaxGC) {
        int gc = G - g0 < kMaxGC ? G - g0 : kMaxGC;
        int pr = prof_begin(c, s, RT_KERNEL_GRADIENT);
        if constexpr (std::is_same<T, float>::value) {
            if (c->tune.gradient_variant == 2 && gc > 1) {
                // warps of 32 / gc particles: ceil(n / (32 / gc)) warps of 32 lanes
                const int64_t warps = (c->n + 32 / gc - 1) / (32 / gc);
                const int gb = grad_block(c);
                unsigned nbs = nblk(warps * 32, gb);
                float* gr = c->grad_t.as<float>();
                switch (gc) {
                    case 2: k_gradient_s<2><<<nbs, gb, 0, s>>>(a, rec, gr, g0); break;
                    case 3: k_gradient_s<3><<<nbs, gb, 0, s>>>(a, rec, gr, g0); break;
                    default: k_gradient_s<4><<<nbs, gb, 0, s>>>(a, rec, gr, g0); break;
                }
                prof_end(c, s, pr);
                ++c->launches;
                continue;
            }
            if (c->tune.gradient_variant >= 1) {
                const int gb = c->tune.gradient_block > 0 ? c->tune.gradient_block : 256;
                unsigned nbg = nblk(c->n * gc, gb);
                float* gr = c->grad_t.as<float>();
                switch (gc) {
                    case 1: k_gradient_g<1><<<nbg, gb, 0, s>>>(a, rec, gr, g0); break;
                    case 2: k_gradient_g<2><<<nbg, gb, 0, s>>>(a, rec, gr, g0); break;
                    case 3: k_gradient_g<3><<<nbg, gb, 0, s>>>(a, rec, gr, g0); break;
                    default: k_gradient_g<4><<<nbg, gb, 0, s>>>(a, rec, gr, g0); break;
                }
                prof_end(c, s, pr);
                ++c->launches;
                continue;
            }
        }
        switch (gc) {
            case 1: k_gradient<T, 1><<<nb, 128, 0, s>>>(a, rec, c->grad_t.as<T>(), g0); break;
            case 2: k_gradient<T, 2><<<nb, 128, 0, s>>>(a, rec, c->grad_t.as<T>(), g0); break;
            case 3: k_gradient<T, 3><<<nb, 128, 0, s>>>(a, rec, c->grad_t.as<T>(), g0); break;
            default: k_gradient<T, 4><<<nb, 128, 0, s>>>(a, rec, c->grad_t.as<T>(), g0); break;
        }
        prof_end(c, s, pr);
        ++c->launches;
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link-time libcuda)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        (void)cudaGetLastError();
    }
    return fn;
}

// tensor map of the packed rows [n][kRowRot + 12 + 16G] floats, box of the 12 + 16G logical
// words of a row (for tile::gather4); encoded again whenever the buffer or its shape changes
static bool packed_rows_map(rt_ctx* c) {
    const int RW = 12 + 16 * c->cfg.n_groups;
    if (c->rows_map_for == c->frec.p && c->rows_map_n == c->n) return true;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || !c->frec.p) return false;
    // rows of kRowRot + RW words (the prefix first); the box is the RW logical words
    cuuint64_t dims[2] = {(cuuint64_t)(RW + kRowRot), (cuuint64_t)c->n};
    cuuint64_t strides[1] = {(cuuint64_t)(RW + kRowRot) * 4};
    cuuint32_t box[2] = {(cuuint32_t)RW, 1};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&c->rows_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->frec.p, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    c->rows_map_for = c->frec.p;
    c->rows_map_n = c->n;
    return true;
}

// float pass 1 and 2 in the variants chosen by the context's tuning
template <int GC, bool HLL>
static void flux_float(rt_ctx* c, cudaStream_t s, const PairArgs<float>& a, const FluxExtra<float>& x,
                       const float* rec, float* pb, float* out, int g0) {
    static bool attr = false;
    if (!attr) {
        attr = true;
        cudaFuncSetAttribute((const void*)k_flux_staged<GC, HLL>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        cudaFuncSetAttribute((const void*)k_flux_gather_g<GC>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
        cudaFuncSetAttribute((const void*)k_flux_tma<GC, HLL>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
        (void)cudaGetLastError();
    }
    unsigned npb = nblk(std::max<int64_t>(a.n_pairs, 1), 128);
    int variant = c->tune.flux_variant;
    if (variant == 2 && !a.frec) variant = 0;
    int pr = prof_begin(c, s, RT_KERNEL_FLUX);
    if (variant == 2) {
        unsigned long long budget = c->cfg.device_wait_budget_cycles ? c->cfg.device_wait_budget_cycles
                                                                     : 4000000000ull;
        const int pw = pair_warps(c);
        k_flux_tma<GC, HLL><<<nblk(std::max<int64_t>(a.n_pairs, 1), pw * 32), pw * 32,
                              (size_t)pw * PackedRows<GC>::WF * sizeof(float) + 128, s>>>(
            a, x, pb, c->rows_map, c->flags.as<int>() + F_TIMEOUT, budget);
    } else if (variant == 1) {
        k_flux_staged<GC, HLL><<<npb, 128, 0, s>>>(a, x, rec, pb, g0);
    } else {
        k_flux<float, GC, HLL><<<npb, 128, 0, s>>>(a, x, rec, pb, g0);
    }
    prof_end(c, s, pr);
    pr = prof_begin(c, s, RT_KERNEL_FLUX_GATHER);
    if (c->tune.gather_variant == 1)
        k_flux_gather_g<GC><<<nblk(c->n * GC, gather_block(c)), gather_block(c), 0, s>>>(a, x, rec, pb, out, g0);
    else
        k_flux_gather<float, GC><<<nblk(c->n, 128), 128, 0, s>>>(a, x, rec, pb, out, g0);
    prof_end(c, s, pr);
    c->launches += 2;
}

template <class T>
static void launch_flux_t(rt_ctx* c, cudaStream_t s, const T* rec, T* out, bool has_alpha, bool packed = false,
                          bool inject_after = false) {
    PairArgs<T> a = pair_args<T>(c);
    if (packed) a.frec = c->frec.as<T>();
    FluxExtra<T> x;
    const bool hll = c->cfg.riemann_solver == RT_RIEMANN_HLL;
    x.wave = hll ? c->wave_t.as<T>() : nullptr;
    x.alpha = has_alpha ? c->alpha_s.as<T>() : nullptr;
    x.alpha_g = c->step_alpha_g ? c->alpha_g_s.as<T>() : nullptr;
    x.acc = nullptr;
    x.inj = inject_after ? c->inj_dense.as<double>() : nullptr;
    x.dt_dev = c->dt_dev.as<double>();
    x.c = (T)c->cfg.c_red;
    x.clamp = c->cfg.clamp_negative;
    x.clamp_count = reinterpret_cast<unsigned long long*>(c->flags.as<int>() + F_CLAMP);
    const int G = c->cfg.n_groups;
    unsigned nb = nblk(c->n, 128);
    T* pb = c->pairbuf.as<T>();
    unsigned npb = nblk(std::max<int64_t>(a.n_pairs, 1), 128);
    for (int g0 = 0; g0 < G; g0 += kMaxGC) {
        int gc = G - g0 < kMaxGC ? G - g0 : kMaxGC;
        if constexpr (std::is_same<T, float>::value) {
            if (hll) {
                switch (gc) {
                    case 1: flux_float<1, true>(c, s, a, x, rec, pb, out, g0); break;
                    case 2: flux_float<2, true>(c, s, a, x, rec, pb, out, g0); break;
                    case 3: flux_float<3, true>(c, s, a, x, rec, pb, out, g0); break;
                    default: flux_float<4, true>(c, s, a, x, rec, pb, out, g0); break;
                }
            } else {
                switch (gc) {
                    case 1: flux_float<1, false>(c, s, a, x, rec, pb, out, g0); break;
                    case 2: flux_float<2, false>(c, s, a, x, rec, pb, out, g0); break;
                    case 3: flux_float<3, false>(c, s, a, x, rec, pb, out, g0); break;
                    default: flux_float<4, false>(c, s, a, x, rec, pb, out, g0); break;
                }
            }
            continue;
        }
        int pr = prof_begin(c, s, RT_KERNEL_FLUX);
        if (hll) {
            switch (gc) {
                case 1: k_flux<T, 1, true><<<npb, 128, 0, s>>>(a, x, rec, pb, g0); break;
                case 2: k_flux<T, 2, true><<<npb, 128, 0, s>>>(a, x, rec, pb, g0); break;
                case 3: k_flux<T, 3, true><<<npb, 128, 0, s>>>(a, x, rec, pb, g0); break;
                default: k_flux<T, 4, true><<<npb, 128, 0, s>>>(a, x, rec, pb, g0); break;
            }
        } else {
            switch (gc) {
                case 1: k_flux<T, 1, false><<<npb, 128, 0, s>>>(a, x, rec, pb, g0); break;
                case 2: k_flux<T, 2, false><<<npb, 128, 0, s>>>(a, x, rec, pb, g0); break;
                case 3: k_flux<T, 3, false><<<npb, 128, 0, s>>>(a, x, rec, pb, g0); break;
                default: k_flux<T, 4, false><<<npb, 128, 0, s>>>(a, x, rec, pb, g0); break;
            }
        }
        prof_end(c, s, pr);
        pr = prof_begin(c, s, RT_KERNEL_FLUX_GATHER);
        switch (gc) {
            case 1: k_flux_gather<T, 1><<<nb, 128, 0, s>>>(a, x, rec, pb, out, g0); break;
            case 2: k_flux_gather<T, 2><<<nb, 128, 0, s>>>(a, x, rec, pb, out, g0); break;
            case 3: k_flux_gather<T, 3><<<nb, 128, 0, s>>>(a, x, rec, pb, out, g0); break;
            default: k_flux_gather<T, 4><<<nb, 128, 0, s>>>(a, x, rec, pb, out, g0); break;
        }
        prof_end(c, s, pr);
        c->launches += 2;
    }
}

template <class T>
static void launch_inject_t(rt_ctx* c, cudaStream_t s, T* rec, const int8_t* bins = nullptr, int step = 0) {
    if (c->n_inj_targets <= 0) return;
    int pr = prof_begin(c, s, RT_KERNEL_INJECT);
    k_inject<T><<<nblk(c->n_inj_targets, 128), 128, 0, s>>>(
        c->inj_targets.as<int32_t>(), c->inj_off.as<int32_t>(), c->inj_src.as<int32_t>(), c->inj_coef.as<double>(),
        c->L_dev.as<double>(), c->cfg.n_groups, c->dt_dev.as<double>(), c->n_inj_targets, 4 * c->cfg.n_groups, rec,
        bins, step);
    prof_end(c, s, pr);
    ++c->launches;
}

rt_status launch_inject(rt_ctx* c, cudaStream_t s, void* rec) {
    if (c->fp64) launch_inject_t<double>(c, s, (double*)rec);
    else launch_inject_t<float>(c, s, (float*)rec);
    RT_CUDA(c, cudaGetLastError());
    return RT_OK;
}

rt_status launch_gradient(rt_ctx* c, cudaStream_t s, void* rec) {
    if (c->fp64) launch_gradient_t<double>(c, s, (double*)rec);
    else launch_gradient_t<float>(c, s, (float*)rec);
    RT_CUDA(c, cudaGetLastError());
    return RT_OK;
}

// packed flux rows from sorted states and gradients given in grad_t (one thread per
// particle and group): what the gradient kernels write beside their gradients
__global__ void k_pack_rows(PairArgs<float> a, const float* __restrict__ rec, const float* __restrict__ grad) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i = t / a.G;
    if (i >= a.n) return;
    const int g = (int)(t - i * a.G);
    float* row = packed_row(a, i);
    float gq[12], u[4];
    vload<12>(grad + i * 12 * a.G + 12 * g, gq);
    vload<4>(rec + i * 4 * a.G + 4 * g, u);
    row_store<12>(a, row, 12 + 4 * a.G + 12 * g, gq);
    row_store<4>(a, row, 12 + 4 * g, u);
    if (g == 0) packed_static(a, i, row);
}

rt_status launch_flux_given(rt_ctx* c, cudaStream_t s, void* Uin, void* Uout, bool has_alpha) {
    if (c->fp64) {
        launch_flux_t<double>(c, s, (const double*)Uin, (double*)Uout, has_alpha);
    } else {
        const bool packed = c->tune.flux_variant == 2 && c->cfg.n_groups <= kMaxGC && packed_rows_map(c);
        if (packed) {
            PairArgs<float> a = pair_args<float>(c);
            a.frec = c->frec.as<float>();
            k_pack_rows<<<nblk(c->n * c->cfg.n_groups, 256), 256, 0, s>>>(a, (const float*)Uin,
                                                                          c->grad_t.as<float>());
            ++c->launches;
        }
        launch_flux_t<float>(c, s, (const float*)Uin, (float*)Uout, has_alpha, packed);
    }
    RT_CUDA(c, cudaGetLastError());
    return RT_OK;
}

// omega, V = 1 / omega and B of caller particles [first, first + count) from the caller
// (omega [count], B [count][3][3], double), with the pair kernels' records derived from them
// as k_geometry derives its own
template <class T>
__global__ void k_set_fields(const double* __restrict__ omega, const double* __restrict__ B9,
                             const int32_t* __restrict__ inv_perm, int64_t first, int64_t count, int64_t n,
                             const double* __restrict__ h, double* omega_d, double* V_d, double* B_d, T* geo_t,
                             T* om_t) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int64_t p = inv_perm[first + k];
    const double om = omega[k];
    const double* b = B9 + 9 * k;
    const double B[6] = {b[0], b[4], b[8], b[1], b[2], b[5]};   // xx yy zz xy xz yz
    const double hi = h[p], H = kKappa * hi, iH = 1.0 / H;
    const double V = 1.0 / om;
    const double bp = V * V * kSigma * iH * iH * iH;
    omega_d[p] = om;
    V_d[p] = V;
    geo_t[8 * p] = (T)iH;
    geo_t[8 * p + 1] = (T)hi;
    for (int e = 0; e < 6; ++e) {
        B_d[e * n + p] = B[e];
        geo_t[8 * p + 2 + e] = (T)(bp * B[e]);
    }
    om_t[p] = (T)om;
}

rt_status set_fields(rt_ctx* c, int64_t first, int64_t count, const double* omega, const double* B) {
    if (count <= 0) return RT_OK;
    const unsigned nb = nblk(count, 128);
    if (c->fp64)
        k_set_fields<double><<<nb, 128, 0, c->stream>>>(omega, B, c->inv_perm.as<int32_t>(), first, count, c->n,
                                                        c->h_d.as<double>(), c->omega_d.as<double>(),
                                                        c->V_d.as<double>(), c->B_d.as<double>(),
                                                        c->geo_t.as<double>(), c->omega_t.as<double>());
    else
        k_set_fields<float><<<nb, 128, 0, c->stream>>>(omega, B, c->inv_perm.as<int32_t>(), first, count, c->n,
                                                       c->h_d.as<double>(), c->omega_d.as<double>(),
                                                       c->V_d.as<double>(), c->B_d.as<double>(),
                                                       c->geo_t.as<float>(), c->omega_t.as<float>());
    ++c->launches;
    RT_CUDA(c, cudaGetLastError());
    return RT_OK;
}

// one min-step of a hydro step with individual time bins, on the active sets only: the
// injection and gradients of the starting particles, the pair fluxes of the pairs with a
// starting member, the gather of the particles they touch (finalising those whose step ends
// now), and the finalisation of the other particles whose step ends now.  In place.
// the time-bin pair pass by row gathers (float, one group chunk); other T: never called
template <int GC, class T>
static void bins_flux_tma(rt_ctx* c, cudaStream_t s, const PairArgs<T>& af, const FluxExtra<T>& x, T* pb, bool hll) {
    if constexpr (std::is_same<T, float>::value) {
        static bool attr = false;
        if (!attr) {
            attr = true;
            cudaFuncSetAttribute((const void*)k_flux_tma<GC, false, true>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
            cudaFuncSetAttribute((const void*)k_flux_tma<GC, true, true>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
            (void)cudaGetLastError();
        }
        const unsigned nbf = nblk(std::max<int64_t>(af.count, 1), 128);
        const unsigned long long budget = c->cfg.device_wait_budget_cycles ? c->cfg.device_wait_budget_cycles
                                                                           : 4000000000ull;
        int* ef = c->flags.as<int>() + F_TIMEOUT;
        const int pw = pair_warps(c);
        const size_t smem = (size_t)pw * PackedRows<GC>::WF * sizeof(float) + 128;
        const unsigned nbt = nblk(std::max<int64_t>(af.count, 1), pw * 32);
        if (hll) k_flux_tma<GC, true, true><<<nbt, pw * 32, smem, s>>>(af, x, pb, c->rows_map, ef, budget);
        else k_flux_tma<GC, false, true><<<nbt, pw * 32, smem, s>>>(af, x, pb, c->rows_map, ef, budget);
    }
}

template <class T>
static void launch_step_bins_t(rt_ctx* c, cudaStream_t s, int step, T* rec, bool has_src, bool has_alpha) {
    set_carveouts<T>();
    const int8_t* bins = c->bins_s.as<int8_t>();
    if (has_src) launch_inject_t<T>(c, s, rec, bins, step);
    const int B = c->bins_max;
    const int tz = step == 0 ? B : __builtin_ctz((unsigned)step);
    const int tz1 = __builtin_ctz((unsigned)(step + 1)) < B ? __builtin_ctz((unsigned)(step + 1)) : B;
    PairArgs<T> a = pair_args<T>(c);
    a.bins = bins;
    a.s = step;
    a.nmin = c->bins_nmin.as<int8_t>();
    a.tz = tz;
    FluxExtra<T> x;
    const bool hll = c->cfg.riemann_solver == RT_RIEMANN_HLL;
    x.wave = hll ? c->wave_t.as<T>() : nullptr;
    x.alpha = has_alpha ? c->alpha_s.as<T>() : nullptr;
    x.alpha_g = c->step_alpha_g ? c->alpha_g_s.as<T>() : nullptr;
    x.acc = c->acc_t.as<T>();
    x.inj = nullptr;
    x.dt_dev = c->dt_dev.as<double>();
    x.c = (T)c->cfg.c_red;
    x.clamp = c->cfg.clamp_negative;
    x.clamp_count = reinterpret_cast<unsigned long long*>(c->flags.as<int>() + F_CLAMP);
    const int G = c->cfg.n_groups;
    T* pb = c->pairbuf.as<T>();
    T* gr = c->grad_t.as<T>();
    const int64_t n_start = c->cum_b[tz], n_touch = c->cum_m[tz], n_pairs = c->cum_q[tz], n_end = c->cum_b[tz1];
    PairArgs<T> ag = a, af = a, ah = a, ae = a;
    ag.order = c->order_b.as<int32_t>();
    ag.count = n_start;
    af.order = c->order_q.as<int32_t>();
    af.count = n_pairs;
    ah.order = c->order_m.as<int32_t>();
    ah.count = n_touch;
    ae.order = c->order_b.as<int32_t>();
    ae.count = n_end;
    const unsigned nbg = nblk(std::max<int64_t>(n_start, 1), 128), nbf = nblk(std::max<int64_t>(n_pairs, 1), 128);
    const unsigned nbh = nblk(std::max<int64_t>(n_touch, 1), 128), nbe = nblk(std::max<int64_t>(n_end, 1), 128);
    // the float pair pass by row gathers of the packed rows: the gradient kernel writes the
    // rows of the particles starting a step (their state after injection and their new
    // gradient); every other particle's row still holds the state and gradient of its own
    // step start, which is what its pairs use until its step ends
    bool packed = false;
    if constexpr (std::is_same<T, float>::value)
        packed = c->tune.flux_variant == 2 && G <= kMaxGC && packed_rows_map(c);
    if (packed) {
        ag.frec = c->frec.as<T>();
        af.frec = c->frec.as<T>();
    }
    for (int g0 = 0; g0 < G; g0 += kMaxGC) {
        const int gc = G - g0 < kMaxGC ? G - g0 : kMaxGC;
        if (n_start == 0) break;
        switch (gc) {
            case 1: k_gradient<T, 1, true><<<nbg, 128, 0, s>>>(ag, rec, gr, g0); break;
            case 2: k_gradient<T, 2, true><<<nbg, 128, 0, s>>>(ag, rec, gr, g0); break;
            case 3: k_gradient<T, 3, true><<<nbg, 128, 0, s>>>(ag, rec, gr, g0); break;
            default: k_gradient<T, 4, true><<<nbg, 128, 0, s>>>(ag, rec, gr, g0); break;
        }
        ++c->launches;
    }
    for (int g0 = 0; g0 < G; g0 += kMaxGC) {
        const int gc = G - g0 < kMaxGC ? G - g0 : kMaxGC;
#define RT_BINS_FLUX(GC_)                                                                    \
    if (n_pairs > 0) {                                                                       \
        if (packed)                                                                          \
            bins_flux_tma<GC_>(c, s, af, x, pb, hll);                                        \
        else if (hll)                                                                        \
            k_flux<T, GC_, true, true><<<nbf, 128, 0, s>>>(af, x, rec, pb, g0);              \
        else                                                                                 \
            k_flux<T, GC_, false, true><<<nbf, 128, 0, s>>>(af, x, rec, pb, g0);             \
        ++c->launches;                                                                       \
    }                                                                                        \
    if (n_touch > 0) {                                                                       \
        k_flux_gather<T, GC_, true><<<nbh, 128, 0, s>>>(ah, x, rec, pb, rec, g0);            \
        ++c->launches;                                                                       \
    }                                                                                        \
    if (n_end > 0) {                                                                         \
        k_finalize_bins<T, GC_><<<nbe, 128, 0, s>>>(ae, x, rec, g0);                         \
        ++c->launches;                                                                       \
    }
        switch (gc) {
            case 1: RT_BINS_FLUX(1) break;
            case 2: RT_BINS_FLUX(2) break;
            case 3: RT_BINS_FLUX(3) break;
            default: RT_BINS_FLUX(4) break;
        }
#undef RT_BINS_FLUX
    }
}

rt_status launch_step_bins(rt_ctx* c, cudaStream_t s, int step, void* U, bool has_src, bool has_alpha) {
    if (c->fp64)
        launch_step_bins_t<double>(c, s, step, (double*)U, has_src, has_alpha);
    else
        launch_step_bins_t<float>(c, s, step, (float*)U, has_src, has_alpha);
    RT_CUDA(c, cudaGetLastError());
    return RT_OK;
}

rt_status launch_step(rt_ctx* c, cudaStream_t s, void* Uin, void* Uout, bool has_src, bool has_alpha,
                      bool inject_first, bool inject_after) {
    inject_first = inject_first && has_src;
    inject_after = inject_after && has_src && c->inj_dense_ready;
    if (c->fp64) {
        if (inject_first) launch_inject_t<double>(c, s, (double*)Uin);
        launch_gradient_t<double>(c, s, (double*)Uin);
        launch_flux_t<double>(c, s, (const double*)Uin, (double*)Uout, has_alpha, false, inject_after);
    } else {
        if (inject_first) launch_inject_t<float>(c, s, (float*)Uin);
        // packed rows for the tensor-memory-accelerator pair pass (one group chunk only)
        const bool packed = c->tune.flux_variant == 2 && c->cfg.n_groups <= kMaxGC && packed_rows_map(c);
        launch_gradient_t<float>(c, s, (float*)Uin, packed);
        launch_flux_t<float>(c, s, (const float*)Uin, (float*)Uout, has_alpha, packed, inject_after);
    }
    RT_CUDA(c, cudaGetLastError());
    return RT_OK;
}

rt_status state_in(rt_ctx* c, const void* U_user, void* rec, int comps, int RS, int off) {
    unsigned nb = nblk(c->n, 256);
    if (c->fp64)
        k_state_in<double><<<nb, 256, 0, c->stream>>>((const double*)U_user, c->perm.as<int32_t>(), c->n, comps, RS,
                                                       off, (double*)rec);
    else
        k_state_in<float><<<nb, 256, 0, c->stream>>>((const float*)U_user, c->perm.as<int32_t>(), c->n, comps, RS, off,
                                                      (float*)rec);
    ++c->launches;
    RT_CUDA(c, cudaGetLastError());
    return RT_OK;
}

rt_status state_out(rt_ctx* c, const void* rec, void* U_user, int comps, int RS, int off) {
    unsigned nb = nblk(c->n, 256);
    if (c->fp64)
        k_state_out<double><<<nb, 256, 0, c->stream>>>((const double*)rec, c->inv_perm.as<int32_t>(), c->n, comps, RS,
                                                        off, (double*)U_user);
    else
        k_state_out<float><<<nb, 256, 0, c->stream>>>((const float*)rec, c->inv_perm.as<int32_t>(), c->n, comps, RS,
                                                       off, (float*)U_user);
    ++c->launches;
    RT_CUDA(c, cudaGetLastError());
    return RT_OK;
}

rt_status field_out(rt_ctx* c, const double* src_sorted, double* dst_user, int comps) {
    k_from_sorted<double><<<nblk(c->n, 256), 256, 0, c->stream>>>(src_sorted, c->inv_perm.as<int32_t>(), c->n, comps,
                                                                  dst_user);
    ++c->launches;
    RT_CUDA(c, cudaGetLastError());
    return RT_OK;
}

rt_status set_step_inputs(rt_ctx* c, double dt, const double* Lsrc, const double* alpha) {
    cudaStream_t s = c->stream;
    k_set_scalar<<<1, 1, 0, s>>>(c->dt_dev.as<double>(), dt);
    ++c->launches;
    if (Lsrc && c->n_src > 0)
        RT_CUDA(c, cudaMemcpyAsync(c->L_dev.p, Lsrc, (size_t)c->n_src * c->cfg.n_groups * sizeof(double),
                                   cudaMemcpyDeviceToDevice, s));
    if (alpha) {
        unsigned nb = nblk(c->n, 256);
        if (c->fp64) k_alpha_sorted<double><<<nb, 256, 0, s>>>(alpha, c->perm.as<int32_t>(), c->n, c->alpha_s.as<double>());
        else k_alpha_sorted<float><<<nb, 256, 0, s>>>(alpha, c->perm.as<int32_t>(), c->n, c->alpha_s.as<float>());
        ++c->launches;
    }
    // the photo-ionisation sink per group applies when no grey alpha is given
    c->step_alpha_g = !alpha && c->has_alpha_g;
    if (c->step_alpha_g) {
        unsigned nb = nblk(c->n, 256);
        const int G = c->cfg.n_groups;
        if (c->fp64)
            k_alpha_g_sorted<double><<<nb, 256, 0, s>>>(c->alpha_g_c.as<double>(), c->perm.as<int32_t>(), c->n, G,
                                                        c->alpha_g_s.as<double>());
        else
            k_alpha_g_sorted<float><<<nb, 256, 0, s>>>(c->alpha_g_c.as<double>(), c->perm.as<int32_t>(), c->n, G,
                                                       c->alpha_g_s.as<float>());
        ++c->launches;
    }
    RT_CUDA(c, cudaGetLastError());
    return RT_OK;
}

// one warp waits on a barrier that nothing completes (rt_wait_selftest)
__global__ void k_wait_selftest(unsigned long long budget, int* ran_out) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_u32(&bar);
    if (threadIdx.x == 0) mbar_init(b, 1);
    __syncwarp();
    const bool done = mbar_wait(b, 0, budget);
    if (!__any_sync(0xffffffffu, done) && threadIdx.x == 0) *ran_out = 1;
}

rt_status wait_selftest(rt_ctx* c, unsigned long long budget, bool* ran_out) {
    int* f = c->flags.as<int>() + F_SELFTEST;
    RT_CUDA(c, cudaMemsetAsync(f, 0, sizeof(int), c->stream));
    k_wait_selftest<<<1, 32, 0, c->stream>>>(budget, f);
    ++c->launches;
    RT_CUDA(c, cudaGetLastError());
    int h = 0;
    RT_CUDA(c, cudaMemcpyAsync(&h, f, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    RT_CUDA(c, cudaStreamSynchronize(c->stream));
    *ran_out = h != 0;
    return RT_OK;
}

rt_status set_dense_injection(rt_ctx* c, bool on) {
    c->inj_dense_ready = false;
    if (!on || c->n_inj_targets <= 0 || !c->inj_dense.p) return RT_OK;
    cudaStream_t s = c->stream;
    const int G = c->cfg.n_groups;
    RT_CUDA(c, cudaMemsetAsync(c->inj_dense.p, 0, (size_t)G * c->n * 8, s));
    k_inject_dense<<<nblk(c->n_inj_targets, 128), 128, 0, s>>>(
        c->inj_targets.as<int32_t>(), c->inj_off.as<int32_t>(), c->inj_src.as<int32_t>(), c->inj_coef.as<double>(),
        c->L_dev.as<double>(), G, c->dt_dev.as<double>(), c->n_inj_targets, c->inj_dense.as<double>());
    ++c->launches;
    RT_CUDA(c, cudaGetLastError());
    c->inj_dense_ready = true;
    return RT_OK;
}

rt_status launch_energy(rt_ctx* c, cudaStream_t s, const void* rec, double* out_dev) {
    double* part = c->energy_part.as<double>();
    int RS = 4 * c->cfg.n_groups;
    const int32_t* perm = c->perm.as<int32_t>();
    if (c->fp64)
        k_energy_part<double><<<kEnergyBlocks, 256, 0, s>>>((const double*)rec, RS, c->V_d.as<double>(), c->n,
                                                            c->cfg.n_groups, perm, c->n_owned, part);
    else
        k_energy_part<float><<<kEnergyBlocks, 256, 0, s>>>((const float*)rec, RS, c->V_d.as<double>(), c->n,
                                                           c->cfg.n_groups, perm, c->n_owned, part);
    k_energy_final<<<1, 32 * ((c->cfg.n_groups + 31) / 32), 0, s>>>(part, kEnergyBlocks, c->cfg.n_groups, out_dev);
    c->launches += 2;
    RT_CUDA(c, cudaGetLastError());
    return RT_OK;
}

}  // namespace rt
