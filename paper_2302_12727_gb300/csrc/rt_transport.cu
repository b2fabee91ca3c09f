// Transport kernels of the FVPM photon-transport step (Ivkovic 2023, Part III,
// "One RT Time Step"): injection, least-squares gradients, the pair flux loop with
// minmod-limited face states, M1 closure and GLF flux, the explicit update, the grey sink
// and the energy diagnostic.
//
// Every pair kernel runs one thread per particle over its symmetric neighbour list in
// cell-sorted order.  The flux of a pair is evaluated by both particles with the same
// operand order (the lower sorted index is the left state k), so the two evaluations are
// bitwise identical and the exchange is exactly antisymmetric without atomics.
#include "rt_internal.cuh"

namespace rt {

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// ------------------------------------------------------------------------------------
// caller order <-> cell-sorted order, component-major arrays of `comps` rows
template <class T>
__global__ void k_to_sorted(const T* __restrict__ src, const int32_t* __restrict__ perm, int64_t n, int comps, T* dst) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t i = perm[p];
    for (int c = 0; c < comps; ++c) dst[c * n + p] = src[c * n + i];
}

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

__global__ void k_set_scalar(double* dst, double v) { *dst = v; }

// ------------------------------------------------------------------------------------
// separation x_l - x_k in the working precision
template <class T>
struct Sep;

template <>
struct Sep<float> {
    const uint32_t* x;
    float s0, s1, s2;
    int64_t n;
    __device__ __forceinline__ void pos(int64_t i, uint32_t& a, uint32_t& b, uint32_t& c) const {
        a = x[i];
        b = x[n + i];
        c = x[2 * n + i];
    }
};

template <>
struct Sep<double> {
    const double* x;
    double b0, b1, b2;
    int periodic;
    int64_t n;
};

__device__ __forceinline__ double wrap_d(double v, double box, int periodic) {
    if (periodic) {
        double h = 0.5 * box;
        if (v > h) v -= box;
        else if (v < -h) v += box;
    }
    return v;
}

template <class T>
struct PosT;
template <>
struct PosT<float> { uint32_t a, b, c; };
template <>
struct PosT<double> { double a, b, c; };

__device__ __forceinline__ void load_pos(const Sep<float>& s, int64_t i, PosT<float>& p) {
    p.a = s.x[i]; p.b = s.x[s.n + i]; p.c = s.x[2 * s.n + i];
}
__device__ __forceinline__ void load_pos(const Sep<double>& s, int64_t i, PosT<double>& p) {
    p.a = s.x[i]; p.b = s.x[s.n + i]; p.c = s.x[2 * s.n + i];
}
// d = x_to - x_from
__device__ __forceinline__ void sep(const Sep<float>& s, const PosT<float>& from, const PosT<float>& to, float& dx,
                                    float& dy, float& dz) {
    dx = (float)(int32_t)(to.a - from.a) * s.s0;
    dy = (float)(int32_t)(to.b - from.b) * s.s1;
    dz = (float)(int32_t)(to.c - from.c) * s.s2;
}
__device__ __forceinline__ void sep(const Sep<double>& s, const PosT<double>& from, const PosT<double>& to,
                                    double& dx, double& dy, double& dz) {
    dx = wrap_d(to.a - from.a, s.b0, s.periodic);
    dy = wrap_d(to.b - from.b, s.b1, s.periodic);
    dz = wrap_d(to.c - from.c, s.b2, s.periodic);
}

template <class T>
struct PairArgs {
    Sep<T> sp;
    const T* invH;
    const T* h;
    const T* omega;
    const T* Bp;          // [6][N]
    const int64_t* row_off;
    const int32_t* cols;
    int64_t n;
};

// symmetric 3x3 (xx, yy, zz, xy, xz, yz) times vector
template <class T>
__device__ __forceinline__ void sym_mv(const T M[6], T x, T y, T z, T& ox, T& oy, T& oz) {
    ox = M[0] * x + M[3] * y + M[4] * z;
    oy = M[3] * x + M[1] * y + M[5] * z;
    oz = M[4] * x + M[5] * y + M[2] * z;
}

// ------------------------------------------------------------------------------------
// a5: injection, one thread per target particle: E_g += dt * sum_e coef_e L[src_e][g]
// (coef = xi / V_target), accumulated in double.
template <class T>
__global__ void k_inject(const int32_t* __restrict__ targets, const int32_t* __restrict__ off,
                         const int32_t* __restrict__ src, const double* __restrict__ coef,
                         const double* __restrict__ L, int G, const double* __restrict__ dt_dev, int64_t n_targets,
                         int64_t n, T* U) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n_targets) return;
    double dt = *dt_dev;
    int64_t p = targets[t];
    for (int g = 0; g < G; ++g) {
        double acc = 0.0;
        for (int e = off[t]; e < off[t + 1]; ++e) acc += coef[e] * L[(int64_t)src[e] * G + g];
        T* E = U + (int64_t)(4 * g) * n + p;
        *E = (T)((double)*E + dt * acc);
    }
}

// ------------------------------------------------------------------------------------
// a6: least-squares gradient (Eq. gradient) of the groups [g0, g0 + GC):
// grad Q_i = omega_i Bp_i sum_j (Q_j - Q_i) w(r_ij / H_i) d_ij,  d_ij = x_j - x_i
template <class T, int GC>
__global__ void __launch_bounds__(128) k_gradient(PairArgs<T> a, const T* __restrict__ U, T* __restrict__ grad, int g0) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = a.n;
    if (i >= n) return;
    constexpr int NC = 4 * GC;
    PosT<T> pi;
    load_pos(a.sp, i, pi);
    T iH = a.invH[i];
    T ui[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) ui[c] = U[(int64_t)(4 * g0 + c) * n + i];
    T acc[NC][3];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c][0] = acc[c][1] = acc[c][2] = T(0);
    const int64_t e0 = a.row_off[i], e1 = a.row_off[i + 1];
    for (int64_t e = e0; e < e1; ++e) {
        int j = a.cols[e];
        PosT<T> pj;
        load_pos(a.sp, j, pj);
        T dx, dy, dz;
        sep(a.sp, pi, pj, dx, dy, dz);
        T r = sqrt(dx * dx + dy * dy + dz * dz);
        T w = spline_w(r * iH);
        if (w == T(0)) continue;
        T wx = w * dx, wy = w * dy, wz = w * dz;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            T dq = U[(int64_t)(4 * g0 + c) * n + j] - ui[c];
            acc[c][0] += dq * wx;
            acc[c][1] += dq * wy;
            acc[c][2] += dq * wz;
        }
    }
    T M[6];
    T om = a.omega[i];
#pragma unroll
    for (int k = 0; k < 6; ++k) M[k] = om * a.Bp[k * n + i];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        T gx, gy, gz;
        sym_mv(M, acc[c][0], acc[c][1], acc[c][2], gx, gy, gz);
        int64_t base = ((int64_t)(4 * g0 + c) * 3) * n + i;
        grad[base] = gx;
        grad[base + n] = gy;
        grad[base + 2 * n] = gz;
    }
}

// ------------------------------------------------------------------------------------
// a7 + a8: pair fluxes, explicit update, grey sink, optional fix-up, groups [g0, g0 + GC).
template <class T>
struct FluxExtra {
    const T* alpha;                 // sorted, or null
    const double* dt_dev;
    T c;
    int clamp;
    unsigned long long* clamp_count;
};

// Flux of pair (k, l) for one group: face states (Eq. rt-riemann-problem with
// s = minmod(grad Q_k . d, grad Q_l . d)), M1 fluxes (Eq. eddington-group), GLF (Eq. riemann-GLF).
template <class T>
__device__ __forceinline__ void pair_flux(const T uk[4], const T ul[4], const T gk[4][3], const T gl[4][3], T dx, T dy,
                                          T dz, T wk, T wl, T Ax, T Ay, T Az, T An, T c, T phi[4]) {
    T L[4], R[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        T dqk = gk[q][0] * dx + gk[q][1] * dy + gk[q][2] * dz;
        T dql = gl[q][0] * dx + gl[q][1] * dy + gl[q][2] * dz;
        T s = minmod(dqk, dql);
        L[q] = uk[q] + wk * s;
        R[q] = ul[q] - wl * s;
    }
    T fL[4], fR[4];
    m1_dot(L[0], L[1], L[2], L[3], Ax, Ay, Az, c, fL[0], fL[1], fL[2], fL[3]);
    m1_dot(R[0], R[1], R[2], R[3], Ax, Ay, Az, c, fR[0], fR[1], fR[2], fR[3]);
    T diss = T(0.5) * c * An;
#pragma unroll
    for (int q = 0; q < 4; ++q) phi[q] = T(0.5) * (fL[q] + fR[q]) - diss * (R[q] - L[q]);
}

// geometry of the pair in canonical roles: A_kl = (Bp_k w_k + Bp_l w_l) d (Eq. HopkinsAij with
// V psitilde = Bp d w), |A|, the interface weights h_k/(h_k+h_l), h_l/(h_k+h_l)
template <class T>
__device__ __forceinline__ void pair_geometry(const T Bk[6], const T Bl[6], T iHk, T iHl, T hk, T hl, T dx, T dy,
                                              T dz, T& Ax, T& Ay, T& Az, T& An, T& wk, T& wl) {
    T r = sqrt(dx * dx + dy * dy + dz * dz);
    T sk = spline_w(r * iHk);
    T sl = spline_w(r * iHl);
    T M[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) M[q] = Bk[q] * sk + Bl[q] * sl;
    sym_mv(M, dx, dy, dz, Ax, Ay, Az);
    An = sqrt(Ax * Ax + Ay * Ay + Az * Az);
    T ih = T(1) / (hk + hl);
    wk = hk * ih;
    wl = hl * ih;
}

template <class T, int GC>
__global__ void __launch_bounds__(128) k_flux(PairArgs<T> a, FluxExtra<T> x, const T* __restrict__ U,
                                              const T* __restrict__ grad, T* __restrict__ Uout, int g0) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = a.n;
    if (i >= n) return;
    constexpr int NC = 4 * GC;
    PosT<T> pi;
    load_pos(a.sp, i, pi);
    const T iHi = a.invH[i], hi = a.h[i];
    T Bi[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) Bi[k] = a.Bp[k * n + i];
    T ui[NC], gi[NC][3];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        int64_t cc = 4 * g0 + c;
        ui[c] = U[cc * n + i];
        gi[c][0] = grad[(cc * 3) * n + i];
        gi[c][1] = grad[(cc * 3 + 1) * n + i];
        gi[c][2] = grad[(cc * 3 + 2) * n + i];
    }
    T acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = T(0);
    const int64_t e0 = a.row_off[i], e1 = a.row_off[i + 1];
    for (int64_t e = e0; e < e1; ++e) {
        const int j = a.cols[e];
        const bool ik = i < j;
        PosT<T> pj;
        load_pos(a.sp, j, pj);
        const T iHj = a.invH[j], hj = a.h[j];
        T Bj[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) Bj[k] = a.Bp[k * n + j];
        // canonical roles: k = lower sorted index (left state), l = higher
        T dx, dy, dz;
        if (ik) sep(a.sp, pi, pj, dx, dy, dz);
        else sep(a.sp, pj, pi, dx, dy, dz);
        T Ax, Ay, Az, An, wk, wl;
        if (ik) pair_geometry(Bi, Bj, iHi, iHj, hi, hj, dx, dy, dz, Ax, Ay, Az, An, wk, wl);
        else pair_geometry(Bj, Bi, iHj, iHi, hj, hi, dx, dy, dz, Ax, Ay, Az, An, wk, wl);
#pragma unroll
        for (int g = 0; g < GC; ++g) {
            T uo[4], go[4][3];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int64_t cc = 4 * (g0 + g) + q;
                uo[q] = U[cc * n + j];
                go[q][0] = grad[(cc * 3) * n + j];
                go[q][1] = grad[(cc * 3 + 1) * n + j];
                go[q][2] = grad[(cc * 3 + 2) * n + j];
            }
            T phi[4];
            if (ik) pair_flux(&ui[4 * g], uo, &gi[4 * g], go, dx, dy, dz, wk, wl, Ax, Ay, Az, An, x.c, phi);
            else pair_flux(uo, &ui[4 * g], go, &gi[4 * g], dx, dy, dz, wk, wl, Ax, Ay, Az, An, x.c, phi);
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[4 * g + q] += ik ? phi[q] : -phi[q];
        }
    }
    // U_i(t + dt) = U_i - dt / V_i sum_l F_il . A_il, then the sink and the fix-up
    const T dt = (T)(*x.dt_dev);
    const T f = dt * a.omega[i];
    T sink = T(1);
    if (x.alpha) {
        sink = T(1) - x.c * x.alpha[i] * dt;
        sink = sink > T(0) ? sink : T(0);
    }
    int nclamp = 0;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        T v = (ui[c] - f * acc[c]) * sink;
        if (x.clamp && (c & 3) == 0 && v < T(0)) {
            v = T(0);
            ++nclamp;
        }
        Uout[(int64_t)(4 * g0 + c) * n + i] = v;
    }
    if (nclamp) atomicAdd(x.clamp_count, (unsigned long long)nclamp);
}

// ------------------------------------------------------------------------------------
// a10: energy per group, sum_i V_i E_i,g in double; fixed grid and tree order.
constexpr int kEnergyBlocks = 512;

template <class T>
__global__ void k_energy_part(const T* __restrict__ U, const double* __restrict__ V, int64_t n, int G,
                              double* part) {
    __shared__ double sm[256];
    for (int g = 0; g < G; ++g) {
        double s = 0.0;
        for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
            s += V[p] * (double)U[(int64_t)(4 * g) * n + p];
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
template <class T>
static PairArgs<T> pair_args(rt_ctx* c) {
    PairArgs<T> a;
    if constexpr (sizeof(T) == 4) {
        a.sp.x = c->xq.as<uint32_t>();
        double units = c->cfg.periodic ? 4294967296.0 : 2147483648.0;
        a.sp.s0 = (float)(c->cfg.box[0] / units);
        a.sp.s1 = (float)(c->cfg.box[1] / units);
        a.sp.s2 = (float)(c->cfg.box[2] / units);
        a.sp.n = c->n;
    } else {
        a.sp.x = c->xs_d.as<double>();
        a.sp.b0 = c->cfg.box[0];
        a.sp.b1 = c->cfg.box[1];
        a.sp.b2 = c->cfg.box[2];
        a.sp.periodic = c->cfg.periodic;
        a.sp.n = c->n;
    }
    a.invH = c->invH_t.as<T>();
    a.h = c->h_t.as<T>();
    a.omega = c->omega_t.as<T>();
    a.Bp = c->Bp_t.as<T>();
    a.row_off = c->row_off.as<int64_t>();
    a.cols = c->cols.as<int32_t>();
    a.n = c->n;
    return a;
}

template <class T>
static void launch_gradient_t(rt_ctx* c, cudaStream_t s, const T* U, T* grad) {
    PairArgs<T> a = pair_args<T>(c);
    const int G = c->cfg.n_groups;
    unsigned nb = nblk(c->n, 128);
    for (int g0 = 0; g0 < G; g0 += kMaxGC) {
        int gc = G - g0 < kMaxGC ? G - g0 : kMaxGC;
        switch (gc) {
            case 1: k_gradient<T, 1><<<nb, 128, 0, s>>>(a, U, grad, g0); break;
            case 2: k_gradient<T, 2><<<nb, 128, 0, s>>>(a, U, grad, g0); break;
            case 3: k_gradient<T, 3><<<nb, 128, 0, s>>>(a, U, grad, g0); break;
            default: k_gradient<T, 4><<<nb, 128, 0, s>>>(a, U, grad, g0); break;
        }
    }
}

template <class T>
static void launch_flux_t(rt_ctx* c, cudaStream_t s, const T* U, const T* grad, T* Uout, bool has_alpha) {
    PairArgs<T> a = pair_args<T>(c);
    FluxExtra<T> x;
    x.alpha = has_alpha ? c->alpha_s.as<T>() : nullptr;
    x.dt_dev = c->dt_dev.as<double>();
    x.c = (T)c->cfg.c_red;
    x.clamp = c->cfg.clamp_negative;
    x.clamp_count = reinterpret_cast<unsigned long long*>(c->flags.as<int>() + 8);
    const int G = c->cfg.n_groups;
    unsigned nb = nblk(c->n, 128);
    for (int g0 = 0; g0 < G; g0 += kMaxGC) {
        int gc = G - g0 < kMaxGC ? G - g0 : kMaxGC;
        switch (gc) {
            case 1: k_flux<T, 1><<<nb, 128, 0, s>>>(a, x, U, grad, Uout, g0); break;
            case 2: k_flux<T, 2><<<nb, 128, 0, s>>>(a, x, U, grad, Uout, g0); break;
            case 3: k_flux<T, 3><<<nb, 128, 0, s>>>(a, x, U, grad, Uout, g0); break;
            default: k_flux<T, 4><<<nb, 128, 0, s>>>(a, x, U, grad, Uout, g0); break;
        }
    }
}

template <class T>
static void launch_inject_t(rt_ctx* c, cudaStream_t s, T* U) {
    if (c->n_inj_targets <= 0) return;
    k_inject<T><<<nblk(c->n_inj_targets, 128), 128, 0, s>>>(
        c->inj_targets.as<int32_t>(), c->inj_off.as<int32_t>(), c->inj_src.as<int32_t>(), c->inj_coef.as<double>(),
        c->L_dev.as<double>(), c->cfg.n_groups, c->dt_dev.as<double>(), c->n_inj_targets, c->n, U);
}

rt_status launch_gradient(rt_ctx* c, cudaStream_t s, const void* U, void* grad) {
    if (c->fp64) launch_gradient_t<double>(c, s, (const double*)U, (double*)grad);
    else launch_gradient_t<float>(c, s, (const float*)U, (float*)grad);
    RT_CUDA(c, cudaGetLastError());
    return RT_OK;
}

rt_status launch_step(rt_ctx* c, cudaStream_t s, void* Uin, void* Uout, bool has_src, bool has_alpha) {
    if (c->fp64) {
        if (has_src) launch_inject_t<double>(c, s, (double*)Uin);
        launch_gradient_t<double>(c, s, (const double*)Uin, c->grad.as<double>());
        launch_flux_t<double>(c, s, (const double*)Uin, c->grad.as<double>(), (double*)Uout, has_alpha);
    } else {
        if (has_src) launch_inject_t<float>(c, s, (float*)Uin);
        launch_gradient_t<float>(c, s, (const float*)Uin, c->grad.as<float>());
        launch_flux_t<float>(c, s, (const float*)Uin, c->grad.as<float>(), (float*)Uout, has_alpha);
    }
    RT_CUDA(c, cudaGetLastError());
    return RT_OK;
}

rt_status to_sorted(rt_ctx* c, const void* U_user, void* U_sorted, int comps) {
    unsigned nb = nblk(c->n, 256);
    if (c->fp64)
        k_to_sorted<double><<<nb, 256, 0, c->stream>>>((const double*)U_user, c->perm.as<int32_t>(), c->n, comps,
                                                        (double*)U_sorted);
    else
        k_to_sorted<float><<<nb, 256, 0, c->stream>>>((const float*)U_user, c->perm.as<int32_t>(), c->n, comps,
                                                       (float*)U_sorted);
    RT_CUDA(c, cudaGetLastError());
    return RT_OK;
}

rt_status from_sorted(rt_ctx* c, const void* U_sorted, void* U_user, int comps) {
    unsigned nb = nblk(c->n, 256);
    if (c->fp64)
        k_from_sorted<double><<<nb, 256, 0, c->stream>>>((const double*)U_sorted, c->inv_perm.as<int32_t>(), c->n,
                                                          comps, (double*)U_user);
    else
        k_from_sorted<float><<<nb, 256, 0, c->stream>>>((const float*)U_sorted, c->inv_perm.as<int32_t>(), c->n,
                                                         comps, (float*)U_user);
    RT_CUDA(c, cudaGetLastError());
    return RT_OK;
}

rt_status set_step_inputs(rt_ctx* c, double dt, const double* Lsrc, const double* alpha) {
    cudaStream_t s = c->stream;
    k_set_scalar<<<1, 1, 0, s>>>(c->dt_dev.as<double>(), dt);
    if (Lsrc && c->n_src > 0)
        RT_CUDA(c, cudaMemcpyAsync(c->L_dev.p, Lsrc, (size_t)c->n_src * c->cfg.n_groups * sizeof(double),
                                   cudaMemcpyDeviceToDevice, s));
    if (alpha) {
        unsigned nb = nblk(c->n, 256);
        if (c->fp64) k_alpha_sorted<double><<<nb, 256, 0, s>>>(alpha, c->perm.as<int32_t>(), c->n, c->alpha_s.as<double>());
        else k_alpha_sorted<float><<<nb, 256, 0, s>>>(alpha, c->perm.as<int32_t>(), c->n, c->alpha_s.as<float>());
    }
    RT_CUDA(c, cudaGetLastError());
    return RT_OK;
}

rt_status launch_energy(rt_ctx* c, cudaStream_t s, const void* U_sorted, double* out_dev) {
    double* part = c->energy_part.as<double>();
    if (c->fp64)
        k_energy_part<double><<<kEnergyBlocks, 256, 0, s>>>((const double*)U_sorted, c->V_d.as<double>(), c->n,
                                                            c->cfg.n_groups, part);
    else
        k_energy_part<float><<<kEnergyBlocks, 256, 0, s>>>((const float*)U_sorted, c->V_d.as<double>(), c->n,
                                                           c->cfg.n_groups, part);
    k_energy_final<<<1, 32 * ((c->cfg.n_groups + 31) / 32), 0, s>>>(part, kEnergyBlocks, c->cfg.n_groups, out_dev);
    RT_CUDA(c, cudaGetLastError());
    return RT_OK;
}

}  // namespace rt
