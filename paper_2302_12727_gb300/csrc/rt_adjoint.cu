// Reverse-mode derivative of n sub-cycles of the transport step (no counterpart in the
// thesis).  Given lambda = dL/dU(final) it returns dL/dU0 and dL/dL_src.
//
// One forward step is  U_inj = U + inj(L);  g = grad(U_inj);  Phi_kl = flux(U_inj, g);
// U~_i = U_inj,i - dt omega_i (sum_{k=i} Phi - sum_{l=i} Phi);  U'_i = U~_i sink_i.
// Its adjoint, for lambda' = dL/dU':
//   lambda~_i = lambda'_i sink_i,  mu_i = -dt omega_i lambda~_i,  Phibar_kl = mu_k - mu_l;
//   through the GLF flux (Eq. riemann-GLF), the M1 closure (Eq. eddington-group) and the
//   limited face states (Eq. rt-riemann-problem, Eq. rt-minmod: the derivative follows the
//   selected slope) to Ubar (direct) and gbar (through the gradients);
//   through the least-squares gradient (Eq. gradient), whose transpose is
//   Ubar_i -= sum_j d_ij . (gamma_i w(r_ij/H_i) + gamma_j w(r_ij/H_j)), gamma = omega Bp gbar;
//   the injection is additive, so lambda passes through and dL/dL_s,g += dt sum_e coef_e lambda_E.
// The fix-up E <- max(E, 0) is treated as inactive.
//
// The forward pass keeps the state every ckpt_every steps; the reverse pass recomputes each
// segment with the forward kernels (bitwise the same states) and walks it backwards.  Pair
// terms are evaluated by both particles in the pair's canonical orientation (k < l), each
// keeping its own side, so the reductions are per particle, fixed-order and atomic-free.
#include "rt_pair.cuh"

namespace rt {

static inline unsigned nblk_(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// J(u)^T pb for the M1 flux contracted with A (m1_dot_): u = (E, F), pb = dL/d(flux).
// Derivatives of (F.A, c^2 E [a(u) A + b(u) u/|F|^2 (F.A) F]) with u = min(|F|^2/(cE)^2, 1),
// a = (1 - chi)/2, b = (3 chi - 1)/(2u), both functions of s = sqrt(4 - 3u).
template <class T>
__device__ __forceinline__ void m1_vjp(const T u4[4], T Ax, T Ay, T Az, T c, const T pb[4], T ub[4]) {
    const T E = u4[0], Fx = u4[1], Fy = u4[2], Fz = u4[3];
    ub[0] = T(0);
    ub[1] = pb[0] * Ax;
    ub[2] = pb[0] * Ay;
    ub[3] = pb[0] * Az;
    if (!(E > T(0))) return;
    const T FA = Fx * Ax + Fy * Ay + Fz * Az;
    const T phA = pb[1] * Ax + pb[2] * Ay + pb[3] * Az;
    const T phF = pb[1] * Fx + pb[2] * Fy + pb[3] * Fz;
    const T F2 = Fx * Fx + Fy * Fy + Fz * Fz;
    const T c2 = c * c;
    const T u = F2 / (c2 * E * E);
    if (u > T(1)) {
        // clamped: flux = c^2 E (F.A) F / |F|^2
        const T iF2 = T(1) / F2;
        ub[0] += c2 * FA * phF * iF2;
        const T k1 = c2 * E * iF2;
        const T k2 = T(2) * c2 * E * FA * phF * iF2 * iF2;
        ub[1] += k1 * (phF * Ax + FA * pb[1]) - k2 * Fx;
        ub[2] += k1 * (phF * Ay + FA * pb[2]) - k2 * Fy;
        ub[3] += k1 * (phF * Az + FA * pb[3]) - k2 * Fz;
        return;
    }
    const T s = sqrt(T(4) - T(3) * u);
    const T sp = T(-1.5) / s;                      // ds/du
    const T q5 = T(5) + T(2) * s, q4 = T(4) + T(2) * s;
    const T a = (T(1) + s - T(2) * u) / q5;
    const T ap = ((sp - T(2)) * q5 - (T(1) + s - T(2) * u) * T(2) * sp) / (q5 * q5);
    const T b = T(6) * (T(1) + T(1) / q4) / q5;
    const T bp = T(6) * ((T(-2) * sp / (q4 * q4)) * q5 - (T(1) + T(1) / q4) * T(2) * sp) / (q5 * q5);
    const T iE = T(1) / E;
    ub[0] += c2 * (a - T(2) * u * ap) * phA - (T(2) * u * bp + b) * FA * phF * iE * iE;
    const T cf = T(2) * ap * iE * phA + T(2) * bp * FA * phF * iE * iE * iE / c2;
    const T bE = b * iE;
    ub[1] += cf * Fx + bE * (phF * Ax + FA * pb[1]);
    ub[2] += cf * Fy + bE * (phF * Ay + FA * pb[2]);
    ub[3] += cf * Fz + bE * (phF * Az + FA * pb[3]);
}

// adjoint of the flux stage for group g0 + g of a group chunk of GC: one thread per (particle i,
// group), over i's whole row; the pair geometry is recomputed by each group's thread
template <class T, int GC>
__global__ void __launch_bounds__(128) k_adj_flux(PairArgs<T> a, FluxExtra<T> x, const T* __restrict__ lam,
                                                  const T* __restrict__ W, T* __restrict__ ubar, T* __restrict__ gam,
                                                  int g0) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i = t / GC;
    if (i >= a.n) return;
    const int gg = g0 + (int)(t - i * GC);
    const T* tag = nullptr;
    const int G = a.G, RS = 4 * G;
    const T dt = (T)(*x.dt_dev);
    auto sink_of = [&](int64_t p) {
        T sk = T(1);
        if (x.alpha) sk = fmax_(T(1) - x.c * x.alpha[p] * dt, T(0));
        return sk;
    };
    const T sink_i = sink_of(i), om_i = a.omega[i];
    T li[4], mui[4], ub[4], gb[4][3];
    vload<4>(lam + i * RS + 4 * gg, li);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        li[q] *= sink_i;
        mui[q] = -dt * om_i * li[q];   // same expression as for the other particle below
        ub[q] = li[q];
        gb[q][0] = gb[q][1] = gb[q][2] = T(0);
    }
    const Pos<T> pi = load_pos(tag, a.pos, i);
    T gi8[8], ui[4], gri[12];
    vload<8>(a.geo + 8 * i, gi8);
    vload<4>(W + i * RS + 4 * gg, ui);
    vload<12>(a.grad + i * 12 * G + 12 * gg, gri);
    for (int64_t e = a.row_off[i]; e < a.row_off[i + 1]; ++e) {
        const int64_t j = a.cols[e];
        const bool ik = i < j;                     // i is the left state k
        const Pos<T> pj = load_pos(tag, a.pos, j);
        T gj8[8];
        vload<8>(a.geo + 8 * j, gj8);
        const T* gk8 = ik ? gi8 : gj8;
        const T* gl8 = ik ? gj8 : gi8;
        T dx, dy, dz;
        if (ik) sep(a.sp, pi, pj, dx, dy, dz);
        else sep(a.sp, pj, pi, dx, dy, dz);       // d = x_l - x_k
        T r = sqrt_(dx * dx + dy * dy + dz * dz);
        T sk = spline_w_(r * gk8[0]), sl = spline_w_(r * gl8[0]);
        T M[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) M[q] = gk8[2 + q] * sk + gl8[2 + q] * sl;
        T Ax, Ay, Az;
        sym_mv(M, dx, dy, dz, Ax, Ay, Az);
        const T diss = T(0.5) * x.c * sqrt_(Ax * Ax + Ay * Ay + Az * Az);
        const T ih = rcp_(gk8[1] + gl8[1]);
        const T wk = gk8[1] * ih, wl = gl8[1] * ih;
        // mu of the other particle
        const T sink_j = sink_of(j), om_j = a.omega[j];
        T lj[4], uj[4], grj[12];
        vload<4>(lam + j * RS + 4 * gg, lj);
        vload<4>(W + j * RS + 4 * gg, uj);
        vload<12>(a.grad + j * 12 * G + 12 * gg, grj);
        const T* uk = ik ? ui : uj;
        const T* ul = ik ? uj : ui;
        const T* gk = ik ? gri : grj;
        const T* gl = ik ? grj : gri;
        T L[4], R[4], s[4];
        int sel[4];                          // 1: slope of k, 2: slope of l, 0: none
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            T dqk = gk[3 * q] * dx + gk[3 * q + 1] * dy + gk[3 * q + 2] * dz;
            T dql = gl[3 * q] * dx + gl[3 * q + 1] * dy + gl[3 * q + 2] * dz;
            s[q] = minmod_(dqk, dql);
            bool pos = dqk > T(0) && dql > T(0), neg = dqk < T(0) && dql < T(0);
            sel[q] = (pos || neg) ? (((pos && dqk < dql) || (neg && dqk > dql)) ? 1 : 2) : 0;
            L[q] = fma_rn(wk, s[q], uk[q]);
            R[q] = fma_rn(-wl, s[q], ul[q]);
        }
        T pb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const T muj = -dt * om_j * (lj[q] * sink_j);
            const T muk = ik ? mui[q] : muj;
            const T mul = ik ? muj : mui[q];
            pb[q] = muk - mul;
        }
        T jL[4], jR[4];
        m1_vjp(L, Ax, Ay, Az, x.c, pb, jL);
        m1_vjp(R, Ax, Ay, Az, x.c, pb, jR);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const T Lb = T(0.5) * jL[q] + diss * pb[q];
            const T Rb = T(0.5) * jR[q] - diss * pb[q];
            const T sb = wk * Lb - wl * Rb;
            ub[q] += ik ? Lb : Rb;
            const bool mine = ik ? (sel[q] == 1) : (sel[q] == 2);
            if (mine) {
                gb[q][0] += sb * dx;
                gb[q][1] += sb * dy;
                gb[q][2] += sb * dz;
            }
        }
    }
    vstore<4>(ubar + i * RS + 4 * gg, ub);
    // gamma_i = omega_i Bp_i gbar_i (the gradient is omega_i Bp_i sum_j (Q_j - Q_i) w d, Bp symmetric)
    T Mi[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) Mi[k] = om_i * gi8[2 + k];
    T out[12];
#pragma unroll
    for (int q = 0; q < 4; ++q) sym_mv(Mi, gb[q][0], gb[q][1], gb[q][2], out[3 * q], out[3 * q + 1], out[3 * q + 2]);
    vstore<12>(gam + i * 12 * G + 12 * gg, out);
}

// transpose of the gradient operator: lambda_i = ubar_i - sum_j d_ij . (gamma_i w_i + gamma_j w_j),
// one thread per (particle i, group g0 + g of a chunk of GC)
template <class T, int GC>
__global__ void __launch_bounds__(128) k_adj_grad(PairArgs<T> a, const T* __restrict__ ubar,
                                                  const T* __restrict__ gam, T* __restrict__ lam_out, int g0) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i = t / GC;
    if (i >= a.n) return;
    const int gg = g0 + (int)(t - i * GC);
    const T* tag = nullptr;
    const int G = a.G, RS = 4 * G;
    const Pos<T> pi = load_pos(tag, a.pos, i);
    const T iHi = a.geo[8 * i];
    T gi[12], acc[4];
    vload<12>(gam + i * 12 * G + 12 * gg, gi);
    vload<4>(ubar + i * RS + 4 * gg, acc);
    for (int64_t e = a.row_off[i]; e < a.row_off[i + 1]; ++e) {
        const int64_t j = a.cols[e];
        const Pos<T> pj = load_pos(tag, a.pos, j);
        T dx, dy, dz;
        sep(a.sp, pi, pj, dx, dy, dz);              // d_ij = x_j - x_i
        const T r = sqrt_(dx * dx + dy * dy + dz * dz);
        const T wi = spline_w_(r * iHi);
        const T wj = spline_w_(r * a.geo[8 * j]);
        T gj[12];
        vload<12>(gam + j * 12 * G + 12 * gg, gj);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const T vx = gi[3 * q] * wi + gj[3 * q] * wj;
            const T vy = gi[3 * q + 1] * wi + gj[3 * q + 1] * wj;
            const T vz = gi[3 * q + 2] * wi + gj[3 * q + 2] * wj;
            acc[q] -= dx * vx + dy * vy + dz * vz;
        }
    }
    vstore<4>(lam_out + i * RS + 4 * gg, acc);
}

// dL/dL_s,g += dt sum over the source's entries of (xi / V_target) lambda_E,g(target): one
// warp per (source, group); its lanes load 32 consecutive entries at a time and every lane adds
// their terms in entry order (the same sum in all lanes)
template <class T>
__global__ void k_adj_inject(const int64_t* __restrict__ src_off, const int32_t* __restrict__ e_gas,
                             const double* __restrict__ e_xi, const double* __restrict__ V, const T* __restrict__ lam,
                             int64_t S, int G, const double* __restrict__ dt_dev, double* dLdL) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= S * G) return;   // whole warps
    const int64_t s = w / G;
    const int g = (int)(w % G);
    const int64_t e0 = src_off[s], e1 = src_off[s + 1];
    double acc = 0.0;
    for (int64_t b = e0; b < e1; b += 32) {
        const int64_t e = b + lane;
        double q = 0.0, l = 0.0;
        if (e < e1) {
            const int64_t p = e_gas[e];
            q = e_xi[e] / V[p];
            l = (double)lam[p * 4 * G + 4 * g];
        }
        const int m = e1 - b < 32 ? (int)(e1 - b) : 32;
        for (int u = 0; u < m; ++u)
            acc = fma(__shfl_sync(0xffffffffu, q, u), __shfl_sync(0xffffffffu, l, u), acc);
    }
    if (lane == 0) dLdL[w] += *dt_dev * acc;
}

template <class T>
static void launch_adj_step(rt_ctx* c, cudaStream_t s, const T* lamN, const T* W, T* ub, T* gam, T* lamO,
                            bool has_alpha) {
    PairArgs<T> a = pair_args<T>(c);
    FluxExtra<T> x;
    x.wave = nullptr;   // GLF only
    x.alpha = has_alpha ? c->alpha_s.as<T>() : nullptr;
    x.alpha_g = nullptr;   // grey sink only
    x.acc = nullptr;
    x.inj = nullptr;
    x.dt_dev = c->dt_dev.as<double>();
    x.c = (T)c->cfg.c_red;
    x.clamp = 0;
    x.clamp_count = nullptr;
    const int G = c->cfg.n_groups;
    for (int g0 = 0; g0 < G; g0 += kMaxGC) {
        int gc = G - g0 < kMaxGC ? G - g0 : kMaxGC;
        const unsigned nbg = nblk_(c->n * gc, 128);
        switch (gc) {
            case 1: k_adj_flux<T, 1><<<nbg, 128, 0, s>>>(a, x, lamN, W, ub, gam, g0); break;
            case 2: k_adj_flux<T, 2><<<nbg, 128, 0, s>>>(a, x, lamN, W, ub, gam, g0); break;
            case 3: k_adj_flux<T, 3><<<nbg, 128, 0, s>>>(a, x, lamN, W, ub, gam, g0); break;
            default: k_adj_flux<T, 4><<<nbg, 128, 0, s>>>(a, x, lamN, W, ub, gam, g0); break;
        }
    }
    for (int g0 = 0; g0 < G; g0 += kMaxGC) {
        int gc = G - g0 < kMaxGC ? G - g0 : kMaxGC;
        const unsigned nbg = nblk_(c->n * gc, 128);
        switch (gc) {
            case 1: k_adj_grad<T, 1><<<nbg, 128, 0, s>>>(a, ub, gam, lamO, g0); break;
            case 2: k_adj_grad<T, 2><<<nbg, 128, 0, s>>>(a, ub, gam, lamO, g0); break;
            case 3: k_adj_grad<T, 3><<<nbg, 128, 0, s>>>(a, ub, gam, lamO, g0); break;
            default: k_adj_grad<T, 4><<<nbg, 128, 0, s>>>(a, ub, gam, lamO, g0); break;
        }
    }
    c->launches += 2 * ((G + kMaxGC - 1) / kMaxGC);
}

rt_status run_adjoint(rt_ctx* c, int n_sub, int k, bool has_src, bool has_alpha, const void* U0s,
                      const void* lam_final, void* lam0, double* dLdL) {
    const int G = c->cfg.n_groups;
    const int64_t n = c->n;
    const size_t ts = c->fp64 ? 8 : 4;
    const size_t S = (size_t)4 * G * n * ts;     // one state, bytes
    const int nck = (n_sub + k - 1) / k;
    const int kseg = k < n_sub ? k : n_sub;
    cudaStream_t st = c->stream;
    RT_TRY(ensure(c, c->ck, (size_t)nck * S, "adjoint checkpoints"));
    RT_TRY(ensure(c, c->seg, (size_t)kseg * S, "adjoint segment"));
    RT_TRY(ensure(c, c->adj_w, S, "adjoint"));
    RT_TRY(ensure(c, c->adj_x, S, "adjoint"));
    RT_TRY(ensure(c, c->adj_ub, S, "adjoint"));
    RT_TRY(ensure(c, c->adj_gam, 3 * S, "adjoint"));
    RT_TRY(ensure(c, c->adj_lam, S, "adjoint"));
    char* ck = c->ck.as<char>();
    char* seg = c->seg.as<char>();
    void* X = c->adj_x.p;
    void* W = c->adj_w.p;

    // forward pass with a checkpoint every k steps
    RT_CUDA(c, cudaMemcpyAsync(X, U0s, S, cudaMemcpyDeviceToDevice, st));
    for (int t = 0; t < n_sub; ++t) {
        if (t % k == 0) RT_CUDA(c, cudaMemcpyAsync(ck + (size_t)(t / k) * S, X, S, cudaMemcpyDeviceToDevice, st));
        if (t == n_sub - 1) break;      // the final state is not needed
        RT_TRY(launch_step(c, st, X, W, has_src, has_alpha));
        std::swap(X, W);
    }

    // reverse pass: lambda ping-pongs between the caller's final-lambda copy and adj_lam
    void* lamN = const_cast<void*>(lam_final);
    void* lamO = c->adj_lam.p;
    for (int m = nck - 1; m >= 0; --m) {
        const int n0 = m * k;
        const int len = (n_sub - n0) < k ? (n_sub - n0) : k;
        RT_CUDA(c, cudaMemcpyAsync(seg, ck + (size_t)m * S, S, cudaMemcpyDeviceToDevice, st));
        for (int t = 0; t + 1 < len; ++t) {
            RT_CUDA(c, cudaMemcpyAsync(c->adj_x.p, seg + (size_t)t * S, S, cudaMemcpyDeviceToDevice, st));
            RT_TRY(launch_step(c, st, c->adj_x.p, seg + (size_t)(t + 1) * S, has_src, has_alpha));
        }
        for (int t = len - 1; t >= 0; --t) {
            RT_CUDA(c, cudaMemcpyAsync(c->adj_w.p, seg + (size_t)t * S, S, cudaMemcpyDeviceToDevice, st));
            if (has_src) RT_TRY(launch_inject(c, st, c->adj_w.p));
            RT_TRY(launch_gradient(c, st, c->adj_w.p));
            if (c->fp64)
                launch_adj_step<double>(c, st, (const double*)lamN, c->adj_w.as<double>(), c->adj_ub.as<double>(),
                                        c->adj_gam.as<double>(), (double*)lamO, has_alpha);
            else
                launch_adj_step<float>(c, st, (const float*)lamN, c->adj_w.as<float>(), c->adj_ub.as<float>(),
                                       c->adj_gam.as<float>(), (float*)lamO, has_alpha);
            if (has_src && dLdL && c->n_inj_entries > 0) {
                int64_t SG = c->n_src * G;   // one warp each
                if (c->fp64)
                    k_adj_inject<double><<<nblk_(SG * 32, 128), 128, 0, st>>>(
                        c->src_off.as<int64_t>(), c->src_entry_gas.as<int32_t>(), c->src_entry_xi.as<double>(),
                        c->V_d.as<double>(), (const double*)lamO, c->n_src, G, c->dt_dev.as<double>(), dLdL);
                else
                    k_adj_inject<float><<<nblk_(SG * 32, 128), 128, 0, st>>>(
                        c->src_off.as<int64_t>(), c->src_entry_gas.as<int32_t>(), c->src_entry_xi.as<double>(),
                        c->V_d.as<double>(), (const float*)lamO, c->n_src, G, c->dt_dev.as<double>(), dLdL);
                ++c->launches;
            }
            RT_CUDA(c, cudaGetLastError());
            std::swap(lamN, lamO);     // lamN: dL/dU at the start of this step
        }
    }
    if (lamN != lam0) RT_CUDA(c, cudaMemcpyAsync(lam0, lamN, S, cudaMemcpyDeviceToDevice, st));
    return RT_OK;
}

}  // namespace rt
