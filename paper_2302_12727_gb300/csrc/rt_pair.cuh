// Device helpers of the pair kernels shared by the forward (rt_transport.cu) and adjoint
// (rt_adjoint.cu) passes: precision primitives, the spline, minmod and M1 closure in
// branch-free form, position / geometry / state record access, and the pair flux.
#pragma once

#include "rt_internal.cuh"

namespace rt {

// ------------------------------------------------------------------------------------
// precision-specific primitives: IEEE in double, approximate reciprocal / square root in
// float (relative error ~1e-7, far inside the float path's tolerance)
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float rcp_(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// explicitly rounded fused multiply-add
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double fmax_(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float fmax_(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double fmin_(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float fmin_(float a, float b) { return fminf(a, b); }

// cubic-spline shape without branches: (1-q)_+^3 - 4 (1/2-q)_+^3 (Eq. cubic-spline-kernel)
template <class T>
__device__ __forceinline__ T spline_w_(T q) {
    T a = fmax_(T(1) - q, T(0));
    T b = fmax_(T(0.5) - q, T(0));
    return a * a * a - T(4) * (b * b * b);
}

// minmod of Eq. rt-minmod (both positive -> min, both negative -> max, else 0) as the median
// of a, b and 0: max(min(a, b), min(max(a, b), 0)), four min/max and no compare or select
template <class T>
__device__ __forceinline__ T minmod_(T a, T b) {
    return fmax_(fmin_(a, b), fmin_(fmax_(a, b), T(0)));
}

// smallest normal number: a product or reciprocal below it is flushed by the approximate
// float instructions, so states below it are treated as vacuum
template <class T>
__device__ __forceinline__ T tiny_();
template <>
__device__ __forceinline__ float tiny_<float>() { return 1.17549435e-38f; }
template <>
__device__ __forceinline__ double tiny_<double>() { return 2.2250738585072014e-308; }
__device__ __forceinline__ double rsqrt_(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float rsqrt_(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// M1 flux of one group contracted with A, in branch-free form (Eq. eddington-group):
// (F . A, c^2 E [(1 - chi)/2 A + (3 chi - 1)/2 (n . A) n]), n = F/|F|, f = |F|/(cE) clipped
// to 1.  The factors are bounded for every state: (1 - chi)/2 = (1 + s - 2u)/(5 + 2s) and
// (3 chi - 1)/2 = 3u/(2 + s) with u = f^2, s = sqrt(4 - 3u), and the direction enters as
// F/|F|, so no (cE)^-2 can overflow.  cE not a normal number (E <= 0 included) gives zero
// pressure; F not normal gives the isotropic closure.
template <class T>
__device__ __forceinline__ void m1_dot_(T E, T Fx, T Fy, T Fz, T Ax, T Ay, T Az, T c, T& oE, T& oFx, T& oFy,
                                        T& oFz) {
    const T FA = Fx * Ax + Fy * Ay + Fz * Az;
    oE = FA;
    const T cE1 = c * E;
    const bool pos = cE1 > tiny_<T>();
    const T F2 = Fx * Fx + Fy * Fy + Fz * Fz;
    const bool dir = F2 > tiny_<T>();
    const T iFn = rsqrt_(dir ? F2 : T(1));
    const T icE = rcp_(pos ? cE1 : T(1));
    const T f = dir ? fmin_(F2 * iFn * icE, T(1)) : T(0);
    const T u = f * f;
    const T s = sqrt_(T(4) - T(3) * u);
    const T a_iso = (T(1) + s - T(2) * u) * rcp_(T(5) + T(2) * s);
    const T a_dir = T(3) * u * rcp_(T(2) + s);
    const T cE = pos ? c * cE1 : T(0);
    const T t = ((a_dir * FA) * iFn) * iFn;
    oFx = cE * (a_iso * Ax + t * Fx);
    oFy = cE * (a_iso * Ay + t * Fy);
    oFz = cE * (a_iso * Az + t * Fz);
}

// ------------------------------------------------------------------------------------
// positions
template <class T>
struct Pos;
template <>
struct Pos<float> {
    uint32_t a, b, c;
};
template <>
struct Pos<double> {
    double a, b, c;
};

__device__ __forceinline__ Pos<float> load_pos(const float*, const void* P, int64_t i) {
    uint4 v = reinterpret_cast<const uint4*>(P)[i];
    return {v.x, v.y, v.z};
}
__device__ __forceinline__ Pos<double> load_pos(const double*, const void* P, int64_t i) {
    const double2* p = reinterpret_cast<const double2*>(P) + 2 * i;
    double2 u = p[0], v = p[1];
    return {u.x, u.y, v.x};
}

struct SepParams {
    float s0, s1, s2;          // float path: fixed-point unit
    double b0, b1, b2;         // double path: box
    int periodic;
};

__device__ __forceinline__ double wrap_d(double v, double box, int periodic) {
    if (periodic) {
        double h = 0.5 * box;
        v = v > h ? v - box : (v < -h ? v + box : v);
    }
    return v;
}

// d = x_to - x_from
__device__ __forceinline__ void sep(const SepParams& s, const Pos<float>& f, const Pos<float>& t, float& dx, float& dy,
                                    float& dz) {
    dx = (float)(int32_t)(t.a - f.a) * s.s0;
    dy = (float)(int32_t)(t.b - f.b) * s.s1;
    dz = (float)(int32_t)(t.c - f.c) * s.s2;
}
__device__ __forceinline__ void sep(const SepParams& s, const Pos<double>& f, const Pos<double>& t, double& dx,
                                    double& dy, double& dz) {
    dx = wrap_d(t.a - f.a, s.b0, s.periodic);
    dy = wrap_d(t.b - f.b, s.b1, s.periodic);
    dz = wrap_d(t.c - f.c, s.b2, s.periodic);
}

// vector loads of K consecutive values (16-byte aligned)
template <int K>
__device__ __forceinline__ void vload(const float* __restrict__ p, float* o) {
    static_assert(K % 4 == 0, "K multiple of 4");
#pragma unroll
    for (int k = 0; k < K; k += 4) {
        float4 v = *reinterpret_cast<const float4*>(p + k);
        o[k] = v.x; o[k + 1] = v.y; o[k + 2] = v.z; o[k + 3] = v.w;
    }
}
template <int K>
__device__ __forceinline__ void vload(const double* __restrict__ p, double* o) {
    static_assert(K % 2 == 0, "K even");
#pragma unroll
    for (int k = 0; k < K; k += 2) {
        double2 v = *reinterpret_cast<const double2*>(p + k);
        o[k] = v.x; o[k + 1] = v.y;
    }
}
// 16-byte asynchronous global -> shared copy (cached in L1), and the wait for all of a
// thread's outstanding copies
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ------------------------------------------------------------------------------------
// TMA row gathers (cp.async.bulk.tensor, tile::gather4) completing on an mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// waits for phase `parity` of the barrier to complete; false once `budget` clock cycles
// have passed without completion.  Each try_wait may suspend the thread for up to 0.1 ms
// (woken early when the phase completes), so waiting warps issue almost no instructions.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long budget) {
    const unsigned long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(bar), "r"(parity), "r"(100000u)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > budget) return false;
    }
}
// four rows (r0..r3) of a 2-D row-major tensor, columns [col, col + box width), into
// consecutive rows at dst; the tensor map's box is one row high
__device__ __forceinline__ void tma_gather4(uint32_t dst, const void* tmap, int col, int r0, int r1, int r2, int r3,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(col), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(bar)
        : "memory");
}

template <int K>
__device__ __forceinline__ void vstore(float* p, const float* o) {
#pragma unroll
    for (int k = 0; k < K; k += 4) *reinterpret_cast<float4*>(p + k) = make_float4(o[k], o[k + 1], o[k + 2], o[k + 3]);
}
template <int K>
__device__ __forceinline__ void vstore(double* p, const double* o) {
#pragma unroll
    for (int k = 0; k < K; k += 2) *reinterpret_cast<double2*>(p + k) = make_double2(o[k], o[k + 1]);
}

template <class T>
struct PairArgs {
    const void* pos;          // uint4[N] or double[4N]
    const T* geo;             // [N][8] {1/H, h, Bp xx yy zz xy xz yz}
    const T* omega;           // [N]
    const int64_t* row_off;
    const int32_t* cols;
    SepParams sp;
    int64_t n;
    const T* grad;            // [N][12G]
    const int32_t* n_low;     // lower neighbours per row (rows ascending)
    const int64_t* up_off;    // first pair slot of each row
    const int32_t* low_slot;  // slot of each lower entry's pair
    const int2* ends;         // (k, l) of each pair slot
    int64_t n_pairs;
    int G;
    // packed flux-input rows [N][kRowRot + RW], RW = 12 + 16G logical words {pos (4), geo
    // (8), U (4G), grad U (12G)} after a prefix that repeats the last kRowRot of them; when
    // set, the gradient kernels write U, grad U and the static part there (instead of grad)
    // for the tensor-memory-accelerator flux pass
    T* frec;
    int RW;
    // individual time bins (bins mode only): sorted bin per particle and the min-step index
    const int8_t* bins;
    int s;
    const int32_t* order;     // the active set of this launch (particles or pair slots)
    int64_t count;
    const int8_t* nmin;       // min bin over each particle and its neighbours
    int tz;                   // interaction level of min-step s
};

// symmetric 3x3 (xx, yy, zz, xy, xz, yz) times vector
template <class T>
__device__ __forceinline__ void sym_mv(const T M[6], T x, T y, T z, T& ox, T& oy, T& oz) {
    ox = M[0] * x + M[3] * y + M[4] * z;
    oy = M[3] * x + M[1] * y + M[5] * z;
    oz = M[4] * x + M[5] * y + M[2] * z;
}

// Angle in [0, pi] of the vector (x, y), y >= 0.  Double: atan2.  Float: the arctangent of
// the smaller over the larger of |x| and y as a q(a^2), q of degree 7 fitted on [0, 1] by
// least squares (fit_atan.py; largest error 1.3e-7 rad in float arithmetic), folded into
// the octant and the half plane without branches; (0, 0) gives 0.  It replaces atan2 in the
// float path's HLL wave speeds, where atan2 cost a third of the pair pass on some states.
__device__ __forceinline__ double angle_0_pi(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float angle_0_pi(float y, float x) {
    const float ax = fabsf(x);
    const float mx = fmaxf(ax, y), mn = fminf(ax, y);
    const float a = mx > 0.f ? mn * rcp_(mx) : 0.f;
    const float t = a * a;
    float q = -0.00405450432f;
    q = fmaf(q, t, 0.021862727f);
    q = fmaf(q, t, -0.0559119885f);
    q = fmaf(q, t, 0.0964217215f);
    q = fmaf(q, t, -0.139086195f);
    q = fmaf(q, t, 0.199465636f);
    q = fmaf(q, t, -0.333298606f);
    q = fmaf(q, t, 0.999999336f);
    float r = a * q;
    r = y > ax ? 1.57079637f - r : r;
    return x < 0.f ? 3.14159274f - r : r;
}

// HLL wave speeds of one face state through A (Eq. riemann-HLL): the largest and smallest
// eigenvalue of the M1 flux Jacobian along n = A/|A|, bilinear in the (f, theta) table of
// rt_wave_table (interleaved (lmax, lmin) per node, units of c); f = |F|/(cE) clipped to 1,
// theta = atan2(|F x A|, F . A) (well conditioned at 0 and pi; 0 for F = 0).  A state with
// E <= 0 has no closure and gets the whole light cone [-c, c].
template <class T>
struct Pair2;
template <>
struct Pair2<float> {
    typedef float2 type;
};
template <>
struct Pair2<double> {
    typedef double2 type;
};

template <class T>
__device__ __forceinline__ void wave_speeds_(const T* __restrict__ tab, T E, T Fx, T Fy, T Fz, T Ax, T Ay, T Az,
                                             T c, T& lmax, T& lmin) {
    if (!(E > T(0))) {
        lmax = c;
        lmin = -c;
        return;
    }
    const T Fn = sqrt_(Fx * Fx + Fy * Fy + Fz * Fz);
    const T f = fmin_(Fn * rcp_(c * E), T(1));
    const T cx = Fy * Az - Fz * Ay, cy = Fz * Ax - Fx * Az, cz = Fx * Ay - Fy * Ax;
    const T th = angle_0_pi(sqrt_(cx * cx + cy * cy + cz * cz), Fx * Ax + Fy * Ay + Fz * Az);
    const T x = f * T(RT_WAVE_NF - 1), y = th / T(3.14159265358979323846) * T(RT_WAVE_NTH - 1);
    const int i = min((int)x, RT_WAVE_NF - 2), j = min((int)y, RT_WAVE_NTH - 2);
    const T t = x - T(i), s = y - T(j);
    typedef typename Pair2<T>::type V;
    const V* tv = reinterpret_cast<const V*>(tab);
    const V a = tv[i * RT_WAVE_NTH + j], b = tv[(i + 1) * RT_WAVE_NTH + j];
    const V d = tv[i * RT_WAVE_NTH + j + 1], e = tv[(i + 1) * RT_WAVE_NTH + j + 1];
    const T w00 = (T(1) - t) * (T(1) - s), w10 = t * (T(1) - s), w01 = (T(1) - t) * s, w11 = t * s;
    lmax = c * (w00 * a.x + w10 * b.x + w01 * d.x + w11 * e.x);
    lmin = c * (w00 * a.y + w10 * b.y + w01 * d.y + w11 * e.y);
}

// Flux of pair (k, l) for one group, k = this particle as the left state: face states
// (Eq. rt-riemann-problem with s = minmod(grad Q_k . d, grad Q_l . d)), M1 fluxes
// (Eq. eddington-group), GLF (Eq. riemann-GLF).  The face states use explicit fma so that
// the evaluation by l (with -d and the roles swapped) gives exactly -phi.
template <bool HLL, class T>
__device__ __forceinline__ void pair_flux(const T uk[4], const T ul[4], const T gk[12], const T gl[12], T dx, T dy,
                                          T dz, T wk, T wl, T Ax, T Ay, T Az, T diss, T c, const T* wave, T An,
                                          T phi[4]) {
    T L[4], R[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        T dqk = gk[3 * q] * dx + gk[3 * q + 1] * dy + gk[3 * q + 2] * dz;
        T dql = gl[3 * q] * dx + gl[3 * q + 1] * dy + gl[3 * q + 2] * dz;
        T s = minmod_(dqk, dql);
        L[q] = fma_rn(wk, s, uk[q]);
        R[q] = fma_rn(-wl, s, ul[q]);
    }
    T fL[4], fR[4];
    m1_dot_(L[0], L[1], L[2], L[3], Ax, Ay, Az, c, fL[0], fL[1], fL[2], fL[3]);
    m1_dot_(R[0], R[1], R[2], R[3], Ax, Ay, Az, c, fR[0], fR[1], fR[2], fR[3]);
    if constexpr (HLL) {
        // HLL (Eq. riemann-HLL): (l+ F_L.A - l- F_R.A + l+ l- |A| (U_R - U_L)) / (l+ - l-),
        // l+ = max(0, lmax_L, lmax_R), l- = min(0, lmin_L, lmin_R); central flux if l+ = l-
        T xL, nL, xR, nR;
        wave_speeds_(wave, L[0], L[1], L[2], L[3], Ax, Ay, Az, c, xL, nL);
        wave_speeds_(wave, R[0], R[1], R[2], R[3], Ax, Ay, Az, c, xR, nR);
        const T lp = fmax_(T(0), fmax_(xL, xR)), lm = fmin_(T(0), fmin_(nL, nR));
        const T den = lp - lm;
        if (den > T(0)) {
            const T jm = lp * lm * An;
            const T iden = T(1) / den;
#pragma unroll
            for (int q = 0; q < 4; ++q) phi[q] = (lp * fL[q] - lm * fR[q] + jm * (R[q] - L[q])) * iden;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) phi[q] = T(0.5) * (fL[q] + fR[q]);
        }
        return;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) phi[q] = T(0.5) * (fL[q] + fR[q]) - diss * (R[q] - L[q]);
}

// update parameters of the flux stage
template <class T>
struct FluxExtra {
    const T* wave;                  // HLL wave-speed table (interleaved); unused by the GLF kernels
    const T* alpha;                 // sorted, or null
    const T* alpha_g;               // sorted per-group absorption [N][G], or null
    T* acc;                         // bins mode: per-particle flux accumulators [N][4G]
    // the next sub-cycle's injection dt sum coef L per (particle, group) [N][G] (zero off the
    // targets), added to E after the update; null when the next sub-cycle injects itself
    const double* inj;
    const double* dt_dev;
    T c;
    int clamp;
    unsigned long long* clamp_count;
};

template <class T>
inline PairArgs<T> pair_args(rt_ctx* c) {
    PairArgs<T> a;
    a.pos = c->pos_t.p;
    a.geo = c->geo_t.as<T>();
    a.omega = c->omega_t.as<T>();
    a.row_off = c->row_off.as<int64_t>();
    a.cols = c->cols.as<int32_t>();
    double units = c->cfg.periodic ? 4294967296.0 : 2147483648.0;
    a.sp.s0 = (float)(c->cfg.box[0] / units);
    a.sp.s1 = (float)(c->cfg.box[1] / units);
    a.sp.s2 = (float)(c->cfg.box[2] / units);
    a.sp.b0 = c->cfg.box[0];
    a.sp.b1 = c->cfg.box[1];
    a.sp.b2 = c->cfg.box[2];
    a.sp.periodic = c->cfg.periodic;
    a.n = c->n;
    a.grad = c->grad_t.as<T>();
    a.n_low = c->n_low.as<int32_t>();
    a.up_off = c->up_off.as<int64_t>();
    a.low_slot = c->low_slot.as<int32_t>();
    a.ends = c->pair_ends.as<int2>();
    a.n_pairs = c->n_directed / 2;
    a.G = c->cfg.n_groups;
    a.frec = nullptr;
    a.RW = 12 + 16 * a.G;
    a.bins = nullptr;
    a.s = 0;
    a.order = nullptr;
    a.count = 0;
    a.nmin = nullptr;
    a.tz = 0;
    return a;
}

}  // namespace rt
