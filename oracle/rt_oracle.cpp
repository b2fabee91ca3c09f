// Plain FP64 CPU oracle for the FVPM photon-transport step of GEAR-RT
// (Ivkovic 2023, arXiv 2302.12727, Part III chapter "One RT Time Step").
//
// TEST INFRASTRUCTURE ONLY.  This file is the correctness reference for the CUDA
// library.  Only the test-suite, the smoke check and the CPU-baseline leg of the
// benchmark may build, load or call it; the library itself never does.  It shares
// no code, header, table or helper with the CUDA sources.
//
// It is deliberately slow and literal: every quantity is computed in double precision
// (compile with -ffp-contract=off), in the order the thesis writes it, with plain
// loops over particles and neighbours.
//
//   cubic-spline kernel W                 Eq. cubic-spline-kernel (Part II, "Partition Of Unity")
//   omega, psi                            Eqs. omega, psi
//   particle volume V = 1/omega           Eq. particle-volume
//   smoothing length h = eta omega^-1/3   Sec. "The Neighbor Search", Eq. number-of-neighbors
//   psi-tilde, E_i, B_i = E_i^-1          Eqs. gradient, psitilde, matrix_B, matrix_E
//   effective surfaces A_ij (Hopkins)     Eq. HopkinsAij
//   interface x_kl, extrapolation         Sec. "Second Step: Transport", Eq. rt-riemann-problem
//   minmod limiter                        Eq. rt-minmod
//   M1 closure, Eddington tensor          Eqs. eddington-group (pressure-tensor-group-*)
//   GLF Riemann flux                      Eq. riemann-GLF
//   HLL Riemann flux, wave speeds         Eq. riemann-HLL (eigenvalue table supplied by the caller,
//                                         built in m1_eigen.py from the M1 flux Jacobian)
//   explicit update                       Eq. transport-update-explicit
//   injection weights xi, octant mu_a     Sec. "Weights For Distribution Of Energy Density",
//                                         Eq. isotropy-correction-with-zero
//   photon removal (grey)                 Sec. "Third step: Thermochemistry" (forward Euler)
//   photon removal per group              Eqs. dEdt-group, dFdt-group (alpha_g = sum_j n_j sigma^N_gj)
//   operator order inject->transport->sink  Sec. "One RT Time Step: Outline"
//   drift correction U + grad U . dx      Sec. "Dealing With Particle Drifts"
//   individual time bins, min(dt_k, dt_l)  Sec. "Individual Timstepping", Eq. transport-update-explicit
//   factor-4 time-step limiter             Sec. "Dynamic Sub-Cycling"
//
// Readings where the thesis is silent or inconsistent:
//   * update sign: U_k(t+dt) = U_k - dt/V_k sum_l F_kl . A_kl (the RT chapter's form; the
//     "+" of the hydro chapter's explicit update contradicts d(UV)/dt + sum F.A = 0).
//   * minmod: s = minmod(grad Q_k . d, grad Q_l . d) with d = x_l - x_k, and both states use s:
//     Q_L = Q_k + s h_k/(h_k+h_l), Q_R = Q_l - s h_l/(h_k+h_l).  Equal magnitudes pick dQ_l.
//   * GLF in 3D: Phi_kl = 1/2 (F(U_L) + F(U_R)) . A_kl - c/2 (U_R - U_L) |A_kl|.
//   * H = 1.825742 h for the 3D cubic spline (Dehnen & Aly 2012, Table 1, cited by the thesis).
//   * W at q = 0 uses the first branch; W = 0 for q >= 1; pair test r^2 < H^2 (strict).
//   * psi_j(x_i) uses h_i; omega_i includes the self term W(0, h_i).
//   * pair set P_i = { j != i : r_ij < max(H_i, H_j) } (A_ij is non-zero if either support covers).
//   * h solve: bisection of f(h) = h - eta * omega(h)^(-1/3) to a relative bracket of h_tol.
//   * source h_s: the same equation over gas particles only (no self term).
//   * octants: sign pattern of x_g - x_s (minimal image); a zero component counts as ">= 0".
//   * injection: Delta E_g = xi_sg L_s dt / V_g (energy -> energy density), no flux injected.
//   * M1: f^2 is clamped to <= 1 inside chi; F = 0 gives D = I/3; E <= 0 gives zero pressure.
//   * grey sink: U <- U * max(0, 1 - c alpha_i dt), alpha_i supplied per particle.
//   * optional negative-energy fix-up: E <- max(E, 0) after the sink (counted).
//   * HLL: l+ = max(0, lmax_L, lmax_R), l- = min(0, lmin_L, lmin_R) over both face states;
//     speeds from the (f, theta) table by bilinear interpolation, theta = atan2(|F x A|, F . A)
//     (0 for F = 0); E <= 0 gives [-c, c]; l+ = l- = 0 gives the central flux.
//
// Parity unpinned (no closed form or paper value reaches them beyond this code itself):
//   the exact value of h where neighbour sets are irregular, B_i of ill-conditioned
//   neighbourhoods, and the long-time state of the unstable configurations.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>

#include <atomic>
#endif

namespace orc {

constexpr double kPi = 3.14159265358979323846;
constexpr double kHoverh = 1.825742;        // H/h, cubic spline, 3D
constexpr double kSigma3 = 16.0 / kPi;      // normalisation in 3D

enum Status { OK = 0, ERR_INVALID = 1, ERR_NOCONV = 4, ERR_GEOMETRY = 5 };

struct Config {
    int32_t n_groups;
    double c_red;
    double eta_res;
    double eta_res_star;
    double box[3];
    int32_t periodic;
    int32_t clamp_negative;
    double h_tol;
    int32_t h_max_iter;
    int32_t brute_force;      // 1: O(N^2) neighbour search, 0: cell list
    int32_t riemann;          // 0: GLF (Eq. riemann-GLF), 1: HLL (Eq. riemann-HLL)
};

// ---------------------------------------------------------------------------------------
// Scalar types: double, and a forward-mode dual number for exact directional derivatives.
struct Dual {
    double v, d;
    Dual() : v(0), d(0) {}
    Dual(double a) : v(a), d(0) {}
    Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
    double q = a.v / b.v;
    return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline Dual sqrt(Dual a) {
    double s = std::sqrt(a.v);
    return Dual(s, s > 0 ? a.d / (2.0 * s) : 0.0);
}
// Kinks of the piecewise-smooth step near a forward-mode evaluation: with g_kink_eps > 0, the
// JVP counts every branch point of the limiter and the closure that a change of the inputs by
// g_kink_eps times the direction could cross (to first order), i.e. where a central
// difference of that step size straddles a kink and so cannot equal the derivative.
static double g_kink_eps = 0.0;
static std::atomic<long> g_kinks{0};
inline void kink_if(double dist, double rate) {
    if (g_kink_eps > 0.0 && std::fabs(dist) <= g_kink_eps * std::fabs(rate)) g_kinks.fetch_add(1);
}

inline double val(double a) { return a; }
inline double val(Dual a) { return a.v; }
inline double sqrt_(double a) { return std::sqrt(a); }
inline Dual sqrt_(Dual a) { return sqrt(a); }

// A double that counts the floating-point operations done on it (add, subtract, multiply,
// divide, square root: one each; comparisons and conversions are not counted).  The pair
// arithmetic instantiated on it measures the work of one pair evaluation (orc_pair_flops).
static long g_flops = 0;
struct Counted {
    double v;
    Counted() : v(0) {}
    Counted(double a) : v(a) {}
};
inline Counted operator+(Counted a, Counted b) { ++g_flops; return Counted(a.v + b.v); }
inline Counted operator-(Counted a, Counted b) { ++g_flops; return Counted(a.v - b.v); }
inline Counted operator-(Counted a) { return Counted(-a.v); }
inline Counted operator*(Counted a, Counted b) { ++g_flops; return Counted(a.v * b.v); }
inline Counted operator/(Counted a, Counted b) { ++g_flops; return Counted(a.v / b.v); }
inline Counted& operator+=(Counted& a, Counted b) { a = a + b; return a; }
inline Counted& operator-=(Counted& a, Counted b) { a = a - b; return a; }
inline Counted& operator*=(Counted& a, Counted b) { a = a * b; return a; }
inline double val(Counted a) { return a.v; }
inline Counted sqrt_(Counted a) { ++g_flops; return Counted(std::sqrt(a.v)); }

// ---------------------------------------------------------------------------------------
// Cubic spline kernel, Eq. cubic-spline-kernel, nu = 3.  H = kHoverh * h.
// (S: the scalar of the distance and the result; H and sigma / H^3 are per-particle constants)
template <class S>
S kernel_W_t(S r, double h) {
    const double H = kHoverh * h;
    const S q = r / S(H);
    S w;
    if (val(q) <= 0.5) {
        w = (S(1.0) - q) * (S(1.0) - q) * (S(1.0) - q) - S(4.0) * (S(0.5) - q) * (S(0.5) - q) * (S(0.5) - q);
    } else if (val(q) < 1.0) {
        w = (S(1.0) - q) * (S(1.0) - q) * (S(1.0) - q);
    } else {
        w = S(0.0);
    }
    return S(kSigma3 / (H * H * H)) * w;
}
double kernel_W(double r, double h) { return kernel_W_t<double>(r, h); }

// ---------------------------------------------------------------------------------------
struct Particles {
    long n = 0;
    double box[3] = {1, 1, 1};
    bool periodic = true;
    std::vector<double> x;   // 3N SoA

    double coord(long i, int a) const { return x[a * n + i]; }
    // minimal-image separation x_j - x_i
    void sep(long i, long j, double d[3]) const {
        for (int a = 0; a < 3; ++a) {
            double v = coord(j, a) - coord(i, a);
            if (periodic) v -= box[a] * std::nearbyint(v / box[a]);
            d[a] = v;
        }
    }
};

// separation from an arbitrary point p to particle j: x_j - p
static void sep_point(const Particles& P, const double p[3], long j, double d[3]) {
    for (int a = 0; a < 3; ++a) {
        double v = P.coord(j, a) - p[a];
        if (P.periodic) v -= P.box[a] * std::nearbyint(v / P.box[a]);
        d[a] = v;
    }
}

template <class S>
static S norm2(const S d[3]) { return d[0] * d[0] + d[1] * d[1] + d[2] * d[2]; }

// Simple uniform cell list used only to find candidates; every candidate is then tested
// with the exact distance.  brute_force bypasses it.
struct CellList {
    int nc[3] = {1, 1, 1};
    double cell[3] = {1, 1, 1};
    std::vector<std::vector<long>> cells;
    const Particles* P = nullptr;
    bool brute = false;

    void build(const Particles& parts, double cell_size, bool brute_force) {
        P = &parts;
        brute = brute_force;
        if (brute) return;
        for (int a = 0; a < 3; ++a) {
            nc[a] = std::max(1, (int)std::floor(parts.box[a] / cell_size));
            nc[a] = std::min(nc[a], 256);
            cell[a] = parts.box[a] / nc[a];
        }
        cells.assign((size_t)nc[0] * nc[1] * nc[2], {});
        for (long i = 0; i < parts.n; ++i) {
            int c[3];
            for (int a = 0; a < 3; ++a) {
                double u = parts.coord(i, a) / cell[a];
                int ci = (int)std::floor(u);
                if (parts.periodic) ci = ((ci % nc[a]) + nc[a]) % nc[a];
                else ci = std::min(std::max(ci, 0), nc[a] - 1);
                c[a] = ci;
            }
            cells[((size_t)c[2] * nc[1] + c[1]) * nc[0] + c[0]].push_back(i);
        }
    }

    // all particle indices within the cells that can hold points closer than R to p
    void candidates(const double p[3], double R, std::vector<long>& out) const {
        out.clear();
        if (brute) {
            for (long j = 0; j < P->n; ++j) out.push_back(j);
            return;
        }
        int lo[3], hi[3];
        bool all[3];
        int c0[3];
        for (int a = 0; a < 3; ++a) {
            int k = (int)std::ceil(R / cell[a]);
            c0[a] = (int)std::floor(p[a] / cell[a]);
            all[a] = (2 * k + 1 >= nc[a]);
            lo[a] = all[a] ? 0 : c0[a] - k;
            hi[a] = all[a] ? nc[a] - 1 : c0[a] + k;
            if (!P->periodic && !all[a]) {
                lo[a] = std::max(lo[a], 0);
                hi[a] = std::min(hi[a], nc[a] - 1);
            }
        }
        for (int cz = lo[2]; cz <= hi[2]; ++cz)
            for (int cy = lo[1]; cy <= hi[1]; ++cy)
                for (int cx = lo[0]; cx <= hi[0]; ++cx) {
                    int w[3] = {cx, cy, cz};
                    for (int a = 0; a < 3; ++a) w[a] = ((w[a] % nc[a]) + nc[a]) % nc[a];
                    const auto& v = cells[((size_t)w[2] * nc[1] + w[1]) * nc[0] + w[0]];
                    out.insert(out.end(), v.begin(), v.end());
                }
    }
};

// ---------------------------------------------------------------------------------------
// Smoothing length: solve h = eta * omega(h)^(-1/3) by bisection.
// omega(h) = sum_j W(|p - x_j|, h) over the candidate particles (self included when p is a
// particle position, since |p - x_i| = 0 is then one of the candidates).
struct HSolve {
    double h = 0, omega = 0;
    int status = OK;
};

static HSolve solve_h(const Particles& P, const CellList& cl, const double p[3], double eta,
                      double h_start, double h_tol, int max_iter, double h_max) {
    HSolve res;
    std::vector<long> cand;
    std::vector<double> r2;
    double R_have = -1.0;
    auto ensure = [&](double h) {
        double R = kHoverh * h;
        if (R <= R_have) return;
        double Rq = R * 1.25;
        cl.candidates(p, Rq, cand);
        r2.clear();
        for (long j : cand) {
            double d[3];
            sep_point(P, p, j, d);
            double q = norm2(d);
            if (q < Rq * Rq) r2.push_back(q);
        }
        R_have = Rq;
    };
    auto omega_of = [&](double h) {
        ensure(h);
        double w = 0.0;
        for (double q : r2) w += kernel_W(std::sqrt(q), h);
        return w;
    };
    auto f = [&](double h, double& om) -> double {
        om = omega_of(h);
        if (om <= 0.0) return -INFINITY;
        return h - eta / std::cbrt(om);
    };
    double om;
    double h_hi = h_start;
    int it = 0;
    while (f(h_hi, om) <= 0.0) {
        if (h_hi >= h_max || ++it > 200) { res.status = ERR_NOCONV; return res; }
        h_hi = std::min(1.25 * h_hi, h_max);
    }
    double h_lo = h_hi;
    it = 0;
    while (f(h_lo, om) > 0.0) {
        h_lo *= 0.5;
        if (++it > 200) { res.status = ERR_NOCONV; return res; }
    }
    for (int k = 0; k < max_iter && (h_hi - h_lo) > h_tol * h_hi; ++k) {
        double hm = 0.5 * (h_lo + h_hi);
        if (f(hm, om) > 0.0) h_hi = hm; else h_lo = hm;
    }
    res.h = 0.5 * (h_lo + h_hi);
    res.omega = omega_of(res.h);
    return res;
}

// omega(h) = sum_j W(|x_j - p|, h) over the particles around p (Eq. omega; p a particle's own
// position includes its self term), for a given h
static double omega_given(const Particles& P, const CellList& cl, const double p[3], double h) {
    std::vector<long> cand;
    const double R = kHoverh * h;
    cl.candidates(p, R * 1.25, cand);
    double w = 0.0;
    for (long j : cand) {
        double d[3];
        sep_point(P, p, j, d);
        double q = norm2(d);
        if (q < R * R * 1.5625) w += kernel_W(std::sqrt(q), h);
    }
    return w;
}

// ---------------------------------------------------------------------------------------
// Symmetric 3x3 helpers
static double det3(const double E[9]) {
    return E[0] * (E[4] * E[8] - E[5] * E[7]) - E[1] * (E[3] * E[8] - E[5] * E[6]) +
           E[2] * (E[3] * E[7] - E[4] * E[6]);
}

// inverse by cofactors (adjugate / determinant)
static void inv3(const double E[9], double det, double B[9]) {
    B[0] = (E[4] * E[8] - E[5] * E[7]) / det;
    B[1] = (E[2] * E[7] - E[1] * E[8]) / det;
    B[2] = (E[1] * E[5] - E[2] * E[4]) / det;
    B[3] = (E[5] * E[6] - E[3] * E[8]) / det;
    B[4] = (E[0] * E[8] - E[2] * E[6]) / det;
    B[5] = (E[2] * E[3] - E[0] * E[5]) / det;
    B[6] = (E[3] * E[7] - E[4] * E[6]) / det;
    B[7] = (E[1] * E[6] - E[0] * E[7]) / det;
    B[8] = (E[0] * E[4] - E[1] * E[3]) / det;
}

// eigenvalues of a symmetric 3x3 matrix by cyclic Jacobi rotations
static void sym_eig3(const double E[9], double ev[3]) {
    double a[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) a[r][c] = E[3 * r + c];
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        if (off < 1e-300) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (a[p][q] == 0.0) continue;
                double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; ++k) {  // A <- A J
                    double akp = a[k][p], akq = a[k][q];
                    a[k][p] = c * akp - s * akq;
                    a[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {  // A <- J^T A
                    double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = c * apk - s * aqk;
                    a[q][k] = s * apk + c * aqk;
                }
            }
    }
    ev[0] = a[0][0]; ev[1] = a[1][1]; ev[2] = a[2][2];
}

// ---------------------------------------------------------------------------------------
struct Target { long g; double xi; };

struct Model {
    Config cfg{};
    Particles P;
    std::vector<double> m;
    std::vector<double> h, omega, V;
    std::vector<double> B;        // 9 per particle, row-major
    std::vector<double> cond;
    std::vector<std::vector<long>> nbr;   // symmetric pair sets, ascending
    long n_src = 0;
    std::vector<double> xsrc;     // 3S SoA
    std::vector<double> hs, omegas;
    std::vector<std::vector<Target>> inj;   // per source: gas targets and their xi
    std::vector<double> octw;     // 8 per source (w_a)
    long n_ill = 0;
    double cond_max = 0;
    // HLL wave-speed table over (f, theta) (units of c), given by the caller
    int wnf = 0, wnth = 0;
    std::vector<double> wmax, wmin;

    double H(long i) const { return kHoverh * h[i]; }
    // smoothing lengths given by the caller instead of solved (a rank of a domain
    // decomposition takes them from the particles' owners); empty: solve
    std::vector<double> h_given, hs_given;
    // the sources' omega_s and octant sums w_a given by the caller (a rank of a domain
    // decomposition takes them from the sources' owners, whose gas neighbourhoods are
    // complete); empty: formed from the model's own gas
    std::vector<double> omegas_given, octw_given;
};

// psi_j(x_i) = W(|x_i - x_j|, h_i) / omega_i     (Eq. psi with h evaluated at x_i)
template <class S>
static S psi_at(const Model& M, long i, S r) { return kernel_W_t<S>(r, M.h[i]) / S(M.omega[i]); }

// psitilde_j(x_i) = B_i (x_j - x_i) psi_j(x_i)     (Eq. psitilde)
template <class S>
static void psitilde(const Model& M, long i, const S d[3], S r, S out[3]) {
    S ps = psi_at<S>(M, i, r);
    const double* Bi = &M.B[9 * i];
    for (int a = 0; a < 3; ++a)
        out[a] = (S(Bi[3 * a]) * d[0] + S(Bi[3 * a + 1]) * d[1] + S(Bi[3 * a + 2]) * d[2]) * ps;
}

// A_ij = V_i psitilde_j(x_i) - V_j psitilde_i(x_j)     (Eq. HopkinsAij), d = x_j - x_i
template <class S>
static void surface(const Model& M, long i, long j, const S d[3], S A[3]) {
    S r = sqrt_(norm2(d));
    S mdv[3] = {-d[0], -d[1], -d[2]};
    S pi_[3], pj_[3];
    psitilde<S>(M, i, d, r, pi_);    // psitilde_j(x_i)
    psitilde<S>(M, j, mdv, r, pj_);  // psitilde_i(x_j)
    for (int a = 0; a < 3; ++a) A[a] = S(M.V[i]) * pi_[a] - S(M.V[j]) * pj_[a];
}

static int build(Model& M) {
    const long n = M.P.n;
    const Config& c = M.cfg;
    double vol = M.P.box[0] * M.P.box[1] * M.P.box[2];
    double h0 = c.eta_res * std::cbrt(vol / (double)n);
    double half_box = 0.5 * std::min(M.P.box[0], std::min(M.P.box[1], M.P.box[2]));
    double h_cap = M.P.periodic ? half_box / kHoverh : 1e300;

    CellList cl;
    cl.build(M.P, kHoverh * h0, c.brute_force != 0);

    M.h.assign(n, 0.0);
    M.omega.assign(n, 0.0);
    int bad = OK;
#pragma omp parallel for schedule(dynamic, 64)
    for (long i = 0; i < n; ++i) {
        double p[3] = {M.P.coord(i, 0), M.P.coord(i, 1), M.P.coord(i, 2)};
        if (!M.h_given.empty()) {
            M.h[i] = M.h_given[i];
            M.omega[i] = omega_given(M.P, cl, p, M.h[i]);
            if (!(M.h[i] > 0.0)) {
#pragma omp critical
                bad = ERR_INVALID;
            }
            continue;
        }
        HSolve s = solve_h(M.P, cl, p, c.eta_res, h0, c.h_tol, c.h_max_iter, h_cap);
        if (s.status != OK) {
#pragma omp critical
            bad = s.status;
        }
        M.h[i] = s.h;
        M.omega[i] = s.omega;
    }
    if (bad != OK) return bad;
    M.V.resize(n);
    double Hmax = 0;
    for (long i = 0; i < n; ++i) {
        M.V[i] = 1.0 / M.omega[i];
        Hmax = std::max(Hmax, M.H(i));
    }
    if (M.P.periodic && Hmax >= half_box) return ERR_GEOMETRY;

    // symmetric pair sets: r_ij < max(H_i, H_j)
    M.nbr.assign(n, {});
#pragma omp parallel for schedule(dynamic, 64)
    for (long i = 0; i < n; ++i) {
        std::vector<long> cand;
        double p[3] = {M.P.coord(i, 0), M.P.coord(i, 1), M.P.coord(i, 2)};
        cl.candidates(p, std::max(M.H(i), Hmax), cand);
        std::vector<long> out;
        for (long j : cand) {
            if (j == i) continue;
            double d[3];
            M.P.sep(i, j, d);
            double r2 = norm2(d);
            double Hm = std::max(M.H(i), M.H(j));
            if (r2 < Hm * Hm) out.push_back(j);
        }
        std::sort(out.begin(), out.end());
        out.erase(std::unique(out.begin(), out.end()), out.end());
        M.nbr[i] = out;
    }

    // E_i = sum_j (x_j - x_i)(x_j - x_i)^T psi_j(x_i);  B_i = E_i^-1     (Eqs. matrix_E, matrix_B)
    M.B.assign(9 * n, 0.0);
    M.cond.assign(n, 0.0);
    for (long i = 0; i < n; ++i) {
        double E[9] = {0};
        for (long j : M.nbr[i]) {
            double d[3];
            M.P.sep(i, j, d);
            double ps = psi_at(M, i, std::sqrt(norm2(d)));
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) E[3 * a + b] += d[a] * d[b] * ps;
        }
        double det = det3(E);
        if (!(det > 0.0)) return ERR_GEOMETRY;
        inv3(E, det, &M.B[9 * i]);
        double ev[3];
        sym_eig3(E, ev);
        double lmin = std::min(ev[0], std::min(ev[1], ev[2]));
        double lmax = std::max(ev[0], std::max(ev[1], ev[2]));
        if (!(lmin > 0.0)) return ERR_GEOMETRY;
        M.cond[i] = lmax / lmin;
        if (M.cond[i] > 1e10) M.n_ill++;
        M.cond_max = std::max(M.cond_max, M.cond[i]);
    }

    // sources: h_s over gas only, octant weights, xi     (Sec. injection weights)
    M.hs.assign(M.n_src, 0.0);
    M.omegas.assign(M.n_src, 0.0);
    M.inj.assign(M.n_src, {});
    M.octw.assign(8 * M.n_src, 0.0);
    for (long s = 0; s < M.n_src; ++s) {
        double p[3] = {M.xsrc[s], M.xsrc[M.n_src + s], M.xsrc[2 * M.n_src + s]};
        HSolve hsol;
        if (!M.hs_given.empty()) {
            hsol.h = M.hs_given[s];
            hsol.omega = M.omegas_given.empty() ? omega_given(M.P, cl, p, hsol.h) : M.omegas_given[s];
            if (!(hsol.h > 0.0) || !(hsol.omega > 0.0)) return ERR_INVALID;
        } else {
            hsol = solve_h(M.P, cl, p, c.eta_res_star, h0, c.h_tol, c.h_max_iter, h_cap);
        }
        if (hsol.status != OK) return hsol.status;
        M.hs[s] = hsol.h;
        M.omegas[s] = hsol.omega;
        double Hs = kHoverh * hsol.h;
        std::vector<long> cand;
        cl.candidates(p, Hs, cand);
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        std::vector<long> gs;
        std::vector<double> psis;
        std::vector<int> oct;
        double w[8] = {0};
        for (long g : cand) {
            double d[3];
            sep_point(M.P, p, g, d);   // x_g - x_s
            double r2 = norm2(d);
            if (!(r2 < Hs * Hs)) continue;
            double ps = kernel_W(std::sqrt(r2), hsol.h) / hsol.omega;
            int a = (d[0] < 0 ? 1 : 0) | (d[1] < 0 ? 2 : 0) | (d[2] < 0 ? 4 : 0);
            gs.push_back(g);
            psis.push_back(ps);
            oct.push_back(a);
            w[a] += ps;
        }
        if (!M.octw_given.empty())
            for (int a = 0; a < 8; ++a) w[a] = M.octw_given[8 * s + a];
        double wsum = 0;
        int qnz = 0;
        for (int a = 0; a < 8; ++a) {
            wsum += w[a];
            if (w[a] > 0) qnz++;
            M.octw[8 * s + a] = w[a];
        }
        for (size_t k = 0; k < gs.size(); ++k) {
            double mu = wsum / (qnz * w[oct[k]]);   // Eq. isotropy-correction-with-zero
            M.inj[s].push_back({gs[k], mu * psis[k]});
        }
    }
    return OK;
}

// ---------------------------------------------------------------------------------------
// Transport pieces, templated on the scalar of the radiation state.

// gradient of every component, Eq. gradient:  grad Q_i = sum_j (Q_j - Q_i) psitilde_j(x_i)
// U: [C][N] (C = 4G components), grad: [C][3][N]
template <class T>
static void gradients(const Model& M, const std::vector<T>& U, std::vector<T>& grad) {
    const long n = M.P.n;
    const int C = 4 * M.cfg.n_groups;
    grad.assign((size_t)C * 3 * n, T(0.0));
#pragma omp parallel for schedule(dynamic, 64)
    for (long i = 0; i < n; ++i) {
        for (long j : M.nbr[i]) {
            double d[3];
            M.P.sep(i, j, d);
            double pt[3];
            psitilde(M, i, d, std::sqrt(norm2(d)), pt);
            for (int cc = 0; cc < C; ++cc) {
                T dq = U[(size_t)cc * n + j] - U[(size_t)cc * n + i];
                for (int a = 0; a < 3; ++a) grad[((size_t)cc * 3 + a) * n + i] += dq * pt[a];
            }
        }
    }
}

// minmod, Eq. rt-minmod
template <class T>
static T minmod(T a, T b) {
    if constexpr (std::is_same<T, Dual>::value) {
        // branch points: either slope changing sign, or their magnitudes changing order
        kink_if(a.v, a.d);
        kink_if(b.v, b.d);
        if (a.v * b.v > 0.0) {
            const double sa = a.v > 0.0 ? 1.0 : -1.0, sb = b.v > 0.0 ? 1.0 : -1.0;
            kink_if(std::fabs(a.v) - std::fabs(b.v), sa * a.d - sb * b.d);
        }
    }
    if (val(a) * val(b) <= 0.0) return T(0.0);
    if (std::fabs(val(a)) < std::fabs(val(b))) return a;
    return b;
}

// M1 flux of one group's state contracted with A:  (F . A,  c^2 D E A)
// D = (1-chi)/2 I + (3chi-1)/2 n n,  n = F/|F|,  chi = (3+4f^2)/(5+2 sqrt(4-3f^2)), f = |F|/(cE)
template <class T>
static void m1_flux_dot(const T u[4], const double A[3], double c, T out[4]) {
    const T& E = u[0];
    out[0] = u[1] * A[0] + u[2] * A[1] + u[3] * A[2];
    if (!(val(E) > 0.0)) {
        out[1] = out[2] = out[3] = T(0.0);
        return;
    }
    T F2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
    if (val(F2) == 0.0) {
        for (int a = 0; a < 3; ++a) out[1 + a] = T(c * c / 3.0) * E * T(A[a]);
        return;
    }
    T Fn = sqrt_(F2);
    T f = Fn / (T(c) * E);
    if constexpr (std::is_same<T, Dual>::value) {
        kink_if(E.v, E.d);            // zero pressure below E = 0
        kink_if(f.v - 1.0, f.d);      // reduced flux clipped to 1
    }
    if (val(f) > 1.0) f = T(1.0);
    T f2 = f * f;
    T chi = (T(3.0) + T(4.0) * f2) / (T(5.0) + T(2.0) * sqrt_(T(4.0) - T(3.0) * f2));
    T n[3] = {u[1] / Fn, u[2] / Fn, u[3] / Fn};
    T nA = n[0] * A[0] + n[1] * A[1] + n[2] * A[2];
    T a_iso = (T(1.0) - chi) / T(2.0);
    T a_dir = (T(3.0) * chi - T(1.0)) / T(2.0);
    for (int a = 0; a < 3; ++a) out[1 + a] = T(c * c) * E * (a_iso * T(A[a]) + a_dir * nA * n[a]);
}

// Left/right states at the interface x_kl = x_k + h_k/(h_k+h_l) (x_l - x_k) for one group
// (Eq. rt-riemann-problem), each component limited with s = minmod(grad Q_k . d, grad Q_l . d).
template <class T>
static void face_states(const T uk[4], const T ul[4], const T gk[4][3], const T gl[4][3], const double d[3],
                        double hk, double hl, T uL[4], T uR[4]) {
    const T hs = T(hk) + T(hl);
    const T wk = T(hk) / hs;
    const T wl = T(hl) / hs;
    for (int q = 0; q < 4; ++q) {
        T dQk = T(0.0), dQl = T(0.0);
        for (int a = 0; a < 3; ++a) {
            dQk += gk[q][a] * T(d[a]);
            dQl += gl[q][a] * T(d[a]);
        }
        T s = minmod(dQk, dQl);
        uL[q] = uk[q] + wk * s;
        uR[q] = ul[q] - wl * s;
    }
}

// GLF flux through A, Eq. riemann-GLF:  1/2 (F(U_L) + F(U_R)) . A - c/2 (U_R - U_L) |A|
template <class T>
static void glf_flux(const T uL[4], const T uR[4], const double A[3], double c, T phi[4]) {
    double Anorm = std::sqrt(norm2(A));
    T fL[4], fR[4];
    m1_flux_dot(uL, A, c, fL);
    m1_flux_dot(uR, A, c, fR);
    for (int q = 0; q < 4; ++q) phi[q] = T(0.5) * (fL[q] + fR[q]) - T(0.5 * c * Anorm) * (uR[q] - uL[q]);
}

// HLL wave speeds of one face state through A (Eq. riemann-HLL): the largest and smallest
// eigenvalue of the M1 flux Jacobian along n = A/|A|, looked up in the (f, theta) table
// with bilinear interpolation; f = |F|/(cE) clipped to 1, theta the angle between F and A,
// taken as atan2(|F x A|, F . A) (well conditioned at theta = 0 and pi, where acos of the
// normalised dot product is not).  A state with E <= 0 has no closure; it gets the whole
// light cone [-c, c].
// The speeds are taken at the state's values (not differentiated).
static void wave_speeds(const Model& M, const double u[4], const double A[3], double c, double& lmax,
                        double& lmin) {
    if (!(u[0] > 0.0)) {
        lmax = c;
        lmin = -c;
        return;
    }
    double Fn = std::sqrt(u[1] * u[1] + u[2] * u[2] + u[3] * u[3]);
    double f = std::min(Fn / (c * u[0]), 1.0);
    double cx = u[2] * A[2] - u[3] * A[1], cy = u[3] * A[0] - u[1] * A[2], cz = u[1] * A[1] - u[2] * A[0];
    double theta = std::atan2(std::sqrt(cx * cx + cy * cy + cz * cz), u[1] * A[0] + u[2] * A[1] + u[3] * A[2]);
    double x = f * (M.wnf - 1), y = theta / M_PI * (M.wnth - 1);
    int i = std::min((int)x, M.wnf - 2), j = std::min((int)y, M.wnth - 2);
    double t = x - i, s = y - j;
    auto at = [&](const std::vector<double>& T, int a, int b) { return T[(size_t)a * M.wnth + b]; };
    auto lerp2 = [&](const std::vector<double>& T) {
        return (1 - t) * (1 - s) * at(T, i, j) + t * (1 - s) * at(T, i + 1, j) + (1 - t) * s * at(T, i, j + 1) +
               t * s * at(T, i + 1, j + 1);
    };
    lmax = c * lerp2(M.wmax);
    lmin = c * lerp2(M.wmin);
}

// HLL flux through A, Eq. riemann-HLL, with the M1 flux contracted with A in place of F and
// |A| on the jump term:  (l+ F_L.A - l- F_R.A + l+ l- |A| (U_R - U_L)) / (l+ - l-),
// l+ = max(0, lmax_L, lmax_R), l- = min(0, lmin_L, lmin_R).  With l+ = l- = 0 (both states
// free-streaming exactly along the surface) the central flux 1/2 (F_L + F_R).A is taken.
template <class T>
static void hll_flux(const Model& M, const T uL[4], const T uR[4], const double A[3], double c, T phi[4]) {
    T fL[4], fR[4];
    m1_flux_dot(uL, A, c, fL);
    m1_flux_dot(uR, A, c, fR);
    double vL[4], vR[4];
    for (int q = 0; q < 4; ++q) {
        vL[q] = val(uL[q]);
        vR[q] = val(uR[q]);
    }
    double xL, nL, xR, nR;
    wave_speeds(M, vL, A, c, xL, nL);
    wave_speeds(M, vR, A, c, xR, nR);
    double lp = std::max(0.0, std::max(xL, xR));
    double lm = std::min(0.0, std::min(nL, nR));
    if (lp - lm > 0.0) {
        double An = std::sqrt(norm2(A));
        for (int q = 0; q < 4; ++q)
            phi[q] = (T(lp) * fL[q] - T(lm) * fR[q] + T(lp * lm * An) * (uR[q] - uL[q])) / T(lp - lm);
    } else {
        for (int q = 0; q < 4; ++q) phi[q] = T(0.5) * (fL[q] + fR[q]);
    }
}

struct StepStats { long clamped = 0; };

// Individual time bins (Sec. "Individual Timstepping"; Eqs. meshless-explicit-individual-
// timesteps and transport-update-explicit): particle i advances in steps of
// dt_i = 2^b_i dt_min over a hydro step of 2^B min-steps.  At min-step s a particle starts
// a step when s mod 2^b_i = 0: it receives its injection for dt_i and a new gradient.  Every
// pair with a starting member exchanges the time-integrated flux
// min(dt_k, dt_l) F_kl . A_kl into both particles' accumulators (k as the left state from
// k's side); a particle applies its accumulator, then its sink over dt_i, when its step ends
// (at min-step s when (s + 1) mod 2^b_i = 0).  Until then its state stays as it was.
// U: [G][4][N]; bins [N]; alpha [N] or null.
template <class T>
static void step_bins(const Model& M, double dt_min, int B, const int* bins, std::vector<T>& U,
                      const std::vector<T>& L, const double* alpha, StepStats* st) {
    const long n = M.P.n;
    const int G = M.cfg.n_groups;
    const int C = 4 * G;
    const double c = M.cfg.c_red;
    std::vector<T> acc((size_t)C * n, T(0.0)), grad, g_now;
    std::vector<char> start(n);
    for (long s = 0; s < (1L << B); ++s) {
        for (long i = 0; i < n; ++i) start[i] = (s % (1L << bins[i])) == 0;
        // injection of the starting particles over their own step
        for (long q = 0; q < M.n_src; ++q)
            for (const Target& t : M.inj[q])
                if (start[t.g]) {
                    const double dti = std::ldexp(dt_min, bins[t.g]);
                    for (int g = 0; g < G; ++g)
                        U[(size_t)(4 * g) * n + t.g] += T(t.xi * dti / M.V[t.g]) * L[(size_t)q * G + g];
                }
        // new gradients of the starting particles; the others keep theirs
        gradients(M, U, g_now);
        if (s == 0) grad = g_now;
        for (long i = 0; i < n; ++i)
            if (start[i])
                for (int cc = 0; cc < C; ++cc)
                    for (int a = 0; a < 3; ++a) grad[((size_t)cc * 3 + a) * n + i] = g_now[((size_t)cc * 3 + a) * n + i];
        // exchanges of the pairs with a starting member
#pragma omp parallel for schedule(dynamic, 64)
        for (long k = 0; k < n; ++k) {
            for (long l : M.nbr[k]) {
                if (!start[k] && !start[l]) continue;
                const double w = std::ldexp(1.0, std::min(bins[k], bins[l]));   // min(dt_k, dt_l) / dt_min
                double d[3];
                M.P.sep(k, l, d);
                double A[3];
                surface(M, k, l, d, A);
                for (int g = 0; g < G; ++g) {
                    T uk[4], ul[4], gk[4][3], gl[4][3], phi[4];
                    for (int q = 0; q < 4; ++q) {
                        const int cc = 4 * g + q;
                        uk[q] = U[(size_t)cc * n + k];
                        ul[q] = U[(size_t)cc * n + l];
                        for (int a = 0; a < 3; ++a) {
                            gk[q][a] = grad[((size_t)cc * 3 + a) * n + k];
                            gl[q][a] = grad[((size_t)cc * 3 + a) * n + l];
                        }
                    }
                    T uL[4], uR[4];
                    face_states(uk, ul, gk, gl, d, M.h[k], M.h[l], uL, uR);
                    if (M.cfg.riemann == 1)
                        hll_flux(M, uL, uR, A, c, phi);
                    else
                        glf_flux(uL, uR, A, c, phi);
                    for (int q = 0; q < 4; ++q) acc[(size_t)(4 * g + q) * n + k] += T(w) * phi[q];
                }
            }
        }
        // particles whose step ends now: update, sink over their step, fix-up
        for (long i = 0; i < n; ++i) {
            if (((s + 1) % (1L << bins[i])) != 0) continue;
            const double dti = std::ldexp(dt_min, bins[i]);
            const double fac = alpha ? std::max(0.0, 1.0 - c * alpha[i] * dti) : 1.0;
            for (int cc = 0; cc < C; ++cc) {
                T& u = U[(size_t)cc * n + i];
                u = (u - T(dt_min / M.V[i]) * acc[(size_t)cc * n + i]) * T(fac);
                acc[(size_t)cc * n + i] = T(0.0);
            }
            if (M.cfg.clamp_negative)
                for (int g = 0; g < G; ++g) {
                    T& E = U[(size_t)(4 * g) * n + i];
                    if (val(E) < 0.0) {
                        E = T(0.0);
                        if (st) st->clamped++;
                    }
                }
        }
    }
}

// Time-step limiter (Sec. "Dynamic Sub-Cycling"): interacting particles differ by at most
// a factor 4 in time step, i.e. 2 bins: b_i <- min(b_i, min_j b_j + 2) until nothing changes.
static void limit_bins(const Model& M, std::vector<int>& b) {
    for (bool changed = true; changed;) {
        changed = false;
        std::vector<int> nb = b;
        for (long i = 0; i < M.P.n; ++i)
            for (long j : M.nbr[i])
                if (b[j] + 2 < nb[i]) {
                    nb[i] = b[j] + 2;
                    changed = true;
                }
        b.swap(nb);
    }
}

// The injection of one step (Sec. "Weights For Distribution Of Energy Density"): each
// source's luminosity times dt, spread over its gas neighbours by the weights xi and turned
// into energy density by the target's volume, E_g += xi_sg L_s dt / V_g.  U: [G][4][N].
template <class T>
static void inject(const Model& M, double dt, std::vector<T>& U, const std::vector<T>& L) {
    const long n = M.P.n;
    const int G = M.cfg.n_groups;
    for (long s = 0; s < M.n_src; ++s)
        for (const Target& t : M.inj[s])
            for (int g = 0; g < G; ++g)
                U[(size_t)(4 * g) * n + t.g] += T(t.xi * dt / M.V[t.g]) * L[(size_t)s * G + g];
}

// One time step: injection -> transport -> grey sink (-> optional fix-up).
// U: [G][4][N] in/out, L: [S][G], alpha: [N] or null.  With grad_given ([G][4][3][N]) the
// step is the transport and sink alone, with those gradients (the caller has injected).
template <class T>
static void step(const Model& M, double dt, std::vector<T>& U, const std::vector<T>& L, const double* alpha,
                 StepStats* st, const double* alpha_g = nullptr, const std::vector<T>* grad_given = nullptr) {
    const long n = M.P.n;
    const int G = M.cfg.n_groups;
    const int C = 4 * G;
    const double c = M.cfg.c_red;

    // 1. injection
    if (!grad_given) inject(M, dt, U, L);

    // 2. gradients of the injected state
    std::vector<T> grad_own;
    if (!grad_given) gradients(M, U, grad_own);
    const std::vector<T>& grad = grad_given ? *grad_given : grad_own;

    // 3. each particle k sums F_kl . A_kl over its neighbours l, with k as the left state
    std::vector<T> Unew(U.size());
#pragma omp parallel for schedule(dynamic, 64)
    for (long k = 0; k < n; ++k) {
        std::vector<T> acc(C, T(0.0));
        for (long l : M.nbr[k]) {
            double d[3];
            M.P.sep(k, l, d);   // x_l - x_k
            double A[3];
            surface(M, k, l, d, A);
            for (int g = 0; g < G; ++g) {
                T uk[4], ul[4], gk[4][3], gl[4][3], phi[4];
                for (int q = 0; q < 4; ++q) {
                    int cc = 4 * g + q;
                    uk[q] = U[(size_t)cc * n + k];
                    ul[q] = U[(size_t)cc * n + l];
                    for (int a = 0; a < 3; ++a) {
                        gk[q][a] = grad[((size_t)cc * 3 + a) * n + k];
                        gl[q][a] = grad[((size_t)cc * 3 + a) * n + l];
                    }
                }
                T uL[4], uR[4];
                face_states(uk, ul, gk, gl, d, M.h[k], M.h[l], uL, uR);
                if (M.cfg.riemann == 1)
                    hll_flux(M, uL, uR, A, c, phi);
                else
                    glf_flux(uL, uR, A, c, phi);
                for (int q = 0; q < 4; ++q) acc[4 * g + q] += phi[q];
            }
        }
        for (int cc = 0; cc < C; ++cc)
            Unew[(size_t)cc * n + k] = U[(size_t)cc * n + k] - T(dt / M.V[k]) * acc[cc];   // Eq. transport-update-explicit
    }

    // 4. sink (forward Euler, clamped at zero): grey alpha_i, or per group alpha_g,i =
    //    sum_j n_j sigma^N_gj (Eqs. dEdt-group, dFdt-group); then the optional fix-up
    long clamped = 0;
    for (long i = 0; i < n; ++i) {
        double fac = 1.0;
        if (alpha) fac = std::max(0.0, 1.0 - c * alpha[i] * dt);
        for (int cc = 0; cc < C; ++cc) {
            double f = alpha_g ? std::max(0.0, 1.0 - c * alpha_g[(size_t)(cc / 4) * n + i] * dt) : fac;
            Unew[(size_t)cc * n + i] *= T(f);
        }
        if (M.cfg.clamp_negative)
            for (int g = 0; g < G; ++g) {
                T& E = Unew[(size_t)(4 * g) * n + i];
                if (val(E) < 0.0) { E = T(0.0); clamped++; }
            }
    }
    if (st) st->clamped += clamped;
    U.swap(Unew);
}

}  // namespace orc

// =========================================================================================
// C interface for the tests (ctypes).
using namespace orc;

extern "C" {

struct orc_config {
    int32_t n_groups;
    double c_red;
    double eta_res;
    double eta_res_star;
    double box[3];
    int32_t periodic;
    int32_t clamp_negative;
    double h_tol;
    int32_t h_max_iter;
    int32_t brute_force;
    int32_t riemann;
};

void* orc_create(const orc_config* cfg, long n, const double* x, const double* m, long n_src, const double* xsrc,
                 int* status) {
    Model* M = new Model();
    M->cfg.n_groups = cfg->n_groups;
    M->cfg.c_red = cfg->c_red;
    M->cfg.eta_res = cfg->eta_res;
    M->cfg.eta_res_star = cfg->eta_res_star;
    for (int a = 0; a < 3; ++a) M->cfg.box[a] = cfg->box[a];
    M->cfg.periodic = cfg->periodic;
    M->cfg.clamp_negative = cfg->clamp_negative;
    M->cfg.h_tol = cfg->h_tol;
    M->cfg.h_max_iter = cfg->h_max_iter;
    M->cfg.brute_force = cfg->brute_force;
    M->cfg.riemann = cfg->riemann;
    M->P.n = n;
    for (int a = 0; a < 3; ++a) M->P.box[a] = cfg->box[a];
    M->P.periodic = cfg->periodic != 0;
    M->P.x.assign(x, x + 3 * n);
    M->m.assign(m, m + n);
    M->n_src = n_src;
    M->xsrc.assign(xsrc, xsrc + 3 * n_src);
    if (n < 2 || cfg->n_groups < 1) {
        *status = ERR_INVALID;
        return M;
    }
    *status = build(*M);
    return M;
}

// as orc_create, with the smoothing lengths given: h [n] for the particles, hs [n_src] for the
// sources (omega then evaluated at them)
void* orc_create_given_h(const orc_config* cfg, long n, const double* x, const double* m, long n_src,
                         const double* xsrc, const double* h, const double* hs, const double* omegas,
                         const double* octw, int* status) {
    Model* M = new Model();
    M->h_given.assign(h, h + n);
    if (n_src > 0) M->hs_given.assign(hs, hs + n_src);
    if (n_src > 0 && omegas) M->omegas_given.assign(omegas, omegas + n_src);
    if (n_src > 0 && octw) M->octw_given.assign(octw, octw + 8 * n_src);
    M->cfg.n_groups = cfg->n_groups;
    M->cfg.c_red = cfg->c_red;
    M->cfg.eta_res = cfg->eta_res;
    M->cfg.eta_res_star = cfg->eta_res_star;
    for (int a = 0; a < 3; ++a) M->cfg.box[a] = cfg->box[a];
    M->cfg.periodic = cfg->periodic;
    M->cfg.clamp_negative = cfg->clamp_negative;
    M->cfg.h_tol = cfg->h_tol;
    M->cfg.h_max_iter = cfg->h_max_iter;
    M->cfg.brute_force = cfg->brute_force;
    M->cfg.riemann = cfg->riemann;
    M->P.n = n;
    for (int a = 0; a < 3; ++a) M->P.box[a] = cfg->box[a];
    M->P.periodic = cfg->periodic != 0;
    M->P.x.assign(x, x + 3 * n);
    M->m.assign(m, m + n);
    M->n_src = n_src;
    M->xsrc.assign(xsrc, xsrc + 3 * n_src);
    if (n < 2 || cfg->n_groups < 1) {
        *status = ERR_INVALID;
        return M;
    }
    *status = build(*M);
    return M;
}

void orc_destroy(void* p) { delete (Model*)p; }

long orc_num_directed_pairs(void* p) {
    Model* M = (Model*)p;
    long s = 0;
    for (auto& v : M->nbr) s += (long)v.size();
    return s;
}

void orc_get_pairs(void* p, long* offsets, int32_t* cols) {
    Model* M = (Model*)p;
    long e = 0;
    offsets[0] = 0;
    for (long i = 0; i < M->P.n; ++i) {
        for (long j : M->nbr[i]) cols[e++] = (int32_t)j;
        offsets[i + 1] = e;
    }
}

// h, omega, V [N]; B [9N] row-major per particle; cond [N]
void orc_get_particles(void* p, double* h, double* omega, double* V, double* B, double* cond) {
    Model* M = (Model*)p;
    long n = M->P.n;
    if (h) std::memcpy(h, M->h.data(), n * sizeof(double));
    if (omega) std::memcpy(omega, M->omega.data(), n * sizeof(double));
    if (V) std::memcpy(V, M->V.data(), n * sizeof(double));
    if (B) std::memcpy(B, M->B.data(), 9 * n * sizeof(double));
    if (cond) std::memcpy(cond, M->cond.data(), n * sizeof(double));
}

// A_ij for every directed entry of the pair sets, [3][P2]
void orc_get_surfaces(void* p, double* A) {
    Model* M = (Model*)p;
    long P2 = orc_num_directed_pairs(p);
    long e = 0;
    for (long i = 0; i < M->P.n; ++i)
        for (long j : M->nbr[i]) {
            double d[3], a[3];
            M->P.sep(i, j, d);
            surface(*M, i, j, d, a);
            for (int k = 0; k < 3; ++k) A[k * P2 + e] = a[k];
            ++e;
        }
}

// psi-tilde_j(x_i) for every directed entry, [3][P2]
void orc_get_psitilde(void* p, double* out) {
    Model* M = (Model*)p;
    long P2 = orc_num_directed_pairs(p);
    long e = 0;
    for (long i = 0; i < M->P.n; ++i)
        for (long j : M->nbr[i]) {
            double d[3], a[3];
            M->P.sep(i, j, d);
            psitilde(*M, i, d, std::sqrt(norm2(d)), a);
            for (int k = 0; k < 3; ++k) out[k * P2 + e] = a[k];
            ++e;
        }
}

long orc_num_injection_entries(void* p) {
    Model* M = (Model*)p;
    long s = 0;
    for (auto& v : M->inj) s += (long)v.size();
    return s;
}

// per source: h_s, omega_s, octant weights (8 per source); per entry (source-major, gas
// ascending): source index, gas index, xi
void orc_get_sources(void* p, double* hs, double* omegas, double* octw, int32_t* e_src, int32_t* e_gas, double* e_xi) {
    Model* M = (Model*)p;
    long e = 0;
    for (long s = 0; s < M->n_src; ++s) {
        if (hs) hs[s] = M->hs[s];
        if (omegas) omegas[s] = M->omegas[s];
        if (octw) for (int a = 0; a < 8; ++a) octw[8 * s + a] = M->octw[8 * s + a];
        for (const Target& t : M->inj[s]) {
            if (e_src) e_src[e] = (int32_t)s;
            if (e_gas) e_gas[e] = (int32_t)t.g;
            if (e_xi) e_xi[e] = t.xi;
            ++e;
        }
    }
}

void orc_geometry_stats(void* p, long* n_ill, double* cond_max) {
    Model* M = (Model*)p;
    *n_ill = M->n_ill;
    *cond_max = M->cond_max;
}

// grad: [4G][3][N]
void orc_gradients(void* p, const double* U, double* grad) {
    Model* M = (Model*)p;
    size_t n = M->P.n, C = 4 * M->cfg.n_groups;
    std::vector<double> u(U, U + C * n), g;
    gradients(*M, u, g);
    std::memcpy(grad, g.data(), C * 3 * n * sizeof(double));
}

// n_sub steps of size dt; U in/out [G][4][N]; L [S][G]; alpha [N] or null; returns clamp count
long orc_run(void* p, int n_sub, double dt, double* U, const double* L, const double* alpha) {
    Model* M = (Model*)p;
    size_t n = M->P.n, C = 4 * M->cfg.n_groups;
    std::vector<double> u(U, U + C * n);
    std::vector<double> l(L, L + (size_t)M->n_src * M->cfg.n_groups);
    StepStats st;
    for (int k = 0; k < n_sub; ++k) step(*M, dt, u, l, alpha, &st);
    std::memcpy(U, u.data(), C * n * sizeof(double));
    return st.clamped;
}

// the transport and sink of one step with the gradients given (the stages after the
// injection and the gradients); U in/out [G][4][N], grad [G][4][3][N], alpha [N] or null;
// returns the fix-up count
long orc_transport_given_gradients(void* p, double dt, double* U, const double* grad, const double* alpha) {
    Model* M = (Model*)p;
    size_t n = M->P.n, C = 4 * M->cfg.n_groups;
    std::vector<double> u(U, U + C * n), g(grad, grad + 3 * C * n), l;
    StepStats st;
    step(*M, dt, u, l, alpha, &st, nullptr, &g);
    std::memcpy(U, u.data(), C * n * sizeof(double));
    return st.clamped;
}

// omega_i (hence V_i = 1 / omega_i) and B_i [3][3] of particles [first, first + count) given by
// the caller instead of the model's own: a rank of a domain decomposition takes them from
// the particles' owners, whose neighbourhoods are complete
void orc_set_fields(void* p, long first, long count, const double* omega, const double* B) {
    Model* M = (Model*)p;
    for (long k = 0; k < count; ++k) {
        const long i = first + k;
        M->omega[i] = omega[k];
        M->V[i] = 1.0 / omega[k];
        for (int e = 0; e < 9; ++e) M->B[9 * i + e] = B[9 * k + e];
    }
}

// the injection of one step alone (the first stage of orc_run's step); U in/out [G][4][N]
void orc_inject(void* p, double dt, double* U, const double* L) {
    Model* M = (Model*)p;
    size_t n = M->P.n, C = 4 * M->cfg.n_groups;
    std::vector<double> u(U, U + C * n);
    std::vector<double> l(L, L + (size_t)M->n_src * M->cfg.n_groups);
    inject(*M, dt, u, l);
    std::memcpy(U, u.data(), C * n * sizeof(double));
}

// as orc_run, with the photo-ionisation sink per group: alpha_g [G][N]
long orc_run_groups(void* p, int n_sub, double dt, double* U, const double* L, const double* alpha_g) {
    Model* M = (Model*)p;
    size_t n = M->P.n, C = 4 * M->cfg.n_groups;
    std::vector<double> u(U, U + C * n);
    std::vector<double> l(L, L + (size_t)M->n_src * M->cfg.n_groups);
    StepStats st;
    for (int k = 0; k < n_sub; ++k) step(*M, dt, u, l, nullptr, &st, alpha_g);
    std::memcpy(U, u.data(), C * n * sizeof(double));
    return st.clamped;
}

// one hydro step with individual time bins; bins [N] in/out (limited in place when
// `limit`); returns the clamp count
long orc_step_bins(void* p, double dt_min, int* bins, int limit, double* U, const double* L, const double* alpha) {
    Model* M = (Model*)p;
    size_t n = M->P.n, C = 4 * M->cfg.n_groups;
    std::vector<int> b(bins, bins + n);
    if (limit) limit_bins(*M, b);
    int B = 0;
    for (int v : b) B = std::max(B, v);
    std::copy(b.begin(), b.end(), bins);
    std::vector<double> u(U, U + C * n);
    std::vector<double> l(L, L + (size_t)M->n_src * M->cfg.n_groups);
    StepStats st;
    step_bins(*M, dt_min, B, b.data(), u, l, alpha, &st);
    std::memcpy(U, u.data(), C * n * sizeof(double));
    return st.clamped;
}

// bins from each particle's CFL step (Eq. rt-cfl): the largest b <= max_bin with
// 2^b dt_min <= cfl dx_i / c, dx_i = (V_i / (4 pi / 3))^(1/3)
void orc_cfl_bins(void* p, double cfl, double dt_min, int max_bin, int* bins) {
    Model* M = (Model*)p;
    for (long i = 0; i < M->P.n; ++i) {
        const double lim = cfl * std::cbrt(M->V[i] / (4.0 * M_PI / 3.0)) / M->cfg.c_red;
        int b = 0;
        while (b < max_bin && std::ldexp(dt_min, b + 1) <= lim) ++b;
        bins[i] = b;
    }
}

// forward-mode derivative of n_sub steps along (dU0, dL): returns U and dU
void orc_jvp(void* p, int n_sub, double dt, const double* U0, const double* dU0, const double* L, const double* dL,
             const double* alpha, double* U, double* dU) {
    Model* M = (Model*)p;
    size_t n = M->P.n, C = 4 * M->cfg.n_groups, SG = (size_t)M->n_src * M->cfg.n_groups;
    std::vector<Dual> u(C * n), l(SG);
    for (size_t k = 0; k < C * n; ++k) u[k] = Dual(U0[k], dU0[k]);
    for (size_t k = 0; k < SG; ++k) l[k] = Dual(L[k], dL[k]);
    for (int k = 0; k < n_sub; ++k) step(*M, dt, u, l, alpha, nullptr);
    for (size_t k = 0; k < C * n; ++k) {
        U[k] = u[k].v;
        dU[k] = u[k].d;
    }
}

// The number of kinks (see kink_if) that n_sub steps along the direction (dU0, dL) pass within
// eps of: central differences of step eps along that direction match the derivative only
// where this is zero.
long orc_jvp_kinks(void* p, int n_sub, double dt, const double* U0, const double* dU0, const double* L,
                   const double* dL, const double* alpha, double eps) {
    Model* M = (Model*)p;
    size_t n = M->P.n, C = 4 * M->cfg.n_groups;
    std::vector<double> U(C * n), dU(C * n);
    g_kinks = 0;
    g_kink_eps = eps;
    orc_jvp(p, n_sub, dt, U0, dU0, L, dL, alpha, U.data(), dU.data());
    g_kink_eps = 0.0;
    return g_kinks.load();
}

// Drift correction (Sec. "Dealing With Particle Drifts"): a particle moved by dx = v dt_drift
// takes the state extrapolated with its gradient (Eq. gradient) at the old position,
// U_i + grad U_i . dx_i, for every component.  U, Uout: [G][4][N]; v: [3][N].
void orc_drift(void* p, const double* U, const double* v, double dt_drift, double* Uout) {
    Model* M = (Model*)p;
    size_t n = M->P.n, C = 4 * M->cfg.n_groups;
    std::vector<double> u(U, U + C * n), g;
    gradients(*M, u, g);
    for (size_t cc = 0; cc < C; ++cc)
        for (size_t i = 0; i < n; ++i) {
            double du = 0.0;
            for (int a = 0; a < 3; ++a) du += g[(cc * 3 + a) * n + i] * (v[a * n + i] * dt_drift);
            Uout[cc * n + i] = u[cc * n + i] + du;
        }
}

// total radiation energy per group, sum_i V_i E_i,g
void orc_energy(void* p, const double* U, double* Etot) {
    Model* M = (Model*)p;
    long n = M->P.n;
    for (int g = 0; g < M->cfg.n_groups; ++g) {
        double s = 0;
        for (long i = 0; i < n; ++i) s += M->V[i] * U[(size_t)(4 * g) * n + i];
        Etot[g] = s;
    }
}

// GLF positivity estimate dt_pos = min_i 2 V_i / (c sum_j |A_ij|)
double orc_dt_positivity(void* p) {
    Model* M = (Model*)p;
    double best = INFINITY;
    for (long i = 0; i < M->P.n; ++i) {
        double s = 0;
        for (long j : M->nbr[i]) {
            double d[3], A[3];
            M->P.sep(i, j, d);
            surface(*M, i, j, d, A);
            s += std::sqrt(norm2(A));
        }
        best = std::min(best, 2.0 * M->V[i] / (M->cfg.c_red * s));
    }
    return best;
}

// M1 flux of a single state for pinning the closure: out = (F.A, c^2 D E A)
void orc_m1_flux(const double* u4, const double* A, double c, double* out) { m1_flux_dot<double>(u4, A, c, out); }

double orc_kernel_W(double r, double h) { return kernel_W(r, h); }

// Floating-point operations of the pair loops, counted by running the oracle's own pair
// arithmetic on the counting scalar (add, subtract, multiply, divide, square root: one each;
// comparisons, conversions and the periodic wrap of separations are not counted):
//   out[0] flux geometry per unordered pair: separation, A_kl (Eq. HopkinsAij), |A_kl| and the
//          GLF dissipation factor c/2 |A_kl|; averaged over the model's pairs (the spline's
//          two branches differ in cost);
//   out[1] flux per unordered pair and group: the face states of Eq. rt-riemann-problem with
//          the minmod slopes and the GLF flux of Eq. riemann-GLF with two M1 closures
//          (Eq. eddington-group), for a state in the general branch (E > 0, 0 < f < 1, slopes
//          of equal sign, so no branch of the closure or the limiter returns early);
//   out[2] accumulation of that flux into both particles' sums, per pair and group;
//   out[3] gradient geometry per directed neighbour entry: separation, |d| and
//          psitilde_j(x_i) (Eq. psitilde); averaged over the model's entries;
//   out[4] gradient per directed entry and group: (Q_j - Q_i) psitilde for the four components
//          (Eq. gradient).
void orc_pair_flops(void* p, double* out) {
    const Model& M = *(const Model*)p;
    const long n = M.P.n;
    const double c = M.cfg.c_red;
    long geo = 0, npair = 0, ggeo = 0, nent = 0;
    for (long i = 0; i < n; ++i)
        for (long j : M.nbr[i]) {
            double dd[3];
            M.P.sep(i, j, dd);
            // x_j - x_i: three subtractions (the periodic wrap is not arithmetic of the method)
            g_flops = 3;
            Counted d[3];
            for (int a = 0; a < 3; ++a) d[a] = Counted(dd[a]);
            Counted r = sqrt_(norm2(d));
            Counted pt[3];
            psitilde<Counted>(M, i, d, r, pt);
            ggeo += g_flops;
            ++nent;
            if (j < i) continue;
            g_flops = 3;
            Counted A[3];
            surface<Counted>(M, i, j, d, A);
            Counted An = sqrt_(norm2(A));
            Counted diss = Counted(0.5 * c) * An;
            (void)diss;
            geo += g_flops;
            ++npair;
        }
    // one pair in the general branch
    long k = -1, l = -1;
    for (long i = 0; i < n && k < 0; ++i)
        if (!M.nbr[i].empty()) { k = i; l = M.nbr[i][0]; }
    double dd[3];
    M.P.sep(k, l, dd);
    const double uk0[4] = {1.0, 0.3 * c, 0.2 * c, -0.1 * c}, ul0[4] = {0.8, 0.1 * c, 0.25 * c, 0.05 * c};
    Counted uk[4], ul[4], gk[4][3], gl[4][3], uL[4], uR[4], phi[4];
    for (int q = 0; q < 4; ++q) {
        uk[q] = uk0[q];
        ul[q] = ul0[q];
        for (int a = 0; a < 3; ++a) {       // grad Q . d = s |d|^2 with s > 0 on both sides
            gk[q][a] = (1.0 + 0.5 * q) * dd[a];
            gl[q][a] = (2.0 + 0.25 * q) * dd[a];
        }
    }
    double A[3];
    surface<double>(M, k, l, dd, A);
    g_flops = 0;
    face_states<Counted>(uk, ul, gk, gl, dd, M.h[k], M.h[l], uL, uR);
    glf_flux<Counted>(uL, uR, A, c, phi);
    const long per_group = g_flops;
    g_flops = 0;
    Counted acc_k[4], acc_l[4];
    for (int q = 0; q < 4; ++q) {
        acc_k[q] += phi[q];
        acc_l[q] -= phi[q];
    }
    const long gather = g_flops;
    g_flops = 0;
    Counted grad[4][3], ps[3] = {Counted(0.1), Counted(0.2), Counted(0.3)};
    for (int q = 0; q < 4; ++q) {
        Counted dq = ul[q] - uk[q];
        for (int a = 0; a < 3; ++a) grad[q][a] += dq * ps[a];
    }
    const long grad_group = g_flops;
    out[0] = npair ? (double)geo / (double)npair : 0.0;
    out[1] = (double)per_group;
    out[2] = (double)gather;
    out[3] = nent ? (double)ggeo / (double)nent : 0.0;
    out[4] = (double)grad_group;
}

// face states of one pair and group: u*/g* per component (E, Fx, Fy, Fz), g* row-major [4][3]
void orc_face_states(const double* uk, const double* ul, const double* gk, const double* gl, const double* d,
                     double hk, double hl, double* uL, double* uR) {
    double GK[4][3], GL[4][3];
    for (int q = 0; q < 4; ++q)
        for (int a = 0; a < 3; ++a) { GK[q][a] = gk[3 * q + a]; GL[q][a] = gl[3 * q + a]; }
    face_states<double>(uk, ul, GK, GL, d, hk, hl, uL, uR);
}

void orc_glf_flux(const double* uL, const double* uR, const double* A, double c, double* phi) {
    glf_flux<double>(uL, uR, A, c, phi);
}

// psi_j(x_i) for every directed entry [P2], and the self weight psi_i(x_i) [N]
void orc_get_psi(void* p, double* psi, double* psi_self) {
    Model* M = (Model*)p;
    long e = 0;
    for (long i = 0; i < M->P.n; ++i) {
        for (long j : M->nbr[i]) {
            double d[3];
            M->P.sep(i, j, d);
            psi[e++] = psi_at(*M, i, std::sqrt(norm2(d)));
        }
        psi_self[i] = psi_at(*M, i, 0.0);
    }
}

double orc_minmod(double a, double b) { return minmod<double>(a, b); }

// HLL wave-speed table (units of c): lmax, lmin [nf][nth] over f = i/(nf-1), theta = j pi/(nth-1)
void orc_set_wave_table(void* p, const double* lmax, const double* lmin, int nf, int nth) {
    Model* M = (Model*)p;
    M->wnf = nf;
    M->wnth = nth;
    M->wmax.assign(lmax, lmax + (size_t)nf * nth);
    M->wmin.assign(lmin, lmin + (size_t)nf * nth);
}

// HLL flux of one pair and group (uses the model's table and c)
void orc_hll_flux(void* p, const double* uL, const double* uR, const double* A, double* phi) {
    Model* M = (Model*)p;
    hll_flux<double>(*M, uL, uR, A, M->cfg.c_red, phi);
}

void orc_wave_speeds(void* p, const double* u, const double* A, double* lmax, double* lmin) {
    Model* M = (Model*)p;
    wave_speeds(*M, u, A, M->cfg.c_red, *lmax, *lmin);
}

int orc_num_threads() {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
}
