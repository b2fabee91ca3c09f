// Photo-ionisation sink of the photon groups (Ivkovic 2023, Part III): the cross-section
// fits of Eq. sigma-parametrizaiton with the parameters of Table tab:cross-sections, their
// averages over a group for an assumed blackbody spectrum (Eq. blackbody; Eqs. sigma_N,
// sigma_E, and the group's mean photon energy), the photon-number to luminosity conversion
// of Appendix "Converting Photon Number Emission Rates to Photon Energy Emission Rates",
// and the per-group absorption alpha_g = sum_j n_j sigma^N_gj of Eqs. dEdt-group and
// dFdt-group, which the gather kernels apply as the sink.
//
// The group integrals are taken on the host by adaptive Gauss-Kronrod (7/15 points) over
// pieces split at the species thresholds, up to h nu = 700 kT (beyond it the spectrum is
// below double range).  The table's sigma_0 is in cm^2 (the fit's "x 1e-18 cm^2" factor
// belongs to sigma_0 in megabarn).  CGS units, frequencies in Hz.
#include <cmath>
#include <vector>

#include "rt_internal.cuh"

namespace rt {

namespace {

const double kH = 6.62607015e-27;     // erg s
const double kK = 1.380649e-16;       // erg / K
const double kEV = 1.602176634e-12;   // erg
// Eqs. nuIonHI, nuIonHeI, nuIonHeII (eV) and Table tab:cross-sections:
// E0 [eV], sigma0 [cm^2], y_a, P, y_w, y_0, y_1 for H0, He0, He+
const double kIon[3] = {13.60, 24.59, 54.42};
const double kFit[3][7] = {{0.4298, 5.475e-14, 32.88, 2.963, 0.0, 0.0, 0.0},
                           {13.61, 9.492e-16, 1.469, 3.188, 2.039, 0.4434, 2.136},
                           {1.720, 1.369e-14, 32.88, 2.963, 0.0, 0.0, 0.0}};

double sigma_fit(int j, double E_eV) {
    if (E_eV < kIon[j]) return 0.0;
    const double* p = kFit[j];
    const double x = E_eV / p[0] - p[5];
    const double y = std::sqrt(x * x + p[6] * p[6]);
    return p[1] * ((x - 1.0) * (x - 1.0) + p[4] * p[4]) * std::pow(y, 0.5 * p[3] - 5.5) *
           std::pow(1.0 + std::sqrt(y / p[2]), -p[3]);
}

// spectral shape nu^3 / (exp(h nu / kT) - 1) (constant factors cancel in every ratio)
double planck(double nu, double T) { return nu * nu * nu / std::expm1(kH * nu / (kK * T)); }

// Gauss-Kronrod 7/15 nodes and weights on [-1, 1]
const double kXgk[8] = {0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
                        0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
                        0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
                        0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
const double kWgk[8] = {0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
                        0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
                        0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
                        0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
const double kWg[4] = {0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
                       0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

template <class F>
double gk15(const F& f, double a, double b, double& err) {
    const double c = 0.5 * (a + b), h = 0.5 * (b - a);
    double fc = f(c);
    double rk = fc * kWgk[7], rg = fc * kWg[3];
    for (int k = 0; k < 7; ++k) {
        const double dx = h * kXgk[k];
        const double s = f(c - dx) + f(c + dx);
        rk += kWgk[k] * s;
        if (k % 2 == 1) rg += kWg[k / 2] * s;
    }
    err = std::fabs((rk - rg) * h);
    return rk * h;
}

template <class F>
double integrate(const F& f, double a, double b, double rel = 1e-12, int depth = 0) {
    double err;
    const double v = gk15(f, a, b, err);
    if (depth >= 40 || err <= rel * std::fabs(v) || err < 1e-300) return v;
    const double m = 0.5 * (a + b);
    return integrate(f, a, m, rel, depth + 1) + integrate(f, m, b, rel, depth + 1);
}

// integral over [a, b) of g, split at the species thresholds inside and truncated at
// h nu = 700 kT
template <class F>
double group_integral(const F& g, double a, double b, double T) {
    const double top = 700.0 * kK * T / kH;
    b = std::isfinite(b) ? std::min(b, top) : top;
    if (!(b > a)) return 0.0;
    std::vector<double> pts{a};
    for (int j = 0; j < 3; ++j) {
        const double nu = kIon[j] * kEV / kH;
        if (nu > a && nu < b) pts.push_back(nu);
    }
    pts.push_back(b);
    double s = 0.0;
    for (size_t k = 0; k + 1 < pts.size(); ++k) s += integrate(g, pts[k], pts[k + 1]);
    return s;
}

bool valid_edges(int G, const double* nu) {
    if (G < 1 || !nu) return false;
    for (int i = 0; i < G; ++i)
        if (!(nu[i] > 0.0) || !std::isfinite(nu[i]) || !(nu[i + 1] > nu[i])) return false;
    return true;
}

}  // namespace

// per-group absorption in caller order: alpha[g][i] = sum_j sigma[g][j] n[j][i]
__global__ void k_absorbers(const double* __restrict__ n_sp, int n_species, const double* __restrict__ sigma,
                            int64_t n, int G, double* __restrict__ alpha) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int g = 0; g < G; ++g) {
        double a = 0.0;
        for (int j = 0; j < n_species; ++j) a += sigma[g * n_species + j] * n_sp[(int64_t)j * n + i];
        alpha[(int64_t)g * n + i] = a;
    }
}

}  // namespace rt

using namespace rt;

extern "C" {

rt_status rt_cross_section(int32_t species, double E_eV, double* sigma_out) {
    if (species < 0 || species > 2 || !sigma_out || !std::isfinite(E_eV)) return RT_ERR_INVALID;
    *sigma_out = sigma_fit(species, E_eV);
    return RT_OK;
}

rt_status rt_blackbody_groups(double T_bb, int32_t n_groups, const double* nu_edges, double* eps_mean,
                              double* sigma_N, double* sigma_E) {
    if (!(T_bb > 0.0) || !std::isfinite(T_bb) || !valid_edges(n_groups, nu_edges) || !eps_mean || !sigma_N ||
        !sigma_E)
        return RT_ERR_INVALID;
    for (int i = 0; i < n_groups; ++i) {
        const double a = nu_edges[i], b = nu_edges[i + 1];
        const double e_int = group_integral([&](double nu) { return planck(nu, T_bb); }, a, b, T_bb);
        const double n_int = group_integral([&](double nu) { return planck(nu, T_bb) / (kH * nu); }, a, b, T_bb);
        if (!(n_int > 0.0)) return RT_ERR_INVALID;
        eps_mean[i] = e_int / n_int;
        for (int j = 0; j < 3; ++j) {
            const double sn = group_integral(
                [&](double nu) { return planck(nu, T_bb) / (kH * nu) * sigma_fit(j, kH * nu / kEV); }, a, b, T_bb);
            const double se =
                group_integral([&](double nu) { return planck(nu, T_bb) * sigma_fit(j, kH * nu / kEV); }, a, b, T_bb);
            sigma_N[i * 3 + j] = sn / n_int;
            sigma_E[i * 3 + j] = se / e_int;
        }
    }
    return RT_OK;
}

rt_status rt_photon_number_to_luminosity(double T_bb, double Ndot, int32_t n_groups, const double* nu_edges,
                                         double* L_out) {
    if (!(T_bb > 0.0) || !std::isfinite(T_bb) || !std::isfinite(Ndot) || !valid_edges(n_groups, nu_edges) ||
        !L_out)
        return RT_ERR_INVALID;
    const double n_all =
        group_integral([&](double nu) { return planck(nu, T_bb) / (kH * nu); }, nu_edges[0], INFINITY, T_bb);
    if (!(n_all > 0.0)) return RT_ERR_INVALID;
    for (int i = 0; i < n_groups; ++i)
        L_out[i] = group_integral([&](double nu) { return planck(nu, T_bb); }, nu_edges[i], nu_edges[i + 1], T_bb) /
                   n_all * Ndot;
    return RT_OK;
}

rt_status rt_set_absorbers(rt_ctx* c, int32_t n_species, const double* n_dev, const double* sigma_host) {
    if (!c) return RT_ERR_INVALID;
    c->err.clear();
    if (!n_dev) {
        c->has_alpha_g = false;
        return RT_OK;
    }
    if (n_species < 1 || n_species > 8 || !sigma_host)
        return fail(c, RT_ERR_INVALID, "rt_set_absorbers: n_species must be in [1, 8] and sigma non-NULL");
    const int G = c->cfg.n_groups;
    for (int k = 0; k < G * n_species; ++k)
        if (!std::isfinite(sigma_host[k]) || sigma_host[k] < 0.0)
            return fail(c, RT_ERR_INVALID, "rt_set_absorbers: cross sections must be finite and >= 0");
    RT_CUDA(c, cudaSetDevice(c->device));
    RT_TRY(ensure(c, c->alpha_g_c, (size_t)G * c->n * sizeof(double), "group absorption"));
    RT_TRY(ensure(c, c->alpha_g_s, (size_t)G * c->n * (c->fp64 ? 8 : 4), "group absorption"));
    RT_TRY(ensure(c, c->sigma_d, (size_t)8 * G * sizeof(double), "cross sections"));
    RT_CUDA(c, cudaMemcpyAsync(c->sigma_d.p, sigma_host, (size_t)G * n_species * sizeof(double),
                               cudaMemcpyHostToDevice, c->stream));
    k_absorbers<<<(unsigned)((c->n + 255) / 256), 256, 0, c->stream>>>(
        n_dev, n_species, c->sigma_d.as<double>(), c->n, G, c->alpha_g_c.as<double>());
    ++c->launches;
    RT_CUDA(c, cudaGetLastError());
    // the host copy of sigma must stay valid until the copy has run
    RT_CUDA(c, cudaStreamSynchronize(c->stream));
    c->has_alpha_g = true;
    return RT_OK;
}

}  // extern "C"
