// HLL wave speeds of the M1 system (Ivkovic 2023, Part III, "Riemann solvers",
// Eq. riemann-HLL): the table of the largest and smallest eigenvalue of the flux Jacobian
// over (f, theta), which the pair-flux kernels interpolate.
//
// Derivation (c = 1; the eigenvalues scale with c and do not depend on E).  The M1 pressure
// P = E D(f) (Eq. eddington) can be written P = a(u) E I + b(u) F F^T / E with u = f^2,
// s = sqrt(4 - 3u), a = (1 + s - 2u) / (5 + 2s) = (1 - chi)/2 and b = 3 / (2 + s)
// = (3 chi - 1) / (2 u).  The flux along the unit normal n is (F . n, P n), so with
// f = F / E its Jacobian with respect to (E, F) is
//   d(F.n)/dE = 0,  d(F.n)/dF = n^T,
//   d(Pn)/dE = (a - 2u a') n - (2u b' + b) (f.n) f,
//   d(Pn)/dF = 2 a' n f^T + 2 b' (f.n) f f^T + b (f n^T + (f.n) I),
// (' = d/du).  In the frame n = e_x, f = f (cos theta, sin theta, 0) the z component of F
// decouples with eigenvalue b f cos theta, and the other three eigenvalues are the roots of
// the characteristic cubic of the 3 x 3 block acting on (E, F_x, F_y).  The cubic is solved
// by the trigonometric form of its three real roots and each root polished by Newton steps,
// in long double: near f = 1 the roots cluster and the cubic's coefficients lose digits in
// double.  At f = 1 (free streaming) all four eigenvalues equal cos theta: that row is set to
// its limit.
#include <cmath>

#include "rt_internal.cuh"

namespace rt {

typedef long double ld;

static void wave_extremes(ld f, ld th, ld& lmax, ld& lmin) {
    if (f >= 1) {
        lmax = lmin = std::cos(th);
        return;
    }
    const ld u = f * f, s = std::sqrt(4 - 3 * u);
    const ld a = (1 + s - 2 * u) / (5 + 2 * s), b = 3 / (2 + s);
    const ld ds = -3 / (2 * s);
    const ld da = ((ds - 2) * (5 + 2 * s) - (1 + s - 2 * u) * 2 * ds) / ((5 + 2 * s) * (5 + 2 * s));
    const ld db = -3 * ds / ((2 + s) * (2 + s));
    const ld fc = f * std::cos(th), fs = f * std::sin(th);
    // 3 x 3 block [[0, 1, 0], [jx, Jxx, Jxy], [jy, Jyx, Jyy]]
    const ld jx = (a - 2 * u * da) - (2 * u * db + b) * fc * fc;
    const ld jy = -(2 * u * db + b) * fc * fs;
    const ld Jxx = 2 * da * fc + 2 * db * fc * fc * fc + 2 * b * fc;
    const ld Jxy = 2 * da * fs + 2 * db * fc * fc * fs;
    const ld Jyx = 2 * db * fc * fc * fs + b * fs;
    const ld Jyy = 2 * db * fc * fs * fs + b * fc;
    const ld lz = b * fc;
    // lambda^3 + A2 lambda^2 + A1 lambda + A0 = det(lambda I - block)
    const ld A2 = -(Jxx + Jyy);
    const ld A1 = -jx + Jxx * Jyy - Jxy * Jyx;
    const ld A0 = jx * Jyy - Jxy * jy;
    // three real roots: lambda = 2 sqrt(-p/3) cos(phi/3 - 2 pi k/3) - A2/3
    const ld p = A1 - A2 * A2 / 3;
    const ld q = 2 * A2 * A2 * A2 / 27 - A2 * A1 / 3 + A0;
    ld root[3];
    if (p < 0) {
        ld arg = (3 * q / (2 * p)) * std::sqrt(-3 / p);
        arg = arg > 1 ? 1 : (arg < -1 ? -1 : arg);
        const ld r = 2 * std::sqrt(-p / 3), ph = std::acos(arg) / 3;
        const ld two_pi_3 = 2 * std::acos((ld)-1) / 3;
        for (int k = 0; k < 3; ++k) root[k] = r * std::cos(ph - two_pi_3 * k) - A2 / 3;
    } else {   // triple root (not reached for f < 1)
        root[0] = root[1] = root[2] = -A2 / 3;
    }
    for (int k = 0; k < 3; ++k)
        for (int it = 0; it < 3; ++it) {
            const ld x = root[k];
            const ld P = ((x + A2) * x + A1) * x + A0, dP = (3 * x + 2 * A2) * x + A1;
            if (dP == 0) break;
            root[k] = x - P / dP;
        }
    lmax = lmin = lz;
    for (int k = 0; k < 3; ++k) {
        lmax = root[k] > lmax ? root[k] : lmax;
        lmin = root[k] < lmin ? root[k] : lmin;
    }
}

void build_wave_table(double* lmax, double* lmin) {
    const ld pi = std::acos((ld)-1);
    for (int i = 0; i < RT_WAVE_NF; ++i)
        for (int j = 0; j < RT_WAVE_NTH; ++j) {
            ld a, b;
            wave_extremes((ld)i / (RT_WAVE_NF - 1), pi * j / (RT_WAVE_NTH - 1), a, b);
            lmax[i * RT_WAVE_NTH + j] = (double)a;
            lmin[i * RT_WAVE_NTH + j] = (double)b;
        }
}

}  // namespace rt

extern "C" rt_status rt_wave_table(double* lmax_host, double* lmin_host) {
    if (!lmax_host || !lmin_host) return RT_ERR_INVALID;
    rt::build_wave_table(lmax_host, lmin_host);
    return RT_OK;
}
