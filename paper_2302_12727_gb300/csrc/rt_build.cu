// Neighbour search and particle geometry of the FVPM photon-transport step:
// cell list, smoothing lengths, symmetric pair lists, E_i / B_i, source injection weights.
//
// Part II of Ivkovic (2023), "The Neighbor Search: Determining the Smoothing Length"
// (Eq. number-of-neighbors), Eqs. omega / particle-volume, matrix_E / matrix_B; Part III,
// "Weights For Distribution Of Energy Density of a Star onto Particles"
// (Eq. isotropy-correction-with-zero).  The thesis runs these as SWIFT cell tasks on CPUs;
// here each is a data-parallel kernel over cell-sorted particles.
#include <cub/cub.cuh>

#include <cmath>
#include <vector>

#include "rt_internal.cuh"

namespace rt {


struct Grid {
    int nc[3];
    double cell[3];
    double inv_cell[3];
    float cellf[3], inv_cellf[3];
    double box[3];
    int periodic;
    const int32_t* cell_start;   // [ncells + 1], lower bound of each cell in sorted order
};

// atomic min / max of positive doubles through their bit patterns (ordered like integers)
__device__ __forceinline__ void atomic_min_pos(unsigned long long* a, double v) {
    atomicMin(a, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void atomic_max_pos(unsigned long long* a, double v) {
    atomicMax(a, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void warp_minmax(double& mn, double& mx) {
    for (int o = 16; o > 0; o >>= 1) {
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
}

__device__ __forceinline__ int wrap_cell(int c, int nc) {
    c %= nc;
    return c < 0 ? c + nc : c;
}

// Visit every particle (sorted index) whose cell can hold points within R of p.  Rows of
// cells along x are contiguous in sorted order; rows whose (y, z) extent is farther than R
// are skipped and each row is clipped to the chord of the sphere, so the visited volume
// is close to the sphere plus one cell layer.  An axis whose span covers the whole grid is
// walked once without clipping.  With ASC the ranges come in ascending cell index (a
// periodic axis is walked from the cell that wraps to the lowest index), so that the
// candidates, being sorted by cell, come in ascending particle index.
__device__ __forceinline__ int first_wrapped(int lo, int hi, int nc) {
    return lo < 0 ? 0 : (hi >= nc ? nc : lo);
}

template <bool ASC = false, class F>
__device__ __forceinline__ void for_each_candidate_range(const Grid& g, float px, float py, float pz, float R,
                                                         F&& fr) {
    // float arithmetic with a relative margin of 1e-4 on R: cells are never missed
    const float Rc = R * 1.0001f + 1e-6f * (g.cellf[0] + g.cellf[1] + g.cellf[2]);
    const float R2 = Rc * Rc;
    const float p[3] = {px, py, pz};
    int lo[3], hi[3];
    bool all[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = (int)floorf((p[a] - Rc) * g.inv_cellf[a]);
        hi[a] = (int)floorf((p[a] + Rc) * g.inv_cellf[a]);
        all[a] = (hi[a] - lo[a] + 1 >= g.nc[a]);
        if (all[a]) {
            lo[a] = 0;
            hi[a] = g.nc[a] - 1;
        } else if (!g.periodic) {
            lo[a] = max(lo[a], 0);
            hi[a] = min(hi[a], g.nc[a] - 1);
        }
    }
    const int nzs = hi[2] - lo[2] + 1, nys = hi[1] - lo[1] + 1;
    const int z0 = ASC ? first_wrapped(lo[2], hi[2], g.nc[2]) : lo[2];
    const int y0 = ASC ? first_wrapped(lo[1], hi[1], g.nc[1]) : lo[1];
    for (int kz = 0; kz < nzs; ++kz) {
        int z = z0 + kz;
        if (z > hi[2]) z -= nzs;
        float dz = 0.f;
        if (!all[2]) dz = fmaxf(0.f, fmaxf(z * g.cellf[2] - pz, pz - (z + 1) * g.cellf[2]));
        if (dz * dz >= R2) continue;
        int zz = wrap_cell(z, g.nc[2]);
        for (int ky = 0; ky < nys; ++ky) {
            int y = y0 + ky;
            if (y > hi[1]) y -= nys;
            float dy = 0.f;
            if (!all[1]) dy = fmaxf(0.f, fmaxf(y * g.cellf[1] - py, py - (y + 1) * g.cellf[1]));
            float rem = R2 - dy * dy - dz * dz;
            if (rem <= 0.f) continue;
            int yy = wrap_cell(y, g.nc[1]);
            int64_t base = ((int64_t)zz * g.nc[1] + yy) * g.nc[0];
            int xa, xb;
            if (all[0]) {
                xa = 0;
                xb = g.nc[0] - 1;
            } else {
                float w = sqrtf(rem);
                xa = (int)floorf((px - w) * g.inv_cellf[0]);
                xb = (int)floorf((px + w) * g.inv_cellf[0]);
                if (!g.periodic) {
                    xa = max(xa, 0);
                    xb = min(xb, g.nc[0] - 1);
                }
            }
            int sl[2], sh[2], ns = 0;
            if (xa < 0) {
                if (ASC) { sl[ns] = 0; sh[ns++] = xb; sl[ns] = xa + g.nc[0]; sh[ns++] = g.nc[0] - 1; }
                else { sl[ns] = xa + g.nc[0]; sh[ns++] = g.nc[0] - 1; sl[ns] = 0; sh[ns++] = xb; }
            } else if (xb >= g.nc[0]) {
                if (ASC) { sl[ns] = 0; sh[ns++] = xb - g.nc[0]; sl[ns] = xa; sh[ns++] = g.nc[0] - 1; }
                else { sl[ns] = xa; sh[ns++] = g.nc[0] - 1; sl[ns] = 0; sh[ns++] = xb - g.nc[0]; }
            } else { sl[ns] = xa; sh[ns++] = xb; }
            for (int sI = 0; sI < ns; ++sI) {
                int b = g.cell_start[base + sl[sI]];
                int e = g.cell_start[base + sh[sI] + 1];
                fr(b, e);
            }
        }
    }
}

// every candidate of for_each_candidate_range, one at a time
template <bool ASC = false, class F>
__device__ __forceinline__ void for_each_candidate(const Grid& g, float px, float py, float pz, float R, F&& f) {
    for_each_candidate_range<ASC>(g, px, py, pz, R, [&](int b, int e) {
        for (int j = b; j < e; ++j) f(j);
    });
}

// every candidate with its quantised position record, read four at a time: the loads of a
// batch are in flight together, and f still sees the candidates one by one, in order
template <bool ASC = false, class F>
__device__ __forceinline__ void for_each_candidate_q(const Grid& g, const uint4* __restrict__ xq, float px, float py,
                                                     float pz, float R, F&& f) {
    for_each_candidate_range<ASC>(g, px, py, pz, R, [&](int b, int e) {
        for (int j0 = b; j0 < e; j0 += 4) {
            uint4 q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (j0 + u < e) q[u] = xq[j0 + u];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (j0 + u < e) f(j0 + u, q[u]);
        }
    });
}

// number of particles in the 3 x 3 x 3 cells around (cx, cy, cz): a local density for the
// first guess of h
__device__ __forceinline__ int count_27(const Grid& g, int cx, int cy, int cz) {
    int cnt = 0;
    for (int dz = -1; dz <= 1; ++dz) {
        int z = cz + dz;
        if (!g.periodic && (z < 0 || z >= g.nc[2])) continue;
        int zz = wrap_cell(z, g.nc[2]);
        for (int dy = -1; dy <= 1; ++dy) {
            int y = cy + dy;
            if (!g.periodic && (y < 0 || y >= g.nc[1])) continue;
            int yy = wrap_cell(y, g.nc[1]);
            int64_t base = ((int64_t)zz * g.nc[1] + yy) * g.nc[0];
            for (int dx = -1; dx <= 1; ++dx) {
                int x = cx + dx;
                if (!g.periodic && (x < 0 || x >= g.nc[0])) continue;
                int xx = wrap_cell(x, g.nc[0]);
                cnt += g.cell_start[base + xx + 1] - g.cell_start[base + xx];
            }
        }
    }
    return cnt;
}

__device__ __forceinline__ int cell_coord(double x, double inv_cell, int nc) {
    int c = (int)floor(x * inv_cell);
    return min(max(c, 0), nc - 1);
}

// exact (no contraction) minimal-image separation, identical to a plain double evaluation
__device__ __forceinline__ double sep_exact(double xj, double xi, double box, int periodic) {
    double v = __dsub_rn(xj, xi);
    if (periodic) v = __dsub_rn(v, __dmul_rn(box, rint(__ddiv_rn(v, box))));
    return v;
}

__device__ __forceinline__ double norm2_exact(double a, double b, double c) {
    return __dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(c, c));
}

// fast minimal image (same value except at exactly half a box, which never neighbours)
__device__ __forceinline__ double sep_fast(double xj, double xi, double box, double half, int periodic) {
    double v = xj - xi;
    if (periodic) {
        if (v > half) v -= box;
        else if (v < -half) v += box;
    }
    return v;
}

// ------------------------------------------------------------------------------------
// a1: cell keys, validation
__global__ void k_keys(const double* __restrict__ x, int64_t n, Grid g, uint32_t* keys, int32_t* idx, int* flags) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c[3];
    bool bad = false;
    for (int a = 0; a < 3; ++a) {
        double v = x[a * n + i];
        if (!(v >= 0.0 && v < g.box[a])) bad = true;
        c[a] = bad ? 0 : cell_coord(v, g.inv_cell[a], g.nc[a]);
    }
    if (bad) atomicExch(&flags[F_BADPOS], 1);
    keys[i] = (uint32_t)(((int64_t)c[2] * g.nc[1] + c[1]) * g.nc[0] + c[0]);
    idx[i] = (int32_t)i;
}

__global__ void k_cell_start(const uint32_t* __restrict__ keys, int64_t n, int64_t ncells, int32_t* cell_start) {
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c > ncells) return;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < (uint32_t)c) lo = mid + 1; else hi = mid;
    }
    cell_start[c] = (int32_t)lo;
}

__global__ void k_gather_positions(const double* __restrict__ x, const double* __restrict__ m,
                                   const int32_t* __restrict__ perm, int64_t n, double q0, double q1, double q2,
                                   double* xs, uint4* xq, double* ms, int32_t* inv_perm) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t i = perm[p];
    double qs[3] = {q0, q1, q2};
    uint32_t qv[3];
    for (int a = 0; a < 3; ++a) {
        double v = x[a * n + i];
        xs[a * n + p] = v;
        double f = floor(v * qs[a]);
        f = fmin(fmax(f, 0.0), 4294967295.0);
        qv[a] = (uint32_t)f;
    }
    xq[p] = make_uint4(qv[0], qv[1], qv[2], 0u);   // one 16-byte record a particle for the walks
    ms[p] = m ? m[i] : 0.0;
    inv_perm[i] = (int32_t)p;
}

// ------------------------------------------------------------------------------------
// a2: smoothing lengths.  f(h) = h - eta * omega(h)^(-1/3), omega(h) = sum_j W(r_ij, h) with
// the self term; safeguarded Newton, first in float on fixed-point separations, then in
// double on the exact separations until the step is below machine precision.  The double
// phase runs for every particle on the FP64 path.  On the float path it runs only for the
// particles that have a candidate within kNearBand of their own support radius at the float
// root (about one in thirty): the float root is within a few 1e-6 of the exact one, so for
// every other particle no neighbour can change side of H_i, and the pair lists, which are
// decided by H_i and H_j, are those of the exact roots.
struct HParams {
    double eta, h0, h_cap;
    float scale[3];
    int max_iter;
    float tol32;
    int refine64;   // 1: Newton in double to machine precision here; 0: flag near-threshold particles
};

// |r^2 - H^2| < kNearBand H^2 at the float root: the particle's h is refined in double
constexpr float kNearBand = 2e-4f;

__device__ __forceinline__ float fsep(uint32_t a, uint32_t b, float scale) { return (float)(int32_t)(a - b) * scale; }

// Newton in double from hd on the exact separations of particle p; returns false if it did
// not converge.  On return hd is the root and om_d = omega(hd).
__device__ bool refine_h_double(const Grid& g, const double* __restrict__ xs, const uint4* __restrict__ xq,
                                int64_t n, const HParams& hp, int64_t p, double& hd, double& om_d) {
    const uint4 q4p = xq[p];
    const uint32_t qx = q4p.x, qy = q4p.y, qz = q4p.z;
    const double px = xs[p], py = xs[n + p], pz = xs[2 * n + p];
    const float pxf = (float)px, pyf = (float)py, pzf = (float)pz;
    double lod = 0.0, hid = INFINITY;
    const double half[3] = {0.5 * g.box[0], 0.5 * g.box[1], 0.5 * g.box[2]};
    bool okd = false, last = false;
    for (int it = 0; it < 60; ++it) {
        double H = kKappa * hd;
        double iH = 1.0 / H;
        double H2 = H * H;
        float Hf = (float)H * 1.001f;
        float H2f = Hf * Hf;
        double sw = 0.0, sdw = 0.0;
        for_each_candidate(g, pxf, pyf, pzf, Hf, [&](int j) {
            float dxf = fsep(xq[j].x, qx, hp.scale[0]);
            float dyf = fsep(xq[j].y, qy, hp.scale[1]);
            float dzf = fsep(xq[j].z, qz, hp.scale[2]);
            if (dxf * dxf + dyf * dyf + dzf * dzf >= H2f) return;
            double dx = sep_fast(xs[j], px, g.box[0], half[0], g.periodic);
            double dy = sep_fast(xs[n + j], py, g.box[1], half[1], g.periodic);
            double dz = sep_fast(xs[2 * n + j], pz, g.box[2], half[2], g.periodic);
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < H2) {
                double q = sqrt(r2) * iH;
                double w = spline_w(q);
                sw += w;
                sdw += 3.0 * w + q * spline_dw(q);
            }
        });
        double om = kSigma * iH * iH * iH * sw;
        double dom = -kKappa * kSigma * iH * iH * iH * iH * sdw;
        double cb = cbrt(om);
        double f = hd - hp.eta / cb;
        double fp = 1.0 + (hp.eta / 3.0) / (cb * om) * dom;
        om_d = om;
        if (last) { okd = true; break; }        // omega evaluated at the final h
        if (f < 0.0) lod = hd; else hid = hd;
        double step = f / fp;
        // once the Newton step is tiny the next iterate is exact to rounding: take it and
        // evaluate omega there once more; a residual at the rounding floor or a collapsed
        // bracket ends the iteration at the current h
        if (fabs(f) <= 1e-15 * hd || (hid - lod) <= 1e-14 * hd) { okd = true; break; }
        if (fp > 0.0 && fabs(step) <= 1e-11 * hd) last = true;
        double hn = hd - step;
        if (!last && (it >= 12 || !(hn > lod && hn < hid) || !(fp > 0.0)))
            hn = isinf(hid) ? 1.01 * hd : 0.5 * (lod + hid);
        hd = hn;
    }
    return okd;
}

// The same Newton in double for particle p, with the 32 lanes of a warp sharing the candidate
// walk (in every contiguous run of candidates, lane l takes the l-th, (l + 32)-th, ...) and
// combining their sums by a fixed butterfly, whose result is the same in every lane: the
// lanes then take the same steps.  Used where few particles need it (k_h_refine), so that the double arithmetic,
// slow on this GPU, is spread over many threads.
__device__ bool refine_h_warp(const Grid& g, const double* __restrict__ xs, const uint4* __restrict__ xq,
                              int64_t n, const HParams& hp, int64_t p, int lane, double& hd, double& om_d) {
    const uint4 q4p = xq[p];
    const uint32_t qx = q4p.x, qy = q4p.y, qz = q4p.z;
    const double px = xs[p], py = xs[n + p], pz = xs[2 * n + p];
    const float pxf = (float)px, pyf = (float)py, pzf = (float)pz;
    double lod = 0.0, hid = INFINITY;
    const double half[3] = {0.5 * g.box[0], 0.5 * g.box[1], 0.5 * g.box[2]};
    bool okd = false, last = false;
    for (int it = 0; it < 60; ++it) {
        double H = kKappa * hd;
        double iH = 1.0 / H;
        double H2 = H * H;
        float Hf = (float)H * 1.001f;
        float H2f = Hf * Hf;
        double sw = 0.0, sdw = 0.0;
        for_each_candidate_range(g, pxf, pyf, pzf, Hf, [&](int b, int e) {
          for (int j = b + lane; j < e; j += 32) {
            float dxf = fsep(xq[j].x, qx, hp.scale[0]);
            float dyf = fsep(xq[j].y, qy, hp.scale[1]);
            float dzf = fsep(xq[j].z, qz, hp.scale[2]);
            if (dxf * dxf + dyf * dyf + dzf * dzf >= H2f) continue;
            double dx = sep_fast(xs[j], px, g.box[0], half[0], g.periodic);
            double dy = sep_fast(xs[n + j], py, g.box[1], half[1], g.periodic);
            double dz = sep_fast(xs[2 * n + j], pz, g.box[2], half[2], g.periodic);
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < H2) {
                double q = sqrt(r2) * iH;
                double w = spline_w(q);
                sw += w;
                sdw += 3.0 * w + q * spline_dw(q);
            }
          }
        });
        for (int o = 16; o > 0; o >>= 1) {
            sw += __shfl_xor_sync(0xffffffffu, sw, o);
            sdw += __shfl_xor_sync(0xffffffffu, sdw, o);
        }
        double om = kSigma * iH * iH * iH * sw;
        double dom = -kKappa * kSigma * iH * iH * iH * iH * sdw;
        double cb = cbrt(om);
        double f = hd - hp.eta / cb;
        double fp = 1.0 + (hp.eta / 3.0) / (cb * om) * dom;
        om_d = om;
        if (last) { okd = true; break; }
        if (f < 0.0) lod = hd; else hid = hd;
        double step = f / fp;
        if (fabs(f) <= 1e-15 * hd || (hid - lod) <= 1e-14 * hd) { okd = true; break; }
        if (fp > 0.0 && fabs(step) <= 1e-11 * hd) last = true;
        double hn = hd - step;
        if (!last && (it >= 12 || !(hn > lod && hn < hid) || !(fp > 0.0)))
            hn = isinf(hid) ? 1.01 * hd : 0.5 * (lod + hid);
        hd = hn;
    }
    return okd;
}

// The same for one warp, walking the candidates once: the double Newton moves h by far less
// than 1e-4 from the float root, so the particles within 1.0009 of its support radius contain
// every neighbour of every iteration.  Their exact distances are dealt to the lanes in walk
// order (candidate c to lane c mod 32) and kept in registers (kRefineSlots a lane); the
// iterations then sum the spline over them.  A lane that would need more slots, or an
// iterate beyond that radius, sends the warp to refine_h_warp.
constexpr int kRefineSlots = 8;

__device__ bool refine_h_warp_cached(const Grid& g, const double* __restrict__ xs, const uint4* __restrict__ xq,
                                     int64_t n, const HParams& hp, int64_t p, int lane, double& hd, double& om_d) {
    const uint4 q4p = xq[p];
    const uint32_t qx = q4p.x, qy = q4p.y, qz = q4p.z;
    const double px = xs[p], py = xs[n + p], pz = xs[2 * n + p];
    const float pxf = (float)px, pyf = (float)py, pzf = (float)pz;
    const double half[3] = {0.5 * g.box[0], 0.5 * g.box[1], 0.5 * g.box[2]};
    const double h_start = hd;
    const double Rc = kKappa * hd * 1.0009, Rc2 = Rc * Rc;
    const float Hf = (float)(kKappa * hd) * 1.001f, H2f = Hf * Hf;
    double r[kRefineSlots];
    int cnt = 0;
    bool over = false;
    int seen = 0;     // candidates of the earlier ranges (walk order)
    for_each_candidate_range(g, pxf, pyf, pzf, Hf, [&](int b, int e) {
        const int first = (lane - seen) & 31;    // this lane's first candidate of the range
        for (int j = b + first; j < e; j += 32) {
            float dxf = fsep(xq[j].x, qx, hp.scale[0]);
            float dyf = fsep(xq[j].y, qy, hp.scale[1]);
            float dzf = fsep(xq[j].z, qz, hp.scale[2]);
            if (dxf * dxf + dyf * dyf + dzf * dzf >= H2f) continue;
            double dx = sep_fast(xs[j], px, g.box[0], half[0], g.periodic);
            double dy = sep_fast(xs[n + j], py, g.box[1], half[1], g.periodic);
            double dz = sep_fast(xs[2 * n + j], pz, g.box[2], half[2], g.periodic);
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < Rc2) {
                if (cnt < kRefineSlots) {
                    const double rr = sqrt(r2);
#pragma unroll
                    for (int k = 0; k < kRefineSlots; ++k)   // static indices keep r in registers
                        if (k == cnt) r[k] = rr;
                    ++cnt;
                } else {
                    over = true;
                }
            }
        }
        seen += e - b;
    });
    if (__any_sync(0xffffffffu, over)) return refine_h_warp(g, xs, xq, n, hp, p, lane, hd, om_d);
    double lod = 0.0, hid = INFINITY;
    bool okd = false, last = false;
    for (int it = 0; it < 60; ++it) {
        double H = kKappa * hd;
        if (H > Rc) {   // beyond the cached radius (never expected): walk again
            hd = h_start;
            return refine_h_warp(g, xs, xq, n, hp, p, lane, hd, om_d);
        }
        double iH = 1.0 / H;
        double sw = 0.0, sdw = 0.0;
#pragma unroll
        for (int k = 0; k < kRefineSlots; ++k) {
            if (k < cnt && r[k] < H) {
                double q = r[k] * iH;
                double w = spline_w(q);
                sw += w;
                sdw += 3.0 * w + q * spline_dw(q);
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            sw += __shfl_xor_sync(0xffffffffu, sw, o);
            sdw += __shfl_xor_sync(0xffffffffu, sdw, o);
        }
        double om = kSigma * iH * iH * iH * sw;
        double dom = -kKappa * kSigma * iH * iH * iH * iH * sdw;
        double cb = cbrt(om);
        double f = hd - hp.eta / cb;
        double fp = 1.0 + (hp.eta / 3.0) / (cb * om) * dom;
        om_d = om;
        if (last) { okd = true; break; }
        if (f < 0.0) lod = hd; else hid = hd;
        double step = f / fp;
        if (fabs(f) <= 1e-15 * hd || (hid - lod) <= 1e-14 * hd) { okd = true; break; }
        if (fp > 0.0 && fabs(step) <= 1e-11 * hd) last = true;
        double hn = hd - step;
        if (!last && (it >= 12 || !(hn > lod && hn < hid) || !(fp > 0.0)))
            hn = isinf(hid) ? 1.0001 * hd : 0.5 * (lod + hid);
        hd = hn;
    }
    return okd;
}

__global__ void k_h_solve(Grid g, const double* __restrict__ xs, const uint4* __restrict__ xq, int64_t n,
                          HParams hp, const double* __restrict__ h_prev, const int32_t* __restrict__ perm,
                          double* h_out, double* omega_out, float* H2f_out, unsigned long long* hminmax, int* flags,
                          int32_t* refine_list, int* refine_count) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double hd = 0.0, om_d = 0.0;
    bool active = p < n;
    if (active) {
        const float kapf = (float)kKappa;
        const float sigf = (float)kSigma;
        const uint4 q4p = xq[p];
        uint32_t qx = q4p.x, qy = q4p.y, qz = q4p.z;
        double px = xs[p], py = xs[n + p], pz = xs[2 * n + p];
        float pxf = (float)px, pyf = (float)py, pzf = (float)pz;

        // first guess: the particle's h of the previous call (particles move little between
        // calls), else the particle count of the surrounding 27 cells
        float h;
        if (h_prev) {
            h = (float)h_prev[perm[p]];
        } else {
            int cnt = count_27(g, cell_coord(px, g.inv_cell[0], g.nc[0]), cell_coord(py, g.inv_cell[1], g.nc[1]),
                               cell_coord(pz, g.inv_cell[2], g.nc[2]));
            double vol27 = 27.0 * g.cell[0] * g.cell[1] * g.cell[2];
            h = cnt > 1 ? (float)(hp.eta * cbrt(vol27 / (double)cnt)) : (float)hp.h0;
        }
        if (!(h > 0.f) || !(h < (float)hp.h_cap)) h = (float)hp.h0;

        // ---- float phase: Newton on float separations, omega summed in double
        float lo = 0.f, hi = INFINITY;
        const float eta = (float)hp.eta;
        bool ok = false, near = false;
        double sw_last = 0.0;
        for (int it = 0; it < hp.max_iter; ++it) {
            float H = kapf * h;
            float iH = 1.f / H;
            float H2 = H * H;
            double sw = 0.0;
            float sdw = 0.f;
            bool nb = false;
            for_each_candidate_q(g, xq, pxf, pyf, pzf, H, [&](int, uint4 qj) {
                float dx = fsep(qj.x, qx, hp.scale[0]);
                float dy = fsep(qj.y, qy, hp.scale[1]);
                float dz = fsep(qj.z, qz, hp.scale[2]);
                float r2 = dx * dx + dy * dy + dz * dz;
                nb |= fabsf(r2 - H2) < kNearBand * H2;
                if (r2 < H2) {
                    float q = sqrtf(r2) * iH;
                    float w = spline_w(q);
                    sw += (double)w;
                    sdw += 3.f * w + q * spline_dw(q);
                }
            });
            sw_last = sw;
            near = nb;
            float om = sigf * iH * iH * iH * (float)sw;
            float dom = -kapf * sigf * iH * iH * iH * iH * sdw;      // d omega / d h
            float cb = cbrtf(om);
            float f = h - eta / cb;
            float fp = 1.f + (eta / 3.f) / (cb * om) * dom;
            if (f < 0.f) lo = h; else hi = h;
            float step = f / fp;
            // converged: residual at the rounding floor, a tiny Newton step, or a collapsed
            // bracket (where f' is small, rounding alone keeps the step above tolerance)
            if (fabsf(f) <= 1e-6f * h || (fp > 0.f && fabsf(step) <= hp.tol32 * h) ||
                (hi - lo) <= hp.tol32 * h) {
                ok = true;
                break;
            }
            float hn = h - step;
            // safeguarded Newton; plain bisection of the bracket after 24 Newton steps
            if (it >= 24 || !(hn > lo && hn < hi) || !(fp > 0.f)) hn = isinf(hi) ? 2.f * h : 0.5f * (lo + hi);
            if (hn > (float)hp.h_cap) hn = (float)hp.h_cap;
            if (hn == h) break;       // no progress possible: reported as not converged
            h = hn;
        }
        if (!ok) atomicExch(&flags[F_NOCONV], 1);
        hd = (double)h;
        {
            double H = kKappa * hd;
            om_d = kSigma / (H * H * H) * sw_last;
        }

        // ---- double phase: Newton on the exact separations to machine precision, here for
        // every particle (FP64 path), else later (k_h_refine) for the near-threshold ones
        if (ok && hp.refine64) {
            if (!refine_h_double(g, xs, xq, n, hp, p, hd, om_d)) atomicExch(&flags[F_NOCONV], 1);
        } else if (ok && near) {
            refine_list[atomicAdd(refine_count, 1)] = (int32_t)p;
        }
        h_out[p] = hd;
        omega_out[p] = om_d;
        double Hd = kKappa * hd;
        H2f_out[p] = (float)(Hd * Hd);
    }
    double mn = active ? hd : INFINITY, mx = active ? hd : 0.0;
    warp_minmax(mn, mx);
    // sum of H^3 (only steers the choice of the pair-search method, never a result)
    double h3 = active ? (kKappa * hd) * (kKappa * hd) * (kKappa * hd) : 0.0;
    for (int o = 16; o > 0; o >>= 1) h3 += __shfl_xor_sync(0xffffffffu, h3, o);
    if ((threadIdx.x & 31) == 0 && mx > 0.0) {
        atomic_min_pos(&hminmax[0], mn);
        atomic_max_pos(&hminmax[1], mx);
        atomicAdd(reinterpret_cast<double*>(&hminmax[4]), h3);
    }
}

// Smoothing lengths given by the caller (rt_neighbours_given_h): h_i from h_in (caller order)
// and omega_i = sum_j W(r_ij, h_i) at it, evaluated like the last iteration of the solve (the
// float path: float weights summed in double; the FP64 path: double).  Non-positive or
// non-finite h sets the F_BADH flag.
__global__ void k_h_given(Grid g, const double* __restrict__ xs, const uint4* __restrict__ xq, int64_t n,
                          HParams hp, const double* __restrict__ h_in, const int32_t* __restrict__ perm,
                          double* h_out, double* omega_out, float* H2f_out, unsigned long long* hminmax, int* flags) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool active = p < n;
    double hd = 0.0;
    if (active) {
        hd = h_in[perm[p]];
        if (!(hd > 0.0) || !(hd < (double)hp.h_cap) || !isfinite(hd)) {
            atomicExch(&flags[F_BADH], 1);
            hd = hp.h0;
        }
        const uint4 q4p = xq[p];
        const uint32_t qx = q4p.x, qy = q4p.y, qz = q4p.z;
        const double px = xs[p], py = xs[n + p], pz = xs[2 * n + p];
        const float pxf = (float)px, pyf = (float)py, pzf = (float)pz;
        const double H = kKappa * hd, iH = 1.0 / H, H2 = H * H;
        double sw = 0.0;
        if (hp.refine64) {
            const double half[3] = {0.5 * g.box[0], 0.5 * g.box[1], 0.5 * g.box[2]};
            const float Hf = (float)H * 1.001f, H2f = Hf * Hf;
            for_each_candidate(g, pxf, pyf, pzf, Hf, [&](int j) {
                float dxf = fsep(xq[j].x, qx, hp.scale[0]);
                float dyf = fsep(xq[j].y, qy, hp.scale[1]);
                float dzf = fsep(xq[j].z, qz, hp.scale[2]);
                if (dxf * dxf + dyf * dyf + dzf * dzf >= H2f) return;
                double dx = sep_fast(xs[j], px, g.box[0], half[0], g.periodic);
                double dy = sep_fast(xs[n + j], py, g.box[1], half[1], g.periodic);
                double dz = sep_fast(xs[2 * n + j], pz, g.box[2], half[2], g.periodic);
                double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 < H2) sw += spline_w(sqrt(r2) * iH);
            });
        } else {
            const float Hf = (float)H, iHf = 1.f / Hf, H2f = Hf * Hf;
            for_each_candidate(g, pxf, pyf, pzf, Hf, [&](int j) {
                float dx = fsep(xq[j].x, qx, hp.scale[0]);
                float dy = fsep(xq[j].y, qy, hp.scale[1]);
                float dz = fsep(xq[j].z, qz, hp.scale[2]);
                float r2 = dx * dx + dy * dy + dz * dz;
                if (r2 < H2f) sw += (double)spline_w(sqrtf(r2) * iHf);
            });
        }
        h_out[p] = hd;
        omega_out[p] = kSigma * iH * iH * iH * sw;
        H2f_out[p] = (float)(H * H);
    }
    double mn = active ? hd : INFINITY, mx = active ? hd : 0.0;
    warp_minmax(mn, mx);
    double h3 = active ? (kKappa * hd) * (kKappa * hd) * (kKappa * hd) : 0.0;
    for (int o = 16; o > 0; o >>= 1) h3 += __shfl_xor_sync(0xffffffffu, h3, o);
    if ((threadIdx.x & 31) == 0 && mx > 0.0) {
        atomic_min_pos(&hminmax[0], mn);
        atomic_max_pos(&hminmax[1], mx);
        atomicAdd(reinterpret_cast<double*>(&hminmax[4]), h3);
    }
}

// Float path: the double phase for the particles k_h_solve flagged, one warp per particle
// (grid-stride over the list; its order is arbitrary, and each particle's result depends on
// its own position and neighbours only).  The smallest and largest h are widened to the
// refined values (the pair search's bound must cover them).
__global__ void k_h_refine(Grid g, const double* __restrict__ xs, const uint4* __restrict__ xq, int64_t n,
                           HParams hp, const int32_t* __restrict__ list, const int* __restrict__ count, double* h_out,
                           double* omega_out, float* H2f_out, unsigned long long* hminmax, int* flags) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int cnt = *count;
    for (int64_t t = w0; t < cnt; t += nw) {
        const int64_t p = list[t];
        double hd = h_out[p], om_d = omega_out[p];
        const bool ok = refine_h_warp_cached(g, xs, xq, n, hp, p, lane, hd, om_d);
        if (lane == 0) {
            if (!ok) atomicExch(&flags[F_NOCONV], 1);
            h_out[p] = hd;
            omega_out[p] = om_d;
            const double Hd = kKappa * hd;
            H2f_out[p] = (float)(Hd * Hd);
            atomic_min_pos(&hminmax[0], hd);
            atomic_max_pos(&hminmax[1], hd);
        }
    }
}

// ------------------------------------------------------------------------------------
// a3: symmetric pair lists { j != i : r_ij < max(H_i, H_j) }.  A float test on the
// fixed-point separation decides all pairs except those within 1e-5 of the threshold,
// which are decided by the exact double test (r^2 and H^2 without contraction).
struct PairParams {
    float scale[3];
    double Hmax;
};

// Local search radii of the direct pair search.  A pair with r_ij < H_j > H_i must be found
// from i, so i searches out to max(H_i, H_j) for every j that can reach it.  Over a coarse
// grid of at most 16^3 blocks, Hb[B] is the largest H in block B and Hreach[A] the largest
// Hb[B] over the blocks B whose box lies within Hb[B] of A's box (A included): every j that
// reaches a particle of A has H_j <= Hreach[A], so max(H_i, Hreach[A]) bounds i's search.
struct Blocks {
    int nb[3];
    double len[3];      // block edge per axis
    int reach[3];       // blocks per axis within H_max of a block (no block farther can qualify)
    int periodic;
};

__device__ __forceinline__ int block_of(const Blocks& bk, double x, double y, double z) {
    const double p[3] = {x, y, z};
    int b[3];
    for (int a = 0; a < 3; ++a) {
        int v = (int)floor(p[a] / bk.len[a]);
        b[a] = v < 0 ? 0 : (v >= bk.nb[a] ? bk.nb[a] - 1 : v);
    }
    return (b[2] * bk.nb[1] + b[1]) * bk.nb[0] + b[0];
}

// Hb (float bits, ordered like integers for H > 0) of every block; the lanes of a warp that
// fall in the same block (particles are sorted by cell) combine before one atomic
// Also stores each particle's float H^2 in the free word of its position record, so that the
// pair search reads a candidate's position and support radius with one 16-byte load.
__global__ void k_block_hmax(const double* __restrict__ xs, const float* __restrict__ H2f, int64_t n, Blocks bk,
                             unsigned* __restrict__ hb, uint4* __restrict__ xq) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool in = p < n;
    const int b = in ? block_of(bk, xs[p], xs[n + p], xs[2 * n + p]) : -1;
    const float h2 = in ? H2f[p] : 0.f;
    if (in) reinterpret_cast<unsigned*>(xq + p)[3] = __float_as_uint(h2);
    const unsigned v = in ? __float_as_uint(sqrtf(h2)) : 0u;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const unsigned m = __reduce_max_sync(peers, v);
    if (in && (threadIdx.x & 31) == __ffs(peers) - 1) atomicMax(&hb[b], m);
}

// Hreach of every block: one warp per block A, its lanes scanning the blocks B within
// bk.reach blocks of A along each axis (each block once, also where that span wraps)
__global__ void k_block_reach(const unsigned* __restrict__ hb, Blocks bk, float* __restrict__ reach) {
    const int nbt = bk.nb[0] * bk.nb[1] * bk.nb[2];
    const int A = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (A >= nbt) return;      // whole warps
    const int a[3] = {A % bk.nb[0], (A / bk.nb[0]) % bk.nb[1], A / (bk.nb[0] * bk.nb[1])};
    const float len[3] = {(float)bk.len[0], (float)bk.len[1], (float)bk.len[2]};
    // the scanned span per axis: [a - k, a + k] wrapped (or clipped), or the whole axis
    int lo[3], w[3];
    for (int x = 0; x < 3; ++x) {
        const int k = bk.reach[x];
        if (2 * k + 1 >= bk.nb[x]) {
            lo[x] = 0;
            w[x] = bk.nb[x];
        } else if (bk.periodic) {
            lo[x] = a[x] - k;
            w[x] = 2 * k + 1;
        } else {
            lo[x] = max(a[x] - k, 0);
            w[x] = min(a[x] + k, bk.nb[x] - 1) - lo[x] + 1;
        }
    }
    const int span = w[0] * w[1] * w[2];
    unsigned r = hb[A];
    for (int t = lane; t < span; t += 32) {
        int b[3] = {lo[0] + t % w[0], lo[1] + (t / w[0]) % w[1], lo[2] + t / (w[0] * w[1])};
        for (int x = 0; x < 3; ++x) b[x] = (b[x] % bk.nb[x] + bk.nb[x]) % bk.nb[x];
        const int Bi = (b[2] * bk.nb[1] + b[1]) * bk.nb[0] + b[0];
        const unsigned hbB = hb[Bi];
        if (hbB <= r) continue;
        const float Hb = __uint_as_float(hbB);
        float d2 = 0.f;
        for (int x = 0; x < 3; ++x) {
            int d = abs(a[x] - b[x]);
            if (bk.periodic) d = min(d, bk.nb[x] - d);
            const float gap = d > 1 ? (d - 1) * len[x] : 0.f;
            d2 += gap * gap;
        }
        // the gap between the boxes, with a relative margin against rounding
        if (d2 < Hb * Hb * 1.0002f) r = hbB;
    }
    r = __reduce_max_sync(0xffffffffu, r);
    if (lane == 0) reach[A] = __uint_as_float(r);
}

// FILL = false counts each row into counts[p]; with cap > 0 it also writes the first cap
// entries of row p to cols[p cap ...] and raises *row_max to the longest row.  FILL = true
// writes row p to cols[row_off[p] ...].  Both walk the candidates in ascending index, so
// every row comes out in ascending column order.
template <bool FILL>
__global__ void k_pairs(Grid g, const double* __restrict__ xs, const uint4* __restrict__ xq,
                        const double* __restrict__ h, const float* __restrict__ H2f, int64_t n, PairParams pp,
                        Blocks bk, const float* __restrict__ reach, int32_t* counts,
                        const int64_t* __restrict__ row_off, int32_t* cols, int cap = 0, int* row_max = nullptr) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int cnt = 0;
    if (p < n) {
        const uint4 q4p = xq[p];
        uint32_t qx = q4p.x, qy = q4p.y, qz = q4p.z;
        double px = xs[p], py = xs[n + p], pz = xs[2 * n + p];
        const float H2i = H2f[p];
        const float Hr = reach[block_of(bk, px, py, pz)];
        float R = sqrtf(fmaxf(H2i, Hr * Hr)) * 1.0001f;
        int64_t base = FILL ? row_off[p] : p * (int64_t)cap;
        for_each_candidate_q<true>(g, xq, (float)px, (float)py, (float)pz, R, [&](int j, uint4 qj) {
            if (j == p) return;
            float dx = fsep(qj.x, qx, pp.scale[0]);
            float dy = fsep(qj.y, qy, pp.scale[1]);
            float dz = fsep(qj.z, qz, pp.scale[2]);
            float r2f = dx * dx + dy * dy + dz * dz;
            float H2m = fmaxf(H2i, __uint_as_float(qj.w));   // H_j^2 (k_block_hmax)
            bool in;
            if (r2f < H2m * (1.f - 1e-5f)) in = true;
            else if (r2f > H2m * (1.f + 1e-5f)) in = false;
            else {
                // exact double test (no contraction), as a plain double evaluation would do it
                double Hm = fmax(__dmul_rn(kKappa, h[p]), __dmul_rn(kKappa, h[j]));
                double ex = sep_exact(xs[j], px, g.box[0], g.periodic);
                double ey = sep_exact(xs[n + j], py, g.box[1], g.periodic);
                double ez = sep_exact(xs[2 * n + j], pz, g.box[2], g.periodic);
                in = norm2_exact(ex, ey, ez) < __dmul_rn(Hm, Hm);
            }
            if (in) {
                if (FILL || cnt < cap) cols[base + cnt] = j;
                ++cnt;
            }
        });
        if (!FILL) counts[p] = cnt;
    }
    if (!FILL && row_max) {   // every lane of the (full) warp takes part
        const int m = __reduce_max_sync(0xffffffffu, cnt);
        if ((threadIdx.x & 31) == 0) atomicMax(row_max, m);
    }
}

// rows of cap entries (k_pairs' counting walk) -> CSR rows at row_off, one warp per row
__global__ void k_rows_compact(const int32_t* __restrict__ cols_cap, int64_t cap, const int64_t* __restrict__ row_off,
                               int64_t n, int32_t* __restrict__ cols) {
    const int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= n) return;
    const int64_t b = row_off[p], m = row_off[p + 1] - b;
    for (int64_t k = lane; k < m; k += 32) cols[b + k] = cols_cap[p * cap + k];
}


// Rows sorted ascending are [lower neighbours j < i | upper neighbours j > i].  Each
// unordered pair is the upper entry of its lower particle; slot(i, j) numbers those entries.
__global__ void k_row_split(const int64_t* __restrict__ row_off, const int32_t* __restrict__ cols, int64_t n,
                            int32_t* n_low, int32_t* n_up) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t lo = row_off[i], hi = row_off[i + 1];
    int64_t b = lo, e = hi;
    while (b < e) {
        int64_t m = (b + e) >> 1;
        if (cols[m] < (int32_t)i) b = m + 1; else e = m;
    }
    n_low[i] = (int32_t)(b - lo);
    n_up[i] = (int32_t)(hi - b);
}

// the two particles of every pair slot
__global__ void k_pair_ends(const int64_t* __restrict__ row_off, const int32_t* __restrict__ cols,
                            const int32_t* __restrict__ n_low, const int64_t* __restrict__ up_off, int64_t n,
                            int2* ends) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t e0 = row_off[i] + n_low[i], e1 = row_off[i + 1], slot = up_off[i];
    for (int64_t e = e0; e < e1; ++e, ++slot) ends[slot] = make_int2((int)i, cols[e]);
}

// for every lower entry (i, k), k < i: the slot of the pair in k's upper list.  One warp per
// particle, its lanes taking the lower entries (each a binary search in row k's upper part).
__global__ void k_low_slots(const int64_t* __restrict__ row_off, const int32_t* __restrict__ cols,
                            const int32_t* __restrict__ n_low, const int64_t* __restrict__ up_off, int64_t n,
                            int32_t* low_slot) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    int64_t r0 = row_off[i];
    int64_t lbase = r0 - up_off[i];       // lower entries before row i
    for (int e = lane; e < n_low[i]; e += 32) {
        int k = cols[r0 + e];
        int64_t b = row_off[k] + n_low[k], hi = row_off[k + 1], t = hi;
        while (b < t) {
            int64_t m = (b + t) >> 1;
            if (cols[m] < (int32_t)i) b = m + 1; else t = m;
        }
        low_slot[lbase + e] = (int32_t)(up_off[k] + (b - row_off[k] - n_low[k]));
    }
}

// Pair search for strongly varying h: each particle lists only { j : r_ij < H_i } (its own
// support) and emits the entry and its transpose as 64-bit keys (row << 32 | col); sorting
// and removing duplicates gives the same symmetric lists, rows ascending, without any
// particle searching out to the largest H of the set.
template <bool FILL>
__global__ void k_pairs_gather(Grid g, const double* __restrict__ xs, const uint4* __restrict__ xq,
                               const double* __restrict__ h, const float* __restrict__ H2f, int64_t n, PairParams pp,
                               int32_t* counts, const int64_t* __restrict__ off, uint64_t* keys) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const uint4 q4p = xq[p];
    uint32_t qx = q4p.x, qy = q4p.y, qz = q4p.z;
    double px = xs[p], py = xs[n + p], pz = xs[2 * n + p];
    const float H2i = H2f[p];
    int cnt = 0;
    int64_t base = FILL ? off[p] : 0;
    for_each_candidate(g, (float)px, (float)py, (float)pz, sqrtf(H2i) * 1.0001f, [&](int j) {
        if (j == p) return;
        float dx = fsep(xq[j].x, qx, pp.scale[0]);
        float dy = fsep(xq[j].y, qy, pp.scale[1]);
        float dz = fsep(xq[j].z, qz, pp.scale[2]);
        float r2f = dx * dx + dy * dy + dz * dz;
        bool in;
        if (r2f < H2i * (1.f - 1e-5f)) in = true;
        else if (r2f > H2i * (1.f + 1e-5f)) in = false;
        else {
            double Hi = __dmul_rn(kKappa, h[p]);
            double ex = sep_exact(xs[j], px, g.box[0], g.periodic);
            double ey = sep_exact(xs[n + j], py, g.box[1], g.periodic);
            double ez = sep_exact(xs[2 * n + j], pz, g.box[2], g.periodic);
            in = norm2_exact(ex, ey, ez) < __dmul_rn(Hi, Hi);
        }
        if (in) {
            if (FILL) {
                keys[2 * (base + cnt)] = ((uint64_t)p << 32) | (uint32_t)j;
                keys[2 * (base + cnt) + 1] = ((uint64_t)(uint32_t)j << 32) | (uint64_t)p;
            }
            ++cnt;
        }
    });
    if (!FILL) counts[p] = cnt;
}

// unique sorted keys -> columns, and the number of entries of every row
__global__ void k_keys_to_csr(const uint64_t* __restrict__ ukeys, const int64_t* __restrict__ nuniq, int32_t* cols,
                              int32_t* counts) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= *nuniq) return;
    uint64_t k = ukeys[e];
    cols[e] = (int32_t)(uint32_t)(k & 0xffffffffu);
    atomicAdd(&counts[(int64_t)(k >> 32)], 1);
}

// ------------------------------------------------------------------------------------
// a4: E_i = sum_j psi_j(x_i) d d^T, B_i = E_i^-1 (double), and the per-particle factors used
// by the pair kernels.
__device__ void sym3_eigs(double a, double b, double c, double d, double e, double f, double ev[3]) {
    // symmetric [[a d e][d b f][e f c]]: trigonometric closed form
    double p1 = d * d + e * e + f * f;
    double q = (a + b + c) / 3.0;
    if (p1 == 0.0) { ev[0] = a; ev[1] = b; ev[2] = c; return; }
    double p2 = (a - q) * (a - q) + (b - q) * (b - q) + (c - q) * (c - q) + 2.0 * p1;
    double p = sqrt(p2 / 6.0);
    double ip = 1.0 / p;
    double B00 = (a - q) * ip, B11 = (b - q) * ip, B22 = (c - q) * ip, B01 = d * ip, B02 = e * ip, B12 = f * ip;
    double detB = B00 * (B11 * B22 - B12 * B12) - B01 * (B01 * B22 - B12 * B02) + B02 * (B01 * B12 - B11 * B02);
    double r = fmin(fmax(detB / 2.0, -1.0), 1.0);
    double phi = acos(r) / 3.0;
    ev[0] = q + 2.0 * p * cos(phi);
    ev[2] = q + 2.0 * p * cos(phi + 2.0943951023931954923);
    ev[1] = 3.0 * q - ev[0] - ev[2];
}

template <class T>
__device__ __forceinline__ void store_pos(void* pos, int64_t p, const double* xs, const uint4* xq, int64_t n);
template <>
__device__ __forceinline__ void store_pos<float>(void* pos, int64_t p, const double*, const uint4* xq, int64_t n) {
    reinterpret_cast<uint4*>(pos)[p] = xq[p];
}
template <>
__device__ __forceinline__ void store_pos<double>(void* pos, int64_t p, const double* xs, const uint4*, int64_t n) {
    double2* d = reinterpret_cast<double2*>(pos) + 2 * p;
    d[0] = make_double2(xs[p], xs[n + p]);
    d[1] = make_double2(xs[2 * n + p], 0.0);
}

// E_i accumulation over the pair list.  Double path: separations and weights in double.
// Float path: separations from the fixed-point positions, weights in float and a
// compensated (Kahan) float sum, so that E_i keeps ~1e-8 relative accuracy before its
// inversion in double.
struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        float y = v - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <class T>
__device__ __forceinline__ void accumulate_E(const double* xs, const uint4* xq, const double* box, int periodic,
                                             float s0, float s1, float s2, int64_t n, int64_t p, double H,
                                             const int64_t* row_off, const int32_t* cols, double E[6]);

template <>
__device__ __forceinline__ void accumulate_E<double>(const double* xs, const uint4*, const double* box,
                                                     int periodic, float, float, float, int64_t n, int64_t p,
                                                     double H, const int64_t* row_off, const int32_t* cols,
                                                     double E[6]) {
    const double half[3] = {0.5 * box[0], 0.5 * box[1], 0.5 * box[2]};
    double px = xs[p], py = xs[n + p], pz = xs[2 * n + p];
    double iH = 1.0 / H, H2 = H * H;
    for (int k = 0; k < 6; ++k) E[k] = 0.0;
    for (int64_t e = row_off[p]; e < row_off[p + 1]; ++e) {
        int j = cols[e];
        double dx = sep_fast(xs[j], px, box[0], half[0], periodic);
        double dy = sep_fast(xs[n + j], py, box[1], half[1], periodic);
        double dz = sep_fast(xs[2 * n + j], pz, box[2], half[2], periodic);
        double r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 < H2)) continue;
        double w = spline_w(sqrt(r2) * iH);
        E[0] += w * dx * dx; E[1] += w * dy * dy; E[2] += w * dz * dz;
        E[3] += w * dx * dy; E[4] += w * dx * dz; E[5] += w * dy * dz;
    }
}

template <>
__device__ __forceinline__ void accumulate_E<float>(const double*, const uint4* xq, const double*, int, float s0,
                                                    float s1, float s2, int64_t n, int64_t p, double H,
                                                    const int64_t* row_off, const int32_t* cols, double E[6]) {
    const uint4 q4p = xq[p];
    uint32_t qx = q4p.x, qy = q4p.y, qz = q4p.z;
    float iH = (float)(1.0 / H), H2 = (float)(H * H);
    Kahan acc[6];
    for (int64_t e = row_off[p]; e < row_off[p + 1]; ++e) {
        int j = cols[e];
        float dx = fsep(xq[j].x, qx, s0), dy = fsep(xq[j].y, qy, s1), dz = fsep(xq[j].z, qz, s2);
        float r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 < H2)) continue;
        float w = spline_w(sqrtf(r2) * iH);
        acc[0].add(w * dx * dx); acc[1].add(w * dy * dy); acc[2].add(w * dz * dz);
        acc[3].add(w * dx * dy); acc[4].add(w * dx * dz); acc[5].add(w * dy * dz);
    }
    for (int k = 0; k < 6; ++k) E[k] = acc[k].value();
}

// Also writes the pair kernels' records: position, {1/H, h, Bp (6)} with
// Bp = V^2 sigma / H^3 B (so that V_i psitilde_j(x_i) = Bp_i d w(q)), and omega; reduces
// max cond_2(E_i) and min V_i into red[2], red[3].
template <class T>
__global__ void k_geometry(const double* __restrict__ xs, const uint4* __restrict__ xq,
                           const double* __restrict__ h, const double* __restrict__ omega,
                           const int64_t* __restrict__ row_off, const int32_t* __restrict__ cols, int64_t n, double b0,
                           double b1, double b2, int periodic, float s0, float s1, float s2, double* V_out,
                           double* B_out, double* cond_out, void* pos_t, T* geo_t, T* om_t,
                           unsigned long long* red, int* flags) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double cond = 0.0, V = INFINITY;
    if (p < n) {
        const double box[3] = {b0, b1, b2};
        double hi = h[p], H = kKappa * hi, iH = 1.0 / H;
        double om = omega[p];
        double E[6];
        accumulate_E<T>(xs, xq, box, periodic, s0, s1, s2, n, p, H, row_off, cols, E);
        double fac = kSigma * iH * iH * iH / om;   // psi = fac * w
        double e_xx = E[0] * fac, e_yy = E[1] * fac, e_zz = E[2] * fac;
        double e_xy = E[3] * fac, e_xz = E[4] * fac, e_yz = E[5] * fac;
        // cofactor inverse of the symmetric matrix
        double c_xx = e_yy * e_zz - e_yz * e_yz;
        double c_xy = e_xz * e_yz - e_xy * e_zz;
        double c_xz = e_xy * e_yz - e_xz * e_yy;
        double det = e_xx * c_xx + e_xy * c_xy + e_xz * c_xz;
        V = 1.0 / om;
        V_out[p] = V;
        store_pos<T>(pos_t, p, xs, xq, n);
        if (!(det > 0.0) || !(om > 0.0)) {
            atomicExch(&flags[F_GEOM], 1);
            for (int k = 0; k < 6; ++k) B_out[k * n + p] = 0.0;
            for (int k = 0; k < 8; ++k) geo_t[8 * p + k] = (T)0;
            om_t[p] = (T)0;
            cond_out[p] = INFINITY;
            cond = INFINITY;
        } else {
            double id = 1.0 / det;
            double B[6];
            B[0] = c_xx * id;
            B[1] = (e_xx * e_zz - e_xz * e_xz) * id;
            B[2] = (e_xx * e_yy - e_xy * e_xy) * id;
            B[3] = c_xy * id;
            B[4] = c_xz * id;
            B[5] = (e_xy * e_xz - e_xx * e_yz) * id;
            double ev[3];
            sym3_eigs(e_xx, e_yy, e_zz, e_xy, e_xz, e_yz, ev);
            double lmin = fmin(ev[0], fmin(ev[1], ev[2])), lmax = fmax(ev[0], fmax(ev[1], ev[2]));
            cond = lmin > 0 ? lmax / lmin : INFINITY;
            cond_out[p] = cond;
            if (!(lmin > 0)) atomicExch(&flags[F_GEOM], 1);
            if (cond > 1e10) atomicAdd(&flags[F_ILL], 1);
            double bp = V * V * kSigma * iH * iH * iH;   // V_i psitilde_j(x_i) = Bp_i d w(q_ij)
            geo_t[8 * p] = (T)iH;
            geo_t[8 * p + 1] = (T)hi;
            for (int k = 0; k < 6; ++k) {
                B_out[k * n + p] = B[k];
                geo_t[8 * p + 2 + k] = (T)(bp * B[k]);
            }
            om_t[p] = (T)om;
        }
    }
    double vmin = V, cmax = cond;
    warp_minmax(vmin, cmax);
    if ((threadIdx.x & 31) == 0) {
        if (cmax > 0.0) atomic_max_pos(&red[2], cmax);
        if (vmin < INFINITY) atomic_min_pos(&red[3], vmin);
    }
}

// ------------------------------------------------------------------------------------
// a5 preparation: per source, h_s = eta_s omega_s(h_s)^(-1/3) over gas only (no self term),
// octant sums w_a of psi, mu_a = sum_b w_b / (q_nz w_a), xi = mu_a psi.  One warp per source.
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct SrcParams {
    double eta, h0, h_cap;
    int max_iter;
    int warm;       // start from the h of the last call (in hs_out), else from h0
    int fixed;      // hs_out holds given smoothing lengths: only omega_s at them
};

// Rows of the culled walk of for_each_candidate handed out round-robin to the threads of a
// block (thread t takes rows t, t + nt, ...).
template <class F>
__device__ __forceinline__ void strided_rows(const Grid& g, float px, float py, float pz, float R, int t, int nt,
                                             F&& f) {
    const float Rc = R * 1.0001f + 1e-6f * (g.cellf[0] + g.cellf[1] + g.cellf[2]);
    const float R2 = Rc * Rc;
    const float p[3] = {px, py, pz};
    int lo[3], hi[3];
    bool all[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = (int)floorf((p[a] - Rc) * g.inv_cellf[a]);
        hi[a] = (int)floorf((p[a] + Rc) * g.inv_cellf[a]);
        all[a] = (hi[a] - lo[a] + 1 >= g.nc[a]);
        if (all[a]) {
            lo[a] = 0;
            hi[a] = g.nc[a] - 1;
        } else if (!g.periodic) {
            lo[a] = max(lo[a], 0);
            hi[a] = min(hi[a], g.nc[a] - 1);
        }
    }
    const int ny = hi[1] - lo[1] + 1;
    const int nrows = (hi[2] - lo[2] + 1) * ny;
    for (int r = t; r < nrows; r += nt) {
        int z = lo[2] + r / ny, y = lo[1] + r % ny;
        float dz = all[2] ? 0.f : fmaxf(0.f, fmaxf(z * g.cellf[2] - pz, pz - (z + 1) * g.cellf[2]));
        float dy = all[1] ? 0.f : fmaxf(0.f, fmaxf(y * g.cellf[1] - py, py - (y + 1) * g.cellf[1]));
        float rem = R2 - dy * dy - dz * dz;
        if (rem <= 0.f) continue;
        int zz = wrap_cell(z, g.nc[2]), yy = wrap_cell(y, g.nc[1]);
        int64_t base = ((int64_t)zz * g.nc[1] + yy) * g.nc[0];
        int xa, xb;
        if (all[0]) {
            xa = 0;
            xb = g.nc[0] - 1;
        } else {
            float w = sqrtf(rem);
            xa = (int)floorf((px - w) * g.inv_cellf[0]);
            xb = (int)floorf((px + w) * g.inv_cellf[0]);
            if (!g.periodic) {
                xa = max(xa, 0);
                xb = min(xb, g.nc[0] - 1);
            }
        }
        int sl[2], sh[2], ns = 0;
        if (xa < 0) { sl[ns] = xa + g.nc[0]; sh[ns++] = g.nc[0] - 1; sl[ns] = 0; sh[ns++] = xb; }
        else if (xb >= g.nc[0]) { sl[ns] = xa; sh[ns++] = g.nc[0] - 1; sl[ns] = 0; sh[ns++] = xb - g.nc[0]; }
        else { sl[ns] = xa; sh[ns++] = xb; }
        for (int sI = 0; sI < ns; ++sI) {
            int b = g.cell_start[base + sl[sI]];
            int e = g.cell_start[base + sh[sI] + 1];
            for (int j = b; j < e; ++j) f(j);
        }
    }
}

constexpr int kSrcThreads = 128;

// one block per source: Newton on h_s = eta_s omega_s(h_s)^(-1/3) over gas only (no self
// term), omega summed over the rows of all threads in a fixed tree order
__global__ void __launch_bounds__(kSrcThreads) k_src_h(Grid g, const double* __restrict__ xs, int64_t n,
                                                       const double* __restrict__ xsrc, int64_t S, SrcParams sp,
                                                       double* hs_out, double* oms_out, int* flags) {
    const int s_id = blockIdx.x;
    const int t = threadIdx.x;
    __shared__ double red_w[kSrcThreads], red_dw[kSrcThreads];
    double p[3] = {xsrc[s_id], xsrc[S + s_id], xsrc[2 * S + s_id]};
    const double half[3] = {0.5 * g.box[0], 0.5 * g.box[1], 0.5 * g.box[2]};
    double h = (sp.warm || sp.fixed) ? hs_out[s_id] : sp.h0, lo = 0.0, hi = INFINITY, om = 0.0;
    bool ok = false;
    if (!(h > 0.0) || !(h < sp.h_cap)) {
        if (sp.fixed && t == 0) atomicExch(&flags[F_BADH], 1);
        h = sp.h0;
    }
    __syncthreads();    // every thread has read the first guess before thread 0 overwrites it
    for (int it = 0; it < sp.max_iter; ++it) {
        double H = kKappa * h, iH = 1.0 / H, H2 = H * H;
        double sw = 0.0, sdw = 0.0;
        strided_rows(g, (float)p[0], (float)p[1], (float)p[2], (float)H, t, kSrcThreads, [&](int j) {
            double dx = sep_fast(xs[j], p[0], g.box[0], half[0], g.periodic);
            double dy = sep_fast(xs[n + j], p[1], g.box[1], half[1], g.periodic);
            double dz = sep_fast(xs[2 * n + j], p[2], g.box[2], half[2], g.periodic);
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < H2) {
                double q = sqrt(r2) * iH;
                double w = spline_w(q);
                sw += w;
                sdw += 3.0 * w + q * spline_dw(q);
            }
        });
        red_w[t] = sw;
        red_dw[t] = sdw;
        __syncthreads();
        for (int w = kSrcThreads / 2; w > 0; w >>= 1) {
            if (t < w) {
                red_w[t] += red_w[t + w];
                red_dw[t] += red_dw[t + w];
            }
            __syncthreads();
        }
        sw = red_w[0];
        sdw = red_dw[0];
        __syncthreads();
        om = kSigma * iH * iH * iH * sw;
        if (sp.fixed) {   // given h: omega there, no iteration
            ok = om > 0.0;
            break;
        }
        double f, fp;
        if (om > 0.0) {
            double dom = -kKappa * kSigma * iH * iH * iH * iH * sdw;
            double cb = cbrt(om);
            f = h - sp.eta / cb;
            fp = 1.0 + (sp.eta / 3.0) / (cb * om) * dom;
        } else {
            f = -INFINITY;
            fp = 0.0;
        }
        if (f < 0.0) lo = h; else hi = h;
        double step = (om > 0.0) ? f / fp : -INFINITY;
        if (om > 0.0 && !(fabs(step) > 2e-16 * h)) { ok = true; break; }
        double hn = h - step;
        if (!(hn > lo && hn < hi) || !(fp > 0.0)) hn = isinf(hi) ? 1.5 * h : 0.5 * (lo + hi);
        if (hn > sp.h_cap) hn = sp.h_cap;
        if (hn == h) { ok = om > 0.0; break; }
        h = hn;
    }
    if (t == 0) {
        if (!ok) atomicExch(&flags[F_SRC_NOCONV], 1);
        hs_out[s_id] = h;
        oms_out[s_id] = om;
    }
}

// The (z, y) rows of the cell cube [c - k, c + k] around a source, numbered
// z-major; row r's particles are one or two contiguous ranges of the sorted order.
struct CubeRows {
    int lo[3], hi[3];
    int ny, rows;
};

__device__ __forceinline__ CubeRows cube_rows(const Grid& g, const int c0[3], const int k[3]) {
    CubeRows cr;
    for (int a = 0; a < 3; ++a) {
        bool all = (2 * k[a] + 1 >= g.nc[a]);
        cr.lo[a] = all ? 0 : c0[a] - k[a];
        cr.hi[a] = all ? g.nc[a] - 1 : c0[a] + k[a];
        if (!g.periodic && !all) {
            cr.lo[a] = max(cr.lo[a], 0);
            cr.hi[a] = min(cr.hi[a], g.nc[a] - 1);
        }
    }
    cr.ny = cr.hi[1] - cr.lo[1] + 1;
    cr.rows = cr.ny * (cr.hi[2] - cr.lo[2] + 1);
    return cr;
}

// every lane walks row r of the cube, lane l taking every 32nd candidate
template <class F>
__device__ __forceinline__ void warp_row(const Grid& g, const CubeRows& cr, int r, int lane, F&& f) {
    const int zz = wrap_cell(cr.lo[2] + r / cr.ny, g.nc[2]);
    const int yy = wrap_cell(cr.lo[1] + r % cr.ny, g.nc[1]);
    const int64_t base = ((int64_t)zz * g.nc[1] + yy) * g.nc[0];
    const int xa = cr.lo[0], xb = cr.hi[0];
    int sl[2], sh[2], ns = 0;
    if (xa < 0) { sl[ns] = xa + g.nc[0]; sh[ns++] = g.nc[0] - 1; sl[ns] = 0; sh[ns++] = xb; }
    else if (xb >= g.nc[0]) { sl[ns] = xa; sh[ns++] = g.nc[0] - 1; sl[ns] = 0; sh[ns++] = xb - g.nc[0]; }
    else { sl[ns] = xa; sh[ns++] = xb; }
    for (int q = 0; q < ns; ++q) {
        const int b = g.cell_start[base + sl[q]];
        const int e = g.cell_start[base + sh[q] + 1];
        for (int j0 = b; j0 < e; j0 += 32) f(j0 + lane, j0 + lane < e);
    }
}

constexpr int kSrcWarps = 8, kSrcRowsMax = 1024;

// Count (FILL = false) or write (FILL = true) the gas entries of every source, one block of
// kSrcWarps warps per source.  The cube's rows are dealt to the warps (row r to warp
// r mod kSrcWarps); the fill pass first counts every row, scans the counts in row order and
// then writes each row's entries from its offset, so the entries come in the row-major
// candidate order of a single warp's walk.  Cubes of more than kSrcRowsMax rows are walked
// by warp 0 alone.  The fill pass also forms xi, from the octant sums of its own entries or,
// when octw_given is set, from the caller's (a source's owner's, over its whole support).
template <bool FILL>
__global__ void __launch_bounds__(kSrcWarps * 32)
k_src_entries(Grid g, const double* __restrict__ xs, int64_t n, const double* __restrict__ xsrc, int64_t S,
              const double* __restrict__ hs, const double* __restrict__ oms, int32_t* counts,
              const int64_t* __restrict__ off, int32_t* e_gas, double* e_xi, double* octw_out,
              const double* __restrict__ octw_given = nullptr) {
    __shared__ int row_n[kSrcRowsMax];
    __shared__ double w8s[kSrcWarps][8];
    __shared__ int total;
    const int src = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const double p[3] = {xsrc[src], xsrc[S + src], xsrc[2 * S + src]};
    int c[3];
    for (int a = 0; a < 3; ++a) c[a] = cell_coord(p[a], g.inv_cell[a], g.nc[a]);
    const double half[3] = {0.5 * g.box[0], 0.5 * g.box[1], 0.5 * g.box[2]};
    const double h = hs[src], H = kKappa * h, iH = 1.0 / H, H2 = H * H;
    const double fac = kSigma * iH * iH * iH / oms[src];
    int k[3];
    for (int a = 0; a < 3; ++a) k[a] = (int)ceil(H * g.inv_cell[a]);
    const CubeRows cr = cube_rows(g, c, k);
    const bool split = cr.rows <= kSrcRowsMax;
    const int nw = split ? kSrcWarps : 1;
    // candidate j of the source's support?  psi and octant when it is
    auto test = [&](int j, bool act, double& ps, int& oct) {
        if (!act) return false;
        const double dx = sep_fast(xs[j], p[0], g.box[0], half[0], g.periodic);
        const double dy = sep_fast(xs[n + j], p[1], g.box[1], half[1], g.periodic);
        const double dz = sep_fast(xs[2 * n + j], p[2], g.box[2], half[2], g.periodic);
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 < H2)) return false;
        ps = fac * spline_w(sqrt(r2) * iH);
        oct = (dx < 0 ? 1 : 0) | (dy < 0 ? 2 : 0) | (dz < 0 ? 4 : 0);
        return true;
    };
    // pass 1: entries per row (per warp when the rows are not split)
    if (threadIdx.x == 0) total = 0;
    __syncthreads();
    int mine = 0;
    if (wid < nw) {
        for (int r = wid; r < cr.rows; r += nw) {
            int cnt = 0;
            warp_row(g, cr, r, lane, [&](int j, bool act) {
                double ps;
                int oct;
                cnt += __popc(__ballot_sync(0xffffffffu, test(j, act, ps, oct)));
            });
            if (split && lane == 0) row_n[r] = cnt;
            mine += cnt;
        }
        if (lane == 0) atomicAdd(&total, mine);
    }
    __syncthreads();
    if (!FILL) {
        if (threadIdx.x == 0) counts[src] = total;
        return;
    }
    // row offsets in row order (exclusive prefix sums of row_n)
    if (split && threadIdx.x == 0) {
        int acc = 0;
        for (int r = 0; r < cr.rows; ++r) {
            const int v = row_n[r];
            row_n[r] = acc;
            acc += v;
        }
    }
    __syncthreads();
    // pass 2: write the entries (psi for now; mu_a applied below) and the octant sums
    const int64_t base = off[src];
    double w8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (wid < nw) {
        int run = 0;
        for (int r = wid; r < cr.rows; r += nw) {
            int pos0 = split ? row_n[r] : run;
            warp_row(g, cr, r, lane, [&](int j, bool act) {
                double ps = 0.0;
                int oct = 0;
                const bool in = test(j, act, ps, oct);
                const unsigned bal = __ballot_sync(0xffffffffu, in);
                if (in) {
                    const int pos = pos0 + __popc(bal & ((1u << lane) - 1u));
                    e_gas[base + pos] = j;
                    e_xi[base + pos] = ps;
                    w8[oct] += ps;
                }
                pos0 += __popc(bal);
            });
            run = pos0;
        }
    }
    for (int a = 0; a < 8; ++a) {
        const double v = warp_sum(w8[a]);
        if (lane == 0) w8s[wid][a] = v;
    }
    __syncthreads();
    // octant sums over the warps in warp order; xi = mu_a psi, mu_a = sum_b w_b / (q_nz w_a)
    double ws8[8], wsum = 0.0;
    int qnz = 0;
    for (int a = 0; a < 8; ++a) {
        double v = 0.0;
        for (int w = 0; w < kSrcWarps; ++w) v += w8s[w][a];
        if (octw_given) v = octw_given[8 * src + a];
        ws8[a] = v;
        wsum += v;
        qnz += (v > 0.0);
    }
    if (threadIdx.x == 0)
        for (int a = 0; a < 8; ++a) octw_out[8 * src + a] = ws8[a];
    __syncthreads();   // the entries of pass 2 are visible to every thread
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int j = e_gas[base + e];
        const double dx = sep_fast(xs[j], p[0], g.box[0], half[0], g.periodic);
        const double dy = sep_fast(xs[n + j], p[1], g.box[1], half[1], g.periodic);
        const double dz = sep_fast(xs[2 * n + j], p[2], g.box[2], half[2], g.periodic);
        const int oct = (dx < 0 ? 1 : 0) | (dy < 0 ? 2 : 0) | (dz < 0 ? 4 : 0);
        e_xi[base + e] = wsum / ((double)qnz * ws8[oct]) * e_xi[base + e];
    }
}

// injection entries keyed by (target, source) so that each target sums its sources in
// source order
__global__ void k_inj_keys(const int32_t* __restrict__ e_gas, const int64_t* __restrict__ off, int64_t S,
                           int64_t total, uint64_t* keys, int32_t* vals) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= total) return;
    // source of entry e by binary search in off
    int64_t lo = 0, hi = S;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= e) lo = mid; else hi = mid;
    }
    keys[e] = ((uint64_t)(uint32_t)e_gas[e] << 32) | (uint64_t)(uint32_t)lo;
    vals[e] = (int32_t)e;
}

__global__ void k_inj_segments(const uint64_t* __restrict__ keys, const int32_t* __restrict__ vals, int64_t total,
                               const double* __restrict__ e_xi, const double* __restrict__ V,
                               int32_t* head_flag, int32_t* inj_src, double* inj_coef) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= total) return;
    uint32_t g = (uint32_t)(keys[e] >> 32);
    head_flag[e] = (e == 0 || (uint32_t)(keys[e - 1] >> 32) != g) ? 1 : 0;
    inj_src[e] = (int32_t)(uint32_t)(keys[e] & 0xffffffffu);
    inj_coef[e] = e_xi[vals[e]] / V[g];   // xi / V_g: E_g += coef * L dt
}

__global__ void k_inj_targets(const uint64_t* __restrict__ keys, const int32_t* __restrict__ head_flag,
                              const int32_t* __restrict__ head_pos, int64_t total, int32_t* targets,
                              int32_t* inj_off) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= total) return;
    if (head_flag[e]) {
        int t = head_pos[e];
        targets[t] = (int32_t)(keys[e] >> 32);
        inj_off[t] = (int32_t)e;
    }
    if (e == total - 1) inj_off[head_pos[e] + head_flag[e]] = (int32_t)total;
}

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// ------------------------------------------------------------------------------------
rt_status build_neighbours(rt_ctx* c, const double* x, const double* m, const double* xsrc, const double* h_in,
                           const double* hs_in, const double* oms_in, const double* octw_in) {
    const int64_t n = c->n, S = c->n_src;
    const rt_config& cfg = c->cfg;
    cudaStream_t st = c->stream;
    const int B = 256;

    // grid: cells of cell_eighths / 8 of the mean-density support radius (default one half)
    double vol = cfg.box[0] * cfg.box[1] * cfg.box[2];
    double h0 = cfg.eta_res * std::cbrt(vol / (double)n);
    double H0 = kKappa * h0;
    const double cell_frac = (c->tune.cell_eighths > 0 ? c->tune.cell_eighths : 4) / 8.0;
    int64_t ncells = 1;
    for (int a = 0; a < 3; ++a) {
        int nca = (int)std::floor(cfg.box[a] / (cell_frac * H0));
        nca = std::max(1, std::min(nca, 1024));
        c->nc[a] = nca;
        c->cell[a] = cfg.box[a] / nca;
        ncells *= nca;
    }
    while (ncells > (int64_t)1 << 27) {   // keep the cell table small
        ncells = 1;
        for (int a = 0; a < 3; ++a) {
            c->nc[a] = std::max(1, c->nc[a] / 2);
            c->cell[a] = cfg.box[a] / c->nc[a];
            ncells *= c->nc[a];
        }
    }
    c->ncells = ncells;
    int bits = 1;
    while (((int64_t)1 << bits) < ncells) ++bits;
    c->key_bits = bits;
    for (int a = 0; a < 3; ++a) c->diag.grid[a] = c->nc[a];

    Grid g;
    for (int a = 0; a < 3; ++a) {
        g.nc[a] = c->nc[a];
        g.cell[a] = c->cell[a];
        g.inv_cell[a] = 1.0 / c->cell[a];
        g.cellf[a] = (float)c->cell[a];
        g.inv_cellf[a] = (float)(1.0 / c->cell[a]);
        g.box[a] = cfg.box[a];
    }
    g.periodic = cfg.periodic;

    // buffers
    RT_TRY(ensure(c, c->keys_in, n * 4, "keys"));
    RT_TRY(ensure(c, c->keys_out, n * 4, "keys"));
    RT_TRY(ensure(c, c->idx_in, n * 4, "idx"));
    RT_TRY(ensure(c, c->perm, n * 4, "perm"));
    RT_TRY(ensure(c, c->inv_perm, n * 4, "inv_perm"));
    RT_TRY(ensure(c, c->cell_start, (ncells + 1) * 4, "cells"));
    RT_TRY(ensure(c, c->xs_d, 3 * n * 8, "positions"));
    RT_TRY(ensure(c, c->xq, 16 * n, "positions"));
    RT_TRY(ensure(c, c->m_s, n * 8, "masses"));
    RT_TRY(ensure(c, c->h_d, n * 8, "h"));
    RT_TRY(ensure(c, c->H2f, n * 4, "h"));
    RT_TRY(ensure(c, c->omega_d, n * 8, "omega"));
    RT_TRY(ensure(c, c->V_d, n * 8, "V"));
    RT_TRY(ensure(c, c->B_d, 6 * n * 8, "B"));
    RT_TRY(ensure(c, c->cond_d, n * 8, "cond"));
    size_t ts = c->fp64 ? 8 : 4;
    RT_TRY(ensure(c, c->pos_t, n * 32, "geom"));
    RT_TRY(ensure(c, c->geo_t, 8 * n * ts, "geom"));
    RT_TRY(ensure(c, c->omega_t, n * ts, "geom"));
    RT_TRY(ensure(c, c->counts, (n + 1) * 4, "counts"));
    RT_TRY(ensure(c, c->row_off, (n + 1) * 8, "row_off"));
    RT_TRY(ensure(c, c->flags, 64, "flags"));
    RT_TRY(ensure(c, c->red_tmp, 64, "reduction"));

    int* flags = c->flags.as<int>();
    RT_CUDA(c, cudaMemsetAsync(flags, 0, 64, st));
    const bool warm = c->has_h_prev;
    c->has_h_prev = false;       // set again only when this call succeeds
    // reductions: [0] min h, [1] max h, [2] max cond, [3] min V (bit patterns of positive doubles)
    unsigned long long* red = reinterpret_cast<unsigned long long*>(c->red_tmp.p);
    RT_CUDA(c, cudaMemsetAsync(red, 0, 40, st));
    RT_CUDA(c, cudaMemsetAsync(red, 0xff, 8, st));
    RT_CUDA(c, cudaMemsetAsync(red + 3, 0xff, 8, st));

    // cub scratch: radix sort of N, scans of N+1 and S+1, radix sort of the injection entries
    size_t t1 = 0, t2 = 0, t3 = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, t1, (const uint32_t*)nullptr, (uint32_t*)nullptr,
                                    (const int32_t*)nullptr, (int32_t*)nullptr, (int)n, 0, bits, st);
    cub::DeviceScan::ExclusiveSum(nullptr, t2, (const int32_t*)nullptr, (int64_t*)nullptr,
                                  (int)(std::max<int64_t>(n, S) + 1), st);
    int64_t Smax = std::max<int64_t>(S, 1) * 4096;
    cub::DeviceRadixSort::SortPairs(nullptr, t3, (const uint64_t*)nullptr, (uint64_t*)nullptr,
                                    (const int32_t*)nullptr, (int32_t*)nullptr, (int)Smax, 0, 64, st);
    RT_TRY(ensure(c, c->cub_tmp, std::max(t1, std::max(t2, t3)) + 256, "cub scratch"));

    // a1: keys, sort, cell table, sorted copies
    k_keys<<<nblk(n, B), B, 0, st>>>(x, n, g, c->keys_in.as<uint32_t>(), c->idx_in.as<int32_t>(), flags);
    size_t tb = c->cub_tmp.bytes;
    RT_CUDA(c, cub::DeviceRadixSort::SortPairs(c->cub_tmp.p, tb, c->keys_in.as<uint32_t>(), c->keys_out.as<uint32_t>(),
                                               c->idx_in.as<int32_t>(), c->perm.as<int32_t>(), (int)n, 0, bits, st));
    k_cell_start<<<nblk(ncells + 1, B), B, 0, st>>>(c->keys_out.as<uint32_t>(), n, ncells, c->cell_start.as<int32_t>());
    g.cell_start = c->cell_start.as<int32_t>();
    double qmul[3];
    float qscale[3];
    for (int a = 0; a < 3; ++a) {
        double units = cfg.periodic ? 4294967296.0 : 2147483648.0;
        qmul[a] = units / cfg.box[a];
        qscale[a] = (float)(cfg.box[a] / units);
    }
    k_gather_positions<<<nblk(n, B), B, 0, st>>>(x, m, c->perm.as<int32_t>(), n, qmul[0], qmul[1], qmul[2],
                                                  c->xs_d.as<double>(), c->xq.as<uint4>(), c->m_s.as<double>(),
                                                  c->inv_perm.as<int32_t>());
    RT_CUDA(c, cudaGetLastError());
    c->launches += 3;   // keys, cell table, gather

    // a2: smoothing lengths
    HParams hp;
    hp.eta = cfg.eta_res;
    hp.h0 = h0;
    double minbox = std::min(cfg.box[0], std::min(cfg.box[1], cfg.box[2]));
    hp.h_cap = cfg.periodic ? 0.5 * minbox / kKappa : 1e30;
    for (int a = 0; a < 3; ++a) hp.scale[a] = qscale[a];
    hp.max_iter = cfg.h_max_iter > 0 ? cfg.h_max_iter : 100;
    hp.tol32 = (float)std::max(cfg.h_tol, 2e-6);
    // the FP64 path refines every h in double; the float path only those of particles with a
    // candidate near their support radius, which is enough for the exact root's pair lists
    hp.refine64 = c->fp64 ? 1 : 0;
    int* refine_count = flags + F_REFINE;
    if (h_in) {
        hp.refine64 = c->fp64 ? 1 : 0;   // omega in the working path's arithmetic
        k_h_given<<<nblk(n, 128), 128, 0, st>>>(g, c->xs_d.as<double>(), c->xq.as<uint4>(), n, hp, h_in,
                                                 c->perm.as<int32_t>(), c->h_d.as<double>(), c->omega_d.as<double>(),
                                                 c->H2f.as<float>(), red, flags);
    } else {
        k_h_solve<<<nblk(n, 128), 128, 0, st>>>(g, c->xs_d.as<double>(), c->xq.as<uint4>(), n, hp,
                                                 warm ? c->h_prev.as<double>() : nullptr, c->perm.as<int32_t>(),
                                                 c->h_d.as<double>(), c->omega_d.as<double>(), c->H2f.as<float>(), red,
                                                 flags, c->idx_in.as<int32_t>(), refine_count);
    }
    RT_CUDA(c, cudaGetLastError());
    c->launches += 1;
    if (!c->fp64 && !h_in) {
        k_h_refine<<<(unsigned)c->sm_count * 8, 256, 0, st>>>(g, c->xs_d.as<double>(), c->xq.as<uint4>(), n, hp,
                                                  c->idx_in.as<int32_t>(), refine_count, c->h_d.as<double>(),
                                                  c->omega_d.as<double>(), c->H2f.as<float>(), red, flags);
        RT_CUDA(c, cudaGetLastError());
        c->launches += 1;
    }
    int hflags[8];
    double hmm[2];
    double sumH3 = 0.0;
    RT_CUDA(c, cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
    RT_CUDA(c, cudaMemcpyAsync(hmm, red, sizeof(hmm), cudaMemcpyDeviceToHost, st));
    RT_CUDA(c, cudaMemcpyAsync(&sumH3, red + 4, 8, cudaMemcpyDeviceToHost, st));
    RT_CUDA(c, cudaStreamSynchronize(st));
    if (hflags[F_BADPOS]) return fail(c, RT_ERR_INVALID, "positions must be finite and inside [0, box)");
    if (hflags[F_NOCONV]) return fail(c, RT_ERR_NOCONV, "smoothing-length iteration did not converge");
    if (hflags[F_BADH]) return fail(c, RT_ERR_INVALID, "given smoothing lengths must be finite, > 0 and below the "
                                                       "quarter of the periodic box over the support ratio");
    c->diag.h_refined = h_in ? 0 : (c->fp64 ? n : (int64_t)hflags[F_REFINE]);
    c->diag.h_min = hmm[0];
    c->diag.h_max = hmm[1];
    double Hmax = kKappa * hmm[1];
    if (cfg.periodic && Hmax >= 0.5 * minbox)
        return fail(c, RT_ERR_GEOMETRY, "support radius reaches half the periodic box");

    // a3: symmetric pair lists
    PairParams pp;
    for (int a = 0; a < 3; ++a) pp.scale[a] = qscale[a];
    pp.Hmax = Hmax;
    // Searching every particle out to max(H_i, H_max) visits H_max^3 / <H^3> times the volume
    // of its own support; above a ratio of 12 the sort-based build is cheaper.
    const double vol_ratio = Hmax * Hmax * Hmax / std::max(sumH3 / (double)n, 1e-300);
    const bool sorted_build = vol_ratio > 12.0;
    c->diag.pair_build = sorted_build ? 1 : 0;
    int64_t P2 = 0;
    if (!sorted_build) {
        // search radii from the coarse blocks' largest H
        Blocks bk;
        int nbt = 1;
        for (int a = 0; a < 3; ++a) {
            bk.nb[a] = std::min(16, c->nc[a]);
            bk.len[a] = cfg.box[a] / bk.nb[a];
            nbt *= bk.nb[a];
        }
        bk.periodic = cfg.periodic;
        for (int a = 0; a < 3; ++a) bk.reach[a] = (int)std::ceil(Hmax / bk.len[a]) + 1;
        RT_TRY(ensure(c, c->blk, (size_t)nbt * 8, "blocks"));
        unsigned* hb = c->blk.as<unsigned>();
        float* reach = reinterpret_cast<float*>(hb + nbt);
        RT_CUDA(c, cudaMemsetAsync(hb, 0, (size_t)nbt * 4, st));
        k_block_hmax<<<nblk(n, 256), 256, 0, st>>>(c->xs_d.as<double>(), c->H2f.as<float>(), n, bk, hb,
                                                   c->xq.as<uint4>());
        k_block_reach<<<nblk((int64_t)nbt * 32, 128), 128, 0, st>>>(hb, bk, reach);
        c->launches += 2;
        // one walk counts the rows and, when the rows of the last call fit row_cap entries,
        // also stores them (then compacted); a longer row needs a second, writing walk
        const int cap = (int)c->row_cap;
        if (cap > 0) RT_TRY(ensure(c, c->cols_cap, (size_t)n * cap * 4, "pair rows"));
        int* row_max = c->flags.as<int>() + F_ROWMAX;
        RT_CUDA(c, cudaMemsetAsync(row_max, 0, 4, st));
        k_pairs<false><<<nblk(n, 128), 128, 0, st>>>(g, c->xs_d.as<double>(), c->xq.as<uint4>(),
                                                      c->h_d.as<double>(), c->H2f.as<float>(), n, pp, bk, reach,
                                                      c->counts.as<int32_t>(), nullptr,
                                                      cap > 0 ? c->cols_cap.as<int32_t>() : nullptr, cap, row_max);
        RT_CUDA(c, cudaMemsetAsync(c->counts.as<int32_t>() + n, 0, 4, st));
        tb = c->cub_tmp.bytes;
        RT_CUDA(c, cub::DeviceScan::ExclusiveSum(c->cub_tmp.p, tb, c->counts.as<int32_t>(), c->row_off.as<int64_t>(),
                                                 (int)(n + 1), st));
        int longest = 0;
        RT_CUDA(c, cudaMemcpyAsync(&P2, c->row_off.as<int64_t>() + n, 8, cudaMemcpyDeviceToHost, st));
        RT_CUDA(c, cudaMemcpyAsync(&longest, row_max, 4, cudaMemcpyDeviceToHost, st));
        RT_CUDA(c, cudaStreamSynchronize(st));
        if (P2 >= ((int64_t)1 << 31)) return fail(c, RT_ERR_INVALID, "more than 2^31 neighbour entries");
        RT_TRY(ensure(c, c->cols, std::max<int64_t>(P2, 1) * 4, "pair lists"));
        // the walks visit the candidates in ascending index: the rows need no sort
        if (cap > 0 && longest <= cap) {
            k_rows_compact<<<nblk(n * 32, 256), 256, 0, st>>>(c->cols_cap.as<int32_t>(), cap,
                                                              c->row_off.as<int64_t>(), n, c->cols.as<int32_t>());
        } else {
            k_pairs<true><<<nblk(n, 128), 128, 0, st>>>(g, c->xs_d.as<double>(), c->xq.as<uint4>(),
                                                         c->h_d.as<double>(), c->H2f.as<float>(), n, pp, bk, reach,
                                                         nullptr, c->row_off.as<int64_t>(), c->cols.as<int32_t>());
        }
        // the next call's rows: the longest row with a quarter to spare, in multiples of 32,
        // while the padded rows stay within eight times the lists (only the filled part of a
        // row is written or read)
        const int64_t next = ((int64_t)longest + longest / 4 + 8 + 31) / 32 * 32;
        c->row_cap = next * n <= 8 * std::max<int64_t>(P2, 1) ? next : 0;
        RT_CUDA(c, cudaGetLastError());
        c->launches += 2;
    } else {
        int64_t* goff = c->row_off.as<int64_t>();      // gather offsets first, CSR offsets after
        k_pairs_gather<false><<<nblk(n, 128), 128, 0, st>>>(g, c->xs_d.as<double>(), c->xq.as<uint4>(),
                                                             c->h_d.as<double>(), c->H2f.as<float>(), n, pp,
                                                             c->counts.as<int32_t>(), nullptr, nullptr);
        RT_CUDA(c, cudaMemsetAsync(c->counts.as<int32_t>() + n, 0, 4, st));
        tb = c->cub_tmp.bytes;
        RT_CUDA(c, cub::DeviceScan::ExclusiveSum(c->cub_tmp.p, tb, c->counts.as<int32_t>(), goff, (int)(n + 1), st));
        int64_t Mg = 0;
        RT_CUDA(c, cudaMemcpyAsync(&Mg, goff + n, 8, cudaMemcpyDeviceToHost, st));
        RT_CUDA(c, cudaStreamSynchronize(st));
        if (2 * Mg >= ((int64_t)1 << 31)) return fail(c, RT_ERR_INVALID, "more than 2^31 neighbour entries");
        const int64_t K = std::max<int64_t>(2 * Mg, 1);
        RT_TRY(ensure(c, c->pkeys, K * 8, "pair keys"));
        RT_TRY(ensure(c, c->pkeys_alt, K * 8, "pair keys"));
        k_pairs_gather<true><<<nblk(n, 128), 128, 0, st>>>(g, c->xs_d.as<double>(), c->xq.as<uint4>(),
                                                            c->h_d.as<double>(), c->H2f.as<float>(), n, pp, nullptr,
                                                            goff, c->pkeys.as<uint64_t>());
        c->launches += 2;
        int key_bits = 32 + c->key_bits;
        {
            int nb = 1;
            while (((int64_t)1 << nb) < n) ++nb;
            key_bits = 32 + nb;
        }
        size_t need = 0;
        cub::DeviceRadixSort::SortKeys(nullptr, need, c->pkeys.as<uint64_t>(), c->pkeys_alt.as<uint64_t>(), (int)K, 0,
                                       key_bits, st);
        size_t need2 = 0;
        cub::DeviceSelect::Unique(nullptr, need2, c->pkeys_alt.as<uint64_t>(), c->pkeys.as<uint64_t>(),
                                  (int64_t*)nullptr, (int)K, st);
        RT_TRY(ensure(c, c->cub_tmp, std::max(need, need2) + 256, "cub scratch"));
        tb = c->cub_tmp.bytes;
        RT_CUDA(c, cub::DeviceRadixSort::SortKeys(c->cub_tmp.p, tb, c->pkeys.as<uint64_t>(), c->pkeys_alt.as<uint64_t>(),
                                                  (int)K, 0, key_bits, st));
        int64_t* nuniq = reinterpret_cast<int64_t*>(red + 5);
        tb = c->cub_tmp.bytes;
        RT_CUDA(c, cub::DeviceSelect::Unique(c->cub_tmp.p, tb, c->pkeys_alt.as<uint64_t>(), c->pkeys.as<uint64_t>(),
                                             nuniq, (int)K, st));
        RT_CUDA(c, cudaMemcpyAsync(&P2, nuniq, 8, cudaMemcpyDeviceToHost, st));
        RT_CUDA(c, cudaStreamSynchronize(st));
        RT_TRY(ensure(c, c->cols, std::max<int64_t>(P2, 1) * 4, "pair lists"));
        RT_CUDA(c, cudaMemsetAsync(c->counts.as<int32_t>(), 0, (n + 1) * 4, st));
        k_keys_to_csr<<<nblk(std::max<int64_t>(P2, 1), 256), 256, 0, st>>>(c->pkeys.as<uint64_t>(), nuniq,
                                                                            c->cols.as<int32_t>(),
                                                                            c->counts.as<int32_t>());
        tb = c->cub_tmp.bytes;
        RT_CUDA(c, cub::DeviceScan::ExclusiveSum(c->cub_tmp.p, tb, c->counts.as<int32_t>(), c->row_off.as<int64_t>(),
                                                 (int)(n + 1), st));
        ++c->launches;
        RT_CUDA(c, cudaGetLastError());
    }
    c->n_directed = P2;
    c->launches += 1;   // geometry below

    // the lower / upper split and the slots of the pairs
    RT_TRY(ensure(c, c->n_low, (n + 1) * 4, "pair split"));
    RT_TRY(ensure(c, c->n_up, (n + 1) * 4, "pair split"));
    RT_TRY(ensure(c, c->up_off, (n + 1) * 8, "pair split"));
    RT_TRY(ensure(c, c->low_slot, std::max<int64_t>(P2 / 2, 1) * 4, "pair split"));
    k_row_split<<<nblk(n, 256), 256, 0, st>>>(c->row_off.as<int64_t>(), c->cols.as<int32_t>(), n,
                                               c->n_low.as<int32_t>(), c->n_up.as<int32_t>());
    RT_CUDA(c, cudaMemsetAsync(c->n_up.as<int32_t>() + n, 0, 4, st));
    tb = c->cub_tmp.bytes;
    RT_CUDA(c, cub::DeviceScan::ExclusiveSum(c->cub_tmp.p, tb, c->n_up.as<int32_t>(), c->up_off.as<int64_t>(),
                                             (int)(n + 1), st));
    k_low_slots<<<nblk(n * 32, 256), 256, 0, st>>>(c->row_off.as<int64_t>(), c->cols.as<int32_t>(),
                                                    c->n_low.as<int32_t>(), c->up_off.as<int64_t>(), n,
                                                    c->low_slot.as<int32_t>());
    RT_TRY(ensure(c, c->pair_ends, std::max<int64_t>(P2 / 2, 1) * 8, "pair split"));
    k_pair_ends<<<nblk(n, 128), 128, 0, st>>>(c->row_off.as<int64_t>(), c->cols.as<int32_t>(), c->n_low.as<int32_t>(),
                                               c->up_off.as<int64_t>(), n, c->pair_ends.as<int2>());
    c->launches += 3;
    RT_CUDA(c, cudaGetLastError());

    // a4: geometry
    if (c->fp64)
        k_geometry<double><<<nblk(n, 128), 128, 0, st>>>(
            c->xs_d.as<double>(), c->xq.as<uint4>(), c->h_d.as<double>(), c->omega_d.as<double>(),
            c->row_off.as<int64_t>(), c->cols.as<int32_t>(), n, cfg.box[0], cfg.box[1], cfg.box[2], cfg.periodic,
            qscale[0], qscale[1], qscale[2], c->V_d.as<double>(), c->B_d.as<double>(), c->cond_d.as<double>(),
            c->pos_t.p, c->geo_t.as<double>(), c->omega_t.as<double>(), red, flags);
    else
        k_geometry<float><<<nblk(n, 128), 128, 0, st>>>(
            c->xs_d.as<double>(), c->xq.as<uint4>(), c->h_d.as<double>(), c->omega_d.as<double>(),
            c->row_off.as<int64_t>(), c->cols.as<int32_t>(), n, cfg.box[0], cfg.box[1], cfg.box[2], cfg.periodic,
            qscale[0], qscale[1], qscale[2], c->V_d.as<double>(), c->B_d.as<double>(), c->cond_d.as<double>(),
            c->pos_t.p, c->geo_t.as<float>(), c->omega_t.as<float>(), red, flags);
    RT_CUDA(c, cudaGetLastError());

    // a5 preparation: sources
    c->n_inj_entries = 0;
    c->n_inj_targets = 0;
    if (S > 0) {
        RT_TRY(ensure(c, c->xsrc_d, 3 * S * 8, "sources"));
        RT_TRY(ensure(c, c->hs_d, S * 8, "sources"));
        RT_TRY(ensure(c, c->omegas_d, S * 8 + 64 * S, "sources"));
        RT_TRY(ensure(c, c->src_counts, (S + 1) * 4, "sources"));
        RT_TRY(ensure(c, c->src_off, (S + 1) * 8, "sources"));
        RT_CUDA(c, cudaMemcpyAsync(c->xsrc_d.p, xsrc, 3 * S * 8, cudaMemcpyDeviceToDevice, st));
        SrcParams sp;
        sp.eta = cfg.eta_res_star;
        sp.h0 = cfg.eta_res_star * std::cbrt(vol / (double)n);
        sp.h_cap = hp.h_cap;
        sp.max_iter = std::max(hp.max_iter, 200);
        sp.warm = c->has_hs_prev ? 1 : 0;
        sp.fixed = hs_in ? 1 : 0;
        c->has_hs_prev = false;     // set again only when this call succeeds
        if (hs_in) RT_CUDA(c, cudaMemcpyAsync(c->hs_d.p, hs_in, S * 8, cudaMemcpyDeviceToDevice, st));
        const unsigned sb = (unsigned)S;   // one block of kSrcWarps warps per source
        k_src_h<<<(unsigned)S, kSrcThreads, 0, st>>>(g, c->xs_d.as<double>(), n, c->xsrc_d.as<double>(), S, sp,
                                                     c->hs_d.as<double>(), c->omegas_d.as<double>(), flags);
        if (hs_in && oms_in)   // the sources' own omega_s, from their owners
            RT_CUDA(c, cudaMemcpyAsync(c->omegas_d.p, oms_in, S * 8, cudaMemcpyDeviceToDevice, st));
        k_src_entries<false><<<sb, kSrcWarps * 32, 0, st>>>(g, c->xs_d.as<double>(), n, c->xsrc_d.as<double>(), S,
                                                 c->hs_d.as<double>(), c->omegas_d.as<double>(),
                                                 c->src_counts.as<int32_t>(), nullptr, nullptr, nullptr, nullptr);
        RT_CUDA(c, cudaMemsetAsync(c->src_counts.as<int32_t>() + S, 0, 4, st));
        tb = c->cub_tmp.bytes;
        RT_CUDA(c, cub::DeviceScan::ExclusiveSum(c->cub_tmp.p, tb, c->src_counts.as<int32_t>(),
                                                 c->src_off.as<int64_t>(), (int)(S + 1), st));
        c->launches += 2;
        int64_t NE = 0;
        RT_CUDA(c, cudaMemcpyAsync(&NE, c->src_off.as<int64_t>() + S, 8, cudaMemcpyDeviceToHost, st));
        RT_CUDA(c, cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
        RT_CUDA(c, cudaStreamSynchronize(st));
        if (hflags[F_BADH]) return fail(c, RT_ERR_INVALID, "given source smoothing lengths must be finite and > 0");
        if (hflags[F_SRC_NOCONV]) return fail(c, RT_ERR_NOCONV, "source smoothing-length iteration did not converge");
        if (NE > Smax) return fail(c, RT_ERR_INVALID, "too many injection entries");
        c->n_inj_entries = NE;
        int64_t NEa = std::max<int64_t>(NE, 1);
        RT_TRY(ensure(c, c->src_entry_gas, NEa * 4, "injection"));
        RT_TRY(ensure(c, c->src_entry_xi, NEa * 8, "injection"));
        RT_TRY(ensure(c, c->inj_key, NEa * 8, "injection"));
        RT_TRY(ensure(c, c->inj_key_out, NEa * 8, "injection"));
        RT_TRY(ensure(c, c->inj_val, NEa * 4, "injection"));
        RT_TRY(ensure(c, c->inj_val_out, NEa * 4, "injection"));
        RT_TRY(ensure(c, c->inj_src, NEa * 4, "injection"));
        RT_TRY(ensure(c, c->inj_coef, NEa * 8, "injection"));
        RT_TRY(ensure(c, c->inj_targets, NEa * 4, "injection"));
        RT_TRY(ensure(c, c->inj_off, (NEa + 1) * 4, "injection"));
        double* octw = c->omegas_d.as<double>() + S;   // 8 per source after omega_s
        k_src_entries<true><<<sb, kSrcWarps * 32, 0, st>>>(g, c->xs_d.as<double>(), n, c->xsrc_d.as<double>(), S,
                                                c->hs_d.as<double>(), c->omegas_d.as<double>(), nullptr,
                                                c->src_off.as<int64_t>(), c->src_entry_gas.as<int32_t>(),
                                                c->src_entry_xi.as<double>(), octw, hs_in ? octw_in : nullptr);
        ++c->launches;
        if (NE > 0) {
            c->launches += 3;
            k_inj_keys<<<nblk(NE, B), B, 0, st>>>(c->src_entry_gas.as<int32_t>(), c->src_off.as<int64_t>(), S, NE,
                                                   c->inj_key.as<uint64_t>(), c->inj_val.as<int32_t>());
            tb = c->cub_tmp.bytes;
            RT_CUDA(c, cub::DeviceRadixSort::SortPairs(c->cub_tmp.p, tb, c->inj_key.as<uint64_t>(),
                                                       c->inj_key_out.as<uint64_t>(), c->inj_val.as<int32_t>(),
                                                       c->inj_val_out.as<int32_t>(), (int)NE, 0, 64, st));
            // head flags into idx_in (free now), positions via scan into counts-sized scratch
            int32_t* head = c->inj_val.as<int32_t>();       // reuse: NE int32
            k_inj_segments<<<nblk(NE, B), B, 0, st>>>(c->inj_key_out.as<uint64_t>(), c->inj_val_out.as<int32_t>(), NE,
                                                       c->src_entry_xi.as<double>(), c->V_d.as<double>(), head,
                                                       c->inj_src.as<int32_t>(), c->inj_coef.as<double>());
            int32_t* hpos = reinterpret_cast<int32_t*>(c->inj_key.as<uint64_t>());   // reuse: NE int32
            tb = c->cub_tmp.bytes;
            RT_CUDA(c, cub::DeviceScan::ExclusiveSum(c->cub_tmp.p, tb, head, hpos, (int)NE, st));
            k_inj_targets<<<nblk(NE, B), B, 0, st>>>(c->inj_key_out.as<uint64_t>(), head, hpos, NE,
                                                      c->inj_targets.as<int32_t>(), c->inj_off.as<int32_t>());
            int32_t lastpos = 0, lasthead = 0;
            RT_CUDA(c, cudaMemcpyAsync(&lastpos, hpos + NE - 1, 4, cudaMemcpyDeviceToHost, st));
            RT_CUDA(c, cudaMemcpyAsync(&lasthead, head + NE - 1, 4, cudaMemcpyDeviceToHost, st));
            RT_CUDA(c, cudaStreamSynchronize(st));
            c->n_inj_targets = lastpos + lasthead;
        }
    }

    // finish: flags, counters (one synchronisation)
    double cv[2];
    RT_CUDA(c, cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, st));
    RT_CUDA(c, cudaMemcpyAsync(cv, red + 2, sizeof(cv), cudaMemcpyDeviceToHost, st));
    RT_CUDA(c, cudaStreamSynchronize(st));
    if (hflags[F_GEOM]) return fail(c, RT_ERR_GEOMETRY, "singular E_i: a particle has fewer than 3 non-coplanar neighbours");
    c->diag.n_ill_conditioned = hflags[F_ILL];
    c->diag.n_directed = P2;
    c->diag.n_pairs = P2 / 2;
    c->diag.n_injection = c->n_inj_entries;
    c->diag.cond_max = cv[0];
    c->diag.dx_min = std::cbrt(cv[1] / (4.0 * M_PI / 3.0));
    // keep h in caller order as the first guess of the next call
    RT_TRY(ensure(c, c->h_prev, n * 8, "h"));
    RT_TRY(field_out(c, c->h_d.as<double>(), c->h_prev.as<double>(), 1));
    c->has_h_prev = true;
    c->has_hs_prev = S > 0;
    return RT_OK;
}

}  // namespace rt
