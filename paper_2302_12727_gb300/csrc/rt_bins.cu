// Individual time bins of the transport step (Ivkovic 2023, Part II Sec. "Individual
// Timstepping" and Eq. transport-update-explicit with min(dt_k, dt_l); Part III
// Sec. "Dynamic Sub-Cycling" for the factor-4 limiter).
//
// Particle i advances in steps dt_i = 2^b_i dt_min; one hydro step is 2^B min-steps,
// B = max b.  At min-step s a particle starts a step when s mod 2^b_i = 0: it receives its
// injection for dt_i and a new gradient; every pair with a starting member exchanges the
// time-integrated flux min(dt_k, dt_l) F_kl . A_kl into both particles' accumulators; a
// particle applies its accumulator and its sink over dt_i when its step ends.  The bins come
// from the caller or from each particle's CFL step (Eq. rt-cfl), and the limiter lowers
// them until interacting particles differ by at most two bins.
#include <cmath>

#include <cub/cub.cuh>

#include "rt_internal.cuh"

namespace rt {

// sorted bins from the caller's (clipped to [0, max_bin]) or from the CFL step: the largest
// b <= max_bin with 2^b dt_min <= cfl dx_i / c, dx_i = (V_i / (4 pi / 3))^(1/3)
__global__ void k_bins_init(const int32_t* __restrict__ bins_in, const int32_t* __restrict__ perm,
                            const double* __restrict__ V, int64_t n, double cfl, double dt_min, double c_red,
                            int max_bin, int8_t* __restrict__ out) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    int b;
    if (bins_in) {
        b = bins_in[perm[p]];
        b = b < 0 ? 0 : (b > max_bin ? max_bin : b);
    } else {
        const double lim = cfl * cbrt(V[p] / (4.0 * 3.14159265358979323846 / 3.0)) / c_red;
        b = 0;
        while (b < max_bin && ldexp(dt_min, b + 1) <= lim) ++b;
    }
    out[p] = (int8_t)b;
}

// one Jacobi sweep of the limiter: b_i <- min(b_i, min_j b_j + 2); flags any change
__global__ void k_limit_bins(const int8_t* __restrict__ b, const int64_t* __restrict__ row_off,
                             const int32_t* __restrict__ cols, int64_t n, int8_t* __restrict__ out, int* changed) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int v = b[i];
    for (int64_t e = row_off[i]; e < row_off[i + 1]; ++e) {
        const int w = b[cols[e]] + 2;
        v = w < v ? w : v;
    }
    out[i] = (int8_t)v;
    if (v != b[i]) atomicExch(changed, 1);
}

__global__ void k_bins_max(const int8_t* __restrict__ b, int64_t n, int* mx) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) atomicMax(mx, (int)b[i]);
}

__global__ void k_bins_out(const int8_t* __restrict__ b, const int32_t* __restrict__ inv_perm, int64_t n,
                           int32_t* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = b[inv_perm[i]];
}

static unsigned nb256(int64_t n) { return (unsigned)((n + 255) / 256); }

// min over a particle's own bin and its neighbours' bins
__global__ void k_bins_nmin(const int8_t* __restrict__ b, const int64_t* __restrict__ row_off,
                            const int32_t* __restrict__ cols, int64_t n, int8_t* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int v = b[i];
    for (int64_t e = row_off[i]; e < row_off[i + 1]; ++e) v = b[cols[e]] < v ? b[cols[e]] : v;
    out[i] = (int8_t)v;
}

// sort keys: a per-particle bin array, or the level min(b_k, b_l) of every pair slot
// (counts per level: a shared histogram per block, added to the global one once per level)
__device__ __forceinline__ void hist_flush(unsigned* sh, unsigned long long* hist) {
    __syncthreads();
    if (threadIdx.x < 32 && sh[threadIdx.x]) atomicAdd(&hist[threadIdx.x], (unsigned long long)sh[threadIdx.x]);
}

__global__ void k_keys_particles(const int8_t* __restrict__ v, int64_t n, uint32_t* __restrict__ keys,
                                 int32_t* __restrict__ vals, unsigned long long* hist) {
    __shared__ unsigned sh[32];
    if (threadIdx.x < 32) sh[threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        keys[i] = (uint32_t)v[i];
        vals[i] = (int32_t)i;
        atomicAdd(&sh[v[i]], 1u);
    }
    hist_flush(sh, hist);
}

__global__ void k_keys_slots(const int8_t* __restrict__ b, const int2* __restrict__ ends, int64_t np,
                             uint32_t* __restrict__ keys, int32_t* __restrict__ vals, unsigned long long* hist) {
    __shared__ unsigned sh[32];
    if (threadIdx.x < 32) sh[threadIdx.x] = 0;
    __syncthreads();
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < np) {
        const int2 kl = ends[t];
        const int q = b[kl.x] < b[kl.y] ? b[kl.x] : b[kl.y];
        keys[t] = (uint32_t)q;
        vals[t] = (int32_t)t;
        atomicAdd(&sh[q], 1u);
    }
    hist_flush(sh, hist);
}

// stable order of `count` entries by their key (< 32), and the cumulative counts per level
static rt_status level_order(rt_ctx* c, int64_t count, DevBuf& order, unsigned long long* hist_dev, int B,
                             std::vector<int64_t>& cum) {
    cudaStream_t s = c->stream;
    size_t tb = 0;
    RT_CUDA(c, cub::DeviceRadixSort::SortPairs(nullptr, tb, (const uint32_t*)nullptr, (uint32_t*)nullptr,
                                               (const int32_t*)nullptr, (int32_t*)nullptr, (int)count, 0, 5, s));
    RT_TRY(ensure(c, c->bin_cub, tb + 256, "time-bin sort scratch"));
    RT_TRY(ensure(c, order, (size_t)std::max<int64_t>(count, 1) * 4, "time-bin order"));
    tb = c->bin_cub.bytes;
    RT_CUDA(c, cub::DeviceRadixSort::SortPairs(c->bin_cub.p, tb, c->bin_keys.as<uint32_t>(),
                                               c->bin_keys2.as<uint32_t>(), c->bin_vals.as<int32_t>(),
                                               order.as<int32_t>(), (int)count, 0, 5, s));
    unsigned long long h[32];
    RT_CUDA(c, cudaMemcpyAsync(h, hist_dev, sizeof(h), cudaMemcpyDeviceToHost, s));
    RT_CUDA(c, cudaStreamSynchronize(s));
    cum.assign(B + 1, 0);
    int64_t run = 0;
    for (int q = 0; q <= B; ++q) {
        run += (int64_t)h[q];
        cum[q] = run;
    }
    return RT_OK;
}

}  // namespace rt

using namespace rt;

extern "C" {

rt_status rt_set_time_bins(rt_ctx* c, const int32_t* bins_dev, double dt_min, double cfl, int32_t max_bin,
                           int32_t limit) {
    if (!c) return RT_ERR_INVALID;
    c->err.clear();
    if (!c->built) return fail(c, RT_ERR_STATE, "rt_neighbours has not been called");
    if (!(dt_min > 0.0) || !std::isfinite(dt_min)) return fail(c, RT_ERR_INVALID, "dt_min must be finite and > 0");
    if (max_bin < 0 || max_bin > RT_MAX_TIME_BIN)
        return fail(c, RT_ERR_INVALID, "max_bin must be in [0, RT_MAX_TIME_BIN]");
    if (!bins_dev && !(cfl > 0.0 && std::isfinite(cfl)))
        return fail(c, RT_ERR_INVALID, "cfl must be finite and > 0 when the bins come from the CFL step");
    RT_CUDA(c, cudaSetDevice(c->device));
    const int64_t n = c->n;
    const int G = c->cfg.n_groups;
    RT_TRY(ensure(c, c->bins_s, (size_t)n, "time bins"));
    RT_TRY(ensure(c, c->bins_tmp, (size_t)n, "time bins"));
    RT_TRY(ensure(c, c->acc_t, (size_t)32 * G * n, "flux accumulators"));   // 32 B per (particle, group)
    cudaStream_t s = c->stream;
    k_bins_init<<<nb256(n), 256, 0, s>>>(bins_dev, c->perm.as<int32_t>(), c->V_d.as<double>(), n, cfl, dt_min,
                                         c->cfg.c_red, max_bin, c->bins_s.as<int8_t>());
    ++c->launches;
    int* flag = c->flags.as<int>() + F_SCRATCH;
    if (limit) {
        // each sweep moves a lowered bin one neighbour further; bins start <= RT_MAX_TIME_BIN
        for (int it = 0; it <= RT_MAX_TIME_BIN; ++it) {
            RT_CUDA(c, cudaMemsetAsync(flag, 0, sizeof(int), s));
            k_limit_bins<<<nb256(n), 256, 0, s>>>(c->bins_s.as<int8_t>(), c->row_off.as<int64_t>(),
                                                  c->cols.as<int32_t>(), n, c->bins_tmp.as<int8_t>(), flag);
            ++c->launches;
            std::swap(c->bins_s, c->bins_tmp);
            int h = 0;
            RT_CUDA(c, cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
            RT_CUDA(c, cudaStreamSynchronize(s));
            if (!h) break;
        }
    }
    RT_CUDA(c, cudaMemsetAsync(flag, 0, sizeof(int), s));
    k_bins_max<<<nb256(n), 256, 0, s>>>(c->bins_s.as<int8_t>(), n, flag);
    ++c->launches;
    int mx = 0;
    RT_CUDA(c, cudaMemcpyAsync(&mx, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    RT_CUDA(c, cudaStreamSynchronize(s));
    RT_CUDA(c, cudaGetLastError());
    c->bins_max = mx;
    c->dt_min = dt_min;
    // active-set orders (see rt_internal.cuh)
    const int64_t np = c->n_directed / 2;
    const int64_t m = std::max<int64_t>(std::max<int64_t>(np, n), 1);
    RT_TRY(ensure(c, c->bins_nmin, (size_t)n, "time bins"));
    RT_TRY(ensure(c, c->bin_keys, (size_t)m * 4, "time-bin keys"));
    RT_TRY(ensure(c, c->bin_keys2, (size_t)m * 4, "time-bin keys"));
    RT_TRY(ensure(c, c->bin_vals, (size_t)m * 4, "time-bin keys"));
    RT_TRY(ensure(c, c->bin_hist, 3 * 32 * 8, "time-bin counts"));
    RT_CUDA(c, cudaMemsetAsync(c->bin_hist.p, 0, 3 * 32 * 8, s));
    unsigned long long* hist = reinterpret_cast<unsigned long long*>(c->bin_hist.p);
    k_bins_nmin<<<nb256(n), 256, 0, s>>>(c->bins_s.as<int8_t>(), c->row_off.as<int64_t>(), c->cols.as<int32_t>(), n,
                                         c->bins_nmin.as<int8_t>());
    k_keys_particles<<<nb256(n), 256, 0, s>>>(c->bins_s.as<int8_t>(), n, c->bin_keys.as<uint32_t>(),
                                              c->bin_vals.as<int32_t>(), hist);
    c->launches += 2;
    RT_TRY(level_order(c, n, c->order_b, hist, mx, c->cum_b));
    k_keys_particles<<<nb256(n), 256, 0, s>>>(c->bins_nmin.as<int8_t>(), n, c->bin_keys.as<uint32_t>(),
                                              c->bin_vals.as<int32_t>(), hist + 32);
    ++c->launches;
    RT_TRY(level_order(c, n, c->order_m, hist + 32, mx, c->cum_m));
    if (np > 0) {
        k_keys_slots<<<nb256(np), 256, 0, s>>>(c->bins_s.as<int8_t>(), c->pair_ends.as<int2>(), np,
                                               c->bin_keys.as<uint32_t>(), c->bin_vals.as<int32_t>(), hist + 64);
        ++c->launches;
        RT_TRY(level_order(c, np, c->order_q, hist + 64, mx, c->cum_q));
    } else {
        c->cum_q.assign(mx + 1, 0);
    }
    RT_CUDA(c, cudaGetLastError());
    c->has_bins = true;
    return RT_OK;
}

rt_status rt_get_time_bins(rt_ctx* c, int32_t* bins_dev, int32_t* max_bin_host) {
    if (!c) return RT_ERR_INVALID;
    c->err.clear();
    if (!c->has_bins) return fail(c, RT_ERR_STATE, "rt_set_time_bins has not been called since rt_neighbours");
    if (bins_dev) {
        k_bins_out<<<nb256(c->n), 256, 0, c->stream>>>(c->bins_s.as<int8_t>(), c->inv_perm.as<int32_t>(), c->n,
                                                        bins_dev);
        ++c->launches;
        RT_CUDA(c, cudaGetLastError());
    }
    if (max_bin_host) *max_bin_host = c->bins_max;
    return RT_OK;
}

}  // extern "C"
