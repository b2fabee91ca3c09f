// Energy sum of a radiation state for callers that cannot allocate device memory.
//
// rt_energy (rt_api.cu) reduces through per-block partial sums held in a workspace that
// rt_create allocates.  This variant keeps those partial sums in a fixed array in the
// library's own device memory instead, so a call allocates nothing and needs no context.
#include <mutex>
#include <vector>

#include "rt_internal.cuh"

namespace rt {
namespace {

constexpr int kStaticBlocks = 256;
constexpr int kStaticThreads = 256;
constexpr int kStaticMaxGroups = 16;

// One partial sum per (group, block): 16 x 256 doubles = 32 KiB, present on every device
// that loads the library until the process exits.  Every call overwrites the slots it uses
// before reading them, so nothing needs clearing between calls; calls that overlap on the
// GPU share these slots and race.
static __device__ __align__(256) double g_energy_scratch[kStaticMaxGroups * kStaticBlocks];

// partial sums of V_i E_i,g over a fixed grid-stride assignment, tree-reduced per block
template <class T>
__global__ void __launch_bounds__(kStaticThreads) k_energy_static_part(const T* __restrict__ U,
                                                                       const double* __restrict__ V, int64_t n, int G,
                                                                       double* __restrict__ part) {
    __shared__ double sm[kStaticThreads];
    for (int g = 0; g < G; ++g) {
        double s = 0.0;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
            s += V[i] * (double)U[(int64_t)(4 * g) * n + i];
        sm[threadIdx.x] = s;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[g * kStaticBlocks + blockIdx.x] = sm[0];
        __syncthreads();
    }
}

__global__ void k_energy_static_final(const double* __restrict__ part, int G, double* __restrict__ out) {
    int g = threadIdx.x;
    if (g >= G) return;
    double s = 0.0;
    for (int b = 0; b < kStaticBlocks; ++b) s += part[g * kStaticBlocks + b];
    out[g] = s;
}

// Device address of g_energy_scratch, looked up once per device with that device current.
// In host code the symbol only names a host-side stand-in, so kernels are given this address.
// The address belongs to the device's current context: a caller that resets the device
// (cudaDeviceReset) gets a new context, in which the array has a new address, so the cache
// remembers the context it was taken in and looks the address up again when that changes.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);

CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<CtxGetCurrentFn>(p);
    }
    return fn;
}

struct ScratchEntry {
    CUcontext ctx = nullptr;
    double* addr = nullptr;
};
std::mutex g_scratch_mu;
std::vector<ScratchEntry> g_scratch;

cudaError_t scratch_address(int device, double** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if ((int)g_scratch.size() <= device) g_scratch.resize(device + 1);
    CUcontext cur = nullptr;
    CtxGetCurrentFn get = ctx_get_current();
    if (get && get(&cur) != CUDA_SUCCESS) cur = nullptr;
    ScratchEntry& e = g_scratch[device];
    if (!e.addr || (cur && cur != e.ctx)) {
        void* p = nullptr;
        cudaError_t r = cudaGetSymbolAddress(&p, g_energy_scratch);
        if (r != cudaSuccess) return r;
        if (!cur && get && get(&cur) != CUDA_SUCCESS) cur = nullptr;   // made current by the lookup
        e.addr = static_cast<double*>(p);
        e.ctx = cur;
    }
    *out = e.addr;
    return cudaSuccess;
}

}  // namespace
}  // namespace rt

extern "C" rt_status rt_energy_static(const void* U_dev, const double* V_dev, int64_t n, int32_t n_groups,
                                      int32_t precision, void* cuda_stream, double* E_tot_dev) {
    using namespace rt;
    if (!U_dev || !V_dev || !E_tot_dev) return RT_ERR_INVALID;
    if (n < 1) return RT_ERR_INVALID;
    if (n_groups < 1 || n_groups > kStaticMaxGroups) return RT_ERR_INVALID;
    if (precision != RT_FP64 && precision != RT_FP32_MIXED) return RT_ERR_INVALID;
    // an error left pending by the caller's earlier CUDA work is reported before any launch
    // (and left pending: this call does not clear what it did not cause)
    if (cudaPeekAtLastError() != cudaSuccess) return RT_ERR_CUDA;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return RT_ERR_CUDA;
    double* part = nullptr;
    if (scratch_address(device, &part) != cudaSuccess) return RT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (precision == RT_FP64)
        k_energy_static_part<double><<<kStaticBlocks, kStaticThreads, 0, s>>>((const double*)U_dev, V_dev, n,
                                                                               n_groups, part);
    else
        k_energy_static_part<float><<<kStaticBlocks, kStaticThreads, 0, s>>>((const float*)U_dev, V_dev, n, n_groups,
                                                                              part);
    if (cudaGetLastError() != cudaSuccess) return RT_ERR_CUDA;
    k_energy_static_final<<<1, 32, 0, s>>>(part, n_groups, E_tot_dev);
    if (cudaGetLastError() != cudaSuccess) return RT_ERR_CUDA;
    return RT_OK;
}
