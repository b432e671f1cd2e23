// imf_penalize_sensitivity_noalloc: the filtered-sensitivity step for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside a host framework that owns every
// device allocation through its own pool and forbids outside ones during its step, and code
// that must never stall the device (cudaMalloc and cudaFree can synchronize the whole
// device). This entry point allocates nothing. Its only scratch is the file-scope array
// below, which every GPU that loads the library holds until the process exits. The caller
// still passes every input and output array.
//
// Scratch contents: one partial maximum of |S_phi| per chunk of kChunk voxels, then the
// final maximum. All calls share the array and each call overwrites what it reads, so
// nothing needs clearing between calls; calls that overlap on the GPU (on different streams,
// or from different host threads) race on the array and must not be issued.
#include <mutex>

#include "imf.h"
#include "imf_internal.cuh"

namespace {

constexpr int kNoallocThreads = 256;
constexpr int kItems = 16;
constexpr long kChunk = (long)kNoallocThreads * kItems;     // voxels reduced per partial
constexpr int kMaxPartials = 65536;                          // 256 KiB of partials
constexpr long kMaxVoxels = kChunk * kMaxPartials;           // 268,435,456 voxels

// partials[0 .. kMaxPartials-1], final maximum at [kMaxPartials]
static __device__ __align__(256) float g_noalloc_scratch[kMaxPartials + 64];

__device__ __forceinline__ float block_max_noalloc(float v)
{
    __shared__ float red[32];
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.f;
        for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    }
    return v;
}

// one partial maximum of |S_phi| over Omega_0 per chunk
__global__ void __launch_bounds__(kNoallocThreads) noalloc_partial_absmax(const float *sens, const uint8_t *fix, long n,
                                                                        float *scratch)
{
    const long base = (long)blockIdx.x * kChunk;
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const long i = base + (long)k * kNoallocThreads + threadIdx.x;
        if (i < n && !(fix && fix[i])) m = fmaxf(m, fabsf(sens[i]));
    }
    m = block_max_noalloc(m);
    if (threadIdx.x == 0) scratch[blockIdx.x] = m;
}

// maximum of the partials, written after them
__global__ void __launch_bounds__(kNoallocThreads) noalloc_final_max(int nparts, float *scratch)
{
    float m = 0.f;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) m = fmaxf(m, scratch[i]);
    m = block_max_noalloc(m);
    if (threadIdx.x == 0) scratch[kMaxPartials] = m;
}

// S = (1 - w) S_phi / max|S_phi| + w S_IMF (Eq. eq_filtered_sens, Eq. eq_accFilter)
__global__ void __launch_bounds__(kNoallocThreads) noalloc_penalize(float *sens, const float *rho, const float *fbar,
                                                                  const uint8_t *sec, long n, const float *scratch,
                                                                  float w, float tau)
{
    const float m = scratch[kMaxPartials];
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        sens[i] = imf::penalized_sensitivity(sens[i], rho[i], fbar[i], sec[i], m, w, tau);
}

// Device address of the scratch array, looked up once per device with that device current.
// The address stays valid for the life of the device's primary context: a caller that resets
// the device (cudaDeviceReset) must not call this entry point again in the same process.
std::mutex g_noalloc_mu;
float *g_noalloc_ptr[256] = {nullptr};

imf_status noalloc_scratch(float **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return IMF_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return IMF_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = (float *)p;
    }
    *out = g_noalloc_ptr[dev];
    return IMF_OK;
}

} // namespace

extern "C" imf_status imf_penalize_sensitivity_noalloc(float *sens, const float *rho_omega, const float *imf_bar,
                                                       const uint8_t *secluded, const uint8_t *fixture, long n,
                                                       double w_acc, double tau, void *cuda_stream)
{
    if (!sens || !rho_omega || !imf_bar || !secluded) return IMF_ERR_INVALID_ARG;
    if (n < 1 || n > kMaxVoxels) return IMF_ERR_INVALID_ARG;
    if (!(w_acc >= 0.0 && w_acc < 1.0) || !(tau >= 0.0 && tau <= 1.0)) return IMF_ERR_INVALID_ARG;
    float *scratch = nullptr;
    const imf_status st = noalloc_scratch(&scratch);
    if (st != IMF_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int nparts = (int)((n + kChunk - 1) / kChunk);
    noalloc_partial_absmax<<<nparts, kNoallocThreads, 0, s>>>(sens, fixture, n, scratch);
    noalloc_final_max<<<1, kNoallocThreads, 0, s>>>(nparts, scratch);
    long blocks = (n + kNoallocThreads - 1) / kNoallocThreads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    noalloc_penalize<<<(int)blocks, kNoallocThreads, 0, s>>>(sens, rho_omega, imf_bar, secluded, n, scratch,
                                                            (float)w_acc, (float)tau);
    return cudaGetLastError() == cudaSuccess ? IMF_OK : IMF_ERR_CUDA;
}
