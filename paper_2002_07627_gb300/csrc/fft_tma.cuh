// TMA-fed persistent axis pass of the two-pass register FFT (fft2.cuh): the y and z passes of
// the collision convolution's transforms (Alg. 1 Convolve; App. B's FFT convolution term),
// with the pointwise product of the design and tool spectra fused into the z pass.
//
// The arithmetic is the one of axis2_kernel (fft2_kernels.cu); what changes is how the pencils
// reach the registers. A block stays resident and walks a strided list of work items (kx
// chunk, orientation, batch row). For each item the tensor memory accelerator copies the W
// pencils of the chunk (and the W pencils of the pointwise factor) into a shared-memory stage
// as [row j][pencil w]; zero padding of short inputs comes from the copy's out-of-bounds fill.
// Two stages alternate: while the block transforms one item, the copy of its next item is in
// flight, so the memory system sees a steady stream instead of the load / compute / store
// phases of one-shot blocks. Results go straight from registers to global memory.
//
// Both factors of the split are template arguments of the loop (a runtime dispatch picks the
// instance before the loop; a loop around two runtime dispatches made the compiler keep every
// case's registers live), and only the splits fft2::choose_split returns are instantiated.
//
// Every wait on a copy is bounded (%globaltimer); on a timeout the block records
// IMF_ERR_TIMEOUT in the status word, waits (bounded again) for the copies it still has in
// flight and returns, so no copy lands in shared memory that a later block owns.
#pragma once
#include <cuda.h>

#include "fft2.cuh"
#include "imf.h"
#include "imf_internal.cuh"
#include "tc_primitives.cuh"

namespace imf {
namespace tma_fft {

constexpr int kStages = 2;

int sm_count();   // multiprocessors of the current device (fft_tma.cu)
// Tiled tensor map of 8-byte elements (complex64): dims innermost first, strides of dims 1.. in
// bytes, box in elements; false when a tensor map cannot describe it (fft_tma.cu).
bool encode_tiled(CUtensorMap *m, const void *ptr, int rank, const uint64_t *dims, const uint64_t *strides_bytes,
                  const uint32_t *box);
// the same for 4-byte elements (the direct path's packed BF16 hi / lo words)
bool encode_tiled_u32(CUtensorMap *m, const void *ptr, int rank, const uint64_t *dims, const uint64_t *strides_bytes,
                      const uint32_t *box);
// shortest pencil of the 16-slot shape the persistent kernel is built for (shorter ones, on
// tiny grids, keep the one-shot kernel; fewer instances keep the build short)
constexpr int kMinLength = 64;

struct Params {
    AxisArgs a;
    int axis_is_plane;   // 1: the FFT axis is the plane dimension of the tensor (z pass), 0: rows
    int nchunks, norient, nbatch;
    long items;
    int box_j, nbox, lrows;
};

template <int W> __host__ __device__ constexpr int threads(bool big) { return W * (big ? 32 : 16); }
static_assert(threads<16>(true) == 512, "the wide big-factor shape runs 512 threads");

__device__ __forceinline__ void decode_item(const Params &P, long it, int &chunk, int &o, int &b)
{
    chunk = (int)(it % P.nchunks);
    const long r = it / P.nchunks;
    o = (int)(r % P.norient);
    b = (int)(r / P.norient);
}

// One thread issues the tensor copies of item `it` into a stage (W pencils of the input, and of
// the factor when MUL), completing on the stage's mbarrier.
template <int MUL, int W>
__device__ __forceinline__ void issue_item(const Params &P, const void *in_map, const void *mul_map, long it,
                                           float2 *din, float2 *dmul, uint64_t *bar)
{
    int chunk, o, b;
    decode_item(P, it, chunk, o, b);
    tc::mbar_expect_tx(bar, (uint32_t)(P.nbox * P.box_j * W * sizeof(float2)) * (MUL ? 2u : 1u));
    const int c0 = chunk * W;
    for (int k = 0; k < P.nbox; ++k) {
        const int j0 = k * P.box_j;
        if (P.axis_is_plane) tc::tma_load_4d(din + (size_t)j0 * W, in_map, c0, b, j0, o, bar);
        else tc::tma_load_4d(din + (size_t)j0 * W, in_map, c0, j0, b, o, bar);
        if (MUL) {
            if (P.axis_is_plane) tc::tma_load_3d(dmul + (size_t)j0 * W, mul_map, c0, b, j0, bar);
            else tc::tma_load_3d(dmul + (size_t)j0 * W, mul_map, c0, j0, b, bar);
        }
    }
}

// The persistent loop for one split L = NA NB.
template <int S, int MUL, int W, int NA, int NB>
__device__ __forceinline__ void run_items(const Params &P, const void *in_map, const void *mul_map, float2 *st,
                                          size_t half, size_t stage, float2 *tile, const float2 *tw, uint64_t *bar)
{
    constexpr int LOGW = W == 8 ? 3 : 4;
    const AxisArgs &a = P.a;
    const int w = threadIdx.x & (W - 1), p = threadIdx.x >> LOGW;
    const long G = gridDim.x, first = blockIdx.x;
    const long mine = (P.items - first + G - 1) / G;      // items of this block: first + k G
    if (threadIdx.x == 0)
        for (int s = 0; s < kStages && s < mine; ++s)
            issue_item<MUL, W>(P, in_map, mul_map, first + s * G, st + s * stage, st + s * stage + half, &bar[s]);
    for (long k = 0; k < mine; ++k) {
        const int s = (int)(k % kStages);
        const bool timeout = !tc::mbar_wait(&bar[s], (uint32_t)((k / kStages) & 1));
        const long it = first + k * G;
        const float2 *sin_ = st + s * stage, *smul = sin_ + half;
        // pass 1: slot p = n1 < NB reads x[n1 + NB n2] (times the factor) from the stage and
        // transforms it in registers (after a timeout the values are not used)
        float2 v[NA];
        const bool act = p < NB;
        if (act) {
#pragma unroll
            for (int n2 = 0; n2 < NA; ++n2) {
                const int j = p + NB * n2;
                v[n2] = sin_[j * W + w];
                if (MUL) v[n2] = c_mul(v[n2], smul[j * W + w]);
            }
            fft2::dft_reg<S, NA>(v);
            fft2::twiddle<S, NA>(v, p, tw);
        }
        // one barrier: the stage is free, the previous item's tile reads are done, and every
        // thread knows whether a copy timed out
        if (__syncthreads_or(timeout)) {
            if (threadIdx.x == 0) {
                if (a.status) atomicCAS(a.status, 0, (int)IMF_ERR_TIMEOUT);
                // drain this block's copies still in flight (bounded) before leaving
                const long issued = k + kStages < mine ? k + kStages : mine;
                for (long q = k; q < issued; ++q) tc::mbar_wait(&bar[q % kStages], (uint32_t)((q / kStages) & 1));
            }
            return;
        }
        if (threadIdx.x == 0 && k + kStages < mine) {
            // generic-proxy reads of the stage above, async-proxy writes into it next
            tc::fence_async_smem();
            issue_item<MUL, W>(P, in_map, mul_map, first + (k + kStages) * G, st + s * stage, st + s * stage + half,
                               &bar[s]);
        }
        if (act) {
#pragma unroll
            for (int k2 = 0; k2 < NA; ++k2) tile[(p * NA + k2) * W + w] = v[k2];
        }
        __syncthreads();
        // pass 2: slot p = k2 < NA, NB-point DFT over n1; X[k2 + NA k1] -> out[j - j0] in the window
        int chunk, o, b;
        decode_item(P, it, chunk, o, b);
        const int c = chunk * W + w;
        if (p < NA && c < a.nx) {
            float2 u[NB];
#pragma unroll
            for (int n1 = 0; n1 < NB; ++n1) u[n1] = tile[(n1 * NA + p) * W + w];
            fft2::dft_reg<S, NB>(u);
            float2 *out = a.out + (long)o * a.out_so + (long)b * a.out_sb + c;
#pragma unroll
            for (int k1 = 0; k1 < NB; ++k1) {
                const int j = p + NA * k1 - a.j0;
                if (j >= 0 && j < a.lout) {
                    float2 y = c_scale(u[k1], a.scale);
                    if (a.conj_out) y.y = -y.y;
                    out[(long)j * a.out_sl] = y;
                }
            }
        }
        // the next iteration's barrier (after its wait) precedes any rewrite of the tile
    }
}

template <int S, bool BIG, int MUL, int W>
__global__ void __launch_bounds__(threads<W>(BIG))
    axis2_tma_kernel(const __grid_constant__ CUtensorMap in_map, const __grid_constant__ CUtensorMap mul_map,
                     Params P)
{
    constexpr int T = threads<W>(BIG);
    extern __shared__ unsigned char smraw[];
    const int A = P.a.A2, B = P.a.B2, L = A * B;
    // 128-byte aligned stages (tensor-copy destinations), then the tile, twiddles and barriers
    unsigned char *base = smraw + ((128 - (tc::smem_addr(smraw) & 127)) & 127);
    const size_t half = (size_t)P.lrows * W;
    const size_t stage = half * (MUL ? 2 : 1);
    float2 *st = reinterpret_cast<float2 *>(base);
    float2 *tile = st + kStages * stage;
    float2 *tw = tile + (size_t)L * W;
    uint64_t *bar = reinterpret_cast<uint64_t *>(tw + L);
    for (int i = threadIdx.x; i < L; i += T) tw[i] = P.a.tw[i];
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) tc::mbar_init(&bar[s], 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    constexpr int maxA = BIG ? fft2::kMaxFactorBig : fft2::kMaxFactor;
    auto outer = [&](auto AA) {
        constexpr int NA = decltype(AA)::value;
        auto inner = [&](auto BB) {
            constexpr int NB = decltype(BB)::value;
            if constexpr (fft2::is_split_choice(NA, NB, maxA) &&
                          (BIG ? NA > fft2::kMaxFactor : NA * NB >= kMinLength))
                run_items<S, MUL, W, NA, NB>(P, &in_map, &mul_map, st, half, stage, tile, tw, bar);
        };
        if constexpr (BIG) fft2::with_size_big(B, inner);
        else fft2::with_size(B, inner);
    };
    if constexpr (BIG) fft2::with_size_big(A, outer);
    else fft2::with_size(A, outer);
}

// ---------------------------------------------------------------------------------------------
// Warp-specialised variant: warp 0 is the producer (one lane issues the tensor copies), the
// other warps are consumers, 8 NA threads of them (pencil w = thread & 7, slot p = thread >> 3),
// so no warp idles through both DFT passes. Each stage has a "full" mbarrier (the copy's bytes)
// and an "empty" one (one arrival per consumer warp once it has read the stage), so the producer
// refills a stage as soon as it is free instead of at a block-wide barrier. Consumers meet once
// per item, at a named reduction barrier after writing the tile, which also makes them agree on a
// timed-out copy; the tile is double-buffered where shared memory allows (else a second named
// barrier guards it). Block barriers are never used after the set-up.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ bool bar_red_or(int id, int nthreads, bool v)
{
    uint32_t r;
    asm volatile("{\n.reg .pred pi, po;\nsetp.ne.u32 pi, %1, 0;\nbar.red.or.pred po, %2, %3, pi;\nselp.u32 %0, 1, 0, po;\n}\n"
                 : "=r"(r)
                 : "r"((uint32_t)v), "r"(id), "r"(nthreads)
                 : "memory");
    return r != 0;
}
__device__ __forceinline__ void bar_named(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}

struct WsLayout {
    int ntiles;           // 1 or 2 tile buffers
};

template <int S, int MUL, int W, int NA, int NB>
__device__ __forceinline__ void ws_items(const Params &P, const void *in_map, const void *mul_map, float2 *st,
                                         size_t half, size_t stage, float2 *tile, int ntiles, const float2 *tw,
                                         uint64_t *full, uint64_t *empty)
{
    constexpr int LOGW = W == 8 ? 3 : 4;
    const AxisArgs &a = P.a;
    const long G = gridDim.x, first = blockIdx.x;
    const long mine = (P.items - first + G - 1) / G;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncons = (int)blockDim.x - 32;
    const size_t tsz = (size_t)NA * NB * W;
    if (warp == 0) {
        // producer: one lane issues every copy of this block, refilling a stage once its empty
        // barrier shows that every consumer warp has read it
        if (lane != 0) return;
        for (long k = 0; k < mine; ++k) {
            const int s = (int)(k % kStages);
            if (k >= kStages && !tc::mbar_wait(&empty[s], (uint32_t)((k / kStages - 1) & 1))) {
                if (a.status) atomicCAS(a.status, 0, (int)IMF_ERR_TIMEOUT);
                // the consumers time out on the stage this copy would have filled
                for (long q = k - kStages + 1; q < k; ++q)
                    if (q >= 0) tc::mbar_wait(&full[q % kStages], (uint32_t)((q / kStages) & 1));
                return;
            }
            tc::fence_async_smem();
            issue_item<MUL, W>(P, in_map, mul_map, first + k * G, st + s * stage, st + s * stage + half, &full[s]);
        }
        return;
    }
    const int ct = threadIdx.x - 32, w = ct & (W - 1), p = ct >> LOGW;
    for (long k = 0; k < mine; ++k) {
        const int s = (int)(k % kStages);
        const bool timeout = !tc::mbar_wait(&full[s], (uint32_t)((k / kStages) & 1));
        const float2 *sin_ = st + s * stage, *smul = sin_ + half;
        float2 v[NA];
        const bool act = p < NB;
        if (act) {
#pragma unroll
            for (int n2 = 0; n2 < NA; ++n2) {
                const int j = p + NB * n2;
                v[n2] = sin_[j * W + w];
                if (MUL) v[n2] = c_mul(v[n2], smul[j * W + w]);
            }
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&empty[s]);
        float2 *tl = tile + (ntiles == 2 ? (size_t)(k & 1) * tsz : 0);
        if (act) {
            fft2::dft_reg<S, NA>(v);
            fft2::twiddle<S, NA>(v, p, tw);
#pragma unroll
            for (int k2 = 0; k2 < NA; ++k2) tl[(p * NA + k2) * W + w] = v[k2];
        }
        if (bar_red_or(1, ncons, timeout)) {
            if (a.status) atomicCAS(a.status, 0, (int)IMF_ERR_TIMEOUT);
            return;
        }
        int chunk, o, b;
        decode_item(P, first + k * G, chunk, o, b);
        const int c = chunk * W + w;
        if (p < NA && c < a.nx) {
            float2 u[NB];
#pragma unroll
            for (int n1 = 0; n1 < NB; ++n1) u[n1] = tl[(n1 * NA + p) * W + w];
            fft2::dft_reg<S, NB>(u);
            float2 *out = a.out + (long)o * a.out_so + (long)b * a.out_sb + c;
#pragma unroll
            for (int k1 = 0; k1 < NB; ++k1) {
                const int j = p + NA * k1 - a.j0;
                if (j >= 0 && j < a.lout) {
                    float2 y = c_scale(u[k1], a.scale);
                    if (a.conj_out) y.y = -y.y;
                    out[(long)j * a.out_sl] = y;
                }
            }
        }
        // one tile: its readers finish before the next item's pass 1 rewrites it
        if (ntiles == 1) bar_named(2, ncons);
    }
}

template <int S, bool BIG, int MUL, int W>
__global__ void __launch_bounds__(256) axis2_ws_kernel(const __grid_constant__ CUtensorMap in_map,
                                                       const __grid_constant__ CUtensorMap mul_map, Params P, int ntiles)
{
    extern __shared__ unsigned char smraw[];
    const int A = P.a.A2, B = P.a.B2, L = A * B;
    unsigned char *base = smraw + ((128 - (tc::smem_addr(smraw) & 127)) & 127);
    const size_t half = (size_t)P.lrows * W;
    const size_t stage = half * (MUL ? 2 : 1);
    float2 *st = reinterpret_cast<float2 *>(base);
    float2 *tile = st + kStages * stage;
    float2 *tw = tile + (size_t)ntiles * L * W;
    uint64_t *full = reinterpret_cast<uint64_t *>(tw + L), *empty = full + kStages;
    const int ncw = ((int)blockDim.x - 32) / 32;
    for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = P.a.tw[i];
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], ncw);
        }
        tc::fence_mbar_init();
    }
    __syncthreads();
    constexpr int maxA = BIG ? fft2::kMaxFactorBig : fft2::kMaxFactor;
    auto outer = [&](auto AA) {
        constexpr int NA = decltype(AA)::value;
        auto inner = [&](auto BB) {
            constexpr int NB = decltype(BB)::value;
            if constexpr (fft2::is_split_choice(NA, NB, maxA) &&
                          (BIG ? NA > fft2::kMaxFactor : NA * NB >= kMinLength))
                ws_items<S, MUL, W, NA, NB>(P, &in_map, &mul_map, st, half, stage, tile, ntiles, tw, full, empty);
        };
        if constexpr (BIG) fft2::with_size_big(B, inner);
        else fft2::with_size(B, inner);
    };
    if constexpr (BIG) fft2::with_size_big(A, outer);
    else fft2::with_size(A, outer);
}

// threads of the warp-specialised block: the producer warp and 8 NA consumer threads in warps
inline int ws_threads(int A) { return 32 + ((8 * A + 31) / 32) * 32; }

inline size_t ws_smem_bytes(const Params &P, int W, bool mul, int ntiles)
{
    const int L = P.a.A2 * P.a.B2;
    return 128 + (size_t)kStages * P.lrows * W * 8 * (mul ? 2 : 1) + (size_t)ntiles * L * W * 8 + (size_t)L * 8 +
           2 * kStages * 8;
}

template <int S, bool BIG, int MUL, int W>
bool launch_ws(const CUtensorMap &in_map, const CUtensorMap &mul_map, Params &P, cudaStream_t s)
{
    static_assert(W == 8, "the warp-specialised pass maps 8 pencils per thread row");
    const int T = ws_threads(P.a.A2);
    if (T > 256) return false;
    auto kernel = axis2_ws_kernel<S, BIG, MUL, W>;
    // two tiles when two blocks of that size still fit an SM, else one
    int ntiles = 2;
    size_t smem = ws_smem_bytes(P, W, MUL != 0, 2);
    if (2 * (smem + 1024) > 228 * 1024) {
        ntiles = 1;
        smem = ws_smem_bytes(P, W, MUL != 0, 1);
    }
    if (smem > 227 * 1024) return false;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, T, smem) != cudaSuccess || per < 1) {
        cudaGetLastError();
        return false;
    }
    const long blocks = P.items < (long)per * sm_count() ? P.items : (long)per * sm_count();
    kernel<<<(unsigned)blocks, T, smem, s>>>(in_map, mul_map, P, ntiles);
    return true;
}

// The six instances (16-slot shape s*, 32-slot shape b*; variant 0 = forward, 1 = inverse,
// 2 = inverse with the pointwise factor), each compiled from fft_tma_inst.cu in its own
// translation unit; false when nothing was launched.
#define IMF_TMA_DECL(name) bool name(const CUtensorMap &in_map, const CUtensorMap &mul_map, Params &P, bool ws, int W, cudaStream_t s);
IMF_TMA_DECL(launch_tma_s0)
IMF_TMA_DECL(launch_tma_s1)
IMF_TMA_DECL(launch_tma_s2)
IMF_TMA_DECL(launch_tma_b0)
IMF_TMA_DECL(launch_tma_b1)
IMF_TMA_DECL(launch_tma_b2)
#undef IMF_TMA_DECL


// Shared memory of one block: 128 bytes of alignment slack, the stages, the tile, the twiddles
// and the barriers.
inline size_t smem_bytes(const Params &P, int W, bool mul)
{
    const int L = P.a.A2 * P.a.B2;
    return 128 + (size_t)kStages * P.lrows * W * 8 * (mul ? 2 : 1) + (size_t)L * W * 8 + (size_t)L * 8 + kStages * 8;
}

template <int S, bool BIG, int MUL, int W>
bool launch_shape(const CUtensorMap &in_map, const CUtensorMap &mul_map, Params &P, cudaStream_t s)
{
    constexpr int T = threads<W>(BIG);
    const size_t smem = smem_bytes(P, W, MUL != 0);
    if (smem > 227 * 1024) return false;
    auto kernel = axis2_tma_kernel<S, BIG, MUL, W>;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, T, smem) != cudaSuccess || per < 1) {
        cudaGetLastError();
        return false;
    }
    const long blocks = P.items < (long)per * sm_count() ? P.items : (long)per * sm_count();
    kernel<<<(unsigned)blocks, T, smem, s>>>(in_map, mul_map, P);
    return true;
}

} // namespace tma_fft
} // namespace imf
