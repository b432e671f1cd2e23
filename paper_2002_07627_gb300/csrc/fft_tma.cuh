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
        if (__syncthreads_or(timeout)) {
            if (threadIdx.x == 0) {
                if (a.status) atomicCAS(a.status, 0, (int)IMF_ERR_TIMEOUT);
                // drain this block's copies still in flight (bounded) before leaving
                const long issued = k + kStages < mine ? k + kStages : mine;
                for (long q = k; q < issued; ++q) tc::mbar_wait(&bar[q % kStages], (uint32_t)((q / kStages) & 1));
            }
            return;
        }
        const long it = first + k * G;
        const float2 *sin_ = st + s * stage, *smul = sin_ + half;
        // pass 1: slot p = n1 < NB reads x[n1 + NB n2] (times the factor) from the stage
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
        // the stage is free (and the previous item's tile reads are done) past this barrier
        __syncthreads();
        if (threadIdx.x == 0 && k + kStages < mine) {
            // generic-proxy reads of the stage above, async-proxy writes into it next
            tc::fence_async_smem();
            issue_item<MUL, W>(P, in_map, mul_map, first + (k + kStages) * G, st + s * stage, st + s * stage + half,
                               &bar[s]);
        }
        if (act) {
            fft2::dft_reg<S, NA>(v);
            fft2::twiddle<S, NA>(v, p, tw);
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

// The six instances (16-slot shape s*, 32-slot shape b*; variant 0 = forward, 1 = inverse,
// 2 = inverse with the pointwise factor), each compiled from fft_tma_inst.cu in its own
// translation unit; false when nothing was launched.
#define IMF_TMA_DECL(name) bool name(const CUtensorMap &in_map, const CUtensorMap &mul_map, Params &P, cudaStream_t s);
IMF_TMA_DECL(launch_tma_s0)
IMF_TMA_DECL(launch_tma_s1)
IMF_TMA_DECL(launch_tma_s2)
IMF_TMA_DECL(launch_tma_b0)
IMF_TMA_DECL(launch_tma_b1)
IMF_TMA_DECL(launch_tma_b2)
#undef IMF_TMA_DECL

int sm_count();

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
