// Inverse x pass with the collision threshold (Eq. eq_conv_D) as a persistent kernel fed by
// tensor copies: the same arithmetic as irfft2_threshold_kernel (fft2_kernels.cu; the helpers
// in xpass.cuh), with the rows reaching shared memory by copy instead of strided loads.
//
// A block stays resident and walks a strided list of items (group of R = 256 / A window rows,
// orientation slot). One thread issues a tiled tensor copy of an item's R rows of half spectrum
// (Hs complex each, contiguous rows) into a shared-memory stage (128-byte aligned, as tensor
// copies require); two stages alternate, so the
// next item's rows are in flight while the current ones are transformed. Both factors of the
// split are template arguments of the loop (only the splits the planner picks are built), and
// every wait on a copy is bounded (IMF_ERR_TIMEOUT, own copies drained, then return).
#include "fft_tma.cuh"
#include "xpass.cuh"

namespace imf {

namespace {

constexpr int kXT = 256;      // threads per block
constexpr int kXStages = 2;

struct XParams {
    IrfftArgs a;
    int hs;                   // complex per row (the row stride)
    int R, ngroups, norient;
    long items;
};

// complex elements per stage: R rows of hs, rounded up to 128 bytes so that every stage (a
// tensor-copy destination) starts on a 128-byte boundary whatever R = 256 / A is
__host__ __device__ inline size_t x_stage(const XParams &P) { return ((size_t)P.R * P.hs + 15) & ~(size_t)15; }

__device__ __forceinline__ void x_issue(const XParams &P, const void *map, long it, float2 *dst, uint64_t *bar)
{
    const int g = (int)(it % P.ngroups), o = (int)(it / P.ngroups);
    tc::mbar_expect_tx(bar, (uint32_t)(P.R * P.hs * sizeof(float2)));
    tc::tma_load_3d(dst, map, 0, g * P.R, o, bar);
}

template <int NA, int NB>
__device__ __forceinline__ void x_items(const XParams &P, const void *map, float2 *st, size_t stage, float2 *tile,
                                        uint8_t *sflag, const float2 *twM, const float2 *twP, uint64_t *bar)
{
    const IrfftArgs &a = P.a;
    constexpr int A = NA, B = NB, Ap = A | 1;
    const int M = a.M, ld = (M > B * Ap ? M : B * Ap) + 1, fp = (2 * M + 31) & ~31;
    const long G = gridDim.x, first = blockIdx.x;
    const long mine = (P.items - first + G - 1) / G;
    if (threadIdx.x == 0)
        for (int s = 0; s < kXStages && s < mine; ++s) x_issue(P, map, first + s * G, st + s * stage, &bar[s]);
    for (long k = 0; k < mine; ++k) {
        const int s = (int)(k % kXStages);
        const bool timeout = !tc::mbar_wait(&bar[s], (uint32_t)((k / kXStages) & 1));
        if (__syncthreads_or(timeout)) {
            if (threadIdx.x == 0) {
                if (a.status) atomicCAS(a.status, 0, (int)IMF_ERR_TIMEOUT);
                const long issued = k + kXStages < mine ? k + kXStages : mine;
                for (long q = k; q < issued; ++q) tc::mbar_wait(&bar[q % kXStages], (uint32_t)((q / kXStages) & 1));
            }
            return;
        }
        const long it = first + k * G;
        const int g = (int)(it % P.ngroups);
        const long o = it / P.ngroups;
        const int r0 = g * P.R, nr = min(P.R, a.rows - r0);
        const float2 *rin = st + s * stage;
        {
            // pass 1: row w gets the threads w B .. w B + B - 1 (samples packed from the stage)
            const int w = threadIdx.x / B, p = threadIdx.x - w * B;
            if (w < nr) {
                float2 v[NA];
                x_pack<NA>(rin + (long)w * P.hs, p, B, M, twP, v);
                fft2::pass1<1, NA>(v, p, twM);
                float2 *line = tile + w * ld;
#pragma unroll
                for (int k2 = 0; k2 < NA; ++k2) line[p * Ap + k2] = v[k2];
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && k + kXStages < mine) {
            // the stage was read above (generic proxy); the copy into it comes next (async proxy)
            tc::fence_async_smem();
            x_issue(P, map, first + (k + kXStages) * G, st + s * stage, &bar[s]);
        }
        {
            // pass 2: row w gets the threads w A .. w A + A - 1, then the threshold epilogue
            const int w = threadIdx.x / A, p = threadIdx.x - w * A;
            const bool act = w < nr;
            const float2 *line = tile + w * ld;
            float2 u[NB];
            if (act) {
#pragma unroll
                for (int n1 = 0; n1 < NB; ++n1) u[n1] = line[n1 * Ap + p];
                fft2::dft_reg<1, NB>(u);
            }
            x_epilogue<NB>(a, u, A, p, act, r0 + w, o, sflag + (act ? w : 0) * fp, threadIdx.x & 31);
        }
        if (a.write_bits) {
            __syncthreads();
            x_pack_bits<kXT>(a, sflag, fp, r0, nr, o);
        }
        // the next iteration's barrier (after its wait) precedes any rewrite of the tile
    }
}

// blocks per SM an instance is compiled for: three (80 registers) where that keeps the split's
// registers without spilling, two for the longest ones (M above 210)
__host__ __device__ constexpr int x_min_blocks(int na, int nb) { return na * nb > 210 ? 2 : 3; }

// one instance per split (A, B) of the x length, so that each gets its own register allocation
template <int NA, int NB>
__global__ void __launch_bounds__(kXT, x_min_blocks(NA, NB)) irfft2_tma_kernel(const __grid_constant__ CUtensorMap map,
                                                                               XParams P)
{
    extern __shared__ unsigned char smraw[];
    const IrfftArgs &a = P.a;
    constexpr int A = NA, B = NB, Ap = A | 1;
    const int M = a.M;
    const int ld = (M > B * Ap ? M : B * Ap) + 1, fp = (2 * M + 31) & ~31;
    unsigned char *base = smraw + ((128 - (tc::smem_addr(smraw) & 127)) & 127);
    const size_t stage = x_stage(P);
    float2 *st = reinterpret_cast<float2 *>(base);
    float2 *tile = st + kXStages * stage;
    float2 *twM = tile + (size_t)P.R * ld, *twP = twM + M;
    uint8_t *sflag = reinterpret_cast<uint8_t *>(twP + M + 1 + 1);    // 16-byte aligned below
    sflag = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(sflag) + 15) & ~uintptr_t(15));
    uint64_t *bar = reinterpret_cast<uint64_t *>(sflag + (size_t)P.R * fp);
    for (int i = threadIdx.x; i < M; i += kXT) twM[i] = a.twM[i];
    for (int i = threadIdx.x; i <= M; i += kXT) twP[i] = a.twP[i];
    if (threadIdx.x == 0) {
        for (int s = 0; s < kXStages; ++s) tc::mbar_init(&bar[s], 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    x_items<NA, NB>(P, &map, st, stage, tile, sflag, twM, twP, bar);
}

size_t x_tma_smem(const XParams &P)
{
    const IrfftArgs &a = P.a;
    const int A = a.A2, B = a.B2, M = a.M, Ap = A | 1;
    const int ld = (M > B * Ap ? M : B * Ap) + 1, fp = (2 * M + 31) & ~31;
    return 128 + (size_t)kXStages * x_stage(P) * 8 + (size_t)P.R * ld * 8 + (size_t)(2 * M + 2) * 8 + 16 +
           (size_t)P.R * fp + 8 * kXStages + 8;
}

} // namespace

bool launch_irfft2_tma(const IrfftArgs &a, int hs, int norient, cudaStream_t s)
{
    if (a.A2 <= 0 || a.B2 <= 0 || a.A2 * a.B2 != a.M) return false;
    if (!fft2::is_split_choice(a.A2, a.B2, fft2::kMaxFactor) || a.M < tma_fft::kMinLength) return false;
    if (hs > 256 || hs < a.M + 1 || (hs & 1) || a.in_sy != hs || a.in_sz != (long)a.rows_y * a.in_sy) return false;
    XParams P{};
    P.a = a;
    P.hs = hs;
    P.R = kXT / a.A2;
    P.ngroups = (a.rows + P.R - 1) / P.R;
    P.norient = norient;
    P.items = (long)P.ngroups * norient;
    if (P.items < 1) return true;
    const long os = a.in_so > 0 ? a.in_so : (long)a.rows * hs;
    const uint64_t dims[3] = {(uint64_t)hs, (uint64_t)a.rows, (uint64_t)norient};
    const uint64_t strides[2] = {(uint64_t)hs * 8, (uint64_t)os * 8};
    const uint32_t box[3] = {(uint32_t)hs, (uint32_t)P.R, 1};
    CUtensorMap map;
    if (!tma_fft::encode_tiled(&map, a.in, 3, dims, strides, box)) return false;
    const size_t smem = x_tma_smem(P);
    if (smem > 227 * 1024) return false;
    bool launched = false;
    fft2::with_size(a.A2, [&](auto AA) {
        constexpr int NA = decltype(AA)::value;
        fft2::with_size(a.B2, [&](auto BB) {
            constexpr int NB = decltype(BB)::value;
            if constexpr (fft2::is_split_choice(NA, NB, fft2::kMaxFactor) && NA * NB >= tma_fft::kMinLength) {
                auto kern = irfft2_tma_kernel<NA, NB>;
                if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
                    cudaGetLastError();
                    return;
                }
                int per = 0;
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kXT, smem) != cudaSuccess || per < 1) {
                    cudaGetLastError();
                    return;
                }
                const long blocks =
                    P.items < (long)per * tma_fft::sm_count() ? P.items : (long)per * tma_fft::sm_count();
                kern<<<(unsigned)blocks, kXT, smem, s>>>(map, P);
                launched = true;
            }
        });
    });
    return launched;
}

} // namespace imf
