// Direct collision convolution on the tcgen05 tensor cores (Eq. eq_ident / eq_imf_4 computed
// as an implicit GEMM instead of through FFTs), for tools whose rotated supports are small.
//
// For a group of orientations r_0 .. r_{N-1} and its union tap list v_0 .. v_{K-1} (every
// offset that lies in at least one R_n T):
//   g_{r_n}(t) = sum_k A[t, k] B[n, k],   A[t, k] = rho_O(t + v_k),   B[n, k] = 1_{R_n T}(v_k).
// A block computes D = A B^T for 128 consecutive translations along x (M = 128) and all N
// orientations of the group, accumulating in TMEM (FP32). rho_O enters as two BF16 terms
// rho_O = hi + lo (the binary tool indicator is exact in BF16), so D = A_hi B^T + A_lo B^T and the
// input error is below 2^-16 of rho_O. B is loaded once per block by a bulk (TMA) copy in
// the K-major canonical layout; A is built in shared memory, chunk by chunk, by eight producer
// warps (two threads per tile row, half a chunk each) from a padded copy of rho_O that holds
// (hi, lo) in one 32-bit word; one thread issues the MMAs; the same eight warps read D back
// with tcgen05.ld (warp w reads TMEM lanes 32 (w mod 4) .. + 31 and half of the columns) and
// write g, the free bits and the near-threshold list in the layout of the FFT path. Every mbarrier wait is bounded; on a
// timeout the block records IMF_ERR_TIMEOUT, stops, and still frees its TMEM.
#include <cfloat>
#include <cuda_bf16.h>

#include "imf_internal.cuh"
#include "tc_primitives.cuh"

namespace imf {

namespace {

constexpr int kDM = 128;          // translations per tile (MMA M)
constexpr int kDKC = 64;          // taps per chunk
constexpr int kDProd = 256;       // 8 producer / epilogue warps: two threads per tile row
constexpr int kDThreads = kDProd + 32;   // + 1 MMA warp
constexpr uint32_t kStageBytes = kDM * kDKC * 2;   // one BF16 operand chunk

__device__ __forceinline__ uint16_t bf16_bits_rn(float x)
{
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

// ---------------------------------------------------------------------------------------
// padded rho_O with (hi, lo) BF16 halves: word = hi | lo << 16, zero outside the grid
// ---------------------------------------------------------------------------------------
__global__ void rho_hl_kernel(const float *rho, const uint8_t *fix, int nx, int ny, int nz, int lox, int loy,
                              int loz, int PX, int PY, int PZ, uint32_t *out)
{
    const long n = (long)PX * PY * PZ;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int x = (int)(i % PX) - lox;
        const int y = (int)((i / PX) % PY) - loy;
        const int z = (int)(i / ((long)PX * PY)) - loz;
        uint32_t w = 0;
        if (x >= 0 && y >= 0 && z >= 0 && x < nx && y < ny && z < nz) {
            const long j = ((long)z * ny + y) * nx + x;
            float r = rho[j];
            if (fix && fix[j]) r = fminf(1.f, r + 1.f);
            const uint16_t h = bf16_bits_rn(r);
            const float hf = __bfloat162float(__ushort_as_bfloat16(h));
            const uint16_t l = bf16_bits_rn(r - hf);
            w = (uint32_t)h | ((uint32_t)l << 16);
        }
        out[i] = w;
    }
}

// ---------------------------------------------------------------------------------------
// the direct kernel
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kDThreads, 2) direct_corr_kernel(DirectArgs a)
{
    extern __shared__ __align__(1024) uint8_t dsm[];
    const uint32_t bbytes = (uint32_t)a.kpad * a.N * 2;
    uint8_t *Bs = dsm;
    uint8_t *Ast = dsm + ((bbytes + 1023) & ~1023u);          // [stage][hi, lo]
    uint64_t *bars = (uint64_t *)(Ast + 4 * kStageBytes);       // full[2], empty[2], bload, dfull, dempty
    uint64_t *full = bars, *empty = bars + 2, *bload = bars + 4, *dfull = bars + 5, *dempty = bars + 6;
    uint32_t *tmem_slot = (uint32_t *)(bars + 8);
    __shared__ int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nchunk = a.kpad / kDKC;
    const int ntiles = a.ntiles_x * a.wy * a.wz;
    uint32_t ncols = 32;
    while (ncols < (uint32_t)a.N) ncols <<= 1;

    if (threadIdx.x == 0) {
        s_abort = 0;
        tc::mbar_init(&full[0], kDProd);
        tc::mbar_init(&full[1], kDProd);
        tc::mbar_init(&empty[0], 1);
        tc::mbar_init(&empty[1], 1);
        tc::mbar_init(bload, 1);
        tc::mbar_init(dfull, 1);
        tc::mbar_init(dempty, kDProd);
        tc::mbar_init(bars + 7, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 8) tc::tmem_alloc(tmem_slot, ncols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 8) {
        // ------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            tc::mbar_expect_tx(bload, bbytes);
            for (uint32_t off = 0; off < bbytes; off += 32768u) {
                const uint32_t n = min(32768u, bbytes - off);
                tc::bulk_g2s(Bs + off, (const uint8_t *)a.bmat + off, n, bload);
            }
            bool ok = tc::mbar_wait(bload, 0);
            const uint32_t idesc = tc::make_idesc_bf16(kDM, a.N);
            const uint32_t bsa = tc::smem_addr(Bs), asa = tc::smem_addr(Ast);
            long gc = 0;
            int tcount = 0;
            for (int t = blockIdx.x; ok && t < ntiles; t += gridDim.x, ++tcount) {
                if (tcount > 0) ok = tc::mbar_wait(dempty, (tcount - 1) & 1);
                tc::fence_after();
                for (int c = 0; ok && c < nchunk; ++c, ++gc) {
                    const int s = (int)(gc & 1);
                    const uint32_t u = (uint32_t)(gc >> 1);
                    if (!(ok = tc::mbar_wait(&full[s], u & 1))) break;
                    tc::fence_after();
#pragma unroll
                    for (int ks = 0; ks < kDKC / 16; ++ks) {
                        const uint32_t ahi = asa + (2 * s) * kStageBytes + ks * 2 * (kDM * 16);
                        const uint32_t alo = ahi + kStageBytes;
                        const uint32_t bk = bsa + (uint32_t)((c * kDKC + ks * 16) / 8) * (a.N * 16);
                        const uint64_t bd = tc::make_desc(bk, a.N * 16, 128);
                        tc::mma_bf16(tmem, tc::make_desc(ahi, kDM * 16, 128), bd, idesc, (c > 0 || ks > 0) ? 1u : 0u);
                        tc::mma_bf16(tmem, tc::make_desc(alo, kDM * 16, 128), bd, idesc, 1u);
                    }
                    tc::mma_commit(&empty[s]);
                }
                if (ok) tc::mma_commit(dfull);
            }
            if (!ok) {
                atomicExch(a.status, kDevTimeout);
                atomicExch(&s_abort, 1);
            }
            // drain: every MMA this thread issued has completed before TMEM is freed
            tc::mma_commit(bars + 7);
            if (!tc::mbar_wait(bars + 7, 0)) atomicExch(a.status, kDevTimeout);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------- producers / epilogue
        const int m = threadIdx.x & (kDM - 1);      // row of the tile = TMEM lane
        const int half = threadIdx.x >> 7;          // which half of each chunk / of the columns
        long gc = 0;
        int tcount = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tcount) {
            const int xs = t % a.ntiles_x, row = t / a.ntiles_x;
            const int y = row % a.wy, z = row / a.wy;
            const int x = xs * kDM + m;
            const int xc = min(x, a.wx - 1);
            // translation t = window index - kmax; padded index = t + lo
            const long pbase = ((long)(z - a.kz + a.loz) * a.PY + (y - a.ky + a.loy)) * a.PX + (xc - a.kx + a.lox);
            for (int c = 0; c < nchunk; ++c, ++gc) {
                const int s = (int)(gc & 1);
                const uint32_t u = (uint32_t)(gc >> 1);
                if (u > 0 && !(ok = tc::mbar_wait(&empty[s], (u - 1) & 1))) break;
                if (*((volatile int *)&s_abort)) { ok = false; break; }
                uint8_t *Ahi = Ast + (2 * s) * kStageBytes, *Alo = Ahi + kStageBytes;
                const int *taps = a.tapoff + c * kDKC;
                // 8 consecutive taps per step: one 16-byte store per operand (a warp writes 512
                // contiguous bytes of the canonical layout, no bank conflicts)
#pragma unroll
                for (int kk = half * (kDKC / 2); kk < (half + 1) * (kDKC / 2); kk += 8) {
                    uint32_t w[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) w[e] = __ldg(a.rhohl + pbase + __ldg(taps + kk + e));
                    uint4 vh, vl;
                    vh.x = (w[0] & 0xffffu) | (w[1] << 16); vl.x = (w[0] >> 16) | (w[1] & 0xffff0000u);
                    vh.y = (w[2] & 0xffffu) | (w[3] << 16); vl.y = (w[2] >> 16) | (w[3] & 0xffff0000u);
                    vh.z = (w[4] & 0xffffu) | (w[5] << 16); vl.z = (w[4] >> 16) | (w[5] & 0xffff0000u);
                    vh.w = (w[6] & 0xffffu) | (w[7] << 16); vl.w = (w[6] >> 16) | (w[7] & 0xffff0000u);
                    const uint32_t off = tc::kmajor_offset(m, kk, kDM);
                    *(uint4 *)(Ahi + off) = vh;
                    *(uint4 *)(Alo + off) = vl;
                }
                tc::fence_async_smem();
                tc::mbar_arrive(&full[s]);
            }
            if (!ok) break;
            if (!(ok = tc::mbar_wait(dfull, tcount & 1))) break;
            tc::fence_after();
            // epilogue: D row m, this warp's half of the columns (= orientations of the group)
            const bool valid = x < a.wx;
            const int q = warp & 3;
            for (int n0 = half * (a.N / 2); n0 < (half + 1) * (a.N / 2); n0 += 8) {
                float v[8];
                tc::tmem_ld8(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)n0, v);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int n = n0 + j;
                    if (n >= a.nb) break;              // uniform across the warp
                    const float gv = fmaxf(v[j], 0.f);
                    float *g = a.g + (long)n * a.g_so + (long)z * a.g_sz + (long)y * a.g_sy;
                    if (valid) g[x] = gv;
                    const unsigned fb = __ballot_sync(0xffffffffu, valid && gv <= a.theta);
                    uint32_t *bw = a.bits + (long)n * a.b_so + (long)z * a.b_sz + (long)y * a.b_sy;
                    if (lane == 0 && xs * kDM + q * 32 < a.wx) bw[(xs * kDM + q * 32) >> 5] = fb;
                    if (a.flag) {
                        const bool near = valid && fabsf(gv - a.theta) <= a.band;
                        const unsigned nm = __ballot_sync(0xffffffffu, near);
                        if (nm) {
                            int base = 0;
                            if (lane == 0) {
                                base = atomicAdd(a.flag_count, __popc(nm));
                                atomicAdd(a.flag_total, __popc(nm));
                            }
                            base = __shfl_sync(0xffffffffu, base, 0);
                            if (near) {
                                const int slot = base + __popc(nm & ((1u << lane) - 1u));
                                if (slot < a.flag_cap) {
                                    const long lin = ((long)z * a.wy + y) * a.wx + x;
                                    a.flags[slot] = make_int2(a.orient_base + n, (int)lin);
                                } else {
                                    atomicExch(a.status, kDevOverflow);
                                }
                            }
                        }
                    }
                }
            }
            tc::fence_before();
            tc::mbar_arrive(dempty);
        }
        if (!ok) {
            atomicExch(a.status, kDevTimeout);
            atomicExch(&s_abort, 1);
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 8) tc::tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------------------------------
// self-test: D[128 x N] = A[128 x K] B[N x K]^T from row-major BF16 inputs
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128, 1) mma_selftest_kernel(const uint16_t *A, const uint16_t *B, float *D, int N,
                                                              int K, int *status)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *As = sm, *Bs = sm + kDM * K * 2;
    uint64_t *bar = (uint64_t *)(Bs + (size_t)N * K * 2);
    uint32_t *tslot = (uint32_t *)(bar + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t ncols = 32;
    while (ncols < (uint32_t)N) ncols <<= 1;
    for (int i = threadIdx.x; i < kDM * K; i += blockDim.x) {
        const int r = i / K, k = i % K;
        *(uint16_t *)(As + tc::kmajor_offset(r, k, kDM)) = A[i];
    }
    for (int i = threadIdx.x; i < N * K; i += blockDim.x) {
        const int r = i / K, k = i % K;
        *(uint16_t *)(Bs + tc::kmajor_offset(r, k, N)) = B[i];
    }
    tc::fence_async_smem();
    if (threadIdx.x == 0) {
        tc::mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    if (threadIdx.x == 0) {
        const uint32_t idesc = tc::make_idesc_bf16(kDM, N);
        for (int ks = 0; ks < K / 16; ++ks) {
            const uint64_t ad = tc::make_desc(tc::smem_addr(As) + ks * 2 * (kDM * 16), kDM * 16, 128);
            const uint64_t bd = tc::make_desc(tc::smem_addr(Bs) + ks * 2 * (N * 16), N * 16, 128);
            tc::mma_bf16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
        }
        tc::mma_commit(bar);
    }
    const bool ok = tc::mbar_wait(bar, 0);
    tc::fence_after();
    if (ok) {
        for (int n0 = 0; n0 < N; n0 += 8) {
            float v[8];
            tc::tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)n0, v);
#pragma unroll
            for (int j = 0; j < 8; ++j) D[(warp * 32 + lane) * N + n0 + j] = v[j];
        }
    } else if (threadIdx.x == 0) {
        *status = kDevTimeout;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

} // namespace

size_t direct_smem_bytes(int kpad, int N)
{
    const size_t b = ((size_t)kpad * N * 2 + 1023) & ~(size_t)1023;
    return b + 4 * (size_t)kStageBytes + 8 * sizeof(uint64_t) + 16;
}

void launch_rho_hl(const float *rho, const uint8_t *fix, int nx, int ny, int nz, int lox, int loy, int loz, int PX,
                   int PY, int PZ, uint32_t *out, cudaStream_t s)
{
    long n = (long)PX * PY * PZ;
    long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    rho_hl_kernel<<<(int)b, 256, 0, s>>>(rho, fix, nx, ny, nz, lox, loy, loz, PX, PY, PZ, out);
}

void launch_direct(const DirectArgs &a, int nsm, cudaStream_t s)
{
    const size_t smem = direct_smem_bytes(a.kpad, a.N);
    cudaFuncSetAttribute(direct_corr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int ntiles = a.ntiles_x * a.wy * a.wz;
    const int grid = ntiles < 2 * nsm ? ntiles : 2 * nsm;
    direct_corr_kernel<<<grid, kDThreads, smem, s>>>(a);
}

int run_mma_selftest(const uint16_t *A, const uint16_t *B, float *D, int N, int K, int *status, cudaStream_t s)
{
    const size_t smem = (size_t)kDM * K * 2 + (size_t)N * K * 2 + 64;
    if (N < 16 || N > 256 || N % 16 || K < 16 || K % 16 || smem > 200 * 1024) return -1;
    cudaFuncSetAttribute(mma_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    mma_selftest_kernel<<<1, 128, smem, s>>>(A, B, D, N, K, status);
    return 0;
}

} // namespace imf
