// Direct collision convolution on the tcgen05 tensor cores (Eq. eq_ident / eq_imf_4 computed
// as an implicit GEMM instead of through FFTs), for tools whose rotated supports are small.
//
// For a group of orientations r_0 .. r_{N-1} and its union tap list v_0 .. v_{K-1} (every
// offset that lies in at least one R_n T):
//   g_{r_n}(t) = sum_k A[t, k] B[n, k],   A[t, k] = rho_O(t + v_k),   B[n, k] = 1_{R_n T}(v_k).
// A block walks tiles of 128 translations (32 consecutive x by 2 y by 2 z, or 32 by 4 by 1 in
// 2D; MMA M = 128) and computes D = A B^T for all N orientations of the group, accumulating in
// TMEM (FP32). rho_O enters as two BF16 terms rho_O = hi + lo (the binary tool indicator is exact
// in BF16), so D = A_hi B^T + A_lo B^T and the input error is below 2^-16 of rho_O.
//
// Data movement: the rho_O neighbourhood a tile reads (a box of (hi, lo) words, the tile
// dilated by the union's extent) arrives by one tiled tensor copy, issued for the next tile as
// soon as every producer has built its last chunk of the current one, so that it lands while the
// last MMAs and the epilogue of the current tile run; B arrives 64 taps at a time by bulk
// copies into four slots (with the chunk's tap offsets), two chunks ahead of the A build; sixteen
// producer warps (four threads per tile row, a quarter of a chunk each) build A in shared memory
// from the box, in the K-major canonical layout, chunk by chunk into two stages; one thread issues
// the MMAs; the same sixteen warps read D back with tcgen05.ld (warp w reads TMEM lanes
// 32 (w mod 4) .. + 31 and every fourth group of 8 columns)
// and write g, the free bits and the near-threshold list in the layout of the FFT path. Every
// mbarrier wait is bounded; on a timeout the block records IMF_ERR_TIMEOUT, stops, waits for its
// own copies and MMAs, and still frees its TMEM.
#include <cfloat>
#include <cuda_bf16.h>

#include "fft_tma.cuh"
#include "imf_internal.cuh"
#include "tc_primitives.cuh"

namespace imf {

namespace {

constexpr int kDM = 128;          // translations per tile (MMA M)
constexpr int kDKC = 64;          // taps per chunk
constexpr int kDProd = 512;       // 16 producer / epilogue warps: four threads per tile row
constexpr int kDThreads = kDProd + 32;   // + 1 MMA warp
constexpr uint32_t kStageBytes = kDM * kDKC * 2;   // one BF16 operand chunk
constexpr int kBSlots = 4;        // B chunk slots
constexpr int kBAhead = 2;        // B copies run this many chunks ahead of the A build (slot reuse:
                                  // chunk gc + kBAhead takes the slot of chunk gc - 2, whose MMAs
                                  // the build of chunk gc has seen complete; six ahead in eight
                                  // slots measured slower: the slots crowd out larger groups)

// byte offsets of the regions of the kernel's dynamic shared memory (after 1024-byte alignment)
struct DirectLayout {
    uint32_t bchunk, box_bytes, b_off, box_off, bar_off, total;
};
__host__ __device__ inline DirectLayout direct_layout(int N, long box_words)
{
    DirectLayout L;
    L.bchunk = (uint32_t)N * 128 + 256;                         // N rows x 64 taps of BF16, then the 64 taps' box offsets
    L.box_bytes = (uint32_t)((box_words * 4 + 127) / 128 * 128);
    L.b_off = 4 * kStageBytes;                                  // A: [stage][hi, lo]
    L.box_off = L.b_off + kBSlots * L.bchunk;
    L.bar_off = L.box_off + L.box_bytes;
    L.total = L.bar_off + (9 + kBSlots) * 8 + 16;
    return L;
}

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
__global__ void __launch_bounds__(kDThreads, 1) direct_corr_kernel(const __grid_constant__ CUtensorMap box_map,
                                                                    DirectArgs a)
{
    extern __shared__ uint8_t dsm_raw[];
    uint8_t *dsm = dsm_raw + ((1024 - (tc::smem_addr(dsm_raw) & 1023)) & 1023);
    const DirectLayout Lo = direct_layout(a.N, (long)a.BX * a.BY * a.BZ);
    uint8_t *Ast = dsm;
    uint8_t *Bst = dsm + Lo.b_off;
    uint32_t *boxes = reinterpret_cast<uint32_t *>(dsm + Lo.box_off);
    uint64_t *bars = reinterpret_cast<uint64_t *>(dsm + Lo.bar_off);
    // full[2] (A built), empty[2] (stage's MMAs done), bfull[4] (B copy), boxfull (box copy),
    // boxfree (every producer done with the box), dfull, dempty, drain
    uint64_t *full = bars, *empty = bars + 2, *bfull = bars + 4, *boxfull = bars + 4 + kBSlots;
    uint64_t *boxfree = boxfull + 1, *dfull = boxfull + 2, *dempty = boxfull + 3, *drain = boxfull + 4;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(boxfull + 5);
    __shared__ int s_abort;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nchunk = a.kpad / kDKC;
    const int ntiles = a.ntx * a.nty * a.ntz;
    const int G = gridDim.x;
    const long mine = (int)blockIdx.x < ntiles ? (ntiles - (int)blockIdx.x + G - 1) / G : 0;
    const long total = mine * nchunk;
    const uint32_t box_words = (uint32_t)a.BX * a.BY * a.BZ;
    uint32_t ncols = 32;
    while (ncols < (uint32_t)a.N) ncols <<= 1;

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&full[i], kDProd);
            tc::mbar_init(&empty[i], 1);
        }
        tc::mbar_init(boxfull, 1);
        tc::mbar_init(boxfree, kDProd);
        for (int i = 0; i < kBSlots; ++i) tc::mbar_init(&bfull[i], 1);
        tc::mbar_init(dfull, 1);
        tc::mbar_init(dempty, kDProd);
        tc::mbar_init(drain, 1);
        tc::fence_mbar_init();
    }
    if (warp == kDProd / 32) tc::tmem_alloc(tmem_slot, ncols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == kDProd / 32) {
        // ------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc::make_idesc_bf16(kDM, a.N);
            const uint32_t asa = tc::smem_addr(Ast), bsa = tc::smem_addr(Bst);
            bool ok = true;
            long gc = 0;
            for (long k = 0; ok && k < mine; ++k) {
                if (k > 0) ok = tc::mbar_wait(dempty, (uint32_t)((k - 1) & 1));
                tc::fence_after();
                for (int c = 0; ok && c < nchunk; ++c, ++gc) {
                    const int s = (int)(gc & 1), bs = (int)(gc % kBSlots);
                    if (!(ok = tc::mbar_wait(&full[s], (uint32_t)((gc >> 1) & 1)))) break;
                    if (!(ok = tc::mbar_wait(&bfull[bs], (uint32_t)((gc / kBSlots) & 1)))) break;
                    tc::fence_after();
#pragma unroll
                    for (int ks = 0; ks < kDKC / 16; ++ks) {
                        const uint32_t ahi = asa + (2 * s) * kStageBytes + ks * 2 * (kDM * 16);
                        const uint32_t alo = ahi + kStageBytes;
                        const uint32_t bk = bsa + bs * Lo.bchunk + (uint32_t)ks * 2 * (a.N * 16);   // 16-byte aligned
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
            tc::mma_commit(drain);
            if (!tc::mbar_wait(drain, 0)) atomicExch(a.status, kDevTimeout);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------- producers / epilogue
        const int m = threadIdx.x & (kDM - 1);      // row of the tile = TMEM lane
        const int quarter = threadIdx.x >> 7;       // which quarter of each chunk / of the column groups
        const int xl = m & 31, yl = (m >> 5) % a.TY, zl = (m >> 5) / a.TY;
        const int base_m = a.sx + xl + a.BX * (yl + a.BY * zl);
        // copies issued by thread 0: the last box use and B use per slot (-1: none)
        long last_box = -1, last_b[kBSlots];
        for (int i = 0; i < kBSlots; ++i) last_b[i] = -1;
        // box use b = (tile k = b / nslab, slab b % nslab)
        auto issue_box = [&](long b) {
            const long k = b / a.nslab;
            const int sl = (int)(b - k * a.nslab);
            const int t = (int)blockIdx.x + (int)k * G;
            const int tx = t % a.ntx, r = t / a.ntx, ty = r % a.nty, tz = r / a.nty;
            const int cx = 32 * tx - a.kx + a.vlo[0] + a.lox - a.sx;     // a multiple of 4
            const int cy = a.TY * ty - a.ky + a.vlo[1] + a.loy;
            const int cz = a.TZ * tz - a.kz + a.vlo[2] + a.loz + a.slab_z0[sl];
            tc::mbar_expect_tx(boxfull, box_words * 4);
            tc::tma_load_3d(boxes, &box_map, cx, cy, cz, boxfull);
            last_box = b;
        };
        auto issue_b = [&](long g2) {
            const int slot = (int)(g2 % kBSlots);
            const int c = (int)(g2 % nchunk);
            const uint32_t bbytes = Lo.bchunk - 256;
            tc::mbar_expect_tx(&bfull[slot], Lo.bchunk);
            tc::bulk_g2s(Bst + slot * Lo.bchunk, reinterpret_cast<const uint8_t *>(a.bmat) + (size_t)c * bbytes, bbytes,
                         &bfull[slot]);
            tc::bulk_g2s(Bst + slot * Lo.bchunk + bbytes, a.tapoff + c * kDKC, 256, &bfull[slot]);
            last_b[slot] = g2;
        };
        if (threadIdx.x == 0) {
            if (mine > 0) issue_box(0);
            for (long g2 = 0; g2 < kBAhead && g2 < total; ++g2) issue_b(g2);
        }
        long gc = 0, bu = 0;                      // chunks and box uses so far
        const long units = mine * a.nslab;
        bool ok = true;
        for (long k = 0; k < mine; ++k) {
          for (int sl = 0; sl < a.nslab; ++sl, ++bu) {
            if (!(ok = tc::mbar_wait(boxfull, (uint32_t)(bu & 1)))) break;
            const uint32_t *box = boxes + base_m;
            for (int c = a.slab_c0[sl]; c < a.slab_c0[sl + 1]; ++c, ++gc) {
                const int s = (int)(gc & 1);
                const uint32_t u = (uint32_t)(gc >> 1);
                if (u > 0 && !(ok = tc::mbar_wait(&empty[s], (u - 1) & 1))) break;
                if (*((volatile int *)&s_abort)) { ok = false; break; }
                // slot (gc + kBAhead) mod kBSlots last held chunk gc - 2, whose MMAs the wait above
                // saw complete
                if (threadIdx.x == 0 && gc + kBAhead < total) {
                    tc::fence_async_smem();      // the slot's tap offsets were read by the generic proxy
                    issue_b(gc + kBAhead);
                }
                // this chunk's tap offsets arrived with its B (issued kBAhead chunks ago)
                const int bs = (int)(gc % kBSlots);
                if (!(ok = tc::mbar_wait(&bfull[bs], (uint32_t)((gc / kBSlots) & 1)))) break;
                uint8_t *Ahi = Ast + (2 * s) * kStageBytes, *Alo = Ahi + kStageBytes;
                const int *taps = reinterpret_cast<const int *>(Bst + bs * Lo.bchunk + (Lo.bchunk - 256));
                // 8 taps per step: eight words of the box, one 16-byte store per operand (a warp
                // reads 32 consecutive words per tap and writes 512 contiguous bytes)
#pragma unroll
                for (int kk = quarter * (kDKC / 4); kk < (quarter + 1) * (kDKC / 4); kk += 8) {
                    const int4 o0 = *reinterpret_cast<const int4 *>(taps + kk);
                    const int4 o1 = *reinterpret_cast<const int4 *>(taps + kk + 4);
                    uint32_t w[8];
                    w[0] = box[o0.x]; w[1] = box[o0.y]; w[2] = box[o0.z]; w[3] = box[o0.w];
                    w[4] = box[o1.x]; w[5] = box[o1.y]; w[6] = box[o1.z]; w[7] = box[o1.w];
                    uint4 vh, vl;
                    vh.x = (w[0] & 0xffffu) | (w[1] << 16); vl.x = (w[0] >> 16) | (w[1] & 0xffff0000u);
                    vh.y = (w[2] & 0xffffu) | (w[3] << 16); vl.y = (w[2] >> 16) | (w[3] & 0xffff0000u);
                    vh.z = (w[4] & 0xffffu) | (w[5] << 16); vl.z = (w[4] >> 16) | (w[5] & 0xffff0000u);
                    vh.w = (w[6] & 0xffffu) | (w[7] << 16); vl.w = (w[6] >> 16) | (w[7] & 0xffff0000u);
                    const uint32_t off = tc::kmajor_offset(m, kk, kDM);
                    *reinterpret_cast<uint4 *>(Ahi + off) = vh;
                    *reinterpret_cast<uint4 *>(Alo + off) = vl;
                }
                tc::fence_async_smem();
                tc::mbar_arrive(&full[s]);
            }
            if (!ok) break;
            // this slab's reads of the box are done: once every producer says so, thread 0 refills
            // it with the next slab's or tile's box (generic-proxy reads before the async-proxy write)
            tc::mbar_arrive(boxfree);
            if (threadIdx.x == 0 && bu + 1 < units) {
                if (!(ok = tc::mbar_wait(boxfree, (uint32_t)(bu & 1)))) break;
                tc::fence_async_smem();
                issue_box(bu + 1);
            }
          }
          if (!ok) break;
            if (!(ok = tc::mbar_wait(dfull, (uint32_t)(k & 1)))) break;
            tc::fence_after();
            // epilogue: D row m, this warp's groups of 8 columns (= orientations of the group)
            const int t = (int)blockIdx.x + (int)k * G;
            const int tx = t % a.ntx, r = t / a.ntx, ty = r % a.nty, tz = r / a.nty;
            const int q = warp & 3;
            const int x = 32 * tx + lane, y = a.TY * ty + q % a.TY, z = a.TZ * tz + q / a.TY;
            const bool rowv = y < a.wy && z < a.wz;             // uniform across the warp
            const bool valid = rowv && x < a.wx;
            for (int n0 = quarter * 8; n0 < a.N; n0 += 32) {
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
                    if (lane == 0 && rowv) bw[tx] = fb;
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
        // no copy of this block may still be landing in shared memory when it ends: wait (bounded)
        // for the last phase of every buffer thread 0 filled
        if (threadIdx.x == 0) {
            if (last_box >= 0) tc::mbar_wait(boxfull, (uint32_t)(last_box & 1));
            for (int i = 0; i < kBSlots; ++i)
                if (last_b[i] >= 0) tc::mbar_wait(&bfull[i], (uint32_t)((last_b[i] / kBSlots) & 1));
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == kDProd / 32) tc::tmem_dealloc(tmem, ncols);
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

size_t direct_smem_bytes(int N, long box_words) { return 1024 + direct_layout(N, box_words).total; }

void launch_rho_hl(const float *rho, const uint8_t *fix, int nx, int ny, int nz, int lox, int loy, int loz, int PX,
                   int PY, int PZ, uint32_t *out, cudaStream_t s)
{
    long n = (long)PX * PY * PZ;
    long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    rho_hl_kernel<<<(int)b, 256, 0, s>>>(rho, fix, nx, ny, nz, lox, loy, loz, PX, PY, PZ, out);
}

bool launch_direct(const DirectArgs &a, int nsm, cudaStream_t s)
{
    CUtensorMap map;
    const uint64_t dims[3] = {(uint64_t)a.PX, (uint64_t)a.PY, (uint64_t)a.PZ};
    const uint64_t strides[2] = {(uint64_t)a.PX * 4, (uint64_t)a.PX * a.PY * 4};
    const uint32_t box[3] = {(uint32_t)a.BX, (uint32_t)a.BY, (uint32_t)a.BZ};
    if (!tma_fft::encode_tiled_u32(&map, a.rhohl, 3, dims, strides, box)) return false;
    const size_t smem = direct_smem_bytes(a.N, (long)a.BX * a.BY * a.BZ);
    if (cudaFuncSetAttribute(direct_corr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int ntiles = a.ntx * a.nty * a.ntz;
    const int grid = ntiles < nsm ? ntiles : nsm;
    if (grid > 0) direct_corr_kernel<<<grid, kDThreads, smem, s>>>(map, a);
    return true;
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
