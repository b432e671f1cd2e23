// Minimum over sharp points, tiled (Eq. eq_imf_2; Alg. 1 "Translate" + "min" over Support(K)).
//
//   gamma_R(x) = min_{k in sharp_R} g_R(x - k),   f(x) <- min(f(x), gamma_R(x))
//
// App. B forms a 4D array of shifted copies of g and reduces it; here the shifted copies are
// never formed. The sharp points of an orientation are split into runs along x (fixed dy,
// dz, consecutive dx); a block stages the g tile its outputs need in shared memory and every
// thread keeps 8 consecutive x outputs in registers, so one run costs 8 + L - 1 shared loads
// and about L/2 three-input minima per output. Runs are grouped in dz-chunks whose tile fits
// the shared-memory budget; the run descriptors of a chunk are staged next to the tile. The
// row pitch is odd and the plane pitch is chosen so that the 32 lanes of a warp (8 rows x 4
// planes) read 32 different banks.
//
// The orientations of a launch may be split into groups, one block per (tile, group), so that
// the grid holds several waves of short units and the uneven cost of the tiles (pruned tiles
// finish early) does not leave SMs idle at the end. Groups of one tile then merge into f with
// an integer atomic minimum, which orders non-negative floats (every g >= 0; -0 is mapped to +0
// first) exactly as the float minimum does, so the result does not depend on the split.
#include <cfloat>

#include "erode.cuh"

namespace imf {

namespace {

__device__ __forceinline__ float fmin3(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Window values of a run of length L that one output combines: the L loaded values themselves
// for L <= 3, else ceil(L / 3) minima of three neighbours T[i] = min(s[i], s[i+1], s[i+2]) (the
// last block starts at L - 3 and may overlap its neighbour; min is exact and idempotent, so the
// cover does not change the result).
template <int L> __host__ __device__ constexpr int nblk() { return L <= 3 ? L : (L + 2) / 3; }
template <int L> __host__ __device__ constexpr int blk(int m) { return L <= 3 ? m : (m + 1 < nblk<L>() ? 3 * m : L - 3); }

// loads the window of one run for XT consecutive outputs and forms its block values V
template <int XT, int L> __device__ __forceinline__ void run_blocks(const float *__restrict__ s, float *V)
{
    float w[XT + L - 1];
#pragma unroll
    for (int i = 0; i < XT + L - 1; ++i) w[i] = s[i];
    if constexpr (L <= 3) {
#pragma unroll
        for (int i = 0; i < XT + L - 1; ++i) V[i] = w[i];
    } else {
#pragma unroll
        for (int i = 0; i < XT + L - 3; ++i) V[i] = fmin3(w[i], w[i + 1], w[i + 2]);
    }
}
template <int XT, int L> __host__ __device__ constexpr int nv() { return L <= 3 ? XT + L - 1 : XT + L - 3; }

// One run of length L for the thread's XT consecutive outputs: acc[j] = min(acc[j], s[j], ...,
// s[j + L - 1]), as three-input minima over the run's block values (XT + L - 1 shared loads,
// nv three-input minima to form the blocks, ceil(nblk / 2) per output).
template <int XT, int L> __device__ __forceinline__ void run_min(const float *__restrict__ s, float *acc)
{
    float V[nv<XT, L>()];
    run_blocks<XT, L>(s, V);
    constexpr int K = nblk<L>();
#pragma unroll
    for (int j = 0; j < XT; ++j) {
        float m = acc[j];
#pragma unroll
        for (int b = 0; b < K; b += 2) {
            if (b + 1 < K) m = fmin3(m, V[j + blk<L>(b)], V[j + blk<L>(b + 1)]);
            else m = fminf(m, V[j + blk<L>(b)]);
        }
        acc[j] = m;
    }
}

// Two runs of the same length with an odd block count, merged so that no output spends a
// two-input minimum on a lone block: K three-input minima per output instead of K + 1.
template <int XT, int L> __device__ __forceinline__ void run_pair(const float *__restrict__ s0, const float *__restrict__ s1,
                                                                float *acc)
{
    float V0[nv<XT, L>()], V1[nv<XT, L>()];
    run_blocks<XT, L>(s0, V0);
    run_blocks<XT, L>(s1, V1);
    constexpr int K = nblk<L>();
#pragma unroll
    for (int j = 0; j < XT; ++j) {
        float m = acc[j];
#pragma unroll
        for (int b = 0; b < 2 * K; b += 2) {
            const float u = b < K ? V0[j + blk<L>(b)] : V1[j + blk<L>(b - K)];
            const float v = b + 1 < K ? V0[j + blk<L>(b + 1)] : V1[j + blk<L>(b + 1 - K)];
            m = fmin3(m, u, v);
        }
        acc[j] = m;
    }
}

// pairing pays where the block count is odd and both windows stay in registers
template <int XT, int L> __host__ __device__ constexpr bool pair_ok()
{
    return (nblk<L>() & 1) && 2 * (XT + L - 1) + XT <= (XT <= 8 ? 48 : 100);
}

template <int XT, int L> __device__ __forceinline__ void run_group(const int2 *sruns, int q0, int q1, const float *tb, float *acc)
{
    int q = q0;
    if constexpr (pair_ok<XT, L>())
        for (; q + 1 < q1; q += 2) run_pair<XT, L>(tb + sruns[q].x, tb + sruns[q + 1].x, acc);
    for (; q < q1; ++q) run_min<XT, L>(tb + sruns[q].x, acc);
}

// Asynchronous fill of a chunk's g tile, one warp per tile row; cells outside the window (read
// only by outputs beyond the grid, which are masked) are zero-filled. Rows are short (a few
// copies per lane), so the row position advances without division and each lane's copies of a
// row are unrolled four at a time. The caller commits and waits.
template <int NT>
__device__ __forceinline__ void fill_tile(const Erode2Args &a, const float *g, const ErodeChunk &ch, int X0, int Y0,
                                          int Z0, uint32_t sbase, int warp, int lane)
{
    const int gx0 = X0 + ch.ox, gy0 = Y0 + ch.oy, gz0 = Z0 + ch.oz;
    const int txh = ch.txh, tyh = ch.tyh, nrow = tyh * ch.tzh;
    const int pz = ch.pitch_z, py = ch.pitch_y;
    const bool xin = gx0 + txh <= a.wx;
    constexpr int NW = NT / 32;
    int iy = warp % tyh, iz = warp / tyh;
    // row pointers advance by NW rows per step (and by one plane minus tyh rows per wrap)
    const long gstep = (long)NW * a.gpx, gwrap = (long)a.gpy * a.gpx - (long)tyh * a.gpx;
    const uint32_t dstep = 4u * (uint32_t)(NW * py), dwrap = 4u * (uint32_t)(pz - tyh * py);
    const float *src = g + ((long)(gz0 + iz) * a.gpy + (gy0 + iy)) * a.gpx + gx0;
    uint32_t drow = sbase + 4u * (uint32_t)(iz * pz + iy * py);
    for (int r = warp; r < nrow; r += NW) {
        const bool rowok = gy0 + iy < a.wy && gz0 + iz < a.wz;
        if (rowok && xin) {
            // whole row inside the window: plain 4-byte copies
            for (int ix0 = lane; ix0 < txh; ix0 += 128) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int ix = ix0 + 32 * k;
                    if (ix < txh)
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(drow + 4u * ix), "l"(src + ix));
                }
            }
        } else {
            for (int ix = lane; ix < txh; ix += 32) {
                const bool ok = rowok && gx0 + ix < a.wx;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(drow + 4u * ix),
                             "l"(ok ? src + ix : g), "r"(ok ? 4 : 0));
            }
        }
        iy += NW;
        src += gstep;
        drow += dstep;
        while (iy >= tyh) {
            iy -= tyh;
            ++iz;
            src += gwrap;
            drow += dwrap;
        }
    }
}

template <int XT> __global__ void __launch_bounds__(er_threads(XT), 1) erode2_kernel(Erode2Args a)
{
    extern __shared__ float tile[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // lane = ty_lo (8) x tz_lo (4); warp = tx (kErTX / XT) x ty_hi (kErTY / 8) x tz_hi
    constexpr int NT = er_threads(XT), NXT = kErTX / XT, NYH = kErTY / 8;
    static_assert(NXT * NYH * (kErTZ / 4) * 32 == NT, "erosion block shape");
    const int tx = warp % NXT, ty = ((warp / NXT) % NYH) * 8 + (lane & 7), tz = (warp / (NXT * NYH)) * 4 + (lane >> 3);
    const int tiles_z = (a.nz + kErTZ - 1) / kErTZ;
    const int grp = blockIdx.z / tiles_z;
    const int X0 = blockIdx.x * kErTX, Y0 = blockIdx.y * kErTY, Z0 = (blockIdx.z - grp * tiles_z) * kErTZ;
    const int ob0 = grp * a.nb / a.ngroups, ob1 = (grp + 1) * a.nb / a.ngroups;
    const int y = Y0 + ty, z = Z0 + tz;
    float *frow = a.f + ((long)z * a.ny + y) * a.nx;
    // the running minimum starts from f; outputs outside the grid start at 0 so that they
    // never keep a warp busy
    float acc[XT];
#pragma unroll
    for (int j = 0; j < XT; ++j) {
        const int x = X0 + tx * XT + j;
        acc[j] = (y < a.ny && z < a.nz && x < a.nx) ? frow[x] : 0.f;
    }
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(tile);
    for (int ob = ob0; ob < ob1; ++ob) {
        const int og = a.orient_base + ob;
        const float *g = a.g + ob * a.g_so;
        // gamma_R >= 0, so outputs whose minimum is already 0 are final: skip work when a whole
        // warp (or the whole block) is done
        bool done = true;
#pragma unroll
        for (int j = 0; j < XT; ++j) done = done && acc[j] <= 0.f;
        if (__syncthreads_and(done)) continue;
        const bool warp_done = __all_sync(0xffffffffu, done);
        for (int c = a.chunk_start[og]; c < a.chunk_start[og + 1]; ++c) {
            const ErodeChunk &ch = a.chunks[c];
            const int pz = ch.pitch_z, py = ch.pitch_y;
            const int run0 = ch.run0, nrun = ch.run1 - ch.run0;
            // the chunk's run descriptors sit behind its tile
            int2 *sruns = reinterpret_cast<int2 *>(tile + er_runs_offset(ch.tzh, pz));
            __syncthreads();
            fill_tile<NT>(a, g, ch, X0, Y0, Z0, sbase, warp, lane);
            for (int q = threadIdx.x; q < nrun; q += NT) sruns[q] = a.runs[run0 + q];
            asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
            __syncthreads();
            if (warp_done) continue;
            const float *tb = tile + tz * pz + ty * py + tx * XT;
            const int *le = ch.lend;
            run_group<XT, 1>(sruns, le[0], le[1], tb, acc);
            run_group<XT, 2>(sruns, le[1], le[2], tb, acc);
            run_group<XT, 3>(sruns, le[2], le[3], tb, acc);
            run_group<XT, 4>(sruns, le[3], le[4], tb, acc);
            run_group<XT, 5>(sruns, le[4], le[5], tb, acc);
            run_group<XT, 6>(sruns, le[5], le[6], tb, acc);
            run_group<XT, 7>(sruns, le[6], le[7], tb, acc);
            run_group<XT, 8>(sruns, le[7], le[8], tb, acc);
            run_group<XT, 9>(sruns, le[8], le[9], tb, acc);
            run_group<XT, 10>(sruns, le[9], le[10], tb, acc);
            run_group<XT, 11>(sruns, le[10], le[11], tb, acc);
            run_group<XT, 12>(sruns, le[11], le[12], tb, acc);
            run_group<XT, 13>(sruns, le[12], le[13], tb, acc);
            run_group<XT, 14>(sruns, le[13], le[14], tb, acc);
            run_group<XT, 15>(sruns, le[14], le[15], tb, acc);
            run_group<XT, 16>(sruns, le[15], le[16], tb, acc);
        }
    }
    if (y < a.ny && z < a.nz) {
        if (a.ngroups == 1) {
#pragma unroll
            for (int j = 0; j < XT; ++j) {
                const int x = X0 + tx * XT + j;
                if (x < a.nx) frow[x] = acc[j];
            }
        } else {
#pragma unroll
            for (int j = 0; j < XT; ++j) {
                const int x = X0 + tx * XT + j;
                if (x < a.nx) atomicMin(reinterpret_cast<unsigned int *>(frow + x), __float_as_uint(__fadd_rn(acc[j], 0.f)));
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------
// The same minimum with dyadic min levels (erode3_kernel). After the fill the tile holds level
// 0, M_0 = g; before the first run of length 2^j the tile is rewritten in place to level j,
// M_j(i) = min(M_{j-1}(i), M_{j-1}(i + 2^(j-1))) = min_{t < 2^j} g(i + t), one warp per tile row
// (a row's cells only depend on the same row, so the warp's own barrier orders the reads before
// the writes). Runs are sorted by length, and a run of length L (2^j <= L < 2^(j+1)) at window
// start s costs one window of 8 + L - 2^j level-j values and one three-input minimum per output:
//   min_{t < L} g(s + o + t) = min(M_j(s + o), M_j(s + o + L - 2^j)).
// Level j at i is read only where i + 2^j - 1 lies in the row (the plan keeps every window in
// the tile), so the cells near a row's end that keep an older level are never read.
// ---------------------------------------------------------------------------------------------
template <int L> __host__ __device__ constexpr int floor_log2() { return L >= 16 ? 4 : L >= 8 ? 3 : L >= 4 ? 2 : L >= 2 ? 1 : 0; }

template <int L> __device__ __forceinline__ void run_lev(const float *__restrict__ s, float *acc)
{
    constexpr int D = L - (1 << floor_log2<L>());
    float w[kErXT + D];
#pragma unroll
    for (int i = 0; i < kErXT + D; ++i) w[i] = s[i];
#pragma unroll
    for (int j = 0; j < kErXT; ++j) acc[j] = D == 0 ? fminf(acc[j], w[j]) : fmin3(acc[j], w[j], w[j + D]);
}

template <int L> __device__ __forceinline__ void lev_group(const int2 *sruns, int q0, int q1, const float *tb, float *acc)
{
    for (int q = q0; q < q1; ++q) run_lev<L>(tb + sruns[q].x, acc);
}

// level j (shift h = 2^(j-1)) of every row of the chunk's tile, in place, one warp per row
__device__ __forceinline__ void build_level(float *tile, const ErodeChunk &ch, int h, int warp, int lane)
{
    constexpr int NW = kErThreads / 32, S = kErMaxRow3 / 32;
    const int txh = ch.txh, tyh = ch.tyh, nrow = tyh * ch.tzh;
    int iy = warp % tyh, iz = warp / tyh;
    for (int r = warp; r < nrow; r += NW) {
        float *row = tile + iz * ch.pitch_z + iy * ch.pitch_y;
        float v[S];
#pragma unroll
        for (int k = 0; k < S; ++k) {
            const int i = lane + 32 * k;
            v[k] = 0.f;
            if (i < txh) v[k] = i + h < txh ? fminf(row[i], row[i + h]) : row[i];
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < S; ++k) {
            const int i = lane + 32 * k;
            if (i < txh) row[i] = v[k];
        }
        __syncwarp();
        iy += NW;
        while (iy >= tyh) {
            iy -= tyh;
            ++iz;
        }
    }
}

__global__ void __launch_bounds__(kErThreads, kErBlocksPerSM) erode3_kernel(Erode2Args a)
{
    extern __shared__ float tile[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NXT = kErTX / kErXT, NYH = kErTY / 8;
    static_assert(NXT * NYH * (kErTZ / 4) * 32 == kErThreads, "erosion block shape");
    const int tx = warp % NXT, ty = ((warp / NXT) % NYH) * 8 + (lane & 7), tz = (warp / (NXT * NYH)) * 4 + (lane >> 3);
    const int tiles_z = (a.nz + kErTZ - 1) / kErTZ;
    const int grp = blockIdx.z / tiles_z;
    const int X0 = blockIdx.x * kErTX, Y0 = blockIdx.y * kErTY, Z0 = (blockIdx.z - grp * tiles_z) * kErTZ;
    const int ob0 = grp * a.nb / a.ngroups, ob1 = (grp + 1) * a.nb / a.ngroups;
    const int y = Y0 + ty, z = Z0 + tz;
    float *frow = a.f + ((long)z * a.ny + y) * a.nx;
    float acc[kErXT];
#pragma unroll
    for (int j = 0; j < kErXT; ++j) {
        const int x = X0 + tx * kErXT + j;
        acc[j] = (y < a.ny && z < a.nz && x < a.nx) ? frow[x] : 0.f;
    }
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(tile);
    for (int ob = ob0; ob < ob1; ++ob) {
        const int og = a.orient_base + ob;
        const float *g = a.g + ob * a.g_so;
        bool done = true;
#pragma unroll
        for (int j = 0; j < kErXT; ++j) done = done && acc[j] <= 0.f;
        if (__syncthreads_and(done)) continue;
        const bool warp_done = __all_sync(0xffffffffu, done);
        for (int c = a.chunk_start[og]; c < a.chunk_start[og + 1]; ++c) {
            const ErodeChunk &ch = a.chunks[c];
            const int run0 = ch.run0, nrun = ch.run1 - ch.run0;
            int2 *sruns = reinterpret_cast<int2 *>(tile + er_runs_offset(ch.tzh, ch.pitch_z));
            __syncthreads();
            fill_tile<kErThreads>(a, g, ch, X0, Y0, Z0, sbase, warp, lane);
            for (int q = threadIdx.x; q < nrun; q += kErThreads) sruns[q] = a.runs[run0 + q];
            asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
            __syncthreads();
            const float *tb = tile + tz * ch.pitch_z + ty * ch.pitch_y + tx * kErXT;
            const int *le = ch.lend;
            if (!warp_done) lev_group<1>(sruns, le[0], le[1], tb, acc);
            // levels 1 .. 4, each only while longer runs remain (uniform over the block)
            if (le[kErMaxL3] > le[1]) {
                __syncthreads();
                build_level(tile, ch, 1, warp, lane);
                __syncthreads();
                if (!warp_done) {
                    lev_group<2>(sruns, le[1], le[2], tb, acc);
                    lev_group<3>(sruns, le[2], le[3], tb, acc);
                }
            }
            if (le[kErMaxL3] > le[3]) {
                __syncthreads();
                build_level(tile, ch, 2, warp, lane);
                __syncthreads();
                if (!warp_done) {
                    lev_group<4>(sruns, le[3], le[4], tb, acc);
                    lev_group<5>(sruns, le[4], le[5], tb, acc);
                    lev_group<6>(sruns, le[5], le[6], tb, acc);
                    lev_group<7>(sruns, le[6], le[7], tb, acc);
                }
            }
            if (le[kErMaxL3] > le[7]) {
                __syncthreads();
                build_level(tile, ch, 4, warp, lane);
                __syncthreads();
                if (!warp_done) {
                    lev_group<8>(sruns, le[7], le[8], tb, acc);
                    lev_group<9>(sruns, le[8], le[9], tb, acc);
                    lev_group<10>(sruns, le[9], le[10], tb, acc);
                    lev_group<11>(sruns, le[10], le[11], tb, acc);
                    lev_group<12>(sruns, le[11], le[12], tb, acc);
                    lev_group<13>(sruns, le[12], le[13], tb, acc);
                    lev_group<14>(sruns, le[13], le[14], tb, acc);
                    lev_group<15>(sruns, le[14], le[15], tb, acc);
                }
            }
            if (le[kErMaxL3] > le[15]) {
                __syncthreads();
                build_level(tile, ch, 8, warp, lane);
                __syncthreads();
                if (!warp_done) {
                    lev_group<16>(sruns, le[15], le[16], tb, acc);
                    lev_group<17>(sruns, le[16], le[17], tb, acc);
                    lev_group<18>(sruns, le[17], le[18], tb, acc);
                    lev_group<19>(sruns, le[18], le[19], tb, acc);
                    lev_group<20>(sruns, le[19], le[20], tb, acc);
                    lev_group<21>(sruns, le[20], le[21], tb, acc);
                    lev_group<22>(sruns, le[21], le[22], tb, acc);
                    lev_group<23>(sruns, le[22], le[23], tb, acc);
                    lev_group<24>(sruns, le[23], le[24], tb, acc);
                    lev_group<25>(sruns, le[24], le[25], tb, acc);
                    lev_group<26>(sruns, le[25], le[26], tb, acc);
                    lev_group<27>(sruns, le[26], le[27], tb, acc);
                    lev_group<28>(sruns, le[27], le[28], tb, acc);
                    lev_group<29>(sruns, le[28], le[29], tb, acc);
                    lev_group<30>(sruns, le[29], le[30], tb, acc);
                    lev_group<31>(sruns, le[30], le[31], tb, acc);
                }
            }
        }
    }
    if (y < a.ny && z < a.nz) {
        if (a.ngroups == 1) {
#pragma unroll
            for (int j = 0; j < kErXT; ++j) {
                const int x = X0 + tx * kErXT + j;
                if (x < a.nx) frow[x] = acc[j];
            }
        } else {
#pragma unroll
            for (int j = 0; j < kErXT; ++j) {
                const int x = X0 + tx * kErXT + j;
                if (x < a.nx) atomicMin(reinterpret_cast<unsigned int *>(frow + x), __float_as_uint(__fadd_rn(acc[j], 0.f)));
            }
        }
    }
}

} // namespace

void launch_erode3(const Erode2Args &a, size_t smem, cudaStream_t s)
{
    cudaFuncSetAttribute(erode3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((a.nx + kErTX - 1) / kErTX, (a.ny + kErTY - 1) / kErTY, ((a.nz + kErTZ - 1) / kErTZ) * a.ngroups);
    erode3_kernel<<<grid, kErThreads, smem, s>>>(a);
}

int erode3_blocks_per_sm(size_t smem)
{
    cudaFuncSetAttribute(erode3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, erode3_kernel, kErThreads, smem) != cudaSuccess) n = 1;
    return n < 1 ? 1 : n;
}

template <int XT> void launch_erode2_xt(const Erode2Args &a, size_t smem, cudaStream_t s)
{
    cudaFuncSetAttribute(erode2_kernel<XT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((a.nx + kErTX - 1) / kErTX, (a.ny + kErTY - 1) / kErTY, ((a.nz + kErTZ - 1) / kErTZ) * a.ngroups);
    erode2_kernel<XT><<<grid, er_threads(XT), smem, s>>>(a);
}

template <int XT> int erode2_bps_xt(size_t smem)
{
    cudaFuncSetAttribute(erode2_kernel<XT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, erode2_kernel<XT>, er_threads(XT), smem) != cudaSuccess)
        n = 1;
    return n < 1 ? 1 : n;
}

void launch_erode2(const Erode2Args &a, size_t smem, int xt, cudaStream_t s)
{
    if (xt == 8) launch_erode2_xt<8>(a, smem, s);
    else launch_erode2_xt<16>(a, smem, s);
}

int erode2_blocks_per_sm(size_t smem, int xt)
{
    return xt == 8 ? erode2_bps_xt<8>(smem) : erode2_bps_xt<16>(smem);
}

} // namespace imf
