// IMF kernels other than the FFT passes: tool resampling, the exact near-threshold
// re-check, the sweep of the cutter over the free translations, the minimum over sharp
// points and orientations, and the normalisation / penalty tail of Alg. 1 and Alg. 2.
#include <algorithm>
#include <cfloat>

#include "imf_internal.cuh"

namespace imf {

namespace {

inline int blocks_for(long n, int per = kThreads, int cap = 152 * 16)
{
    long b = (n + per - 1) / per;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

// ---------------------------------------------------------------------------------------
// Rotate (Alg. 1): nearest neighbour, inverse map about the origin voxel.
// u_c = floor((R_0c v_0 + R_1c v_1) + R_2c v_2 + 1/2), every operation rounded to nearest
// in FP64 with no contraction, so the set of resampled voxels is reproducible exactly.
// ---------------------------------------------------------------------------------------
__global__ void rotate_kernel(RotateArgs a)
{
    const int o = blockIdx.y;
    const int *bx = a.box + 6 * o;
    const long vol = (long)bx[3] * bx[4] * bx[5];
    const double *R = a.R + 9 * o;
    uint8_t *oT = a.outT + a.box_off[o], *oK = a.outK + a.box_off[o], *oS = a.outS + a.box_off[o];
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < vol; idx += (long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % bx[3]);
        const int j = (int)((idx / bx[3]) % bx[4]);
        const int k = (int)(idx / ((long)bx[3] * bx[4]));
        const double v0 = bx[0] + i, v1 = bx[1] + j, v2 = bx[2] + k;
        int u[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double p = __dadd_rn(__dadd_rn(__dmul_rn(R[c], v0), __dmul_rn(R[3 + c], v1)), __dmul_rn(R[6 + c], v2));
            u[c] = (int)floor(__dadd_rn(p, 0.5));
        }
        const int ax = a.ox + u[0], ay = a.oy + u[1], az = a.oz + u[2];
        uint8_t t = 0, kk = 0, ss = 0;
        if (ax >= 0 && ax < a.tx && ay >= 0 && ay < a.ty && az >= 0 && az < a.tz) {
            const long src = ((long)az * a.ty + ay) * a.tx + ax;
            t = a.T[src];
            kk = a.K[src];
            ss = a.Sm[src];
        }
        oT[idx] = t;
        oK[idx] = kk;
        oS[idx] = ss;
    }
}

__global__ void scatter_tool_kernel(float *dst, int Px, int Py, int Pz, const uint32_t *off, int n, int kx,
                                    int ky, int kz)
{
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
        const uint32_t p = off[m];
        int x = (int)(p & 1023u) - 512 - kx, y = (int)((p >> 10) & 1023u) - 512 - ky, z = (int)((p >> 20) & 1023u) - 512 - kz;
        x %= Px; if (x < 0) x += Px;
        y %= Py; if (y < 0) y += Py;
        z %= Pz; if (z < 0) z += Pz;
        dst[((long)z * Py + y) * Px + x] = 1.0f;
    }
}

// ---------------------------------------------------------------------------------------
// Near-threshold re-check: g(t) = sum_{v in RT} rho_O(t + v) by a compensated FP32 sum
// (Neumaier), compared with theta in FP64 (recheck_blocks_kernel below: one warp per flagged
// translation).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// ---------------------------------------------------------------------------------------
// Sweep (Eq. eq_conv_A): A_R(x) = OR_{k in RK} free(x - k), on bit-packed rows. RK is a
// union of runs [a, b] along x at fixed (dy, dz) (at most 32 long); a run contributes the
// sliding OR of length L = b - a + 1 of one source row. With the dilation levels
// D_j(i) = OR_{t < 2^j} free(i + t) (D_0 = free), the sliding OR of length L at i is
// D_j(i) | D_j(i + L - 2^j) for 2^j <= L <= 2^(j+1), so every run costs two 32-bit windows.
// ---------------------------------------------------------------------------------------

// Levels 1..4 of the free bits of slots [0, nb): word i of level j at bits + j * lstride + i.
// Bits past the end of a row count as 0; a row's window words only reach its padding words.
__global__ void sweep_levels_kernel(SweepLevelsArgs a)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < a.n; i += (long)gridDim.x * blockDim.x) {
        const int w = (int)(i % a.wpr);
        uint32_t lev[kSweepLevels - 1];
        sweep_level_words(a.bits[i], w + 1 < a.wpr ? a.bits[i + 1] : 0u, lev);
#pragma unroll
        for (int j = 1; j < kSweepLevels; ++j) a.bits[j * a.lstride + i] = lev[j - 1];
    }
}

// One thread per (output word, orientation of the batch); results are OR-ed into A. The run
// descriptors of the orientation are staged in shared memory (see SweepArgs::pairs).
constexpr int kSweepStage = 512;

__global__ void __launch_bounds__(256) sweep_kernel(SweepArgs a)
{
    __shared__ int4 sp[kSweepStage];
    const long total = (long)a.awords * a.ny * a.nz;
    const int ob = blockIdx.y;
    const int og = a.orient_base + ob;
    const int m0 = a.pair_start[og], m1 = a.pair_start[og + 1];
    const long tstride = (long)gridDim.x * blockDim.x;
    for (long tb = (long)blockIdx.x * blockDim.x; tb < total; tb += tstride) {
        const long t = tb + threadIdx.x;
        const bool live = t < total;
        const int q = live ? (int)(t % a.awords) : 0;
        const int y = live ? (int)((t / a.awords) % a.ny) : 0;
        const int z = live ? (int)(t / ((long)a.awords * a.ny)) : 0;
        // word q of the output row, in window coordinates of slot ob (run offsets added below)
        const uint32_t *base = a.bits + ob * a.b_so + (long)z * a.b_sz + (long)y * a.b_sy + q;
        uint32_t *dstw = a.A + ((long)z * a.ny + y) * a.awords + q;
        const int rem = a.nx - 32 * q;
        const uint32_t full = rem < 32 ? (1u << rem) - 1u : 0xffffffffu;
        // A only grows: words already fully accessible need no more work (unless this
        // orientation's own set is wanted, which starts empty)
        const uint32_t old = live ? *dstw : full;
        const bool per = a.A_per != nullptr;
        uint32_t acc = per ? 0u : old;
        for (int c0 = m0; c0 < m1; c0 += kSweepStage) {
            const int cn = min(kSweepStage, m1 - c0);
            __syncthreads();
            for (int i = threadIdx.x; i < cn; i += blockDim.x) sp[i] = a.pairs[c0 + i];
            __syncthreads();
            if (!live || (acc & full) == full) continue;
            // unrolled so that the loads of several runs are in flight at once
#pragma unroll 8
            for (int i = 0; i < cn; ++i) {
                const int4 d = sp[i];
                acc |= sweep_pair_bits(base + (long)d.w * a.lstride + d.x, d);
            }
        }
        if (live) {
            const uint32_t add = acc & full & ~old;
            if (add) atomicOr(dstw, add);
            if (per) a.A_per[(long)a.perm[og] * a.a_per_so + ((long)z * a.ny + y) * a.awords + q] = acc & full;
        }
    }
}

// The same sweep with the orientations of the batch walked inside the thread: one thread per
// output word and orientation group (blockIdx.y of `ngroups`), which stops as soon as its word
// is fully accessible, so most words of the air around a part leave after a few orientations
// instead of being swept by every orientation of the batch in parallel. A block stages each
// orientation's runs and leaves the group's loop once all its words are full. The groups of a
// word merge with an atomic OR; A only grows, so the result does not depend on the grouping.
__global__ void __launch_bounds__(256) sweep_loop_kernel(SweepArgs a, int ngroups)
{
    __shared__ int4 sp[kSweepStage];
    const long total = (long)a.awords * a.ny * a.nz;
    const int grp = blockIdx.y;
    const int ob0 = grp * a.nb / ngroups, ob1 = (grp + 1) * a.nb / ngroups;
    const long tstride = (long)gridDim.x * blockDim.x;
    for (long tb = (long)blockIdx.x * blockDim.x; tb < total; tb += tstride) {
        const long t = tb + threadIdx.x;
        const bool live = t < total;
        const int q = live ? (int)(t % a.awords) : 0;
        const int y = live ? (int)((t / a.awords) % a.ny) : 0;
        const int z = live ? (int)(t / ((long)a.awords * a.ny)) : 0;
        uint32_t *dstw = a.A + ((long)z * a.ny + y) * a.awords + q;
        const int rem = a.nx - 32 * q;
        const uint32_t full = rem < 32 ? (1u << rem) - 1u : 0xffffffffu;
        const uint32_t old = live ? *dstw : full;
        uint32_t acc = old;
        for (int ob = ob0; ob < ob1; ++ob) {
            if (__syncthreads_and((acc & full) == full)) break;
            const int og = a.orient_base + ob;
            const int m0 = a.pair_start[og], m1 = a.pair_start[og + 1];
            const uint32_t *base = a.bits + ob * a.b_so + (long)z * a.b_sz + (long)y * a.b_sy + q;
            for (int c0 = m0; c0 < m1; c0 += kSweepStage) {
                const int cn = min(kSweepStage, m1 - c0);
                __syncthreads();
                for (int i = threadIdx.x; i < cn; i += blockDim.x) sp[i] = a.pairs[c0 + i];
                __syncthreads();
                if ((acc & full) == full) continue;
#pragma unroll 4
                for (int i = 0; i < cn; ++i) {
                    const int4 d = sp[i];
                    acc |= sweep_pair_bits(base + (long)d.w * a.lstride + d.x, d);
                }
            }
        }
        if (live) {
            const uint32_t add = acc & full & ~old;
            if (add) atomicOr(dstw, add);
        }
    }
}

// ---------------------------------------------------------------------------------------
// Greedy process plan (Sec. 3.4.1): the negative space as bits, the part of it each
// orientation's accessible set covers, and its removal.
// ---------------------------------------------------------------------------------------
__global__ void plan_init_kernel(const float *rho, const uint8_t *fix, int nx, int ny, int nz, int awords,
                                 float tau, uint32_t *rem)
{
    const long total = (long)awords * ny * nz;
    for (long w = blockIdx.x * (long)blockDim.x + threadIdx.x; w < total; w += (long)gridDim.x * blockDim.x) {
        const int q = (int)(w % awords);
        const long row = w / awords;
        uint32_t bits = 0;
        for (int b = 0; b < 32; ++b) {
            const int x = 32 * q + b;
            if (x >= nx) break;
            const long idx = row * nx + x;
            if (!(fix && fix[idx]) && rho[idx] <= tau) bits |= 1u << b;
        }
        rem[w] = bits;
    }
}

__global__ void __launch_bounds__(256) plan_count_kernel(const uint32_t *sets, long set_words, const uint32_t *rem,
                                                         unsigned long long *counts)
{
    __shared__ unsigned long long part[8];
    const uint32_t *s = sets + (long)blockIdx.y * set_words;
    unsigned long long c = 0;
    for (long w = blockIdx.x * (long)blockDim.x + threadIdx.x; w < set_words; w += (long)gridDim.x * blockDim.x)
        c += __popc(s[w] & rem[w]);
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += part[i];
        if (t) atomicAdd(counts + blockIdx.y, t);
    }
}

__global__ void plan_remove_kernel(const uint32_t *set, long words, uint32_t *rem)
{
    for (long w = blockIdx.x * (long)blockDim.x + threadIdx.x; w < words; w += (long)gridDim.x * blockDim.x)
        rem[w] &= ~set[w];
}

// Warp-per-point re-check: the 32 lanes of a warp split the tool voxels of one flagged
// translation (eight taps per lane in flight at once: the gathers of rho and of the fixture mostly
// miss in L2), each lane keeps a compensated FP32 sum, the warp combines them with compensated
// shuffles and lane 0 compares the total with theta in FP64.
__global__ void __launch_bounds__(256) recheck_blocks_kernel(RecheckArgs a)
{
    const int n = min(*a.count, a.cap);
    const int lane = threadIdx.x & 31;
    const int warps = (int)(gridDim.x * (blockDim.x >> 5));
    for (int e = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); e < n; e += warps) {
        const int2 fl = a.flags[e];
        const int og = fl.x, lin = fl.y;
        const int i = lin % a.wx, y = (lin / a.wx) % a.wy, z = lin / (a.wx * a.wy);
        const int tx = i - a.kx, ty = y - a.ky, tz = z - a.kz;
        float s = 0.f, c = 0.f;
        const int m1 = a.rt_start[og + 1];
        // rho_O at tool voxel m (0 outside the grid: adding it is exact, so the sum is the sum
        // over the voxels inside)
        auto tap = [&](int m) -> float {
            const uint32_t p = __ldg(a.rt_off + m);
            const int x = tx + (int)(p & 1023u) - 512;
            const int yy = ty + (int)((p >> 10) & 1023u) - 512;
            const int zz = tz + (int)((p >> 20) & 1023u) - 512;
            if (x < 0 || yy < 0 || zz < 0 || x >= a.nx || yy >= a.ny || zz >= a.nz) return 0.f;
            const long idx = ((long)zz * a.ny + yy) * a.nx + x;
            float r = __ldg(a.rho + idx);
            if (a.fix && a.fix[idx]) r = fminf(1.f, r + 1.f);
            return r;
        };
        constexpr int U = 8;
        int m = a.rt_start[og] + lane;
        for (; m + (U - 1) * 32 < m1; m += U * 32) {
            float r[U];
#pragma unroll
            for (int u = 0; u < U; ++u) r[u] = tap(m + u * 32);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                float t, err;
                two_sum(s, r[u], t, err);
                s = t;
                c += err;
            }
        }
        for (; m < m1; m += 32) {
            float t, err;
            two_sum(s, tap(m), t, err);
            s = t;
            c += err;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const float s2 = __shfl_down_sync(0xffffffffu, s, off);
            const float c2 = __shfl_down_sync(0xffffffffu, c, off);
            float t, err;
            two_sum(s, s2, t, err);
            s = t;
            c = c + c2 + err;
        }
        if (lane == 0) {
            const double tot = (double)s + (double)c;
            const long slot = og - a.orient_base;
            a.g[slot * a.g_so + (long)z * a.g_sz + (long)y * a.g_sy + i] = (float)tot;
            uint32_t *w = a.bits + slot * a.b_so + (long)z * a.b_sz + (long)y * a.b_sy + (i >> 5);
            const uint32_t bit = 1u << (i & 31);
            if (tot <= a.theta) atomicOr(w, bit);
            else atomicAnd(w, ~bit);
        }
    }
}

__global__ void fill_f32_kernel(float *p, float v, long n)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) p[i] = v;
}

__device__ __forceinline__ float block_max(float v)
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

// max over Omega_0 (non-fixture cells) of a nonnegative field, as an unsigned bit pattern
__global__ void max_omega0_kernel(const float *f, const uint8_t *fix, long n, unsigned *maxbits, int absval)
{
    float m = 0.f;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        if (fix && fix[i]) continue;
        float v = f[i];
        if (absval) v = fabsf(v);
        m = fmaxf(m, v);
    }
    m = block_max(m);
    if (threadIdx.x == 0) atomicMax(maxbits, __float_as_uint(m));
}

// Alg. 1 tail: f_bar = f / M (FP64, as f times the FP64 reciprocal of M: within one FP64 ulp of
// the quotient, and FP64 division per voxel is slow on this part), B = [f_bar > lambda],
// f_bar <- f_bar B, Gamma = Omega_0 [rho <= tau] B; outputs on fixture cells are 0.
__global__ void finalize_kernel(FinalizeArgs a)
{
    const long n = (long)a.nx * a.ny * a.nz;
    const float Mf = __uint_as_float(*a.maxbits);
    const bool ok = Mf > 0.f && Mf <= FLT_MAX;
    const double invM = ok ? 1.0 / (double)Mf : 0.0;
    for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < n; idx += (long)gridDim.x * blockDim.x) {
        const float f = a.f[idx];
        const bool fixc = a.fix && a.fix[idx];
        double fb = (ok && !fixc) ? (double)f * invM : 0.0;
        const bool B = fb > a.lambda;
        if (!B) fb = 0.0;
        a.fbar[idx] = (float)fb;
        a.secluded[idx] = (uint8_t)(B && !((double)a.rho[idx] > a.tau));
        if (a.raw) a.raw[idx] = f;
        if (a.acc) {
            if (a.acc_from_f) {
                // sharp points = the whole cutter, one tool: some cutter point lies on a free
                // translation iff the minimum over sharp points is <= theta (Eq. eq_imf_2 vs
                // Eq. eq_conv_A; the FP32 comparison of the free bits)
                a.acc[idx] = (uint8_t)(!fixc && f <= a.theta);
            } else {
                const int x = (int)(idx % a.nx);
                const long row = idx / a.nx;
                const uint32_t w = a.A[row * a.awords + (x >> 5)];
                a.acc[idx] = (uint8_t)(!fixc && ((w >> (x & 31)) & 1u));
            }
        }
    }
}

// Eq. eq_filtered_sens with Eq. eq_accFilter (FP32).
__global__ void penalize_kernel(float *sens, const float *rho, const float *fbar, const uint8_t *sec, long n,
                                const unsigned *maxbits, float w, float tau)
{
    const float m = __uint_as_float(*maxbits);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        sens[i] = penalized_sensitivity(sens[i], rho[i], fbar[i], sec[i], m, w, tau);
}

} // namespace

void launch_rotate(const RotateArgs &a, cudaStream_t s)
{
    dim3 grid(blocks_for(a.max_box, kThreads, 4096), a.n_orient);
    rotate_kernel<<<grid, kThreads, 0, s>>>(a);
}

void launch_scatter_tool(float *dst, int Px, int Py, int Pz, const uint32_t *off, int n, int kx, int ky, int kz,
                         cudaStream_t s)
{
    scatter_tool_kernel<<<blocks_for(n), kThreads, 0, s>>>(dst, Px, Py, Pz, off, n, kx, ky, kz);
}

void launch_sweep_levels(const SweepLevelsArgs &a, cudaStream_t s)
{
    sweep_levels_kernel<<<blocks_for(a.n, kThreads, 152 * 8), kThreads, 0, s>>>(a);
}

void launch_sweep_loop(const SweepArgs &a, int nsm, cudaStream_t s)
{
    // about 2048 resident threads per SM: as many orientation groups as that takes
    const long words = (long)a.awords * a.ny * a.nz;
    const long want = (long)nsm * 2048;
    int groups = (int)std::min<long>(a.nb, std::max<long>(1, (want + words - 1) / words));
    dim3 grid(blocks_for(words, kThreads, 1 << 20), groups);
    sweep_loop_kernel<<<grid, kThreads, 0, s>>>(a, groups);
}

void launch_sweep(const SweepArgs &a, cudaStream_t s)
{
    dim3 grid(blocks_for((long)a.awords * a.ny * a.nz, kThreads, 152 * 4), a.nb);
    sweep_kernel<<<grid, kThreads, 0, s>>>(a);
}

void launch_plan_init(const float *rho, const uint8_t *fix, int nx, int ny, int nz, int awords, double tau,
                      uint32_t *remaining, cudaStream_t s)
{
    plan_init_kernel<<<blocks_for((long)awords * ny * nz), kThreads, 0, s>>>(rho, fix, nx, ny, nz, awords, (float)tau,
                                                                            remaining);
}

void launch_plan_count(const uint32_t *sets, long set_words, int n_sets, const uint32_t *remaining,
                       unsigned long long *counts, cudaStream_t s)
{
    dim3 grid(blocks_for(set_words, 256, 152 * 2), n_sets);
    plan_count_kernel<<<grid, 256, 0, s>>>(sets, set_words, remaining, counts);
}

void launch_plan_remove(const uint32_t *set, long words, uint32_t *remaining, cudaStream_t s)
{
    plan_remove_kernel<<<blocks_for(words), kThreads, 0, s>>>(set, words, remaining);
}

void launch_recheck_blocks(const RecheckArgs &a, int max_points, cudaStream_t s)
{
    // eight points (warps) per block, at most eight blocks per SM
    const int want = (max_points + 7) / 8;
    int blocks = want < 1 ? 1 : (want > 152 * 8 ? 152 * 8 : want);
    recheck_blocks_kernel<<<blocks, 256, 0, s>>>(a);
}

void launch_fill_f32(float *p, float v, long n, cudaStream_t s)
{
    fill_f32_kernel<<<blocks_for(n), kThreads, 0, s>>>(p, v, n);
}

void launch_max_omega0(const float *f, const uint8_t *fix, long n, unsigned *maxbits, cudaStream_t s)
{
    max_omega0_kernel<<<blocks_for(n, kThreads, 152 * 4), kThreads, 0, s>>>(f, fix, n, maxbits, 0);
}

void launch_absmax_omega0(const float *v, const uint8_t *fix, long n, unsigned *maxbits, cudaStream_t s)
{
    max_omega0_kernel<<<blocks_for(n, kThreads, 152 * 4), kThreads, 0, s>>>(v, fix, n, maxbits, 1);
}

void launch_finalize(const FinalizeArgs &a, cudaStream_t s)
{
    finalize_kernel<<<blocks_for((long)a.nx * a.ny * a.nz), kThreads, 0, s>>>(a);
}

void launch_penalize(float *sens, const float *rho, const float *fbar, const uint8_t *sec, long n,
                     const unsigned *maxbits, double w, double tau, cudaStream_t s)
{
    penalize_kernel<<<blocks_for(n), kThreads, 0, s>>>(sens, rho, fbar, sec, n, maxbits, (float)w, (float)tau);
}

} // namespace imf
