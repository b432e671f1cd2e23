// Two-pass register FFT kernels (fft2.cuh) for the hot passes of the collision convolution
// (Alg. 1 Convolve; App. B): the y and z passes over columns of the half spectrum, with the
// pointwise product of the design and tool spectra fused into the z pass, and the inverse x
// pass with the collision threshold (Eq. eq_conv_D) fused in.
//
// A pencil of length L = A B is loaded straight from global memory into registers (B threads
// of A samples each), transformed, twiddled and written to shared memory once; A threads then
// read it back, finish it with B-point DFTs and store the result straight to global memory.
#include <algorithm>

#include "fft2.cuh"
#include "imf_internal.cuh"
#include "tc_primitives.cuh"
#include "threshold_row.cuh"
#include "xpass.cuh"

namespace imf {

namespace {

constexpr int kW2 = 16;          // pencils (axis passes) or rows (x pass) per block
constexpr int kT2 = 256;         // threads per block: kW2 pencils x 16 slots

// Columns [z][y][kx] of W consecutive kx per block; a pencil is one (batch row b, kx) pair.
// With factors up to 16 a block has W = 16 pencils of 16 slots; with factors up to 24 (BIG)
// W = 8 pencils of 32 slots, or 16 (WIDE: 512 threads, 128-byte rows of kx per load instead of
// 64). When nx is not a multiple of W, the last grid column of blocks takes the remaining ntail
// kx columns of W batch rows at a time, so no block transforms empty pencils.
// Grid: x = kx chunk (fastest), y = orientation, z = batch row: the chunks of one row run
// together (adjacent 64 / 128-byte pieces of the same DRAM pages), and the orientations of one
// batch row follow each other, so a pointwise factor shared by the orientations (the design
// spectrum of the z pass) is read from DRAM once and from L2 after.
template <bool BIG, bool WIDE = false> struct AxisShape {
    static constexpr int W = BIG ? (WIDE ? 16 : 8) : kW2;       // pencils per block
    static constexpr int LOGW = BIG ? (WIDE ? 4 : 3) : 4;
    static constexpr int T = BIG ? W * 32 : kT2;                 // threads per block
    template <typename F> __device__ __forceinline__ static void with(int n, F &&f)
    {
        if constexpr (BIG) fft2::with_size_big(n, f);
        else fft2::with_size(n, f);
    }
};

// MUL: whether the pointwise factor a.mul is applied on load (the inverse z pass): 1 always,
// 0 never, -1 decided at run time. The small shape (axis2_kernel) decides at run time (62
// registers, four blocks per SM); the big shape (axis2_big_kernel) is specialised, so that
// without the factor it fits three blocks per SM (80 registers) while the z pass keeps its 120.
template <int S, bool BIG, int MUL, bool WIDE = false>
__device__ __forceinline__ void axis2_body(const AxisArgs &a, int nbatch, int nfull, int ntail)
{
    using Sh = AxisShape<BIG, WIDE>;
    constexpr int kW = Sh::W;
    extern __shared__ float2 sm[];
    const int A = a.A2, B = a.B2, L = A * B;
    float2 *tile = sm, *tw = sm + (size_t)L * kW;
    const int w = threadIdx.x & (kW - 1), p = threadIdx.x >> Sh::LOGW;
    const int chunk = blockIdx.x, row = blockIdx.z;
    long b;
    int c;
    bool ok;
    if (chunk < nfull) {
        b = row;
        c = chunk * kW + w;
        ok = true;
    } else {
        const long f0 = (long)row * kW;
        if (f0 >= (long)nbatch * ntail) return;  // whole block idle (uniform)
        const long f = f0 + w;
        b = f / ntail;
        c = nfull * kW + (int)(f - b * ntail);
        ok = b < nbatch;
    }
    for (int i = threadIdx.x; i < L; i += Sh::T) tw[i] = a.tw[i];
    const long o = blockIdx.y;
    // pass 1: slot p = n1 < B loads x[n1 + B n2] (times the pointwise factor) and runs the
    // A-point DFT while the twiddle table is still being staged; after the barrier it applies
    // the twiddles and stores tile element (n1, k2) of pencil w at (n1 A + k2) W + w. Every
    // thread enters (the size is uniform), so the barrier inside is reached by all.
    const bool act1 = p < B && ok;
    const float2 *in = a.in + o * a.in_so + b * a.in_sb + c;
    const float2 *mul = (MUL != 0 && a.mul) ? a.mul + o * a.mul_so + b * a.mul_sb + c : nullptr;
    Sh::with(A, [&](auto AA) {
        constexpr int NA = decltype(AA)::value;
        float2 v[NA];
        if (act1) {
            if (MUL == 1 || mul) {
                float2 m[NA];
#pragma unroll
                for (int n2 = 0; n2 < NA; ++n2) {
                    const int j = p + B * n2;
                    v[n2] = make_float2(0.f, 0.f);
                    m[n2] = make_float2(0.f, 0.f);
                    if (j < a.lin) {
                        v[n2] = in[(long)j * a.in_sl];
                        m[n2] = mul[(long)j * a.mul_sl];
                    }
                }
#pragma unroll
                for (int n2 = 0; n2 < NA; ++n2) v[n2] = c_mul(v[n2], m[n2]);
            } else {
#pragma unroll
                for (int n2 = 0; n2 < NA; ++n2) {
                    const int j = p + B * n2;
                    v[n2] = j < a.lin ? in[(long)j * a.in_sl] : make_float2(0.f, 0.f);
                }
            }
            fft2::dft_reg<S, NA>(v);
        }
        __syncthreads();
        if (act1) {
            fft2::twiddle<S, NA>(v, p, tw);
#pragma unroll
            for (int k2 = 0; k2 < NA; ++k2) tile[(p * NA + k2) * kW + w] = v[k2];
        }
    });
    __syncthreads();
    // pass 2: slot p = k2 < A, B-point DFT over n1; X[k2 + A k1] -> out[j - j0] if in window
    if (p < A && ok) {
        float2 *out = a.out + o * a.out_so + b * a.out_sb + c;
        Sh::with(B, [&](auto BB) {
            constexpr int NB = decltype(BB)::value;
            float2 u[NB];
#pragma unroll
            for (int n1 = 0; n1 < NB; ++n1) u[n1] = tile[(n1 * A + p) * kW + w];
            fft2::dft_reg<S, NB>(u);
#pragma unroll
            for (int k1 = 0; k1 < NB; ++k1) {
                const int j = p + A * k1 - a.j0;
                if (j >= 0 && j < a.lout) {
                    float2 v = c_scale(u[k1], a.scale);
                    if (a.conj_out) v.y = -v.y;
                    out[(long)j * a.out_sl] = v;
                }
            }
        });
    }
}

template <int S> __global__ void __launch_bounds__(kT2) axis2_kernel(AxisArgs a, int nbatch, int nfull, int ntail)
{
    axis2_body<S, false, -1>(a, nbatch, nfull, ntail);
}

template <int S, int MUL>
__global__ void __launch_bounds__(kT2, MUL == 0 ? 3 : 1) axis2_big_kernel(AxisArgs a, int nbatch, int nfull, int ntail)
{
    axis2_body<S, true, MUL>(a, nbatch, nfull, ntail);
}

// 16 pencils of 32 slots (512 threads): rows of 16 kx (128 bytes) per load
template <int S, int MUL>
__global__ void __launch_bounds__(512, 1) axis2_big_wide_kernel(AxisArgs a, int nbatch, int nfull, int ntail)
{
    axis2_body<S, true, MUL, true>(a, nbatch, nfull, ntail);
}

// Inverse x pass of nr <= NT / A consecutive window rows r0 .. r0 + nr - 1 of orientation slot
// o; row r0 + w's half spectrum starts at rin + w * rstride. The M-point inverse DFT of the
// packed samples runs in two passes: pass 1 gives row w the threads w B .. w B + B - 1 and
// pass 2 the threads w A .. w A + A - 1, so the slots a pass does not need are whole idle
// warps. Row w's line of the tile holds pass-1 element (n1, k2) at n1 Ap + k2 with Ap = A | 1
// odd (stores of consecutive n1 fall in different bank pairs).
template <int NT>
__device__ __forceinline__ void x_rows2(const IrfftArgs &a, const float2 *rin, long rstride, int r0, int nr, long o,
                                        float2 *tile, const float2 *twM, const float2 *twP, uint8_t *sflag)
{
    const int A = a.A2, B = a.B2, M = a.M, Ap = A | 1;
    const int ld = max(M, B * Ap) + 1, fp = (2 * M + 31) & ~31;
    {
        const int w = threadIdx.x / B, p = threadIdx.x - w * B;
        if (w < nr) {
            float2 *line = tile + w * ld;
            fft2::with_size(A, [&](auto AA) {
                constexpr int NA = decltype(AA)::value;
                float2 v[NA];
                x_pack<NA>(rin + w * rstride, p, B, M, twP, v);
                fft2::pass1<1, NA>(v, p, twM);
#pragma unroll
                for (int k2 = 0; k2 < NA; ++k2) line[p * Ap + k2] = v[k2];
            });
        }
    }
    __syncthreads();
    // pass 2 (every thread enters the uniform size dispatch; inactive threads store nothing)
    {
        const int w = threadIdx.x / A, p = threadIdx.x - w * A;
        const bool act = w < nr;
        const float2 *line = tile + w * ld;
        fft2::with_size(B, [&](auto BB) {
            constexpr int NB = decltype(BB)::value;
            float2 u[NB];
            if (act) {
#pragma unroll
                for (int n1 = 0; n1 < NB; ++n1) u[n1] = line[n1 * Ap + p];
                fft2::dft_reg<1, NB>(u);
            }
            x_epilogue<NB>(a, u, A, p, act, r0 + w, o, sflag + w * fp, threadIdx.x & 31);
        });
    }
    if (!a.write_bits) return;   // uniform
    __syncthreads();
    x_pack_bits<NT>(a, sflag, fp, r0, nr, o);
}

// Shared-memory layout of x_rows2 after `base` float2 of other data: the tile (R lines of ld)
// from the next even offset, then R rows of flag bytes (fp each) from a 16-byte boundary.
struct XLayout {
    long tile, flags, end;   // offsets in float2
};
__host__ __device__ inline XLayout x_layout(long base, int NT, int M, int A, int B)
{
    const int R = NT / A, ld = (M > B * (A | 1) ? M : B * (A | 1)) + 1, fp = (2 * M + 31) & ~31;
    XLayout l;
    l.tile = (base + 1) & ~1L;
    l.flags = (l.tile + (long)R * ld + 1) & ~1L;
    l.end = l.flags + ((long)R * fp + 7) / 8;
    return l;
}

// Inverse x pass over R = 256 / A consecutive window rows per block (rows of the input evenly
// spaced: in_sz = rows_y in_sy).
__global__ void __launch_bounds__(kT2) irfft2_threshold_kernel(IrfftArgs a)
{
    extern __shared__ float2 sm[];
    const int M = a.M, R = kT2 / a.A2;
    const XLayout l = x_layout(2 * M + 1, kT2, M, a.A2, a.B2);
    float2 *twM = sm, *twP = sm + M, *tile = sm + l.tile;
    uint8_t *sflag = reinterpret_cast<uint8_t *>(sm + l.flags);
    for (int i = threadIdx.x; i < M; i += kT2) twM[i] = a.twM[i];
    for (int i = threadIdx.x; i <= M; i += kT2) twP[i] = a.twP[i];
    __syncthreads();
    const int r0 = (int)blockIdx.x * R;
    const long o = blockIdx.z;
    x_rows2<kT2>(a, a.in + o * a.in_so + (long)r0 * a.in_sy, a.in_sy, r0, min(R, a.rows - r0), o, tile, twM, twP,
                 sflag);
}

// Inverse y pass and inverse x pass (with the threshold) of one z-plane of one orientation slot
// per block, the plane staying in shared memory between them (no y-pass output in HBM). The
// plane of the inverse-z output (P1 rows ky of hs complex kx, contiguous) arrives in one bulk
// copy and every step runs in place on it:
//   y pass 1 / y pass 2: per group of 32 columns kx (lane = column, warp = slot), all groups of
//     one pass before the next pass; pass 2 keeps the window rows y < lout;
//   x pass 1 / x pass 2: per round of rows y < lout; pass 1 writes its elements (n1, k2) at
//     n1 A + k2 of the row itself (A B = M <= hs); pass 2 ends in the threshold epilogue.
// Each pass loops inside one size case of the uniform dispatch (a loop around the dispatch
// would keep every case's registers live); the free-bit words are packed at the end.
constexpr int kYX = 512;

__host__ __device__ inline long yx2_flags_offset(int Ly, int hs, int M)
{
    return ((long)Ly * hs + Ly + 2 * M + 1 + 1) & ~1L;   // float2 offset, 16-byte aligned
}

__global__ void __launch_bounds__(kYX) yx2_threshold_kernel(AxisArgs ay, IrfftArgs a, int hs)
{
    extern __shared__ float2 sm[];
    __shared__ uint64_t bar;
    const int Ay = ay.A2, By = ay.B2, Ly = Ay * By, Hx = ay.nx;
    const int Ax = a.A2, Bx = a.B2, M = a.M, fp = (2 * M + 31) & ~31, nrow = a.rows_y;
    const long pl = (long)Ly * hs;
    float2 *plane = sm, *twy = sm + pl, *twM = twy + Ly, *twP = twM + M;
    uint8_t *sflag = reinterpret_cast<uint8_t *>(sm + yx2_flags_offset(Ly, hs, M));
    const int z = blockIdx.x;
    const long o = blockIdx.y;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        const uint32_t bytes = (uint32_t)(pl * sizeof(float2));
        tc::mbar_expect_tx(&bar, bytes);
        tc::bulk_g2s(plane, ay.in + o * ay.in_so + (long)z * ay.in_sb, bytes, &bar);
    }
    for (int i = threadIdx.x; i < Ly; i += kYX) twy[i] = ay.tw[i];
    for (int i = threadIdx.x; i < M; i += kYX) twM[i] = a.twM[i];
    for (int i = threadIdx.x; i <= M; i += kYX) twP[i] = a.twP[i];
    __syncthreads();
    if (!tc::mbar_wait(&bar, 0)) {
        // the copy did not land in time: report it, give it one more bounded wait, stop
        if (threadIdx.x == 0) atomicExch(a.status, kDevTimeout);
        tc::mbar_wait(&bar, 0);
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // y pass 1: slot p = warp < By loads x[p + By n2] of column c, A-point DFT and twiddles,
    // element (n1, k2) back to row n1 Ay + k2 of the column
    fft2::with_size(Ay, [&](auto AA) {
        constexpr int NA = decltype(AA)::value;
        for (int c0 = 0; c0 < Hx; c0 += 32) {
            const int c = c0 + lane;
            const bool act = warp < By && c < Hx;
            float2 v[NA];
            if (act) {
#pragma unroll
                for (int n2 = 0; n2 < NA; ++n2) v[n2] = plane[(long)(warp + By * n2) * hs + c];
                fft2::pass1<1, NA>(v, warp, twy);
            }
            __syncthreads();
            if (act) {
#pragma unroll
                for (int k2 = 0; k2 < NA; ++k2) plane[(long)(warp * NA + k2) * hs + c] = v[k2];
            }
        }
    });
    __syncthreads();
    // y pass 2: slot p = warp < Ay, By-point DFT over n1, X[p + Ay k1] to row p + Ay k1 < lout
    fft2::with_size(By, [&](auto BB) {
        constexpr int NB = decltype(BB)::value;
        for (int c0 = 0; c0 < Hx; c0 += 32) {
            const int c = c0 + lane;
            const bool act = warp < Ay && c < Hx;
            float2 u[NB];
            if (act) {
#pragma unroll
                for (int n1 = 0; n1 < NB; ++n1) u[n1] = plane[(long)(n1 * Ay + warp) * hs + c];
                fft2::dft_reg<1, NB>(u);
            }
            __syncthreads();
            if (act) {
#pragma unroll
                for (int k1 = 0; k1 < NB; ++k1) {
                    const int y = warp + Ay * k1;
                    if (y < ay.lout) plane[(long)y * hs + c] = u[k1];
                }
            }
        }
    });
    __syncthreads();
    // x pass 1: rows of Bx threads, kYX / Bx rows per round
    fft2::with_size(Ax, [&](auto AA) {
        constexpr int NA = decltype(AA)::value;
        const int w0 = threadIdx.x / Bx, p = threadIdx.x - w0 * Bx, rpr = kYX / Bx;
        for (int y0 = 0; y0 < nrow; y0 += rpr) {
            const int y = y0 + w0;
            const bool act = w0 < rpr && y < nrow;
            float2 v[NA];
            if (act) {
                x_pack<NA>(plane + (long)y * hs, p, Bx, M, twP, v);
                fft2::pass1<1, NA>(v, p, twM);
            }
            __syncthreads();
            if (act) {
#pragma unroll
                for (int k2 = 0; k2 < NA; ++k2) plane[(long)y * hs + p * NA + k2] = v[k2];
            }
        }
    });
    __syncthreads();
    // x pass 2 and the threshold epilogue: rows of Ax threads, kYX / Ax rows per round
    fft2::with_size(Bx, [&](auto BB) {
        constexpr int NB = decltype(BB)::value;
        const int w0 = threadIdx.x / Ax, p = threadIdx.x - w0 * Ax, rpr = kYX / Ax;
        for (int y0 = 0; y0 < nrow; y0 += rpr) {
            const int y = y0 + w0;
            const bool act = w0 < rpr && y < nrow;
            float2 u[NB];
            if (act) {
#pragma unroll
                for (int n1 = 0; n1 < NB; ++n1) u[n1] = plane[(long)y * hs + n1 * Ax + p];
                fft2::dft_reg<1, NB>(u);
            }
            x_epilogue<NB>(a, u, Ax, p, act, z * nrow + y, o, sflag + (long)(act ? y : 0) * fp, lane);
        }
    });
    if (!a.write_bits) return;   // uniform
    __syncthreads();
    x_pack_bits<kYX>(a, sflag, fp, z * nrow, nrow, o);
}

template <typename K> void set_smem2(K kernel, size_t bytes)
{
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

} // namespace

// the BIG kernel has lengths up to 24 x 24 and 8 (or 16, wide) pencils per block
static size_t axis2_smem_for(int A, int B, int W)
{
    return (size_t)(A * B * W + A * B) * sizeof(float2);
}

size_t irfft2_smem(int M, int A, int B) { return (size_t)x_layout(2 * M + 1, kT2, M, A, B).end * sizeof(float2); }

size_t yx2_smem(int Ly, int hs, int M, int rows)
{
    return (size_t)(yx2_flags_offset(Ly, hs, M) + ((long)rows * ((2 * M + 31) & ~31) + 7) / 8) * sizeof(float2);
}

template <bool BIG, bool WIDE>
static void launch_axis2_shape(int sign, const AxisArgs &a, int nbatch, int norient, cudaStream_t s)
{
    using Sh = AxisShape<BIG, WIDE>;
    constexpr int kW = Sh::W;
    const size_t smem = axis2_smem_for(a.A2, a.B2, kW);
    const int nfull = a.nx / kW, ntail = a.nx % kW;
    // the tail column handles ntail kx of kW rows at a time (nbatch blocks cover them)
    dim3 grid(nfull + (ntail ? 1 : 0), norient, nbatch);
    auto go = [&](auto kernel) {
        set_smem2(kernel, smem);
        kernel<<<grid, Sh::T, smem, s>>>(a, nbatch, nfull, ntail);
    };
    if constexpr (BIG && WIDE) {
        if (sign < 0) go(axis2_big_wide_kernel<-1, 0>);
        else if (a.mul) go(axis2_big_wide_kernel<1, 1>);
        else go(axis2_big_wide_kernel<1, 0>);
    } else if constexpr (BIG) {
        if (sign < 0) go(axis2_big_kernel<-1, 0>);
        else if (a.mul) go(axis2_big_kernel<1, 1>);
        else go(axis2_big_kernel<1, 0>);
    } else {
        if (sign < 0) go(axis2_kernel<-1>);
        else go(axis2_kernel<1>);
    }
}

void launch_axis2(int sign, const AxisArgs &a, int nbatch, int norient, cudaStream_t s)
{
    if (a.tma && launch_axis2_tma(sign, a, nbatch, norient, s)) return;
    if (a.A2 > fft2::kMaxFactor) {
        // big factors: 16 pencils per block where the option asks for it (wider rows of kx per
        // load, one 512-thread block per SM), else 8
        const bool wide = a.mul ? (a.wide & 1) != 0 : (a.wide & 2) != 0;
        if (wide) launch_axis2_shape<true, true>(sign, a, nbatch, norient, s);
        else launch_axis2_shape<true, false>(sign, a, nbatch, norient, s);
    } else {
        launch_axis2_shape<false, false>(sign, a, nbatch, norient, s);
    }
}

void launch_irfft2_threshold(const IrfftArgs &a, int norient, cudaStream_t s)
{
    const size_t smem = irfft2_smem(a.M, a.A2, a.B2);
    set_smem2(irfft2_threshold_kernel, smem);
    const int R = kT2 / a.A2;
    dim3 grid((a.rows + R - 1) / R, 1, norient);
    irfft2_threshold_kernel<<<grid, kT2, smem, s>>>(a);
}

} // namespace imf

namespace imf {

bool yx2_fits(const AxisArgs &ay, const IrfftArgs &a, int hs)
{
    // y pass slots are the block's 16 warps, x pass factors those of the x-pass kernel
    if (ay.A2 <= 0 || a.A2 <= 0 || ay.A2 > fft2::kMaxFactor || a.A2 > fft2::kMaxFactor || ay.in_sl != hs || ay.scale != 1.f || ay.conj_out || ay.mul || ay.j0 != 0 ||
        ay.lin != ay.A2 * ay.B2 || ay.in_sb != (long)ay.lin * hs || (hs & 1))
        return false;
    // x pass 1 writes its elements into the row itself: M = A B must fit the row
    if (a.M > hs) return false;
    return yx2_smem(ay.A2 * ay.B2, hs, a.M, a.rows_y) <= (size_t)(227 * 1024 - 64);
}

void launch_yx2_threshold(const AxisArgs &ay, const IrfftArgs &a, int hs, int nz, int norient, cudaStream_t s)
{
    const size_t smem = yx2_smem(ay.A2 * ay.B2, hs, a.M, a.rows_y);
    set_smem2(yx2_threshold_kernel, smem);
    yx2_threshold_kernel<<<dim3(nz, norient), kYX, smem, s>>>(ay, a, hs);
}

} // namespace imf
