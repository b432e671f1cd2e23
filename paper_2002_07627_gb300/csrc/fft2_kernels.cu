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
#include "threshold_row.cuh"

namespace imf {

namespace {

constexpr int kW2 = 16;          // pencils (axis passes) or rows (x pass) per block
constexpr int kT2 = 256;         // threads per block: kW2 pencils x 16 slots

// Columns [z][y][kx] of W = 16 consecutive kx per block; a pencil is one (batch row b, kx)
// pair. When nx is not a multiple of 16, the last grid column of blocks takes the remaining
// ntail kx columns of 16 batch rows at a time, so no block transforms empty pencils.
template <int S> __global__ void __launch_bounds__(kT2) axis2_kernel(AxisArgs a, int nbatch, int nfull, int ntail)
{
    extern __shared__ float2 sm[];
    const int A = a.A2, B = a.B2, L = A * B;
    float2 *tile = sm, *tw = sm + (size_t)L * kW2;
    const int w = threadIdx.x & (kW2 - 1), p = threadIdx.x >> 4;
    long b;
    int c;
    bool ok;
    if ((int)blockIdx.x < nfull) {
        b = blockIdx.y;
        c = (int)blockIdx.x * kW2 + w;
        ok = true;
    } else {
        const long f0 = (long)blockIdx.y * kW2;
        if (f0 >= (long)nbatch * ntail) return;  // whole block idle (uniform)
        const long f = f0 + w;
        b = f / ntail;
        c = nfull * kW2 + (int)(f - b * ntail);
        ok = b < nbatch;
    }
    for (int i = threadIdx.x; i < L; i += kT2) tw[i] = a.tw[i];
    const long o = blockIdx.z;
    // pass 1: slot p = n1 < B loads x[n1 + B n2] (times the pointwise factor) and runs the
    // A-point DFT while the twiddle table is still being staged; after the barrier it applies
    // the twiddles and stores tile element (n1, k2) of pencil w at (n1 A + k2) W + w. Every
    // thread enters (the size is uniform), so the barrier inside is reached by all.
    const bool act1 = p < B && ok;
    const float2 *in = a.in + o * a.in_so + b * a.in_sb + c;
    const float2 *mul = a.mul ? a.mul + o * a.mul_so + b * a.mul_sb + c : nullptr;
    fft2::with_size(A, [&](auto AA) {
        constexpr int NA = decltype(AA)::value;
        float2 v[NA];
        if (act1) {
            if (mul) {
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
            for (int k2 = 0; k2 < NA; ++k2) tile[(p * NA + k2) * kW2 + w] = v[k2];
        }
    });
    __syncthreads();
    // pass 2: slot p = k2 < A, B-point DFT over n1; X[k2 + A k1] -> out[j - j0] if in window
    if (p < A && ok) {
        float2 *out = a.out + o * a.out_so + b * a.out_sb + c;
        fft2::with_size(B, [&](auto BB) {
            constexpr int NB = decltype(BB)::value;
            float2 u[NB];
#pragma unroll
            for (int n1 = 0; n1 < NB; ++n1) u[n1] = tile[(n1 * A + p) * kW2 + w];
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

// Inverse x pass over R = 256 / A window rows per block: the half spectrum X[0..M] of a row is
// packed into M complex samples Z[k] = (X[k] + conj X[M-k]) + i exp(+2 pi i k / P)
// (X[k] - conj X[M-k]) as pass 1 loads it, the M-point inverse DFT runs in two passes, the
// samples are written back to the row's shared-memory line in natural order and the threshold
// epilogue reads them. Pass 1 gives row w the threads w B .. w B + B - 1 and pass 2 the threads
// w A .. w A + A - 1, so the slots a pass does not need are whole idle warps. Row w's line
// holds pass-1 element (n1, k2) at n1 Ap + k2 with Ap = A | 1 odd (stores of consecutive n1
// fall in different bank pairs).
__global__ void __launch_bounds__(kT2) irfft2_threshold_kernel(IrfftArgs a)
{
    extern __shared__ float2 sm[];
    const int A = a.A2, B = a.B2, M = a.M, Ap = A | 1, R = kT2 / A;
    const int ld = max(M, B * Ap) + 1;
    float2 *tile = sm, *twM = sm + R * ld, *twP = twM + M;
    // free flags of the block's rows, one byte per translation; rows of fp >= 2 M >= nout bytes,
    // 16-byte aligned
    const int fp = (2 * M + 31) & ~31;
    uint8_t *sflag = reinterpret_cast<uint8_t *>(sm + ((R * ld + 2 * M + 2) & ~1));
    for (int i = threadIdx.x; i < M; i += kT2) twM[i] = a.twM[i];
    for (int i = threadIdx.x; i <= M; i += kT2) twP[i] = a.twP[i];
    __syncthreads();
    const int r0 = (int)blockIdx.x * R;
    const long o = blockIdx.z;
    {
        const int w = threadIdx.x / B, p = threadIdx.x - w * B;
        const int r = r0 + w;
        if (w < R && r < a.rows) {
            const int y = r % a.rows_y, z = r / a.rows_y;
            const float2 *row = a.in + o * a.in_so + z * a.in_sz + y * a.in_sy;
            float2 *line = tile + w * ld;
            fft2::with_size(A, [&](auto AA) {
                constexpr int NA = decltype(AA)::value;
                float2 v[NA], xc[NA];
#pragma unroll
                for (int n2 = 0; n2 < NA; ++n2) {
                    const int k = p + B * n2;
                    v[n2] = row[k];
                    xc[n2] = row[M - k];
                }
#pragma unroll
                for (int n2 = 0; n2 < NA; ++n2) {
                    const int k = p + B * n2;
                    const float2 xk = v[n2], xcc = c_conj(xc[n2]);
                    const float2 e = c_add(xk, xcc);
                    const float2 od = c_mul(c_conj(twP[k]), c_sub(xk, xcc));
                    v[n2] = c_add(e, c_mul_si<1>(od));
                }
                fft2::pass1<1, NA>(v, p, twM);
#pragma unroll
                for (int k2 = 0; k2 < NA; ++k2) line[p * Ap + k2] = v[k2];
            });
        }
    }
    __syncthreads();
    // pass 2 (every thread enters the uniform size dispatch; inactive threads store nothing)
    const int lane = threadIdx.x & 31;
    {
        const int w = threadIdx.x / A, p = threadIdx.x - w * A;
        const bool act = w < R && r0 + w < a.rows;
        float2 *line = tile + w * ld;
        fft2::with_size(B, [&](auto BB) {
            constexpr int NB = decltype(BB)::value;
            float2 u[NB];
            if (act) {
#pragma unroll
                for (int n1 = 0; n1 < NB; ++n1) u[n1] = line[n1 * Ap + p];
                fft2::dft_reg<1, NB>(u);
            }
            // thread (row w, k2 = p) holds z[p + A k1]: g[2j] = Re, g[2j+1] = Im for j = p + A k1,
            // clamped at 0, written straight from registers (consecutive lanes, consecutive j);
            // the free flags g <= theta go to shared memory as bytes and near-threshold
            // translations are listed for the re-check
            int y = 0, z = 0;
            if (act) {
                y = (r0 + w) % a.rows_y;
                z = (r0 + w) / a.rows_y;
            }
            float *grow = a.g + o * a.g_so + z * a.g_sz + y * a.g_sy;
            const long lrow = ((long)z * a.rows_y + y) * a.nout;
#pragma unroll
            for (int k1 = 0; k1 < NB; ++k1) {
                const int i0 = 2 * (p + A * k1);
                const bool v0 = act && i0 < a.nout, v1 = act && i0 + 1 < a.nout;
                const float g0 = fmaxf(u[k1].x, 0.f), g1 = fmaxf(u[k1].y, 0.f);
                if (v1) *reinterpret_cast<float2 *>(grow + i0) = make_float2(g0, g1);
                else if (v0) grow[i0] = g0;
                if (a.write_bits && v0)
                    *reinterpret_cast<uint16_t *>(sflag + w * fp + i0) =
                        (uint16_t)((g0 <= a.theta ? 1u : 0u) | (v1 && g1 <= a.theta ? 0x100u : 0u));
                if (a.flag)
                    record_near(a, o, lrow + i0, v0 && fabsf(g0 - a.theta) <= a.band,
                                v1 && fabsf(g1 - a.theta) <= a.band, lane);
            }
        });
    }
    if (!a.write_bits) return;   // uniform
    __syncthreads();
    // one free-bit word (32 translations along x) per thread, packed from its 32 flag bytes:
    // for a 4-byte group v with bytes b_i in {0, 1}, the multiplier 0x01020408 = 2^24 + 2^17 +
    // 2^10 + 2^3 moves byte i (bit 8 i) to bit 24 + i and every cross term to a distinct bit
    // below 24 (no carries); bytes past nout are masked off
    const int nwq = (a.nout + 31) >> 5;
    for (int i = threadIdx.x; i < R * nwq; i += kT2) {
        const int ww = i / nwq, q = i - ww * nwq, rr = r0 + ww;
        if (rr >= a.rows) break;   // later i only have larger rows
        const uint4 *fw = reinterpret_cast<const uint4 *>(sflag + ww * fp + 32 * q);
        uint32_t word = 0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint4 v = fw[h];
            const uint32_t g4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                word |= (((g4[k] & 0x01010101u) * 0x01020408u) >> 24 & 0xfu) << (16 * h + 4 * k);
        }
        const int rem = a.nout - 32 * q;
        if (rem < 32) word &= (1u << rem) - 1u;
        const int y = rr % a.rows_y, z = rr / a.rows_y;
        a.bits[o * a.b_so + z * a.b_sz + y * a.b_sy + q] = word;
    }
}

template <typename K> void set_smem2(K kernel, size_t bytes)
{
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

} // namespace

size_t axis2_smem(int L) { return (size_t)(L * kW2 + L) * sizeof(float2); }

size_t irfft2_smem(int M, int A, int B)
{
    // R rows of flag bytes (the window has at most 2 M translations along x, rows padded to 32
    // bytes) after the tables, starting on a 16-byte boundary
    const int R = kT2 / A, ld = std::max(M, B * (A | 1)) + 1, fp = (2 * M + 31) & ~31;
    return (size_t)(((R * ld + 2 * M + 2) & ~1) + (R * fp + 7) / 8) * sizeof(float2);
}

void launch_axis2(int sign, const AxisArgs &a, int nbatch, int norient, cudaStream_t s)
{
    const size_t smem = axis2_smem(a.A2 * a.B2);
    const int nfull = a.nx / kW2, ntail = a.nx % kW2;
    dim3 grid(nfull + (ntail ? 1 : 0), nbatch, norient);
    if (sign < 0) {
        set_smem2(axis2_kernel<-1>, smem);
        axis2_kernel<-1><<<grid, kT2, smem, s>>>(a, nbatch, nfull, ntail);
    } else {
        set_smem2(axis2_kernel<1>, smem);
        axis2_kernel<1><<<grid, kT2, smem, s>>>(a, nbatch, nfull, ntail);
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
