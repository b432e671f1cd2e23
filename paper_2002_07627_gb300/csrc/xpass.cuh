// Pieces of the inverse x pass of the two-pass register FFT shared by the one-shot kernels
// (fft2_kernels.cu) and the persistent kernel fed by tensor copies (fft_tma_x.cu): the packing of
// a row's half spectrum into complex samples, the threshold epilogue (Eq. eq_conv_D) and the
// packing of the free flags into bits.
#pragma once
#include "fft2.cuh"
#include "imf_internal.cuh"
#include "threshold_row.cuh"

namespace imf {
namespace {

// Pass-1 input of the inverse x pass for thread p of a row: the half spectrum X[0..M] of the
// row (at `row`, global or shared memory) packed into the complex samples
// Z[k] = (X[k] + conj X[M-k]) + i exp(+2 pi i k / P) (X[k] - conj X[M-k]), k = p + B n2.
template <int NA>
__device__ __forceinline__ void x_pack(const float2 *row, int p, int B, int M, const float2 *twP, float2 *v)
{
    float2 xc[NA];
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
}

// Threshold epilogue of pass 2 for thread (window row r, k2 = p) holding z[p + A k1] (act:
// the thread has a row): g[2j] = Re, g[2j+1] = Im for j = p + A k1, clamped at 0, written
// straight from registers (consecutive lanes, consecutive j); the free flags g <= theta go to
// the row's flag bytes in shared memory (when bits are wanted) and near-threshold translations
// are listed for the re-check. Called by all 32 lanes of a warp.
template <int NB>
__device__ __forceinline__ void x_epilogue(const IrfftArgs &a, const float2 *u, int A, int p, bool act, int r, long o,
                                           uint8_t *frow, int lane)
{
    int y = 0, z = 0;
    if (act) {
        y = r % a.rows_y;
        z = r / a.rows_y;
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
            *reinterpret_cast<uint16_t *>(frow + i0) =
                (uint16_t)((g0 <= a.theta ? 1u : 0u) | (v1 && g1 <= a.theta ? 0x100u : 0u));
        if (a.flag)
            record_near(a, o, lrow + i0, v0 && fabsf(g0 - a.theta) <= a.band, v1 && fabsf(g1 - a.theta) <= a.band,
                        lane);
    }
}

// Free-bit words of nr window rows r0 .. from their flag bytes (rows fp bytes apart), one word
// (32 translations along x) per thread and step (pack_flag_bytes); bytes past nout are masked
// off.
template <int NT>
__device__ __forceinline__ void x_pack_bits(const IrfftArgs &a, const uint8_t *sflag, int fp, int r0, int nr, long o)
{
    const int nwq = (a.nout + 31) >> 5;
    for (int i = threadIdx.x; i < nr * nwq; i += NT) {
        const int ww = i / nwq, q = i - ww * nwq, rr = r0 + ww;
        const uint4 *fw = reinterpret_cast<const uint4 *>(sflag + (long)ww * fp + 32 * q);
        const uint4 f0 = fw[0], f1 = fw[1];
        const uint32_t g8[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
        uint32_t word = pack_flag_bytes(g8);
        const int rem = a.nout - 32 * q;
        if (rem < 32) word &= (1u << rem) - 1u;
        const int y = rr % a.rows_y, z = rr / a.rows_y;
        a.bits[o * a.b_so + z * a.b_sz + y * a.b_sy + q] = word;
    }
}

} // namespace
} // namespace imf
