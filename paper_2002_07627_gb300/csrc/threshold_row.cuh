// Epilogue of the inverse x pass (both FFT variants): the collision measure of one window row
// from its complex half-length samples, with the threshold of Eq. eq_conv_D fused in.
#pragma once
#include "imf_internal.cuh"

namespace imf {

// Near-threshold translations of one warp step: lanes whose output `near` is set append
// (orientation, window index) to the re-check list; overflow is reported through the status
// word, never written past.
__device__ __forceinline__ void record_near(const IrfftArgs &a, long o, long lin0, bool n0, bool n1, int lane)
{
    const unsigned nm0 = __ballot_sync(0xffffffffu, n0), nm1 = __ballot_sync(0xffffffffu, n1);
    if (!(nm0 | nm1)) return;
    int base = 0;
    if (lane == 0) {
        const int cnt = __popc(nm0) + __popc(nm1);
        base = atomicAdd(a.flag_count, cnt);
        atomicAdd(a.flag_total, cnt);
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    const unsigned lt = (1u << lane) - 1u;
    int slot = base + __popc(nm0 & lt) + __popc(nm1 & lt);
    if (n0) {
        if (slot < a.flag_cap) a.flags[slot] = make_int2(a.orient_base + (int)o, (int)lin0);
        else atomicExch(a.status, kDevOverflow);
        ++slot;
    }
    if (n1) {
        if (slot < a.flag_cap) a.flags[slot] = make_int2(a.orient_base + (int)o, (int)(lin0 + 1));
        else atomicExch(a.status, kDevOverflow);
    }
}

// Row r (window row index y + rows_y z) of orientation slot o; z[n] is at zrow[n * zs].
// g[i] = Re z[i/2] (i even) or Im z[i/2] (i odd), clamped at 0 (g >= 0 exactly); when BITS,
// bit i of the row's free mask is g[i] <= theta; translations with |g - theta| <= band go to
// the re-check list. Called by all 32 lanes of a warp.
template <bool BITS>
__device__ __forceinline__ void threshold_row(const IrfftArgs &a, const float2 *zrow, int zs, long o, int r, int lane)
{
    const int y = r % a.rows_y, z = r / a.rows_y;
    float *grow = a.g + o * a.g_so + z * a.g_sz + y * a.g_sy;
    const long lrow = ((long)z * a.rows_y + y) * a.nout;
    if constexpr (BITS) {
        // one output per lane, one free-bit word per warp step
        const int nwords = (a.nout + 31) >> 5;
        uint32_t *brow = a.bits + o * a.b_so + z * a.b_sz + y * a.b_sy;
        for (int q = 0; q < nwords; ++q) {
            const int i = q * 32 + lane;
            const bool valid = i < a.nout;
            float gv = 0.f;
            if (valid) {
                const float2 zz = zrow[(i >> 1) * zs];
                gv = fmaxf((i & 1) ? zz.y : zz.x, 0.f);
                grow[i] = gv;
            }
            const unsigned freeb = __ballot_sync(0xffffffffu, valid && gv <= a.theta);
            if (lane == 0) brow[q] = freeb;
            if (a.flag) record_near(a, o, lrow + i, valid && fabsf(gv - a.theta) <= a.band, false, lane);
        }
    } else {
        // no free bits wanted: each lane takes one complex sample, i.e. two outputs
        for (int s = 0; 64 * s < a.nout; ++s) {
            const int i0 = 64 * s + 2 * lane;
            const bool v0 = i0 < a.nout, v1 = i0 + 1 < a.nout;
            float g0 = 0.f, g1 = 0.f;
            if (v0) {
                const float2 zz = zrow[(32 * s + lane) * zs];
                g0 = fmaxf(zz.x, 0.f);
                g1 = fmaxf(zz.y, 0.f);
                if (v1) *reinterpret_cast<float2 *>(grow + i0) = make_float2(g0, g1);
                else grow[i0] = g0;
            }
            if (a.flag)
                record_near(a, o, lrow + i0, v0 && fabsf(g0 - a.theta) <= a.band,
                            v1 && fabsf(g1 - a.theta) <= a.band, lane);
        }
    }
}

// Dispatch on whether the free bits are wanted (uniform across the launch).
__device__ __forceinline__ void threshold_row_any(const IrfftArgs &a, const float2 *zrow, int zs, long o, int r, int lane)
{
    if (a.write_bits) threshold_row<true>(a, zrow, zs, o, r, lane);
    else threshold_row<false>(a, zrow, zs, o, r, lane);
}

} // namespace imf
