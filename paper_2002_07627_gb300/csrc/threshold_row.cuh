// Epilogue of the inverse x pass (both FFT variants): the collision measure of one window row
// from its complex half-length samples, with the threshold of Eq. eq_conv_D fused in.
#pragma once
#include "imf_internal.cuh"

namespace imf {

// Row r (window row index y + rows_y z) of orientation slot o; z[n] is at zrow[n * zs].
// g[i] = Re z[i/2] (i even) or Im z[i/2] (i odd), clamped at 0 (g >= 0 exactly); bit i of the
// row's free mask is g[i] <= theta; translations with |g - theta| <= band are appended to
// the re-check list (overflow is reported through the status word, never written past).
// Called by all 32 lanes of a warp.
__device__ __forceinline__ void threshold_row(const IrfftArgs &a, const float2 *zrow, int zs, long o, int r, int lane)
{
    const int nwords = (a.nout + 31) >> 5;
    const int y = r % a.rows_y, z = r / a.rows_y;
    float *grow = a.g + o * a.g_so + z * a.g_sz + y * a.g_sy;
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
                        const long lin = ((long)z * a.rows_y + y) * a.nout + i;
                        a.flags[slot] = make_int2(a.orient_base + (int)o, (int)lin);
                    } else {
                        atomicExch(a.status, kDevOverflow);
                    }
                }
            }
        }
    }
}

} // namespace imf
