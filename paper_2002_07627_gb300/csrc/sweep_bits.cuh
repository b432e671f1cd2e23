// Bit arithmetic of the sweep (Eq. eq_conv_A) on rows of free translations packed 32 per word
// along x (bit t of word w is translation 32 w + t). Shared by the kernels and the host tests.
//
// Dilation levels: D_j(i) = OR_{t < 2^j} free(i + t), D_0 = free. A sliding OR of length L at
// position s is D_j(s) | D_j(s + L - 2^j) for 2^j <= L <= 2^(j+1): the two windows of length 2^j
// cover [s, s + L) and overlap in the middle.
#pragma once
#include <cstdint>
#include <vector_types.h>

namespace imf {

constexpr int kSweepLevels = 5;   // D_0 .. D_4: runs up to 32 long need windows of at most 16

// Levels 1..4 of word w of a row from the word itself and the next one (0 past the row's end):
// after the shift-OR by 2^(j-1), bit t < 32 of v is the OR of source bits t .. t + 2^j - 1 of
// (lo, hi), all below bit 64 for j <= 4.
__host__ __device__ __forceinline__ void sweep_level_words(uint32_t lo, uint32_t hi, uint32_t *lev)
{
    uint64_t v = (uint64_t)lo | ((uint64_t)hi << 32);
#pragma unroll
    for (int j = 1; j < kSweepLevels; ++j) {
        v |= v >> (1 << (j - 1));
        lev[j - 1] = (uint32_t)v;
    }
}

// Level of a run of length L (1 <= L <= 32): the largest j <= 4 with 2^j <= L.
__host__ __device__ __forceinline__ int sweep_level(int L)
{
    int j = 0;
    while (j < kSweepLevels - 1 && (2 << j) <= L) ++j;
    return j;
}

// 32 bits starting at bit s of a row (s >= 0): two words and a funnel shift.
__host__ __device__ __forceinline__ uint32_t bit_window(const uint32_t *row, int s)
{
    const uint32_t u0 = row[s >> 5], u1 = row[(s >> 5) + 1];
    const int sh = s & 31;
    return sh ? (u0 >> sh) | (u1 << (32 - sh)) : u0;
}

// Low 32 bits of the 64-bit (hi:lo) shifted right by sh & 31.
__host__ __device__ __forceinline__ uint32_t funnel_r(uint32_t lo, uint32_t hi, int sh)
{
#ifdef __CUDA_ARCH__
    return __funnelshift_r(lo, hi, sh);
#else
    return (uint32_t)((((uint64_t)hi << 32) | lo) >> (sh & 31));
#endif
}

// Descriptor of one cutter run for the sweep kernel: the run is [a, b] along x in the row at
// word offset `row` of a level plane, seen from output word q at shift s = kx - b >= 0 (kx: the
// largest cutter x offset). x = row + word of s, y = word distance from s to s + L - 2^j,
// z = (s & 31) | ((s + L - 2^j) & 31) << 8, w = level j.
__host__ __device__ inline int4 sweep_pair(long row, int s, int L)
{
    const int j = sweep_level(L), s2 = s + L - (1 << j);
    return make_int4((int)(row + (s >> 5)), (s2 >> 5) - (s >> 5), (s & 31) | ((s2 & 31) << 8), j);
}

// Bits of one run for the output word whose descriptor-relative base in level d.w is p
// (p = level plane + output row + output word + d.x): the OR of the two windows.
__host__ __device__ __forceinline__ uint32_t sweep_pair_bits(const uint32_t *p, int4 d)
{
    return funnel_r(p[0], p[1], d.z & 31) | funnel_r(p[d.y], p[d.y + 1], d.z >> 8);
}

// Pack 32 flag bytes (each 0 or 1; only the low bit of each byte is read) into one word, byte
// b -> bit b. For a 4-byte group v with bytes c_i in {0, 1}, the multiplier 0x01020408 =
// 2^24 + 2^17 + 2^10 + 2^3 moves byte i (bit 8 i) to bit 24 + i and every cross term to a
// distinct bit below 24, so there are no carries.
__host__ __device__ __forceinline__ uint32_t pack_flag_bytes(const uint32_t *g8)
{
    uint32_t word = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) word |= (((g8[k] & 0x01010101u) * 0x01020408u) >> 24 & 0xfu) << (4 * k);
    return word;
}

} // namespace imf
