// One instance of the TMA-fed persistent axis pass (fft_tma.cuh), chosen by the build:
// IMF_TMA_BIG = 0 (16 pencils of 16 slots, factors <= 16) or 1 (8 pencils of 32 slots, a factor
// above 16); IMF_TMA_VARIANT = 0 (forward), 1 (inverse), 2 (inverse with the pointwise factor).
// The build compiles this file six times, in parallel.
#include "fft_tma.cuh"

#if !defined(IMF_TMA_BIG) || !defined(IMF_TMA_VARIANT)
#error "IMF_TMA_BIG and IMF_TMA_VARIANT are set by the build"
#endif

#define IMF_TMA_CAT2(a, b, c) a##b##c
#define IMF_TMA_CAT(a, b, c) IMF_TMA_CAT2(a, b, c)
#if IMF_TMA_BIG
#define IMF_TMA_NAME IMF_TMA_CAT(launch_tma_b, IMF_TMA_VARIANT, )
#else
#define IMF_TMA_NAME IMF_TMA_CAT(launch_tma_s, IMF_TMA_VARIANT, )
#endif

namespace imf {
namespace tma_fft {

bool IMF_TMA_NAME(const CUtensorMap &in_map, const CUtensorMap &mul_map, Params &P, bool ws, int W, cudaStream_t s)
{
    constexpr int S = IMF_TMA_VARIANT == 0 ? -1 : 1;
    constexpr int MUL = IMF_TMA_VARIANT == 2 ? 1 : 0;
    constexpr bool BIG = IMF_TMA_BIG != 0;
    if (ws) return W == 8 && launch_ws<S, BIG, MUL, 8>(in_map, mul_map, P, s);
    if (BIG && W == 16) return launch_shape<S, true, MUL, 16>(in_map, mul_map, P, s);
    return W == (BIG ? 8 : 16) && launch_shape<S, BIG, MUL, BIG ? 8 : 16>(in_map, mul_map, P, s);
}

} // namespace tma_fft
} // namespace imf
