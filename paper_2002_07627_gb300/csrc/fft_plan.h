// Padded FFT lengths of a tool plan (imf_set_tool): smooth lengths chosen by a cost model that
// prefers lengths the two-pass register transform splits. Shared by the library (imf_api.cu)
// and the CPU tests (hosttest.cu).
#pragma once
#include "fft.cuh"
#include "fft2.cuh"

namespace imf {

inline bool is_smooth(long n)
{
    for (long p : {2L, 3L, 5L, 7L})
        while (n % p == 0) n /= p;
    return n == 1;
}
inline int next_smooth(int n)
{
    if (n < 1) n = 1;
    while (!is_smooth(n)) ++n;
    return n;
}

// Relative cost of one length-L pass: L times the summed per-point cost of its radix stages
// (radix-8 and radix-4 butterflies are the cheapest per point, 7 and 5 the dearest), or a
// flat per-point cost for lengths the two-pass register transform handles with factors up to
// maxA (16 for the x pass, 24 for the y and z passes).
inline double fft_cost(int L, int maxA)
{
    int A = 0, B = 0;
    // a length with a two-pass split crosses shared memory once and runs unrolled DFTs
    if (fft2::choose_split(L, &A, &B, maxA)) return L * (A > fft2::kMaxFactor ? 1.2 : 1.1);
    FftPlan p;
    if (!make_plan(L, &p)) return 1e300;
    double c = 0;
    for (int s = 0; s < p.nrad; ++s) {
        switch (p.rad[s]) {
        case 8: c += 1.0; break;
        case 4: c += 0.9; break;
        case 2: c += 0.8; break;
        case 3: c += 1.0; break;
        case 5: c += 1.25; break;
        default: c += 1.45; break;
        }
    }
    return L * c;
}

// FFT plan choice: among smooth lengths from the minimum up to 12 % above it, the cheapest
// by fft_cost (a padded transform is correct for any length at or above the minimum).
inline int best_smooth(int n, int maxA)
{
    const int n0 = next_smooth(n);
    int best = n0;
    double bc = fft_cost(n0, maxA);
    for (int m = n0 + 1; m <= n0 + n0 / 8; ++m) {
        if (!is_smooth(m)) continue;
        const double c = fft_cost(m, maxA);
        if (c < bc) { bc = c; best = m; }
    }
    return best;
}

} // namespace imf
