// Internal order of a tool's orientations (imf_set_tool). Results never depend on it; it only
// groups device work. Shared by the library (imf_api.cu) and the CPU tests (hosttest.cu).
#pragma once
#include <algorithm>
#include <utility>
#include <vector>

namespace imf {

// Greedy nearest-neighbour chain over the rotations (Frobenius distance), so that consecutive
// orientations, and therefore every group of the direct path, have overlapping supports.
inline std::vector<int> locality_order(const std::vector<double> &R, int n)
{
    std::vector<int> order;
    std::vector<char> used(n, 0);
    int cur = 0;
    for (int step = 0; step < n; ++step) {
        order.push_back(cur);
        used[cur] = 1;
        int best = -1;
        double bd = 1e300;
        for (int j = 0; j < n; ++j) {
            if (used[j]) continue;
            double d = 0;
            for (int e = 0; e < 9; ++e) d += (R[9 * cur + e] - R[9 * j + e]) * (R[9 * cur + e] - R[9 * j + e]);
            if (d < bd) { bd = d; best = j; }
        }
        if (best < 0) break;
        cur = best;
    }
    return order;
}

// Chain positions in the order of the base-2 radical inverse of their index (van der Corput):
// every prefix of the result is spread evenly along the chain.
inline std::vector<int> spread_order(const std::vector<int> &chain)
{
    const int n = (int)chain.size();
    std::vector<std::pair<double, int>> key(n);
    for (int i = 0; i < n; ++i) {
        double v = 0, b = 0.5;
        for (unsigned k = (unsigned)i; k; k >>= 1, b *= 0.5)
            if (k & 1) v += b;
        key[i] = {v, i};
    }
    std::sort(key.begin(), key.end());
    std::vector<int> out(n);
    for (int i = 0; i < n; ++i) out[i] = chain[key[i].second];
    return out;
}

} // namespace imf
