// Host-side plan of the tiled minimum over sharp points (erode.cu): runs of sharp points along
// x, their shared-memory offsets and the dz-chunks whose tile fits the budget. Shared by the
// library (imf_api.cu) and the CPU tests (hosttest.cu), which check the plan without a GPU.
#pragma once
#include <algorithm>
#include <cstdint>
#include <map>
#include <utility>
#include <vector>

#include "erode.cuh"

namespace imf {

// Bank layout of a tile with row pitch P and plane pitch Q (floats): the 32 lanes of a warp
// (8 rows ty x 4 planes tz, same x) read 32 different banks.
inline bool bank_free(int P, int Q)
{
    bool seen[32] = {false};
    for (int tz = 0; tz < 4; ++tz)
        for (int ty = 0; ty < 8; ++ty) {
            const int b = ((tz * Q + ty * P) % 32 + 32) % 32;
            if (seen[b]) return false;
            seen[b] = true;
        }
    return true;
}

// Runs along x (at most maxL long) of the sharp points `sh` (offset triples) of one orientation,
// grouped in dz-chunks whose g tile and run descriptors fit kErodeBudget bytes together (each
// chunk takes as many dz as fit, from the largest down); appends the chunks and their (tile
// offset, length) runs and raises smem_max to the largest tile plus descriptors. K = kmax of the
// tool's cutter offsets (the translation window starts at t = -K).

inline void plan_erode(const std::vector<int32_t> &sh, const int K[3], std::vector<ErodeChunk> &chunks,
                std::vector<int2> &runs, size_t &smem_max, int maxL = kErMaxL)
{
    if (sh.empty()) return;
    int kmn[3] = {1 << 30, 1 << 30, 1 << 30}, kmx[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
    std::map<std::pair<int, int>, std::vector<int>> rows;   // (dz, dy) -> dx
    for (size_t m = 0; m < sh.size(); m += 3) {
        for (int c = 0; c < 3; ++c) { kmn[c] = std::min(kmn[c], sh[m + c]); kmx[c] = std::max(kmx[c], sh[m + c]); }
        rows[{sh[m + 2], sh[m + 1]}].push_back(sh[m]);
    }
    struct Run { int dz, dy, a, L; };
    std::vector<Run> rr;
    for (auto &kv : rows) {
        auto &v = kv.second;
        std::sort(v.begin(), v.end());
        size_t i = 0;
        while (i < v.size()) {
            size_t j = i;
            while (j + 1 < v.size() && v[j + 1] == v[j] + 1) ++j;
            for (int a0 = v[i]; a0 <= v[j]; a0 += maxL)
                rr.push_back({kv.first.first, kv.first.second, a0, std::min(maxL, v[j] - a0 + 1)});
            i = j + 1;
        }
    }
    const int Ex = kmx[0] - kmn[0] + 1, Ey = kmx[1] - kmn[1] + 1;
    const int txh = kErTX + Ex - 1, tyh = kErTY + Ey - 1;
    const int P = txh | 1;
    int Q = tyh * P;
    while (!bank_free(P, Q)) ++Q;
    std::map<int, int> runs_at;                               // dz -> runs
    for (const Run &r : rr) ++runs_at[r.dz];
    const int planes = (int)(kErodeBudget / (4 * (size_t)Q));
    const int dzc_max = std::max(1, planes - kErTZ + 1);
    int dzc = dzc_max;
    for (int hi = kmx[2]; hi >= kmn[2]; hi -= dzc) {
        // the most dz (down from hi) whose tile and descriptors fit the budget together
        dzc = 1;
        for (int d = 1; d <= dzc_max && hi - d + 1 >= kmn[2]; ++d) {
            long nr = 0;
            for (int z = hi - d + 1; z <= hi; ++z) {
                auto it = runs_at.find(z);
                if (it != runs_at.end()) nr += it->second;
            }
            const size_t bytes = 4 * (size_t)er_runs_offset(kErTZ + d - 1, Q) +
                                 8 * (size_t)std::min<long>(nr, kErMaxRunsPerChunk);
            if (bytes > kErodeBudget) break;
            dzc = d;
        }
        const int lo = std::max(kmn[2], hi - dzc + 1);
        std::vector<int2> cr;
        for (const Run &r : rr) {
            if (r.dz < lo || r.dz > hi) continue;
            const int off = (hi - r.dz) * Q + (kmx[1] - r.dy) * P + (kmx[0] - (r.a + r.L - 1));
            cr.push_back(make_int2(off, r.L));
        }
        if (cr.empty()) continue;
        std::stable_sort(cr.begin(), cr.end(), [](const int2 &x, const int2 &y) { return x.y < y.y; });
        for (size_t b = 0; b < cr.size(); b += kErMaxRunsPerChunk) {
            const size_t e = std::min(cr.size(), b + (size_t)kErMaxRunsPerChunk);
            ErodeChunk ch{};
            ch.run0 = (int)runs.size();
            for (size_t i = b; i < e; ++i) runs.push_back(cr[i]);
            ch.run1 = (int)runs.size();
            ch.lend[0] = 0;
            for (int L = 1; L <= kErMaxL3; ++L) {
                int c = ch.lend[L - 1];
                while (ch.run0 + c < ch.run1 && runs[ch.run0 + c].y == L) ++c;
                ch.lend[L] = c;
            }
            ch.txh = txh; ch.tyh = tyh; ch.tzh = kErTZ + (hi - lo);
            ch.pitch_y = P; ch.pitch_z = Q;
            ch.ox = K[0] - kmx[0]; ch.oy = K[1] - kmx[1]; ch.oz = K[2] - hi;
            chunks.push_back(ch);
        }
        for (size_t b = 0; b < cr.size(); b += kErMaxRunsPerChunk) {
            const size_t nr = std::min(cr.size(), b + (size_t)kErMaxRunsPerChunk) - b;
            smem_max = std::max(smem_max, 4 * (size_t)er_runs_offset(kErTZ + (hi - lo), Q) + 8 * nr);
        }
    }
}

} // namespace imf
