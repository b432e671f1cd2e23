// Host-only exports that run the kernels' building blocks (fft.cuh, fft2.cuh, erode_plan.h,
// fft_plan.h, orient_order.h, sweep_bits.cuh) on the CPU, for the CPU unit tests. Not part of
// libimf and never loaded by the product path.
#include <cmath>
#include <cstring>
#include <vector>

#include "fft.cuh"
#include "fft2.cuh"
#include "erode_plan.h"
#include "fft_plan.h"
#include "orient_order.h"
#include "sweep_bits.cuh"

extern "C" int imf_host_fft(int L, int sign, const float *in, float *out)
{
    imf::FftPlan p;
    if (L < 1 || !imf::make_plan(L, &p)) return -1;
    std::vector<float2> tw(L), a(L), b(L);
    for (int m = 0; m < L; ++m) {
        const double ang = -2.0 * M_PI * (double)m / (double)L;
        tw[m] = make_float2((float)std::cos(ang), (float)std::sin(ang));
        a[m] = make_float2(in[2 * m], in[2 * m + 1]);
    }
    float2 *r = sign < 0 ? imf::fft_pencil_host<-1>(p, a.data(), b.data(), tw.data())
                         : imf::fft_pencil_host<1>(p, a.data(), b.data(), tw.data());
    for (int m = 0; m < L; ++m) {
        out[2 * m] = r[m].x;
        out[2 * m + 1] = r[m].y;
    }
    return p.nrad;
}

// Number of (d, j) pairs, 2 <= d <= maxd, 0 <= j < maxj, where the stage reciprocal disagrees
// with integer division.
extern "C" long imf_host_check_div(int maxd, int maxj)
{
    long bad = 0;
    for (int d = 1; d <= maxd; ++d) {
        const unsigned mul = imf::div_magic((unsigned)d);
        for (int j = 0; j < maxj; ++j)
            if (imf::fast_div((unsigned)j, mul) != (unsigned)(j / d)) ++bad;
    }
    return bad;
}

// The two-pass register transform of fft2.cuh on one pencil. Returns 100 A + B for the split
// it used, or -1 when L has no supported split.
extern "C" int imf_host_fft2(int L, int sign, const float *in, float *out)
{
    int A = 0, B = 0;
    if (L < 4 || !imf::fft2::choose_split(L, &A, &B, imf::fft2::kMaxFactorBig)) return -1;
    std::vector<float2> tw(L), x(L), X(L), T(L);
    for (int m = 0; m < L; ++m) {
        const double ang = -2.0 * M_PI * (double)m / (double)L;
        tw[m] = make_float2((float)std::cos(ang), (float)std::sin(ang));
        x[m] = make_float2(in[2 * m], in[2 * m + 1]);
    }
    if (sign < 0) imf::fft2::fft2_pencil_host<-1>(A, B, x.data(), X.data(), T.data(), tw.data());
    else imf::fft2::fft2_pencil_host<1>(A, B, x.data(), X.data(), T.data(), tw.data());
    for (int m = 0; m < L; ++m) {
        out[2 * m] = X[m].x;
        out[2 * m + 1] = X[m].y;
    }
    return 100 * A + B;
}

// The plan of the tiled minimum over sharp points for one orientation's sharp offsets
// (n_pts triples x, y, z), window origin K and longest run maxL (16 or 31). Writes per chunk 44
// ints (run0, run1, txh, tyh, tzh, pitch_y, pitch_z, ox, oy, oz, lend[0..31], 0, 0) and per run
// 2 ints (tile offset, length). Returns the number of chunks, or -1 when the output arrays are
// too small; *smem gets the largest tile in bytes and *nruns the number of runs.
extern "C" int imf_host_plan_erode(const int *sh, int n_pts, const int *K, int maxL, int max_chunks, int *chunk_out,
                                   int max_runs, int *runs_out, long *smem, int *nruns)
{
    std::vector<int32_t> v(sh, sh + 3 * (size_t)n_pts);
    std::vector<imf::ErodeChunk> chunks;
    std::vector<int2> runs;
    size_t sm = 0;
    imf::plan_erode(v, K, chunks, runs, sm, maxL);
    *smem = (long)sm;
    *nruns = (int)runs.size();
    if ((int)chunks.size() > max_chunks || (int)runs.size() > max_runs) return -1;
    for (size_t c = 0; c < chunks.size(); ++c) {
        const imf::ErodeChunk &ch = chunks[c];
        int *o = chunk_out + 44 * c;
        const int head[10] = {ch.run0, ch.run1, ch.txh, ch.tyh, ch.tzh, ch.pitch_y, ch.pitch_z, ch.ox, ch.oy, ch.oz};
        for (int i = 0; i < 10; ++i) o[i] = head[i];
        for (int i = 0; i <= imf::kErMaxL3; ++i) o[10 + i] = ch.lend[i];
        o[42] = o[43] = 0;
    }
    for (size_t r = 0; r < runs.size(); ++r) {
        runs_out[2 * r] = runs[r].x;
        runs_out[2 * r + 1] = runs[r].y;
    }
    return (int)chunks.size();
}

// Tile geometry constants of the plan (kErTX, kErTY, kErTZ, kErXT, kErMaxL, budget bytes,
// runs per chunk).
extern "C" void imf_host_erode_constants(long *out)
{
    out[0] = imf::kErTX; out[1] = imf::kErTY; out[2] = imf::kErTZ; out[3] = imf::kErXT;
    out[4] = imf::kErMaxL; out[5] = (long)imf::kErodeBudget; out[6] = imf::kErMaxRunsPerChunk;
}

// One cutter run of the sweep as the kernels compute it (sweep_bits.cuh): the dilation levels
// of a row of wpr words, then the two windows of the run's descriptor for output word q at
// shift s >= 0 and length L (1 .. 32). Returns 1 for arguments out of range (reads past the row).
extern "C" int imf_host_sweep_run(const uint32_t *row, int wpr, int q, int s, int L, uint32_t *out)
{
    if (!row || !out || wpr < 2 || q < 0 || s < 0 || L < 1 || L > 32) return 1;
    const int4 d = imf::sweep_pair(0, s, L);
    if (q + d.x + d.y + 1 >= wpr) return 1;
    std::vector<uint32_t> lev((size_t)imf::kSweepLevels * wpr);
    for (int w = 0; w < wpr; ++w) {
        uint32_t l[imf::kSweepLevels - 1];
        imf::sweep_level_words(row[w], w + 1 < wpr ? row[w + 1] : 0u, l);
        lev[w] = row[w];
        for (int j = 1; j < imf::kSweepLevels; ++j) lev[(size_t)j * wpr + w] = l[j - 1];
    }
    *out = imf::sweep_pair_bits(lev.data() + (size_t)d.w * wpr + q + d.x, d);
    return 0;
}

// The x pass's packing of 32 free-flag bytes into one word (pack_flag_bytes).
extern "C" uint32_t imf_host_pack_flags(const uint8_t *bytes32)
{
    uint32_t g8[8];
    std::memcpy(g8, bytes32, sizeof g8);
    return imf::pack_flag_bytes(g8);
}

// The padded length the planner picks for a minimum length n with two-pass factors up to maxA,
// and the split it then uses (A, B; 0 when the length runs the radix-stage kernels).
extern "C" int imf_host_plan_length(int n, int maxA, int *A, int *B)
{
    const int L = imf::best_smooth(n, maxA);
    *A = *B = 0;
    if (!imf::fft2::choose_split(L, A, B, maxA)) *A = *B = 0;
    return L;
}

// The internal orientation order for n rotations (row-major 3 x 3 each): the nearest-neighbour
// chain, interleaved by spread_order when `spread` is set.
extern "C" void imf_host_orient_order(const double *R, int n, int spread, int *out)
{
    std::vector<double> r(R, R + 9 * (size_t)n);
    std::vector<int> o = imf::locality_order(r, n);
    if (spread) o = imf::spread_order(o);
    for (int i = 0; i < n; ++i) out[i] = o[i];
}
