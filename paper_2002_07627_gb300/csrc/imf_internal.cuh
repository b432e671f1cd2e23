// Internal kernel interface of libimf (not part of the C ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "erode.cuh"
#include "fft.cuh"
#include "sweep_bits.cuh"

namespace imf {

constexpr int kThreads = 256;

// Device status word values (mirror imf_status).
constexpr int kDevOk = 0;
constexpr int kDevTimeout = 4;
constexpr int kDevOverflow = 7;

// ---------------------------------------------------------------------------------------
// FFT passes
// ---------------------------------------------------------------------------------------

// Complex FFT along a strided axis (y or z of the half-spectrum [z][y][kx]). A block
// transforms W consecutive kx columns of one batch row `b` of one orientation `o`.
struct AxisArgs {
    const float2 *in;
    float2 *out;
    const float2 *mul;           // optional pointwise factor applied on load
    long in_so, in_sb, in_sl;    // strides in complex elements: orientation, batch, axis
    long out_so, out_sb, out_sl;
    long mul_so, mul_sb, mul_sl;
    int nx;                      // contiguous extent (number of kx columns)
    int lin;                     // input samples j < lin are read, the rest are zero
    int j0, lout;                // output samples j0 .. j0+lout-1 are written
    float scale;
    int conj_out;
    const float2 *tw;            // exp(-2 pi i m / L), m < L
    FftPlan plan;
    int A2, B2;                  // two-pass split L = A2 B2 (fft2.cuh), or 0: Stockham stages
    int wide;                    // big-factor shape: bit 0 = 16 pencils per block for passes with
                                 // a pointwise factor, bit 1 = for the others (else 8)
    int tma;                     // 1: the persistent TMA-fed kernel (fft_tma.cu) where it applies
    int *status;                 // device status word for bounded-wait timeouts, or NULL
};

// Real-to-complex FFT along x (rows of a real grid), packed as a half-length complex FFT.
struct RfftArgs {
    const float *src;            // real rows
    const uint8_t *fix;          // optional fixture: the row value becomes min(1, src + fix)
    long src_sy, src_sz;         // row strides (elements)
    int rows_y, rows;            // rows per z-plane, total rows
    int nin;                     // valid samples per row (<= 2M), the rest are zero
    float2 *out;
    long out_sy, out_sz;         // complex row strides
    int M;                       // half length: P = 2M
    const float2 *twM;           // exp(-2 pi i m / M)
    const float2 *twP;           // exp(-2 pi i k / P), k <= M
    FftPlan plan;                // length M
};

// Complex-to-real inverse FFT along x with the collision threshold fused in (Sec. 2.1.1:
// free translations are those with g <= theta).
struct IrfftArgs {
    const float2 *in;
    long in_sy, in_sz, in_so;    // rows evenly spaced: in_sz = rows_y * in_sy
    int rows_y, rows;            // window rows per z-plane, total window rows
    int nout;                    // window extent along x
    float *g;
    long g_sy, g_sz, g_so;
    uint32_t *bits;              // free bits, 32 translations per word along x
    long b_sy, b_sz, b_so;
    float theta, band;
    int flag;                    // record translations with |g - theta| <= band
    int2 *flags;
    int *flag_count;
    int *flag_total;
    int flag_cap;
    int *status;
    int orient_base;
    int M;
    const float2 *twM, *twP;
    FftPlan plan;
    int A2, B2;                  // two-pass split M = A2 B2 (fft2.cuh), or 0: Stockham stages
    int write_bits;              // store the free bits (the sweep or a debug copy reads them)
};

void launch_axis_fft(int sign, const AxisArgs &a, int nbatch, int norient, cudaStream_t s);
void launch_rfft_fwd(const RfftArgs &a, cudaStream_t s);
void launch_irfft_threshold(const IrfftArgs &a, int norient, cudaStream_t s);
// The same inverse x pass as a persistent kernel fed by tensor copies of whole rows (hs complex
// each, contiguous); false (nothing launched) where it does not apply.
bool launch_irfft2_tma(const IrfftArgs &a, int hs, int norient, cudaStream_t s);
// two-pass register variants (fft2_kernels.cu); the dispatchers above call them when A2 > 0
void launch_axis2(int sign, const AxisArgs &a, int nbatch, int norient, cudaStream_t s);
// The same pass as a persistent kernel fed by tensor copies; false (nothing launched) where
// a tensor map cannot describe the arrays or the stages do not fit.
bool launch_axis2_tma(int sign, const AxisArgs &a, int nbatch, int norient, cudaStream_t s);
void launch_irfft2_threshold(const IrfftArgs &a, int norient, cudaStream_t s);
// the inverse y and x passes of one z-plane per block (fft2_kernels.cu); yx2_fits says whether
// the plane (and the x pass scratch) fits in shared memory for these arguments
bool yx2_fits(const AxisArgs &ay, const IrfftArgs &a, int hs);
void launch_yx2_threshold(const AxisArgs &ay, const IrfftArgs &a, int hs, int nz, int norient, cudaStream_t s);
size_t irfft2_smem(int M, int A, int B);

// ---------------------------------------------------------------------------------------
// IMF kernels
// ---------------------------------------------------------------------------------------

// Rotation and resampling of the tool (Alg. 1 Rotate): nearest neighbour, inverse map.
struct RotateArgs {
    const uint8_t *T, *K, *Sm;   // tool assembly, cutter, sharp-point mask [tz][ty][tx]
    int tx, ty, tz, ox, oy, oz;
    const double *R;             // 9 per orientation, row major
    const int *box;              // 6 per orientation: lo[3], ext[3]
    const long *box_off;         // start of each orientation's boxes in `out*`
    uint8_t *outT, *outK, *outS;
    int n_orient;
    long max_box;                // largest box volume
};
void launch_rotate(const RotateArgs &a, cudaStream_t s);

// Dense padded real tool array for the spectrum: ones at (v - kmax) mod P for v in R T.
void launch_scatter_tool(float *dst, int Px, int Py, int Pz, const uint32_t *off, int n,
                         int kx, int ky, int kz, cudaStream_t s);

struct RecheckArgs {
    const int2 *flags;
    const int *count;
    int cap;
    const float *rho;
    const uint8_t *fix;
    int nx, ny, nz;
    const uint32_t *rt_off;      // packed offsets of R T, all orientations
    const int *rt_start;         // n_orient + 1
    int wx, wy;                  // window extents (x, y)
    int kx, ky, kz;              // kmax: window index = t + kmax
    float *g;
    long g_sy, g_sz, g_so;
    uint32_t *bits;
    long b_sy, b_sz, b_so;
    double theta;
    int orient_base;
};
void launch_recheck_blocks(const RecheckArgs &a, int max_points, cudaStream_t s);

// Free bits with their dilation levels (sweep_bits.cuh): level j (0 .. kSweepLevels - 1) of
// every slot lives at bits + j * lstride, bit t of word i of level j being the OR of the free
// bits 32 i + t .. 32 i + t + 2^j - 1.
struct SweepLevelsArgs {
    uint32_t *bits;              // level 0 of slot 0 (the free bits)
    long lstride;                // words between levels
    long n;                      // words of the batch's slots (rows of wpr words)
    int wpr;
};
struct SweepArgs {
    const uint32_t *bits;        // level 0 of slot 0; level j at + j * lstride
    long lstride;
    long b_sy, b_sz, b_so;
    // per cutter run, sweep_pair(row, s, L) with row = (kz - dz) b_sz + (ky - dy) b_sy
    const int4 *pairs;
    const int *pair_start;       // n_orient + 1
    int nx, ny, nz, awords;
    int orient_base, nb;
    uint32_t *A;                 // accessible bits [nz][ny][awords], OR-accumulated
    // optional per-orientation sets: A_R of internal orientation og is stored (not OR-ed) at
    // A_per + perm[og] * a_per_so (the caller's orientation index), or nothing when NULL
    uint32_t *A_per;
    long a_per_so;
    const int *perm;
};
void launch_sweep_levels(const SweepLevelsArgs &a, cudaStream_t s);
void launch_sweep(const SweepArgs &a, cudaStream_t s);
// the sweep with the batch's orientations walked inside each thread (early exit per word)
void launch_sweep_loop(const SweepArgs &a, int nsm, cudaStream_t s);

// Greedy machining process plan (Sec. 3.4.1) over per-orientation accessible sets.
// remaining[w] = bits of the negative space Omega_0 and [rho <= tau] in word w of [nz][ny][awords]
void launch_plan_init(const float *rho, const uint8_t *fix, int nx, int ny, int nz, int awords, double tau,
                      uint32_t *remaining, cudaStream_t s);
// counts[s] += popcount(sets[s] & remaining) for s < n_sets (counts zeroed by the caller)
void launch_plan_count(const uint32_t *sets, long set_words, int n_sets, const uint32_t *remaining,
                       unsigned long long *counts, cudaStream_t s);
// remaining &= ~sets[pick]
void launch_plan_remove(const uint32_t *set, long words, uint32_t *remaining, cudaStream_t s);


// Tiled minimum over sharp points: erode.cuh.

// Direct collision convolution on the tensor cores (direct_tc.cu).
// most z-slabs the direct path splits one orientation group's union into
constexpr int kDirectMaxSlabs = 32;
struct DirectArgs {
    const uint32_t *rhohl;       // padded rho_O as (hi | lo << 16) BF16 pairs, [PZ][PY][PX], PX % 4 == 0
    int PX, PY, PZ;              // padded extents
    int lox, loy, loz;           // padding before the grid along x, y, z
    const int *tapoff;           // union taps of the group as word offsets in the tile's box
    int kpad;                    // taps, padded to a multiple of 64 (padding taps have B = 0)
    const uint16_t *bmat;        // B [N x kpad] BF16 0/1 in the K-major canonical layout
    int N, nb;                   // MMA N (multiple of 16) and orientations in the group
    int vlo[3];                  // smallest union offset of the group (x, y, z)
    int BX, BY, BZ;              // box of rho_O words a tile reads per z-slab (BX % 4 == 0)
    int nslab;                   // z-slabs of the union: the box is loaded once per tile and slab
    int slab_c0[kDirectMaxSlabs + 1];  // first 64-tap chunk of each slab (slab_c0[nslab] = kpad / 64)
    int slab_z0[kDirectMaxSlabs];      // first union z offset of each slab, relative to vlo[2]
    int sx;                      // x offset of the tile's first translation in its box (0..3)
    int TY, TZ;                  // tile of 32 x TY x TZ = 128 translations (TY TZ = 4)
    int wx, wy, wz, kx, ky, kz;  // translation window and kmax (t = window index - kmax)
    int ntx, nty, ntz;           // tiles along x, y, z
    float *g;
    long g_sy, g_sz, g_so;
    uint32_t *bits;
    long b_sy, b_sz, b_so;
    float theta, band;
    int flag;
    int2 *flags;
    int *flag_count, *flag_total;
    int flag_cap;
    int *status;
    int orient_base;
};
// dynamic shared memory of the direct kernel for a group with MMA N and a box of `box_words`
size_t direct_smem_bytes(int N, long box_words);
void launch_rho_hl(const float *rho, const uint8_t *fix, int nx, int ny, int nz, int lox, int loy, int loz, int PX,
                   int PY, int PZ, uint32_t *out, cudaStream_t s);
// false when the box cannot be described by a tensor map (the caller reports it)
bool launch_direct(const DirectArgs &a, int nsm, cudaStream_t s);
int run_mma_selftest(const uint16_t *A, const uint16_t *B, float *D, int N, int K, int *status, cudaStream_t s);

void launch_fill_f32(float *p, float v, long n, cudaStream_t s);
void launch_max_omega0(const float *f, const uint8_t *fix, long n, unsigned *maxbits, cudaStream_t s);
struct FinalizeArgs {
    const float *f;
    const float *rho;
    const uint8_t *fix;
    const uint32_t *A;
    int nx, ny, nz, awords;
    const unsigned *maxbits;
    double lambda, tau;
    float *fbar;
    uint8_t *secluded;
    float *raw;
    uint8_t *acc;
    int acc_from_f;              // acc = [f <= theta] instead of the swept bits A
    float theta;
};
void launch_finalize(const FinalizeArgs &a, cudaStream_t s);
void launch_absmax_omega0(const float *v, const uint8_t *fix, long n, unsigned *maxbits, cudaStream_t s);
void launch_penalize(float *sens, const float *rho, const float *fbar, const uint8_t *sec, long n,
                     const unsigned *maxbits, double w, double tau, cudaStream_t s);

// Eq. eq_filtered_sens with the filter of Eq. eq_accFilter at one voxel (FP32):
// S = (1 - w) S_phi / m + w S_IMF with S_IMF = f_bar where rho > tau, 1 on Gamma, 0 elsewhere;
// S_phi stays unnormalised when m = max |S_phi| over Omega_0 is 0. Shared by the handle's
// penalty kernel and the allocation-free one.
__device__ __forceinline__ float penalized_sensitivity(float s, float rho, float fbar, uint8_t sec, float m, float w,
                                                       float tau)
{
    const float sb = m > 0.f ? s * (1.f / m) : s;
    const float simf = rho > tau ? fbar : (sec ? 1.f : 0.f);
    return (1.f - w) * sb + w * simf;
}

} // namespace imf
