/*
 * libimf: inaccessibility measure field (IMF) on one GB300 GPU (sm_103a).
 *
 * The IMF is defined in Mirzendehdel, Behandish, Nelaturi, "Topology Optimization with
 * Accessibility Constraint for Multi-Axis Machining" (arXiv 2002.07627), Sec. 2.1:
 *
 *   f(x) = min_i min_{R in Theta_i} min_{k in K_i} (rho_O * reflected 1_{R T_i})(x - R k)
 *                                                   (Eq. eq_imf_4 and Eq. eq_imf_5)
 *
 * with rho_O = rho_Omega + 1_F (part density plus fixture), T_i = H_i u K_i (holder plus cutter)
 * and the accessible set A = U_R (free translations of R T) + R K (Eq. eq_A / eq_conv_A).
 * Algorithm 1 of the paper normalises f by its maximum, applies the allowance lambda and
 * returns the secluded region Gamma; Eq. eq_filtered_sens / eq_accFilter turn that into the
 * penalty on the compliance sensitivity.
 *
 * Discrete readings used by this library (the paper leaves these open):
 *   - grids are C order [nz][ny][nx], x fastest; nz = 1 is a 2D problem;
 *   - everything outside the grid is empty air (linear, not circular, correlation);
 *   - Omega_0 (the design domain) is the set of grid cells outside the fixture;
 *   - rho_O = min(1, rho_Omega + 1_F) and 1_T = 1_H OR 1_K;
 *   - rotation and resampling: nearest neighbour, inverse map about the tool origin voxel o:
 *     for an integer offset v, u = floor(R^T v + 1/2) (FP64), 1_RT(v) = 1_T(o + u);
 *     R is built from the normalised unit quaternion (w, x, y, z) in the standard way;
 *   - a translation t is collision-free iff g(t) <= theta_i with theta_i = theta_rel * |T_i|
 *     (|T_i| = voxel count of the unrotated tool);
 *   - sharp points default to every voxel of the resampled cutter R K;
 *   - f_bar = f / M with M = max over Omega_0 of f (f_bar = 0 when M = 0); B = [f_bar > lambda];
 *     f_bar <- f_bar * B; Gamma = Omega_0 * [rho_Omega <= tau] * B; fixture cells get
 *     f_bar = 0, Gamma = 0 and A = 0.
 *
 * Ownership: the caller owns every input and output array (device memory unless stated);
 * the library never frees them. The library owns the tool spectra and its scratch buffers,
 * which imf_destroy frees. Calls do not block the host unless stated; errors found on the
 * host are returned at once, errors found on the device are reported by imf_sync_status.
 * A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef IMF_H
#define IMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct imf_handle_s *imf_handle;

typedef enum {
    IMF_OK = 0,
    IMF_ERR_INVALID_ARG = 1, /* a host-side argument check failed (see imf_last_error)       */
    IMF_ERR_OOM = 2,         /* a device allocation failed                                  */
    IMF_ERR_CUDA = 3,        /* a CUDA runtime call failed                                  */
    IMF_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up                          */
    IMF_ERR_NOT_READY = 5,   /* imf_compute before any imf_set_tool                         */
    IMF_ERR_BUDGET = 6,      /* the working set does not fit in hbm_budget_bytes            */
    IMF_ERR_OVERFLOW = 7     /* the near-threshold re-check list overflowed on the device   */
} imf_status;

/* collision-convolution path */
enum { IMF_AUTO = 0, IMF_FP32_FFT = 1, IMF_BF16_DIRECT = 2 };

/* sharp-point sampling of a cutter given without a sharp_mask (Sec. 2.1.5, remark on sampling
 * the cutter boundary; App. B, n_K = O(1) representative points); in the tool frame, before
 * rotation, then resampled like the cutter */
enum { IMF_SHARP_ALL = 0,       /* every cutter voxel (exact IMF)                               */
       IMF_SHARP_BOUNDARY = 1,  /* cutter voxels with a face neighbour outside the cutter      */
       IMF_SHARP_NEAREST = 2 }; /* the sharp_k boundary voxels nearest the tool origin
                                   (squared distance, ties by linear index; nested in k)       */

typedef struct {
    int nx, ny, nz;          /* design grid; nz = 1 is 2D                                       */
    double voxel;            /* voxel edge length; f is reported in voxel volumes (Sec. 2.1.5) */
    double lambda;           /* allowance lambda of Alg. 1 (0.01 in Sec. 2.1.5)                */
    double tau;              /* density threshold tau of Sec. 2.1.5 / Eq. eq_accFilter (0.5)  */
    double theta_rel;        /* collision threshold theta_i = theta_rel * |T_i| (0.01)         */
    int precision;           /* IMF_AUTO | IMF_FP32_FFT | IMF_BF16_DIRECT (collision path)     */
    int recheck;             /* 1: re-check translations with |g - theta| <= band exactly      */
    double recheck_band;     /* band half-width in voxel volumes; <= 0 picks a default         */
    int orient_batch;        /* orientations per batch of device work; 0 = 64 (fewer if the
                                HBM budget needs it)                                           */
    size_t hbm_budget_bytes; /* cap on library-owned device memory; 0 = no cap (App. B)        */
    int erode_groups;        /* orientation groups per tile of the minimum over sharp points
                                (work-unit granularity only; the result does not depend on it);
                                0 = chosen from the grid and the SM count                      */
    int fft_stages_only;     /* 1: every FFT pass uses radix stages (2..8) even where a two-pass
                                register split exists (comparisons, tests, the autotuner); read
                                at every launch; 0 = default                                  */
    int accessible_by_sweep; /* the accessible output of imf_compute: 0 = with one tool whose
                                sharp points are its whole cutter, A = [f <= theta] (exact:
                                both say "some cutter point lies on a free translation"; the
                                route of App. A), else the sweep of Eq. eq_conv_A; 1 = always
                                the sweep                                                      */
    int separate_yx_passes;  /* 1: the inverse y and x passes run as two kernels with the y
                                output in HBM; 0 = one kernel per z-plane that keeps the plane
                                in shared memory, wherever it fits (same arithmetic, same
                                results)                                                       */
    int plan_only;           /* 1: imf_set_tool resamples the tool and plans every size on the
                                host and touches no device (no allocation, no kernel); the
                                handle then answers imf_get_tool_info and imf_footprint but
                                refuses imf_compute (admission planning); 0 = default          */
    int sharp_sampling;      /* IMF_SHARP_ALL (default) | IMF_SHARP_BOUNDARY | IMF_SHARP_NEAREST:
                                sharp points of tools set without a sharp_mask; fewer points
                                can only raise the IMF (conservative, Sec. 2.1.5)             */
    int sharp_k;             /* points kept by IMF_SHARP_NEAREST (>= 1; default 1)             */
    int fft_wide_pencils;    /* launch shape of the y / z FFT passes whose padded length has a
                                factor above 16 (same arithmetic, same results): bit 0 = 16
                                pencils per block or per copy-fed item (128-byte rows) for the z
                                pass with the spectral product, bit 1 = for the other passes,
                                else 8; -1 = library default (16 for every pass)               */
    int fft_tma;             /* launch form of the two-pass y / z FFT passes (same arithmetic,
                                same results): bits 0-1 for the z pass with the spectral
                                product, bits 2-3 for the other passes; 0 = one-shot blocks that
                                load their pencils into registers, 1 = persistent blocks fed by
                                tensor-memory-accelerator copies through a two-stage shared-
                                memory pipeline, 2 = the same with a producer warp and consumer
                                warps that meet once per item; -1 = library default (1 for
                                every pass)                                                    */
    int erode_levels;        /* minimum over sharp points: 1 = dyadic min levels built in the
                                shared-memory tile (one three-input minimum per output and run
                                of any length, but every row's levels rebuilt per chunk), 0
                                (default) = pairwise minima over each run; same results. Tiles
                                with rows above 128 cells use 0                                */
    int fft_tma_x;           /* the inverse x pass with the threshold, where it runs on its own
                                (planes too large for the fused y + x pass): 1 = persistent
                                blocks fed by tensor copies of whole rows, 0 = one-shot blocks;
                                same results; -1 = library default (1)                        */
    int sweep_loop;          /* the sweep of Eq. eq_conv_A: 0 (default) = one thread per output
                                word and orientation of the batch; 1 = each thread walks the
                                batch's orientations for its word and stops once the word is
                                fully accessible (same results; slower where measured)         */
    int erode_xt;            /* minimum over sharp points, pairwise form: consecutive x outputs
                                per thread, 8 (1024 threads per block) or 16 (512 threads, fewer
                                shared loads per output and run, half the resident warps; slower
                                where measured); same results; 0 = library default (8)         */
} imf_options;

/* Fill *opt with the defaults above (grid 0x0x0, which imf_create rejects). */
void imf_default_options(imf_options *opt);

/* Create a handle for one design grid. Allocates nothing on the device yet.
 * Errors: IMF_ERR_INVALID_ARG for non-positive extents or parameters out of range. */
imf_status imf_create(const imf_options *opt, imf_handle *out);

/*
 * Set tool assembly `tool_id` (0 <= tool_id < 64; ids must be set densely from 0) with its
 * orientation set Theta_i (Alg. 1 inputs [1_H_i], [1_K_i], Theta_i; Sec. 2.1.4-2.1.5).
 *   holder, cutter : HOST uint8 arrays [tz][ty][tx], nonzero = inside; copied.
 *   sharp_mask     : HOST uint8 [tz][ty][tx] subset of the cutter used as sharp points, or
 *                    NULL for the handle's sharp_sampling rule (every cutter voxel by
 *                    default); resampled like the cutter.
 *   origin         : tool-frame origin voxel (x, y, z); rotations are about it.
 *   quats          : HOST double [n_orient][4] unit quaternions (w, x, y, z).
 * Resamples the tool on the device, builds the conjugated FFT spectra of every orientation
 * (the reflection of Alg. 1 becomes a conjugation; footnote of Sec. 2.1.5) and keeps them
 * resident. Synchronous (setup call). Errors: IMF_ERR_INVALID_ARG (empty cutter, bad
 * sizes, a cutter that vanishes under every orientation), IMF_ERR_OOM, IMF_ERR_BUDGET,
 * IMF_ERR_CUDA. */
imf_status imf_set_tool(imf_handle h, int tool_id, const uint8_t *holder, const uint8_t *cutter,
                        const uint8_t *sharp_mask, int tx, int ty, int tz, const int origin[3],
                        const double *quats, int n_orient);

/*
 * Algorithm 1 for the current design, asynchronously on `cuda_stream` (a cudaStream_t;
 * NULL = legacy default stream).
 *   rho_omega     : DEVICE float [nz][ny][nx], rho_Omega in [0, 1].
 *   fixture       : DEVICE uint8 [nz][ny][nx] (nonzero = fixture) or NULL.
 *   imf_bar       : DEVICE float [nz][ny][nx] out, f_bar after the allowance.
 *   secluded      : DEVICE uint8 [nz][ny][nx] out, 1_Gamma.
 *   imf_raw       : DEVICE float out, f before normalisation (voxel volumes), or NULL.
 *   accessible    : DEVICE uint8 out, 1_A (A = U_i U_R A_i,R on Omega_0), or NULL.
 * Errors: IMF_ERR_NOT_READY, IMF_ERR_INVALID_ARG (NULL required pointer), IMF_ERR_OOM,
 * IMF_ERR_CUDA; device-side errors via imf_sync_status. */
imf_status imf_compute(imf_handle h, const float *rho_omega, const uint8_t *fixture, float *imf_bar,
                       uint8_t *secluded, float *imf_raw, uint8_t *accessible, void *cuda_stream);

/*
 * Same as imf_compute with HOST arrays (pageable or pinned): copies the inputs to
 * library-owned device buffers, computes, copies the outputs back and waits for the stream.
 * Synchronous. imf_raw and accessible may be NULL. */
imf_status imf_compute_host(imf_handle h, const float *rho_omega, const uint8_t *fixture,
                            float *imf_bar, uint8_t *secluded, float *imf_raw, uint8_t *accessible,
                            void *cuda_stream);

/*
 * Filtered sensitivity of Eq. eq_filtered_sens with the accessibility filter of
 * Eq. eq_accFilter, in place, asynchronously on `cuda_stream`:
 *   S = (1 - w_acc) S_phi / max_{Omega_0} |S_phi| + w_acc S_IMF,
 *   S_IMF = f_bar where rho_Omega > tau, 1 where Gamma, 0 elsewhere.
 *   sens     : DEVICE float [nz][ny][nx], S_phi in, S out (left unnormalised if max = 0).
 *   rho_omega, imf_bar, secluded, fixture (or NULL): DEVICE, as in imf_compute.
 * Errors: IMF_ERR_INVALID_ARG (NULL pointer, w_acc outside [0, 1)), IMF_ERR_CUDA. */
imf_status imf_penalize_sensitivity(imf_handle h, float *sens, const float *rho_omega,
                                    const float *imf_bar, const uint8_t *secluded,
                                    const uint8_t *fixture, double w_acc, void *cuda_stream);

/*
 * Same filtered sensitivity as imf_penalize_sensitivity, for callers that cannot allocate
 * device memory (a host framework that owns all device memory through its own pool, or code
 * that must not stall the device, which cudaMalloc / cudaFree can do). The paper has no
 * counterpart: this is a deployment variant of the step above.
 *   Allocates nothing and needs no handle. Its reduction scratch is a fixed array of
 *   65,600 floats (256 KiB) inside the library, held by every GPU that loads the library
 *   until the process exits; it limits n to 268,435,456 voxels.
 *   sens, rho_omega, imf_bar, secluded, fixture (or NULL): DEVICE arrays of n elements, as in
 *   imf_penalize_sensitivity; tau is the density threshold (0.5 in the paper).
 *   The first call on a device looks up the scratch address on that device (the device that
 *   is current). With lazy module loading (the CUDA default) that lookup may load the
 *   library's device code, which allocates the scratch array and can synchronize the device:
 *   make the first call on each device during set-up, before any stream capture and outside
 *   any section that must not allocate. The address is cached for the life of the device's
 *   context; after a cudaDeviceReset this entry point must not be called again in the process.
 *   Every call shares the scratch array: calls that overlap on the GPU (other streams or
 *   other host threads) race and must not be issued. Asynchronous on cuda_stream.
 * Errors: IMF_ERR_INVALID_ARG (NULL array, n < 1 or n above the limit, w_acc outside [0, 1),
 * tau outside [0, 1]), IMF_ERR_CUDA. */
imf_status imf_penalize_sensitivity_noalloc(float *sens, const float *rho_omega, const float *imf_bar,
                                            const uint8_t *secluded, const uint8_t *fixture, long n,
                                            double w_acc, double tau, void *cuda_stream);

/*
 * Per-orientation accessible sets for machining process planning (Sec. 3.4.1). Runs
 * imf_compute (outputs as there; the accessible set is built by the sweep of Eq. eq_conv_A) and
 * also stores every orientation's own accessible set A_{i,R} before the union of Eq. eq_A_multi:
 *   sets : DEVICE uint32 [n][nz][ny][(nx + 31) / 32], n = total orientations of all tools in
 *          tool order and, within a tool, the caller's orientation order; bit x & 31 of word
 *          x >> 5 of row (y, z) is A_{i,R}(x, y, z). Fixture cells are not masked. Caller-owned;
 *          cleared and written asynchronously on cuda_stream.
 * Errors: as imf_compute; IMF_ERR_INVALID_ARG for a NULL sets pointer. */
imf_status imf_compute_accessible_sets(imf_handle h, const float *rho_omega, const uint8_t *fixture, float *imf_bar,
                                       uint8_t *secluded, uint32_t *sets, void *cuda_stream);

/*
 * Greedy machining process plan (Sec. 3.4.1): the negative space N = Omega_0 and [rho <= tau]
 * (the cells to machine away from the design domain) is removed step by step; each step picks
 * the oriented tool whose accessible set covers the most of what is left of N (ties: the lowest
 * index) and removes that part, until N is empty, no set covers any of the rest, or max_steps.
 *   sets       : DEVICE, as written by imf_compute_accessible_sets (n_sets of them).
 *   rho_omega, fixture (or NULL): DEVICE, the final design, as in imf_compute.
 *   order, removed : HOST int / int64 [max_steps]: set index and voxels removed per step.
 *   n_steps    : HOST out, steps taken; negative / left (or NULL): HOST out, |N| and the
 *                voxels no set can reach (inaccessible negative space).
 * Synchronous (one count per step is read back). Uses handle-owned scratch (grown on demand).
 * Errors: IMF_ERR_INVALID_ARG (NULL, n_sets < 1, max_steps < 0), IMF_ERR_OOM, IMF_ERR_CUDA. */
imf_status imf_process_plan(imf_handle h, const uint32_t *sets, int n_sets, const float *rho_omega,
                            const uint8_t *fixture, int max_steps, int *order, long long *removed, int *n_steps,
                            long long *negative, long long *left, void *cuda_stream);

/*
 * Batched and served forms (not in the paper; they reshape how Alg. 1 is launched).
 *
 * imf_capture_graph records one imf_compute with these exact arrays into a CUDA graph owned by
 * the handle (it first runs imf_compute once on `cuda_stream` so every buffer exists, then
 * captures on that stream). imf_launch_graph replays it on any stream; the arrays given at
 * capture must stay valid and are read / written in place on every replay. Profiling is
 * suspended during capture. Synchronous capture; asynchronous replay.
 * Errors: IMF_ERR_NOT_READY, IMF_ERR_INVALID_ARG, IMF_ERR_CUDA. */
imf_status imf_capture_graph(imf_handle h, const float *rho_omega, const uint8_t *fixture, float *imf_bar,
                             uint8_t *secluded, float *imf_raw, uint8_t *accessible, void *cuda_stream);
imf_status imf_launch_graph(imf_handle h, void *cuda_stream);

/*
 * Autotuner: times imf_compute on these arrays for each orientation-batch size in
 * {4, 8, 16, 32, 64, 128} (capped by the orientation count and the HBM budget) and keeps the
 * fastest; then, by coordinate descent from the handle's options, the FFT form (two-pass
 * register splits or radix stages), the launch form of the y / z passes (fft_tma), their
 * pencils per block (fft_wide_pencils), the x pass's form (fft_tma_x) and the orientation groups
 * of the minimum over sharp points (erode_groups), keeping a change only when it is 3 % faster;
 * then, with IMF_AUTO, the collision path. Every choice selects among equivalent kernels, so
 * the results do not change. The chosen batch goes to *best (NULL allowed); imf_get_options
 * reads the rest. Synchronous; it replaces a captured graph, which must be captured again. */
imf_status imf_autotune(imf_handle h, const float *rho_omega, const uint8_t *fixture, float *imf_bar,
                        uint8_t *secluded, void *cuda_stream, int *best);

/* The handle's current options (after imf_autotune: the tuned ones). */
imf_status imf_get_options(imf_handle h, imf_options *out);

/* Wait for the last stream used by the handle and return the device-side status
 * (IMF_OK, IMF_ERR_OVERFLOW, IMF_ERR_TIMEOUT) or IMF_ERR_CUDA; clears it. */
imf_status imf_sync_status(imf_handle h);

/* Last error message of the handle (static storage owned by the handle; never NULL). */
const char *imf_last_error(imf_handle h);

/* A second handle for the same grid and tools, for concurrent computes of one design (the
 * served form runs several requests of a design at once): it shares the tool spectra and tables
 * (read-only) and owns its own work buffers, allocated at its first imf_compute. The shared
 * tools are freed with the last handle that holds them, whichever is destroyed last; imf_set_tool
 * is refused on a handle whose tools are shared. Computes on the handles may overlap on the GPU.
 * Synchronous. Errors: IMF_ERR_INVALID_ARG, IMF_ERR_NOT_READY (no tool), IMF_ERR_OOM. */
imf_status imf_clone(imf_handle h, imf_handle *out);

/* Free every library-owned device buffer and the handle (tools shared with a clone stay until
 * the last handle holding them is destroyed). NULL is a no-op. */
void imf_destroy(imf_handle h);

/* ---------------------------------------------------------------------------------------
 * Introspection for tests and benchmarks.
 * ------------------------------------------------------------------------------------- */

typedef struct {
    int n_orient;            /* orientations of the tool                                  */
    int P[3];                /* padded FFT extents (x, y, z)                              */
    int kmax[3];             /* max over orientations of the cutter/sharp offsets          */
    int win[3];              /* extents of the translation window t in [-kmax, n-1-kmin]   */
    long size_T;             /* |T_i|, voxels of the unrotated tool                       */
    double theta;            /* theta_i                                                   */
    double band;             /* re-check band half-width                                  */
    long n_rt, n_rk, n_sharp;/* total resampled voxels over all orientations             */
    int path;                /* IMF_FP32_FFT or IMF_BF16_DIRECT                           */
    size_t spectra_bytes;    /* resident tool-spectrum bytes                              */
} imf_tool_info;

imf_status imf_get_tool_info(imf_handle h, int tool_id, imf_tool_info *out);

/* Select the collision path of a tool: IMF_FP32_FFT (needs the spectra, i.e. the handle was not
 * created with IMF_BF16_DIRECT) or IMF_BF16_DIRECT (available when every orientation group's
 * union of rotated tool voxels fits the tensor-core kernel in at most 32 z-slabs of a tile's
 * shared-memory box, which holds for tools tens of voxels across). Synchronous. With IMF_AUTO the
 * path starts as IMF_FP32_FFT and imf_autotune keeps the faster of the two.
 * Errors: IMF_ERR_INVALID_ARG when the path is not available. */
imf_status imf_set_path(imf_handle h, int tool_id, int path);

/* Tensor-core self-test: D[128 x N] = A[128 x K] B[N x K]^T for HOST row-major BF16 bit
 * patterns A, B and a HOST FP32 result D, computed by the same tcgen05 / TMEM / descriptor
 * code the direct path uses (N a multiple of 16 in [16, 256], K a multiple of 16, both operands
 * within 200 KB of shared memory: (128 + N) K 2 bytes). Synchronous; not tied to a handle.
 * Errors: IMF_ERR_INVALID_ARG (NULL, N or K out of range; checked before any allocation),
 * IMF_ERR_OOM, IMF_ERR_CUDA, IMF_ERR_TIMEOUT (a bounded wait of the kernel ran out). */
imf_status imf_selftest_mma(int N, int K, const uint16_t *A, const uint16_t *B, float *D);

/* Copy the resampled offsets of one orientation to HOST int32 [n][3] (x, y, z) arrays:
 * which = 0 (R T), 1 (R K), 2 (sharp points). *n receives the count; `out` may be NULL to
 * query it; `cap` is the capacity of `out` in triples. Synchronous.
 * Errors: IMF_ERR_INVALID_ARG (NULL h or n, tool not set, orient or which out of range, cap
 * below the count). */
imf_status imf_get_offsets(imf_handle h, int tool_id, int orient, int which, int32_t *out,
                           long cap, long *n);

/* Copy the last batch's collision field g (FP32, the translation window of `tool_id`) and
 * its free bits into HOST buffers, for tests: the last orientation batch of the last
 * imf_compute is kept when `keep` was enabled with imf_set_debug. g_out may be NULL to read
 * only the caller's orientation index of the slot. Synchronous.
 * Errors: IMF_ERR_INVALID_ARG (NULL handle, no batch computed yet, slot out of range, cap
 * below the window's floats). */
imf_status imf_set_debug(imf_handle h, int keep_last_g);
imf_status imf_get_last_g(imf_handle h, int slot, float *g_out, long cap, int *orient_out);

/* Copy the free bits of slot `slot` of the last batch into a HOST buffer, for tests: word
 * [z][y][w] (z < win[2], y < win[1], w < (win[0] + 31) / 32 + 2), bit i & 31 of word i >> 5 is
 * [g(t) <= theta] for the translation at window index (i, y, z), after the near-threshold
 * re-check (Eq. eq_conv_D). Available when imf_set_debug(h, 1) was set before the compute (or on
 * the sweep route). `orient_out` receives the caller's orientation index. Synchronous.
 * Errors: IMF_ERR_INVALID_ARG (bad slot, capacity), IMF_ERR_NOT_READY (bits not kept). */
imf_status imf_get_last_bits(imf_handle h, int slot, uint32_t *bits_out, long cap, int *orient_out);

typedef struct {
    long launches;           /* kernels launched by the library since creation             */
    long computes;           /* imf_compute calls                                          */
    long flagged;            /* near-threshold translations re-checked (last compute)      */
    long flagged_total;      /* since creation                                             */
    int n_kernels;           /* entries filled in the per-kernel timing table              */
    size_t owned_bytes;      /* device bytes the handle owns now                           */
} imf_stats;

/* Errors: IMF_ERR_INVALID_ARG (NULL). */
imf_status imf_get_stats(imf_handle h, imf_stats *out);

/* Device footprint of a handle, from the plan of its tools (the sizes App. B's memory-budgeted
 * batching needs before committing memory). Works on a plan_only handle, which holds nothing.
 *   slots : orientation slots of the work buffers (orientations per device batch); 0 = what
 *           the first imf_compute without an HBM budget uses (orient_batch, 64 by default,
 *           capped by the orientation count).
 * Fills resident (tool spectra and tables of every set tool), work (the work buffers the first
 * imf_compute allocates with that many slots), setup_peak (the largest footprint during the
 * imf_set_tool calls, transient rotation and spectrum buffers included) and total =
 * max(resident + work, setup_peak): the most the handle holds through its first compute, not
 * counting imf_compute_host's staging buffers. Synchronous, host only.
 * Errors: IMF_ERR_INVALID_ARG (NULL, slots < 0), IMF_ERR_NOT_READY (no tool set). */
typedef struct {
    size_t resident, work, setup_peak, total;
    int slots;
} imf_footprint_info;
imf_status imf_footprint(imf_handle h, int slots, imf_footprint_info *out);

/* Per-kernel timing with CUDA events on the launching stream (off by default). When on,
 * every launch is bracketed by events; imf_get_kernel_times accumulates their durations. */
imf_status imf_set_profiling(imf_handle h, int on);
/* name/ms/count of kernel class `i` (0 <= i < n_kernels); synchronizes the handle's stream.
 * These three return IMF_ERR_INVALID_ARG for a NULL handle (and i out of range). */
imf_status imf_get_kernel_time(imf_handle h, int i, const char **name, double *total_ms,
                               long *count);
imf_status imf_reset_kernel_times(imf_handle h);

#ifdef __cplusplus
}
#endif

#endif /* IMF_H */
