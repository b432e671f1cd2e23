// C ABI of libimf (include/imf.h): handle, tool setup, planning and the launch sequence of
// Algorithm 1 on one GPU. Host code only; kernels live in fft_kernels.cu and imf_kernels.cu.
//
// Data layout in device memory (per tool plan, x fastest everywhere):
//   spectra   [n_orient][Pz][Py][Hs] complex64, conj(FFT(1_RT)) / (Px Py Pz), resident
//   rho spec  [Pz][Py][Hs]            FFT(rho_O), once per imf_compute and plan
//   per batch slot (orientations processed together):
//     Y1 [Wz][Py][Hs], Y2 [Wz][Wy][Hs] complex64 (inverse-FFT intermediates)
//     g  [Wz][Wy][gpx] float  collision measure on the translation window
//     free bits [Wz][Wy][wpr] uint32
//   f [nz][ny][nx] float running minimum; A bits [nz][ny][awords]
// The translation window holds t in [-kmax, n - 1 - kmin] per axis at index t + kmax, where
// kmin / kmax bound the cutter and sharp-point offsets of every orientation of the tool.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <map>
#include <memory>
#include <unordered_map>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "imf.h"
#include "fft2.cuh"
#include "imf_internal.cuh"
#include "erode_plan.h"
#include "fft_plan.h"
#include "orient_order.h"

using namespace imf;

namespace {

// defaults of imf_options::fft_wide_pencils and fft_tma: every big-factor y / z pass fed by
// tensor copies with 16 pencils per item (128-byte rows per copy). Measured at 256^3 x 128 on one
// box: z pass 10.6 ms (copies, 8 pencils) -> 7.8 ms (16 pencils); y pass 9.0 ms (one-shot, 8
// pencils) -> 6.4 ms (copies, 16 pencils); the warp-specialised form with 8 pencils was slower
constexpr int kFftWideDefault = 3;
constexpr int kFftTmaDefault = 5;

enum KernelId {
    KID_ROTATE, KID_SPEC, KID_RFFT_FWD, KID_AXIS_FWD, KID_AXIS_INV_MUL, KID_AXIS_INV, KID_IRFFT_THRESH,
    KID_RECHECK, KID_SWEEP, KID_ERODE, KID_INIT, KID_MAX, KID_FINALIZE, KID_ABSMAX, KID_PENALIZE, KID_RHO_HL,
    KID_DIRECT, KID_SWEEP_LEVELS, KID_YX, KID_PLAN, KID_COUNT
};
const char *kKernelNames[KID_COUNT] = {
    "rotate_resample", "tool_spectrum", "rfft_x_fwd", "fft_axis_fwd", "fft_z_inv_mul", "fft_y_inv",
    "irfft_x_threshold", "recheck_near_threshold", "sweep_dilate", "erode_min", "init", "max_omega0",
    "finalize", "absmax_omega0", "penalize", "rho_hi_lo", "direct_corr_tcgen05", "sweep_levels", "fft_yx_inv_threshold",
    "process_plan"};

// Geometry of one orientation group of the direct path: the union's smallest offset, the box of
// rho_O words a tile reads per z-slab, the tile's x offset in it, and the slabs (first chunk and
// first union z offset of each).
struct DirectGroup {
    int glo[3] = {0, 0, 0};
    int BX = 0, BY = 0, BZ = 0, sx = 0, nslab = 1;
    int c0[kDirectMaxSlabs + 1] = {0};
    int z0[kDirectMaxSlabs] = {0};
};

struct Tool {
    bool set = false;
    int tx = 0, ty = 0, tz = 0, o[3] = {0, 0, 0}, n_orient = 0;
    long size_T = 0;
    double theta = 0, band = 0;
    std::vector<std::vector<int32_t>> rt, rk, sh;   // per-orientation offset triples
    int kmin[3] = {0, 0, 0}, kmax[3] = {0, 0, 0};
    int P[3] = {1, 1, 1}, M = 1, Hx = 2, Hs = 2;
    int win[3] = {1, 1, 1}, gpx = 4, wpr = 3;
    FftPlan plM{}, ply{}, plz{};
    int sM[2] = {0, 0}, sy[2] = {0, 0}, sz[2] = {0, 0};  // two-pass splits (A, B), or 0
    float2 *twM = nullptr, *twP = nullptr, *twy = nullptr, *twz = nullptr;
    float2 *spec = nullptr;
    size_t spec_bytes = 0;
    uint32_t *rt_off = nullptr;
    int *rt_start = nullptr;
    int4 *sw_pairs = nullptr;            // sweep run descriptors (SweepArgs::pairs), all orientations
    int *sw_start = nullptr;
    ErodeChunk *er_chunks = nullptr;
    int *er_chunk_start = nullptr;
    int2 *er_runs = nullptr;
    size_t erode_smem = 0;
    int erode_bps = 1;                   // resident erosion blocks per SM
    bool erode_levels = false;           // plan and kernel of the dyadic-level minimum (erode3)
    long n_rt = 0, n_rk = 0, n_sh = 0;
    std::vector<int> perm, iperm;        // internal orientation order -> caller's index, and back
    int *perm_dev = nullptr;             // perm on the device (per-orientation outputs)
    int path = IMF_FP32_FFT;             // collision path in use
    bool sharp_is_cutter = true;         // sharp points = every cutter voxel (no proper subset)
    bool has_spec = false;               // FFT spectra built
    // direct tensor-core path
    bool dir_ok = false;
    int dG = 0;                          // orientations per group
    std::vector<int> grp_start, grp_kpad, grp_N;
    std::vector<long> grp_tap_off, grp_b_off;
    std::vector<DirectGroup> grp_geo;    // per group: union minimum, box, z-slabs
    int dTY = 2, dTZ = 2;                // tile of 32 x dTY x dTZ translations
    int *d_taps = nullptr;
    uint16_t *d_bmat = nullptr;
    int dlo[3] = {0, 0, 0}, dP[3] = {1, 1, 1};
    double direct_macs = 0;              // tensor MACs per compute (both BF16 halves)
    // device bytes of this tool: resident tables (offset lists, run descriptors, twiddles,
    // direct-path taps) and the largest footprint of its imf_set_tool beyond what was owned
    // before (transient rotation and spectrum buffers included)
    size_t table_bytes = 0, setup_bytes = 0;
    bool planned_only = false;           // sizes planned on the host, nothing on the device
};

struct ProfRec {
    int kid;
    cudaEvent_t a, b;
};

} // namespace

struct imf_handle_s {
    imf_options opt{};
    std::string err = "";
    Tool tools[64];
    int n_tools = 0;
    // compute work buffers (grow only)
    float2 *rho_spec = nullptr, *X1 = nullptr, *X2 = nullptr;
    size_t rho_spec_n = 0, X1_n = 0, X2_n = 0;
    uint32_t *rhohl = nullptr;
    size_t rhohl_n = 0;
    int nsm = 152;
    float2 *Y1 = nullptr, *Y2 = nullptr;
    float *g = nullptr;
    uint32_t *bits = nullptr;
    size_t Y1_n = 0, Y2_n = 0, g_n = 0, bits_n = 0;  // per slot
    int slots = 0;
    float *f = nullptr;
    uint32_t *A = nullptr;
    int awords = 0;
    int2 *flags = nullptr;
    int flag_cap = 0;
    int *dev_small = nullptr;   // [0] status, [1] flag count of the batch, [2] maxbits,
                                // [3] maxbits (penalize), [4] flags of the last compute
    // host staging for imf_compute_host
    float *h_rho = nullptr, *h_fbar = nullptr, *h_raw = nullptr;
    uint8_t *h_fix = nullptr, *h_sec = nullptr, *h_acc = nullptr;
    cudaStream_t last_stream = nullptr;
    bool used_stream = false;
    size_t owned_bytes = 0;
    std::unordered_map<void *, size_t> sizes;
    // stats
    long launches = 0, computes = 0, flagged_last = 0, flagged_total = 0;
    // profiling
    bool prof = false;
    std::vector<ProfRec> prof_pending;
    std::vector<cudaEvent_t> ev_pool;
    double prof_ms[KID_COUNT] = {0};
    long prof_cnt[KID_COUNT] = {0};
    // captured graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    // per-orientation accessible sets (imf_compute_accessible_sets): bits of all orientations
    uint32_t *aset = nullptr;
    long aset_so = 0;
    // greedy process plan work buffers
    uint32_t *plan_rem = nullptr;
    unsigned long long *plan_cnt = nullptr;
    size_t plan_rem_n = 0, plan_cnt_n = 0;
    // tools shared with clones (imf_clone): the last handle holding a reference frees them
    std::shared_ptr<int> tool_refs;
    // debug
    bool keep_g = false;
    bool run_sweep = true;      // this compute builds A by the sweep (else A = [f <= theta])
    int last_batch_base = -1, last_batch_n = 0, last_tool = -1;
};

namespace {

imf_status fail(imf_handle h, imf_status st, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
imf_status fail(imf_handle h, imf_status st, const char *fmt, ...)
{
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return st;
}

#define CU(call)                                                                                    \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess)                                                                      \
            return fail(h, e_ == cudaErrorMemoryAllocation ? IMF_ERR_OOM : IMF_ERR_CUDA, "%s: %s (%s:%d)", \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                         \
    } while (0)

template <typename T> imf_status dalloc(imf_handle h, T **p, size_t n)
{
    *p = nullptr;
    if (n == 0) n = 1;
    const size_t bytes = n * sizeof(T);
    if (h->opt.hbm_budget_bytes && h->owned_bytes + bytes > h->opt.hbm_budget_bytes)
        return fail(h, IMF_ERR_BUDGET, "device allocation of %zu bytes exceeds hbm_budget_bytes (%zu owned)",
                    bytes, h->owned_bytes);
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(h, IMF_ERR_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    h->owned_bytes += bytes;
    h->sizes[(void *)*p] = bytes;
    return IMF_OK;
}

template <typename T> void dfree(imf_handle h, T *&p, size_t = 0)
{
    if (p) {
        cudaFree(p);
        auto it = h->sizes.find((void *)p);
        if (it != h->sizes.end()) {
            h->owned_bytes -= std::min(h->owned_bytes, it->second);
            h->sizes.erase(it);
        }
    }
    p = nullptr;
}

#define TRY(x)                                                                                      \
    do {                                                                                            \
        imf_status s_ = (x);                                                                        \
        if (s_ != IMF_OK) return s_;                                                                \
    } while (0)

// ----------------------------------------------------------------------------- profiling
cudaEvent_t get_event(imf_handle h)
{
    if (!h->ev_pool.empty()) {
        cudaEvent_t e = h->ev_pool.back();
        h->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

struct Launch {
    imf_handle h;
    int kid;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    Launch(imf_handle h_, int kid_, cudaStream_t s_) : h(h_), kid(kid_), s(s_)
    {
        if (h->prof) {
            a = get_event(h);
            cudaEventRecord(a, s);
        }
    }
    ~Launch()
    {
        h->launches++;
        if (h->prof) {
            cudaEvent_t b = get_event(h);
            cudaEventRecord(b, s);
            h->prof_pending.push_back({kid, a, b});
        }
    }
};

void drain_profile(imf_handle h)
{
    for (auto &r : h->prof_pending) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        h->prof_ms[r.kid] += ms;
        h->prof_cnt[r.kid] += 1;
        h->ev_pool.push_back(r.a);
        h->ev_pool.push_back(r.b);
    }
    h->prof_pending.clear();
}

// R from the unit quaternion (w, x, y, z), normalised first; row major, v = R u.
void quat_to_R(const double *q, double *R)
{
    const double n = std::sqrt(((q[0] * q[0] + q[1] * q[1]) + q[2] * q[2]) + q[3] * q[3]);
    const double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
    R[0] = 1.0 - 2.0 * (y * y + z * z);
    R[1] = 2.0 * (x * y - w * z);
    R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);
    R[4] = 1.0 - 2.0 * (x * x + z * z);
    R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);
    R[7] = 2.0 * (y * z + w * x);
    R[8] = 1.0 - 2.0 * (x * x + y * y);
}

// Host copy of rotate_kernel's arithmetic for one orientation (the same FP64 operation order,
// host code compiled without contraction), so the plan-only path resamples the tool on the CPU
// with the same result as the device.
void rotate_host(const uint8_t *T, const uint8_t *K, const uint8_t *S, int tx, int ty, int tz, const int *o,
                 const double *R, const int *bx, uint8_t *oT, uint8_t *oK, uint8_t *oS)
{
    const long vol = (long)bx[3] * bx[4] * bx[5];
    for (long idx = 0; idx < vol; ++idx) {
        const int i = (int)(idx % bx[3]);
        const int j = (int)((idx / bx[3]) % bx[4]);
        const int k = (int)(idx / ((long)bx[3] * bx[4]));
        const double v0 = bx[0] + i, v1 = bx[1] + j, v2 = bx[2] + k;
        int u[3];
        for (int c = 0; c < 3; ++c) {
            const double a0 = R[c] * v0, a1 = R[3 + c] * v1, a2 = R[6 + c] * v2;
            const double p = (a0 + a1) + a2;
            u[c] = (int)std::floor(p + 0.5);
        }
        const int ax = o[0] + u[0], ay = o[1] + u[1], az = o[2] + u[2];
        uint8_t t = 0, kk = 0, ss = 0;
        if (ax >= 0 && ax < tx && ay >= 0 && ay < ty && az >= 0 && az < tz) {
            const long src = ((long)az * ty + ay) * tx + ax;
            t = T[src];
            kk = K[src];
            ss = S[src];
        }
        oT[idx] = t;
        oK[idx] = kk;
        oS[idx] = ss;
    }
}

// Sharp-point sampling of the cutter (Sec. 2.1.5 remark on sampling the cutter boundary; App. B
// on n_K = O(1) representative points), in the tool frame before rotation: IMF_SHARP_BOUNDARY
// keeps the cutter voxels with a face neighbour outside the cutter (or outside the array);
// IMF_SHARP_NEAREST keeps the k boundary voxels nearest the tool origin (squared distance, ties
// by linear index), so the sets for growing k are nested. Fewer sharp points can only raise the
// IMF (a conservative approximation).
void sample_sharp_points(const std::vector<uint8_t> &K, int tx, int ty, int tz, const int *o, int mode, int k,
                         std::vector<uint8_t> &S)
{
    auto in = [&](int x, int y, int z) {
        return x >= 0 && y >= 0 && z >= 0 && x < tx && y < ty && z < tz && K[((long)z * ty + y) * tx + x];
    };
    std::vector<std::pair<long, long>> cand;   // (squared distance to the origin, linear index)
    std::fill(S.begin(), S.end(), 0);
    for (int z = 0; z < tz; ++z)
        for (int y = 0; y < ty; ++y)
            for (int x = 0; x < tx; ++x) {
                if (!in(x, y, z)) continue;
                const bool surf = !in(x - 1, y, z) || !in(x + 1, y, z) || !in(x, y - 1, z) || !in(x, y + 1, z) ||
                                  !in(x, y, z - 1) || !in(x, y, z + 1);
                if (!surf) continue;
                const long id = ((long)z * ty + y) * tx + x;
                if (mode == IMF_SHARP_BOUNDARY) S[id] = 1;
                const long dx = x - o[0], dy = y - o[1], dz = z - o[2];
                cand.push_back({dx * dx + dy * dy + dz * dz, id});
            }
    if (mode == IMF_SHARP_NEAREST) {
        std::sort(cand.begin(), cand.end());
        for (size_t i = 0; i < cand.size() && (long)i < (long)k; ++i) S[cand[i].second] = 1;
    }
}

// Scan box of the rotated array: the tool's voxel cubes rotate into the hull of the rotated
// corners of its voxel-edge box; one voxel of margin on every side.
void scan_box(const double *R, int tx, int ty, int tz, const int *o, int *box)
{
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    const double ex[3][2] = {{-o[0] - 0.5, tx - o[0] - 0.5}, {-o[1] - 0.5, ty - o[1] - 0.5}, {-o[2] - 0.5, tz - o[2] - 0.5}};
    for (int c = 0; c < 8; ++c) {
        const double u[3] = {ex[0][c & 1], ex[1][(c >> 1) & 1], ex[2][(c >> 2) & 1]};
        for (int r = 0; r < 3; ++r) {
            const double v = R[3 * r] * u[0] + R[3 * r + 1] * u[1] + R[3 * r + 2] * u[2];
            lo[r] = std::min(lo[r], v);
            hi[r] = std::max(hi[r], v);
        }
    }
    for (int r = 0; r < 3; ++r) {
        box[r] = (int)std::floor(lo[r]) - 1;
        box[3 + r] = (int)std::ceil(hi[r]) + 1 - box[r] + 1;
    }
}

void twiddles(int L, int denom, int count, std::vector<float2> &out)
{
    out.resize(std::max(count, 1));
    for (int m = 0; m < count; ++m) {
        const double a = -2.0 * M_PI * (double)m / (double)denom;
        out[m] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    (void)L;
}

template <typename T> imf_status upload(imf_handle h, T **dst, const std::vector<T> &src)
{
    TRY(dalloc(h, dst, src.size()));
    if (!src.empty()) CU(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return IMF_OK;
}

void free_tool(imf_handle h, Tool &t)
{
    dfree(h, t.twM, (size_t)t.M);
    dfree(h, t.twP, (size_t)t.M + 1);
    dfree(h, t.twy, (size_t)t.P[1]);
    dfree(h, t.twz, (size_t)t.P[2]);
    dfree(h, t.spec, t.spec_bytes / sizeof(float2));
    dfree(h, t.rt_off, (size_t)t.n_rt);
    dfree(h, t.rt_start, (size_t)t.n_orient + 1);
    dfree(h, t.sw_pairs, (size_t)0);
    dfree(h, t.sw_start, (size_t)t.n_orient + 1);
    dfree(h, t.er_chunks);
    dfree(h, t.er_chunk_start);
    dfree(h, t.er_runs);
    dfree(h, t.d_taps);
    dfree(h, t.d_bmat);
    dfree(h, t.perm_dev);
    t = Tool();
}

constexpr size_t kDirectSmemLimit = 224 * 1024;

// byte offset of element (row r, column k) in a K-major canonical tile with R rows
inline size_t tc_kmajor(int r, int k, int R) { return (size_t)(k >> 3) * (R * 16) + (r >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

// Groups of consecutive orientations, their union tap lists (word offsets in the box of rho_O a
// tile of the direct kernel reads) and B matrices (BF16 0/1, K-major canonical layout, N rows).
// A union too tall for one box in shared memory is cut into z-slabs (balanced, each slab's taps
// padded to whole 64-tap chunks); the box is then loaded once per tile and slab. The group size
// minimises a cost model of the kernel: per tile and 64 taps of the union, the A build (about 512
// shared-memory wavefronts, whatever N) or the MMAs and their operand reads (about 4.6 N + 256
// cycles), whichever is larger, summed over the groups.
bool plan_direct(Tool &t, const int n[3], int vlo[3], int vhi[3], std::vector<int> &taps, std::vector<uint16_t> &bm)
{
    for (int c = 0; c < 3; ++c) {
        t.dlo[c] = std::max(0, t.kmax[c] - vlo[c]);
        const int hi = std::max(0, vhi[c] - t.kmin[c]);
        t.dP[c] = n[c] + t.dlo[c] + hi;
    }
    t.dP[0] = (t.dP[0] + 3) & ~3;           // rows of 16-byte multiples (tensor-map stride)
    t.dTY = n[2] == 1 ? 4 : 2;
    t.dTZ = n[2] == 1 ? 1 : 2;
    const int EX = vhi[0] - vlo[0] + 1, EY = vhi[1] - vlo[1] + 1;
    auto key = [&](const int32_t *v) {
        return ((long)(v[2] - vlo[2]) * EY + (v[1] - vlo[1])) * EX + (v[0] - vlo[0]);
    };
    auto unkey = [&](long k, int v[3]) {
        v[0] = (int)(k % EX) + vlo[0];
        v[1] = (int)((k / EX) % EY) + vlo[1];
        v[2] = (int)(k / ((long)EX * EY)) + vlo[2];
    };
    // union of a group as sorted keys (z-major), with its bounds
    auto group_union = [&](int o0, int nb, std::vector<long> &uni, int glo[3], int ghi[3]) {
        uni.clear();
        for (int c = 0; c < 3; ++c) { glo[c] = 1 << 30; ghi[c] = -(1 << 30); }
        for (int i = o0; i < o0 + nb; ++i)
            for (size_t m = 0; m < t.rt[i].size(); m += 3) {
                uni.push_back(key(&t.rt[i][m]));
                for (int c = 0; c < 3; ++c) {
                    glo[c] = std::min(glo[c], t.rt[i][m + c]);
                    ghi[c] = std::max(ghi[c], t.rt[i][m + c]);
                }
            }
        std::sort(uni.begin(), uni.end());
        uni.erase(std::unique(uni.begin(), uni.end()), uni.end());
    };
    // box and slabs of a group with MMA N: the tallest slab whose box fits, then balanced slabs
    auto geometry = [&](const int glo[3], const int ghi[3], int N, DirectGroup &gg) {
        gg.BX = (3 + 32 + ghi[0] - glo[0] + 3) & ~3;
        gg.BY = t.dTY + ghi[1] - glo[1];
        const int EZ = ghi[2] - glo[2] + 1;
        int sz = 0;
        for (int h = 1; h <= EZ; ++h) {
            const int bz = t.dTZ + h - 1;
            if (bz > 256 || direct_smem_bytes(N, (long)gg.BX * gg.BY * bz) > kDirectSmemLimit) break;
            sz = h;
        }
        if (gg.BX > 256 || gg.BY > 256 || sz < 1) return false;
        gg.nslab = (EZ + sz - 1) / sz;
        if (gg.nslab > kDirectMaxSlabs) return false;
        sz = (EZ + gg.nslab - 1) / gg.nslab;
        gg.BZ = t.dTZ + sz - 1;
        for (int c = 0; c < 3; ++c) gg.glo[c] = glo[c];
        gg.sx = (((glo[0] - t.kmax[0] + t.dlo[0]) % 4) + 4) % 4;
        for (int sl = 0; sl < gg.nslab; ++sl) gg.z0[sl] = sl * sz;
        return true;
    };
    // padded tap order of a group: per slab, its taps (box word offsets) padded to whole chunks;
    // pos[i] = padded index of union entry i
    auto layout = [&](const std::vector<long> &uni, DirectGroup &gg, std::vector<int> *offs, std::vector<int> &pos) {
        pos.assign(uni.size(), 0);
        int np = 0;
        size_t i = 0;
        const int sz = gg.nslab > 1 ? gg.z0[1] : gg.BZ - t.dTZ + 1;
        for (int sl = 0; sl < gg.nslab; ++sl) {
            gg.c0[sl] = np / 64;
            int v[3];
            for (; i < uni.size(); ++i) {
                unkey(uni[i], v);
                if ((v[2] - gg.glo[2]) / sz != sl) break;
                pos[i] = np++;
                if (offs)
                    offs->push_back((v[0] - gg.glo[0]) + gg.BX * ((v[1] - gg.glo[1]) + gg.BY * (v[2] - gg.glo[2] - gg.z0[sl])));
            }
            while (np % 64 || np == gg.c0[sl] * 64) {
                ++np;
                if (offs) offs->push_back(0);
            }
        }
        gg.c0[gg.nslab] = np / 64;
        return np;
    };
    int bestG = 0;
    double best = 1e300;
    std::vector<long> uni;
    std::vector<int> pos;
    for (int G = std::min(256, (t.n_orient + 15) / 16 * 16); G >= 16; G -= 16) {
        bool fits = true;
        double cost = 0;
        for (int o0 = 0; o0 < t.n_orient && fits; o0 += G) {
            const int nb = std::min(G, t.n_orient - o0), N = (nb + 15) / 16 * 16;
            int glo[3], ghi[3];
            DirectGroup gg;
            group_union(o0, nb, uni, glo, ghi);
            fits = geometry(glo, ghi, N, gg);
            if (!fits) break;
            const int kpad = layout(uni, gg, nullptr, pos);
            cost += kpad * std::max(512.0, 4.6 * N + 256.0);
        }
        if (fits && cost < best) {
            best = cost;
            bestG = G;
        }
    }
    if (!bestG) return false;
    const int G = bestG;
    std::vector<int> gs, gk, gn;
    std::vector<long> gto, gbo;
    std::vector<DirectGroup> geo;
    std::vector<int> tp;
    std::vector<uint16_t> b;
    double macs = 0;
    for (int o0 = 0; o0 < t.n_orient; o0 += G) {
        const int nb = std::min(G, t.n_orient - o0), N = (nb + 15) / 16 * 16;
        int glo[3], ghi[3];
        DirectGroup gg;
        group_union(o0, nb, uni, glo, ghi);
        geometry(glo, ghi, N, gg);
        gs.push_back(o0);
        gto.push_back((long)tp.size());
        gbo.push_back((long)b.size());
        const int kpad = layout(uni, gg, &tp, pos);
        gk.push_back(kpad);
        gn.push_back(N);
        geo.push_back(gg);
        const size_t b0 = b.size();
        b.resize(b0 + (size_t)N * kpad, 0);
        for (int i = o0; i < o0 + nb; ++i)
            for (size_t m = 0; m < t.rt[i].size(); m += 3) {
                const int k = (int)(std::lower_bound(uni.begin(), uni.end(), key(&t.rt[i][m])) - uni.begin());
                b[b0 + tc_kmajor(i - o0, pos[k], N) / 2] = 0x3F80;    // BF16 1.0
            }
        const long tiles = (long)((t.win[0] + 31) / 32) * ((t.win[1] + t.dTY - 1) / t.dTY) *
                           ((t.win[2] + t.dTZ - 1) / t.dTZ);
        macs += 2.0 * tiles * 128.0 * N * kpad;
    }
    gs.push_back(t.n_orient);
    t.dG = G;
    t.grp_start = gs;
    t.grp_kpad = gk;
    t.grp_N = gn;
    t.grp_tap_off = gto;
    t.grp_b_off = gbo;
    t.grp_geo = geo;
    t.direct_macs = macs;
    taps.swap(tp);
    bm.swap(b);
    return true;
}

// Sizes of the per-handle work buffers for the current tools (elements; see ensure_work).
struct WorkSizes {
    size_t rs = 0, x1 = 0, x2 = 0, y1 = 0, y2 = 0, gn = 0, bn = 0, hl = 0;
    int maxo = 1, min_slots = 1;
};

WorkSizes work_sizes(imf_handle h)
{
    const imf_options &op = h->opt;
    WorkSizes w;
    for (int i = 0; i < h->n_tools; ++i) {
        const Tool &t = h->tools[i];
        w.rs = std::max(w.rs, (size_t)t.P[2] * t.P[1] * t.Hs);
        w.x1 = std::max(w.x1, (size_t)op.nz * op.ny * t.Hs);
        w.x2 = std::max(w.x2, (size_t)op.nz * t.P[1] * t.Hs);
        w.y1 = std::max(w.y1, (size_t)t.win[2] * t.P[1] * t.Hs);
        w.y2 = std::max(w.y2, (size_t)t.win[2] * t.win[1] * t.Hs);
        w.gn = std::max(w.gn, (size_t)t.win[2] * t.win[1] * t.gpx);
        w.bn = std::max(w.bn, (size_t)t.win[2] * t.win[1] * t.wpr);
        w.maxo = std::max(w.maxo, t.n_orient);
        if (t.path == IMF_BF16_DIRECT) {
            w.hl = std::max(w.hl, (size_t)t.dP[0] * t.dP[1] * t.dP[2]);
            w.min_slots = std::max(w.min_slots, std::min(t.dG, t.n_orient));
        }
    }
    return w;
}

// Orientation slots of the first imf_compute without an HBM budget: the requested batch (64 by
// default), at most the largest orientation count, at least one direct-path group.
int default_slots(imf_handle h, const WorkSizes &w)
{
    int want = h->opt.orient_batch > 0 ? h->opt.orient_batch : 64;
    return std::max(std::min(want, w.maxo), w.min_slots);
}

// Bytes the work buffers of a first imf_compute with `slots` orientation slots allocate
// (each allocation as dalloc makes it: at least one element).
size_t work_bytes(imf_handle h, const WorkSizes &w, int slots)
{
    const imf_options &op = h->opt;
    auto b = [](size_t n, size_t e) { return std::max<size_t>(n, 1) * e; };
    const size_t N = (size_t)op.nx * op.ny * op.nz;
    const size_t awords = (size_t)(op.nx + 31) / 32;
    size_t t = 0;
    if (w.hl) t += b(w.hl, 4);
    t += b(N, 4) + b((size_t)op.nz * op.ny * awords, 4) + b(8, 4);
    t += b(w.rs, 8) + b(w.x1, 8) + b(w.x2, 8);
    t += b(w.y1 * slots, 8) + b(w.y2 * slots, 8) + b(w.gn * slots, 4) + b(w.bn * slots * kSweepLevels, 4);
    const long wcap = std::max<long>(1 << 16, (long)(w.gn * slots / 32));
    t += b((size_t)wcap, 8);
    return t;
}

imf_status ensure_work(imf_handle h)
{
    const imf_options &op = h->opt;
    const long N = (long)op.nx * op.ny * op.nz;
    const WorkSizes ws = work_sizes(h);
    const size_t rs = ws.rs, x1 = ws.x1, x2 = ws.x2, y1 = ws.y1, y2 = ws.y2, gn = ws.gn, bn = ws.bn, hl = ws.hl;
    const int min_slots = ws.min_slots;
    if (hl > h->rhohl_n) { dfree(h, h->rhohl); h->rhohl_n = 0; TRY(dalloc(h, &h->rhohl, hl)); h->rhohl_n = hl; }
    if (!h->f) {
        TRY(dalloc(h, &h->f, (size_t)N));
        h->awords = (op.nx + 31) / 32;
        TRY(dalloc(h, &h->A, (size_t)op.nz * op.ny * h->awords));
        TRY(dalloc(h, &h->dev_small, (size_t)8));
        CU(cudaMemset(h->dev_small, 0, 8 * sizeof(int)));
    }
    if (rs > h->rho_spec_n) { dfree(h, h->rho_spec, h->rho_spec_n); TRY(dalloc(h, &h->rho_spec, rs)); h->rho_spec_n = rs; }
    if (x1 > h->X1_n) { dfree(h, h->X1, h->X1_n); TRY(dalloc(h, &h->X1, x1)); h->X1_n = x1; }
    if (x2 > h->X2_n) { dfree(h, h->X2, h->X2_n); TRY(dalloc(h, &h->X2, x2)); h->X2_n = x2; }
    // default batch: 64 orientations (larger batches prune more in the minimum and the sweep,
    // since outputs that reach 0 skip the rest of their orientation group, and leave fewer
    // partial waves; 128^3 x 64: 5.9 ms per step against 6.3 with 16)
    int want = default_slots(h, ws);
    // per orientation slot: Y1, Y2, g, free bits and its share of the near-threshold list
    const size_t per_slot = y1 * 8 + y2 * 8 + gn * 4 + bn * 4 * kSweepLevels + (gn / 32 + 1) * sizeof(int2);
    if (op.hbm_budget_bytes) {
        const size_t have = op.hbm_budget_bytes > h->owned_bytes ? op.hbm_budget_bytes - h->owned_bytes : 0;
        const size_t cur = (size_t)h->slots * (h->Y1_n * 8 + h->Y2_n * 8 + h->g_n * 4 + h->bits_n * 4 * kSweepLevels) +
                           (size_t)h->flag_cap * sizeof(int2);
        const size_t fixed = (size_t)(1 << 16) * sizeof(int2);
        const long fit = (long)((have + cur > fixed ? have + cur - fixed : 0) / std::max<size_t>(per_slot, 1));
        if (fit < min_slots)
            return fail(h, IMF_ERR_BUDGET, "%d orientation slots need %zu bytes; budget has %zu", min_slots,
                        per_slot * min_slots, have + cur);
        want = (int)std::min<long>(want, fit);
    }
    if (y1 > h->Y1_n || y2 > h->Y2_n || gn > h->g_n || bn > h->bits_n || want != h->slots) {
        dfree(h, h->Y1);
        dfree(h, h->Y2);
        dfree(h, h->g);
        dfree(h, h->bits);
        dfree(h, h->flags);
        h->flag_cap = 0;
        h->slots = 0;          // consistent if an allocation below fails: the next call retries
        h->Y1_n = std::max(y1, h->Y1_n);
        h->Y2_n = std::max(y2, h->Y2_n);
        h->g_n = std::max(gn, h->g_n);
        h->bits_n = std::max(bn, h->bits_n);
        TRY(dalloc(h, &h->Y1, h->Y1_n * want));
        TRY(dalloc(h, &h->Y2, h->Y2_n * want));
        TRY(dalloc(h, &h->g, h->g_n * want));
        TRY(dalloc(h, &h->bits, h->bits_n * want * kSweepLevels));   // free bits and their dilation levels
        CU(cudaMemset(h->bits, 0, h->bits_n * want * kSweepLevels * sizeof(uint32_t)));
        CU(cudaMemset(h->g, 0, h->g_n * want * sizeof(float)));
        h->slots = want;
    }
    const long wcap = std::max<long>(1 << 16, (long)(h->g_n * h->slots / 32));
    if (!h->flags || wcap > h->flag_cap) {
        dfree(h, h->flags);
        h->flag_cap = 0;
        TRY(dalloc(h, &h->flags, (size_t)wcap));
        h->flag_cap = (int)std::min<long>(wcap, 1L << 30);
    }
    return IMF_OK;
}

// Pencils per block of the big-factor axis kernel (AxisArgs::wide): the option, or the default.
int fft_wide(imf_handle h) { return h->opt.fft_wide_pencils >= 0 ? h->opt.fft_wide_pencils : kFftWideDefault; }
// consecutive x outputs per thread of the pairwise minimum over sharp points
int erode_xt(const imf_options &o) { return o.erode_xt > 0 ? o.erode_xt : 8; }

// the two-pass split of a pass, or none (radix stages) when the handle asks for stages only
template <typename Args> void set_split(imf_handle h, Args &a, const int *sp)
{
    const bool stages = h->opt.fft_stages_only != 0;
    a.A2 = stages ? 0 : sp[0];
    a.B2 = stages ? 0 : sp[1];
}

// launch options shared by every axis pass of the handle
void axis_opts(imf_handle h, AxisArgs &a)
{
    a.wide = fft_wide(h);
    // bits 0-1: the pass with the pointwise factor (the z pass of the collision convolution),
    // bits 2-3: the others; 0 = one-shot blocks, 1 = tensor-copy pipeline with block barriers,
    // 2 = warp-specialised tensor-copy pipeline
    const int m = h->opt.fft_tma < 0 ? kFftTmaDefault : h->opt.fft_tma;
    a.tma = a.mul ? (m & 3) : ((m >> 2) & 3);
    a.status = h->dev_small;
}

// forward 3D real FFT of a real grid [nz][ny][nx] (optionally min(1, x + fixture)) into the
// half spectrum [Pz][Py][Hs] of plan `t`, using X1 / X2 as intermediates
imf_status forward_real_3d(imf_handle h, const Tool &t, const float *src, const uint8_t *fix, int nx, int ny, int nz,
                           float2 *X1, float2 *X2, float2 *out, float scale, int conj_out, cudaStream_t s)
{
    {
        RfftArgs a{};
        a.src = src; a.fix = fix; a.src_sy = nx; a.src_sz = (long)nx * ny; a.rows_y = ny; a.rows = ny * nz;
        a.nin = nx; a.out = X1; a.out_sy = t.Hs; a.out_sz = (long)ny * t.Hs; a.M = t.M; a.twM = t.twM; a.twP = t.twP;
        a.plan = t.plM;
        Launch L(h, KID_RFFT_FWD, s);
        launch_rfft_fwd(a, s);
    }
    {
        AxisArgs a{};
        a.in = X1; a.in_sb = (long)ny * t.Hs; a.in_sl = t.Hs;
        a.out = X2; a.out_sb = (long)t.P[1] * t.Hs; a.out_sl = t.Hs;
        a.nx = t.Hx; a.lin = ny; a.j0 = 0; a.lout = t.P[1]; a.scale = 1.f; a.tw = t.twy; a.plan = t.ply;
        set_split(h, a, t.sy); axis_opts(h, a);
        Launch L(h, KID_AXIS_FWD, s);
        launch_axis_fft(-1, a, nz, 1, s);
    }
    {
        AxisArgs a{};
        a.in = X2; a.in_sb = t.Hs; a.in_sl = (long)t.P[1] * t.Hs;
        a.out = out; a.out_sb = t.Hs; a.out_sl = (long)t.P[1] * t.Hs;
        a.nx = t.Hx; a.lin = nz; a.j0 = 0; a.lout = t.P[2]; a.scale = scale; a.conj_out = conj_out;
        a.tw = t.twz; a.plan = t.plz;
        set_split(h, a, t.sz); axis_opts(h, a);
        Launch L(h, KID_AXIS_FWD, s);
        launch_axis_fft(-1, a, t.P[1], 1, s);
    }
    return IMF_OK;
}

} // namespace

// ============================================================================== C ABI

extern "C" {

void imf_default_options(imf_options *opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof *opt);
    opt->voxel = 1.0;
    opt->lambda = 0.01;
    opt->tau = 0.5;
    opt->theta_rel = 0.01;
    opt->precision = IMF_AUTO;
    opt->recheck = 1;
    opt->recheck_band = 0.0;
    opt->orient_batch = 0;
    opt->hbm_budget_bytes = 0;
    opt->erode_groups = 0;
    opt->fft_stages_only = 0;
    opt->accessible_by_sweep = 0;
    opt->separate_yx_passes = 0;
    opt->plan_only = 0;
    opt->sharp_sampling = IMF_SHARP_ALL;
    opt->sharp_k = 1;
    opt->fft_wide_pencils = -1;
    opt->fft_tma = -1;
    opt->erode_levels = 0;
    opt->fft_tma_x = -1;
    opt->sweep_loop = 0;
    opt->erode_xt = 0;
}

imf_status imf_create(const imf_options *opt, imf_handle *out)
{
    if (!out) return IMF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!opt) return IMF_ERR_INVALID_ARG;
    if (opt->nx < 1 || opt->ny < 1 || opt->nz < 1) return IMF_ERR_INVALID_ARG;
    if ((long)opt->nx * opt->ny * opt->nz > (1L << 31) - 1) return IMF_ERR_INVALID_ARG;
    if (!(opt->lambda >= 0 && opt->lambda < 1) || !(opt->tau >= 0 && opt->tau <= 1) || !(opt->theta_rel >= 0) ||
        !(opt->voxel > 0))
        return IMF_ERR_INVALID_ARG;
    if (opt->precision < IMF_AUTO || opt->precision > IMF_BF16_DIRECT) return IMF_ERR_INVALID_ARG;
    if (opt->erode_groups < 0) return IMF_ERR_INVALID_ARG;
    if (opt->sharp_sampling < IMF_SHARP_ALL || opt->sharp_sampling > IMF_SHARP_NEAREST) return IMF_ERR_INVALID_ARG;
    if (opt->fft_wide_pencils < -1 || opt->fft_wide_pencils > 3) return IMF_ERR_INVALID_ARG;
    if (opt->fft_tma_x < -1 || opt->fft_tma_x > 1) return IMF_ERR_INVALID_ARG;
    if (opt->erode_xt != 0 && opt->erode_xt != 8 && opt->erode_xt != 16) return IMF_ERR_INVALID_ARG;
    if (opt->fft_tma < -1 || opt->fft_tma > 15 || (opt->fft_tma >= 0 && ((opt->fft_tma & 3) == 3 || (opt->fft_tma >> 2) == 3)))
        return IMF_ERR_INVALID_ARG;
    if (opt->sharp_sampling == IMF_SHARP_NEAREST && opt->sharp_k < 1) return IMF_ERR_INVALID_ARG;
    imf_handle h = new (std::nothrow) imf_handle_s();
    if (!h) return IMF_ERR_OOM;
    h->opt = *opt;
    *out = h;
    return IMF_OK;
}

imf_status imf_clone(imf_handle h, imf_handle *out)
{
    if (!out) return IMF_ERR_INVALID_ARG;
    *out = nullptr;
    if (!h) return IMF_ERR_INVALID_ARG;
    if (h->n_tools == 0) return fail(h, IMF_ERR_NOT_READY, "imf_clone before imf_set_tool");
    for (int i = 0; i < h->n_tools; ++i)
        if (h->tools[i].planned_only)
            return fail(h, IMF_ERR_INVALID_ARG, "a plan-only handle has no device tools to share");
    if (h->used_stream) CU(cudaStreamSynchronize(h->last_stream));
    imf_handle c = new (std::nothrow) imf_handle_s();
    if (!c) return IMF_ERR_OOM;
    if (!h->tool_refs) h->tool_refs = std::make_shared<int>(0);
    c->opt = h->opt;
    c->n_tools = h->n_tools;
    for (int i = 0; i < h->n_tools; ++i) c->tools[i] = h->tools[i];   // device pointers shared
    c->tool_refs = h->tool_refs;
    c->nsm = h->nsm;
    *out = c;
    return IMF_OK;
}

void imf_destroy(imf_handle h)
{
    if (!h) return;
    if (h->used_stream) cudaStreamSynchronize(h->last_stream);
    // tools shared with a clone stay for the handles that still hold them
    const bool last_owner = !h->tool_refs || h->tool_refs.use_count() == 1;
    if (last_owner)
        for (auto &t : h->tools) free_tool(h, t);
    h->tool_refs.reset();
    dfree(h, h->rho_spec, h->rho_spec_n);
    dfree(h, h->rhohl);
    dfree(h, h->X1, h->X1_n);
    dfree(h, h->X2, h->X2_n);
    dfree(h, h->Y1, h->Y1_n * h->slots);
    dfree(h, h->Y2, h->Y2_n * h->slots);
    dfree(h, h->g, h->g_n * h->slots);
    dfree(h, h->bits, h->bits_n * h->slots * kSweepLevels);
    dfree(h, h->f, 0);
    dfree(h, h->A, 0);
    dfree(h, h->flags, (size_t)h->flag_cap);
    dfree(h, h->dev_small, 8);
    dfree(h, h->plan_rem);
    dfree(h, h->plan_cnt);
    for (float **p : {&h->h_rho, &h->h_fbar, &h->h_raw}) dfree(h, *p, 0);
    for (uint8_t **p : {&h->h_fix, &h->h_sec, &h->h_acc}) dfree(h, *p, 0);
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    for (auto &r : h->prof_pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    delete h;
}

const char *imf_last_error(imf_handle h)
{
    if (!h) return "null handle";
    return h->err.c_str();
}

imf_status imf_set_tool(imf_handle h, int tool_id, const uint8_t *holder, const uint8_t *cutter,
                        const uint8_t *sharp_mask, int tx, int ty, int tz, const int origin[3], const double *quats,
                        int n_orient)
{
    if (!h) return IMF_ERR_INVALID_ARG;
    if (tool_id < 0 || tool_id >= 64 || tool_id > h->n_tools)
        return fail(h, IMF_ERR_INVALID_ARG, "tool_id %d: ids are set densely from 0 (have %d)", tool_id, h->n_tools);
    if (!holder || !cutter || !origin || !quats) return fail(h, IMF_ERR_INVALID_ARG, "NULL tool argument");
    if (tx < 1 || ty < 1 || tz < 1 || tx > 340 || ty > 340 || tz > 340)
        return fail(h, IMF_ERR_INVALID_ARG, "tool extents %dx%dx%d outside [1, 340]", tx, ty, tz);
    if (n_orient < 1 || n_orient > 4096) return fail(h, IMF_ERR_INVALID_ARG, "n_orient %d outside [1, 4096]", n_orient);
    const long tv = (long)tx * ty * tz;
    std::vector<uint8_t> T(tv), K(tv), S(tv);
    long nK = 0, nT = 0;
    for (long i = 0; i < tv; ++i) {
        K[i] = cutter[i] ? 1 : 0;
        T[i] = (holder[i] || cutter[i]) ? 1 : 0;
        S[i] = sharp_mask ? (uint8_t)(sharp_mask[i] && cutter[i]) : K[i];
        nK += K[i];
        nT += T[i];
    }
    if (nK == 0) return fail(h, IMF_ERR_INVALID_ARG, "empty cutter");
    if (!sharp_mask && h->opt.sharp_sampling != IMF_SHARP_ALL)
        sample_sharp_points(K, tx, ty, tz, origin, h->opt.sharp_sampling, h->opt.sharp_k, S);
    bool sharp_all = true;
    for (long i = 0; i < tv; ++i) sharp_all = sharp_all && S[i] == K[i];
    for (int i = 0; i < n_orient; ++i) {
        const double *q = quats + 4 * i;
        const double nn = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
        if (!(nn > 1e-300) || !std::isfinite(nn)) return fail(h, IMF_ERR_INVALID_ARG, "quaternion %d is zero or not finite", i);
    }
    if (h->tool_refs && h->tool_refs.use_count() > 1)
        return fail(h, IMF_ERR_INVALID_ARG, "the tools of this handle are shared with a clone (imf_clone)");
    if (h->used_stream) CU(cudaStreamSynchronize(h->last_stream));
    Tool &t = h->tools[tool_id];
    if (t.set) free_tool(h, t);
    t.tx = tx; t.ty = ty; t.tz = tz;
    t.o[0] = origin[0]; t.o[1] = origin[1]; t.o[2] = origin[2];
    t.n_orient = n_orient;
    t.size_T = nT;
    t.theta = h->opt.theta_rel * (double)nT;
    t.sharp_is_cutter = sharp_all;

    // --- orientation order: nearest-neighbour chain (groups of the direct path stay compact);
    // on the FFT path the chain is interleaved so that every orientation batch spreads over all
    // directions and design voxels reach f = 0 (which prunes the minimum) after fewer batches.
    // Results never depend on the order, only the grouping of device work does.
    std::vector<double> R(9 * (size_t)n_orient);
    for (int i = 0; i < n_orient; ++i) quat_to_R(quats + 4 * i, &R[9 * i]);
    t.perm = locality_order(R, n_orient);
    if (h->opt.precision == IMF_FP32_FFT) t.perm = spread_order(t.perm);
    t.iperm.assign(n_orient, 0);
    std::vector<double> qint(4 * (size_t)n_orient);
    for (int i = 0; i < n_orient; ++i) {
        t.iperm[t.perm[i]] = i;
        for (int c = 0; c < 4; ++c) qint[4 * i + c] = quats[4 * t.perm[i] + c];
    }
    quats = qint.data();

    // --- rotate and resample on the device (Alg. 1 Rotate)
    std::vector<int> box(6 * (size_t)n_orient);
    std::vector<long> boff(n_orient + 1, 0);
    long maxb = 0;
    for (int i = 0; i < n_orient; ++i) {
        quat_to_R(quats + 4 * i, &R[9 * i]);
        scan_box(&R[9 * i], tx, ty, tz, t.o, &box[6 * i]);
        const long v = (long)box[6 * i + 3] * box[6 * i + 4] * box[6 * i + 5];
        boff[i + 1] = boff[i] + v;
        maxb = std::max(maxb, v);
    }
    const long tot = boff[n_orient];
    uint8_t *dT = nullptr, *dK = nullptr, *dS = nullptr, *dout = nullptr;
    double *dR = nullptr;
    int *dbox = nullptr;
    long *dboff = nullptr;
    imf_status st = IMF_OK;
    std::vector<uint8_t> hout;
    const bool plan_only = h->opt.plan_only != 0;
    auto vbytes = [](size_t n, size_t e) { return std::max<size_t>(n, 1) * e; };
    const size_t rot_bytes = 3 * vbytes((size_t)tv, 1) + vbytes(R.size(), 8) + vbytes(box.size(), 4) +
                             vbytes(boff.size(), 8) + vbytes((size_t)tot * 3, 1);
    if (plan_only) {
        // resample on the host (same arithmetic as rotate_kernel); nothing touches the device
        hout.assign((size_t)tot * 3, 0);
        for (int i = 0; i < n_orient; ++i)
            rotate_host(T.data(), K.data(), S.data(), tx, ty, tz, t.o, &R[9 * i], &box[6 * i], hout.data() + boff[i],
                        hout.data() + tot + boff[i], hout.data() + 2 * tot + boff[i]);
    } else {
        auto cleanup = [&]() {
            dfree(h, dT, (size_t)tv); dfree(h, dK, (size_t)tv); dfree(h, dS, (size_t)tv);
            dfree(h, dout, (size_t)tot * 3); dfree(h, dR, R.size()); dfree(h, dbox, box.size());
            dfree(h, dboff, boff.size());
        };
        if ((st = upload(h, &dT, T)) || (st = upload(h, &dK, K)) || (st = upload(h, &dS, S)) ||
            (st = upload(h, &dR, R)) || (st = upload(h, &dbox, box)) || (st = upload(h, &dboff, boff)) ||
            (st = dalloc(h, &dout, (size_t)tot * 3))) {
            cleanup();
            return st;
        }
        RotateArgs a{};
        a.T = dT; a.K = dK; a.Sm = dS; a.tx = tx; a.ty = ty; a.tz = tz; a.ox = t.o[0]; a.oy = t.o[1]; a.oz = t.o[2];
        a.R = dR; a.box = dbox; a.box_off = dboff; a.outT = dout; a.outK = dout + tot; a.outS = dout + 2 * tot;
        a.n_orient = n_orient; a.max_box = maxb;
        {
            Launch L(h, KID_ROTATE, 0);
            launch_rotate(a, 0);
        }
        hout.resize((size_t)tot * 3);
        cudaError_t e = cudaMemcpy(hout.data(), dout, (size_t)tot * 3, cudaMemcpyDeviceToHost);
        cleanup();
        if (e != cudaSuccess) return fail(h, IMF_ERR_CUDA, "rotate: %s", cudaGetErrorString(e));
    }
    // --- offset lists, cutter row intervals
    t.rt.assign(n_orient, {});
    t.rk.assign(n_orient, {});
    t.sh.assign(n_orient, {});
    std::vector<std::vector<int32_t>> ivs(n_orient);
    int vlo[3] = {1 << 30, 1 << 30, 1 << 30}, vhi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
    std::vector<int> rvlo(3 * n_orient), rvhi(3 * n_orient);
    bool anyK = false;
    for (int k = 0; k < 3; ++k) { t.kmin[k] = 1 << 30; t.kmax[k] = -(1 << 30); }
    for (int i = 0; i < n_orient; ++i) {
        const int *b = &box[6 * i];
        const uint8_t *bT = hout.data() + boff[i], *bK = hout.data() + tot + boff[i], *bS = hout.data() + 2 * tot + boff[i];
        int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
        for (int z = 0; z < b[5]; ++z)
            for (int y = 0; y < b[4]; ++y) {
                int run = -1;
                for (int x = 0; x <= b[3]; ++x) {
                    const long id = ((long)z * b[4] + y) * b[3] + x;
                    const int v[3] = {b[0] + x, b[1] + y, b[2] + z};
                    const bool inK = x < b[3] && bK[id];
                    if (x < b[3] && bT[id]) {
                        t.rt[i].insert(t.rt[i].end(), v, v + 3);
                        for (int c = 0; c < 3; ++c) { lo[c] = std::min(lo[c], v[c]); hi[c] = std::max(hi[c], v[c]); }
                    }
                    if (inK) {
                        t.rk[i].insert(t.rk[i].end(), v, v + 3);
                        for (int c = 0; c < 3; ++c) { t.kmin[c] = std::min(t.kmin[c], v[c]); t.kmax[c] = std::max(t.kmax[c], v[c]); }
                        if (run < 0) run = x;
                    } else if (run >= 0) {
                        for (int r0 = run; r0 <= x - 1; r0 += 32)   // sweep runs of at most 32
                            ivs[i].insert(ivs[i].end(), {b[0] + r0, b[0] + std::min(x - 1, r0 + 31), b[1] + y, b[2] + z});
                        run = -1;
                    }
                    if (x < b[3] && bS[id]) t.sh[i].insert(t.sh[i].end(), v, v + 3);
                }
            }
        for (int c = 0; c < 3; ++c) { rvlo[3 * i + c] = lo[c]; rvhi[3 * i + c] = hi[c]; }
        if (!t.rk[i].empty()) anyK = true;
        for (int c = 0; c < 3; ++c) { vlo[c] = std::min(vlo[c], lo[c]); vhi[c] = std::max(vhi[c], hi[c]); }
    }
    if (!anyK) {
        free_tool(h, t);
        return fail(h, IMF_ERR_INVALID_ARG, "the cutter vanishes under every orientation");
    }
    // --- plan: padded sizes and the translation window
    const int n[3] = {h->opt.nx, h->opt.ny, h->opt.nz};
    int req[3];
    for (int c = 0; c < 3; ++c) {
        t.win[c] = n[c] + t.kmax[c] - t.kmin[c];
        int r = t.win[c];
        for (int i = 0; i < n_orient; ++i) {
            if (t.rk[i].empty()) continue;
            r = std::max(r, n[c] + std::max(t.kmax[c] - rvlo[3 * i + c], rvhi[3 * i + c] - t.kmin[c]));
        }
        req[c] = r;
        if (vlo[c] < -511 || vhi[c] > 511) {
            free_tool(h, t);
            return fail(h, IMF_ERR_INVALID_ARG, "rotated tool offsets exceed +-511 voxels");
        }
    }
    t.M = best_smooth((req[0] + 1) / 2, fft2::kMaxFactor);
    t.P[0] = 2 * t.M;
    t.P[1] = best_smooth(req[1], fft2::kMaxFactorBig);
    t.P[2] = best_smooth(req[2], fft2::kMaxFactorBig);
    t.Hx = t.M + 1;
    t.Hs = (t.Hx + 1) & ~1;
    t.gpx = (t.win[0] + 3) & ~3;
    t.wpr = (t.win[0] + 31) / 32 + 2;
    // two-pass splits where they exist; launches use them unless fft_stages_only is set (then
    // every pass runs radix stages), so the choice can change after planning
    if (!fft2::choose_split(t.M, &t.sM[0], &t.sM[1])) t.sM[0] = t.sM[1] = 0;
    if (!fft2::choose_split(t.P[1], &t.sy[0], &t.sy[1], fft2::kMaxFactorBig)) t.sy[0] = t.sy[1] = 0;
    if (!fft2::choose_split(t.P[2], &t.sz[0], &t.sz[1], fft2::kMaxFactorBig)) t.sz[0] = t.sz[1] = 0;
    if (!make_plan(t.M, &t.plM) || !make_plan(t.P[1], &t.ply) || !make_plan(t.P[2], &t.plz)) {
        free_tool(h, t);
        return fail(h, IMF_ERR_INVALID_ARG, "no FFT plan for %d x %d x %d", t.P[0], t.P[1], t.P[2]);
    }
    const double ptot = (double)t.P[0] * t.P[1] * t.P[2];
    const double band_auto = 4e-6 * (double)nT + 1e-3;
    t.band = h->opt.recheck_band > 0 ? h->opt.recheck_band : band_auto;
    // --- device tables
    std::vector<float2> tw;
    std::vector<uint32_t> rto;
    std::vector<int> rts(n_orient + 1, 0), ivst(n_orient + 1, 0);
    std::vector<int4> ivv;
    for (int i = 0; i < n_orient; ++i) {
        for (size_t m = 0; m < t.rt[i].size(); m += 3)
            rto.push_back((uint32_t)(t.rt[i][m] + 512) | ((uint32_t)(t.rt[i][m + 1] + 512) << 10) |
                          ((uint32_t)(t.rt[i][m + 2] + 512) << 20));
        rts[i + 1] = (int)rto.size();
        // cutter run [a, b] at (dy, dz): sliding OR of length L at shift s = kx - b >= 0 from
        // level j with 2^j <= L <= 2^(j+1) (runs are at most 32 long), windows s and s + L - 2^j
        for (size_t m = 0; m < ivs[i].size(); m += 4) {
            const int a0 = ivs[i][m], b0 = ivs[i][m + 1], dy = ivs[i][m + 2], dz = ivs[i][m + 3];
            const int L = b0 - a0 + 1, sa = t.kmax[0] - b0;
            const long row = (long)(t.kmax[2] - dz) * t.win[1] * t.wpr + (long)(t.kmax[1] - dy) * t.wpr;
            if (row + (sa >> 5) > 0x7fffffffL) {
                free_tool(h, t);
                return fail(h, IMF_ERR_INVALID_ARG, "translation window too large for the sweep descriptors");
            }
            ivv.push_back(sweep_pair(row, sa, L));
        }
        ivst[i + 1] = (int)ivv.size();
        t.n_sh += (long)t.sh[i].size() / 3;
    }
    t.n_rt = (long)rto.size();
    t.n_rk = 0;
    for (auto &v : t.rk) t.n_rk += (long)v.size() / 3;
    std::vector<ErodeChunk> chunks;
    std::vector<int2> eruns;
    std::vector<int> chst(n_orient + 1, 0);
    // the dyadic-level kernel (runs up to kErMaxL3) where every tile row fits its level build,
    // else the pairwise kernel (runs up to kErMaxL)
    t.erode_levels = h->opt.erode_levels != 0;
    for (int pass = 0; pass < 2; ++pass) {
        chunks.clear();
        eruns.clear();
        t.erode_smem = 0;
        for (int i = 0; i < n_orient; ++i) {
            plan_erode(t.sh[i], t.kmax, chunks, eruns, t.erode_smem, t.erode_levels ? kErMaxL3 : kErMaxL);
            chst[i + 1] = (int)chunks.size();
        }
        bool rows_fit = true;
        for (const ErodeChunk &c : chunks) rows_fit = rows_fit && c.txh <= kErMaxRow3;
        if (!t.erode_levels || rows_fit) break;
        t.erode_levels = false;
    }
    if (t.erode_smem > 227 * 1024) {
        free_tool(h, t);
        return fail(h, IMF_ERR_INVALID_ARG, "sharp-point set too wide for the tiled minimum (%zu bytes of tile)",
                    t.erode_smem);
    }
    if (!plan_only) {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
            h->nsm = n;
        t.erode_bps = t.erode_levels ? erode3_blocks_per_sm(t.erode_smem)
                                      : erode2_blocks_per_sm(t.erode_smem, erode_xt(h->opt));
    }
    st = IMF_OK;
    auto bail = [&](imf_status s2) { free_tool(h, t); return s2; };
    // resident tables: twiddles, offset lists, sweep and erosion descriptors (counted the same
    // way whether they are uploaded or only planned)
    t.table_bytes = vbytes((size_t)t.M, 8) + vbytes((size_t)t.M + 1, 8) + vbytes((size_t)t.P[1], 8) +
                    vbytes((size_t)t.P[2], 8) + vbytes(rto.size(), 4) + vbytes(rts.size(), 4) +
                    vbytes(ivv.size(), sizeof(int4)) + vbytes(ivst.size(), 4) +
                    vbytes(chunks.size(), sizeof(ErodeChunk)) + vbytes(chst.size(), 4) +
                    vbytes(eruns.size(), sizeof(int2)) + vbytes(t.perm.size(), 4);
    if (!plan_only) {
        twiddles(t.M, t.M, t.M, tw);
        if ((st = upload(h, &t.twM, tw))) return bail(st);
        twiddles(t.P[0], t.P[0], t.M + 1, tw);
        if ((st = upload(h, &t.twP, tw))) return bail(st);
        twiddles(t.P[1], t.P[1], t.P[1], tw);
        if ((st = upload(h, &t.twy, tw))) return bail(st);
        twiddles(t.P[2], t.P[2], t.P[2], tw);
        if ((st = upload(h, &t.twz, tw))) return bail(st);
        if ((st = upload(h, &t.rt_off, rto)) || (st = upload(h, &t.rt_start, rts)) ||
            (st = upload(h, &t.sw_pairs, ivv)) || (st = upload(h, &t.sw_start, ivst)) ||
            (st = upload(h, &t.er_chunks, chunks)) || (st = upload(h, &t.er_chunk_start, chst)) ||
            (st = upload(h, &t.er_runs, eruns)) || (st = upload(h, &t.perm_dev, t.perm)))
            return bail(st);
    }
    // --- direct tensor-core path: groups, union taps, B matrices
    const int prec = h->opt.precision;
    if (prec != IMF_FP32_FFT) {
        std::vector<int> taps;
        std::vector<uint16_t> bm;
        t.dir_ok = plan_direct(t, n, vlo, vhi, taps, bm);
        if (t.dir_ok) t.table_bytes += vbytes(taps.size(), 4) + vbytes(bm.size(), 2);
        if (t.dir_ok && !plan_only && ((st = upload(h, &t.d_taps, taps)) || (st = upload(h, &t.d_bmat, bm))))
            return bail(st);
    }
    if (prec == IMF_BF16_DIRECT && !t.dir_ok)
        return bail(fail(h, IMF_ERR_INVALID_ARG, "tool too large for the direct tensor-core path"));
    t.path = prec == IMF_BF16_DIRECT ? IMF_BF16_DIRECT : IMF_FP32_FFT;
    if (prec == IMF_BF16_DIRECT) {
        t.setup_bytes = std::max(rot_bytes, t.table_bytes);
        t.planned_only = plan_only;
        t.set = true;
        if (tool_id == h->n_tools) h->n_tools++;
        return IMF_OK;
    }

    // --- tool spectra: conj(FFT(1_RT)) / Ptot (reflection as conjugation, Alg. 1 footnote)
    const size_t per = (size_t)t.P[2] * t.P[1] * t.Hs;
    t.spec_bytes = per * n_orient * sizeof(float2);
    // transient buffers of the spectrum build: the dense padded tool and two intermediates
    t.setup_bytes = std::max(rot_bytes, t.table_bytes + t.spec_bytes + (size_t)t.P[0] * t.P[1] * t.P[2] * 4 +
                                            2 * per * sizeof(float2));
    if (plan_only) {
        t.planned_only = true;
        t.has_spec = true;
        t.set = true;
        if (tool_id == h->n_tools) h->n_tools++;
        return IMF_OK;
    }
    if ((st = dalloc(h, &t.spec, per * n_orient))) return bail(st);
    float *dense = nullptr;
    float2 *s1 = nullptr, *s2 = nullptr;
    const size_t dn = (size_t)t.P[0] * t.P[1] * t.P[2];
    if ((st = dalloc(h, &dense, dn)) || (st = dalloc(h, &s1, per)) || (st = dalloc(h, &s2, per))) {
        dfree(h, dense, dn); dfree(h, s1, per); dfree(h, s2, per);
        return bail(st);
    }
    for (int i = 0; i < n_orient && st == IMF_OK; ++i) {
        cudaMemsetAsync(dense, 0, dn * sizeof(float), 0);
        const int cnt = rts[i + 1] - rts[i];
        {
            Launch L(h, KID_SPEC, 0);
            if (cnt > 0) launch_scatter_tool(dense, t.P[0], t.P[1], t.P[2], t.rt_off + rts[i], cnt, t.kmax[0], t.kmax[1], t.kmax[2], 0);
        }
        st = forward_real_3d(h, t, dense, nullptr, t.P[0], t.P[1], t.P[2], s1, s2, t.spec + per * i, (float)(1.0 / ptot), 1, 0);
    }
    cudaError_t e = cudaDeviceSynchronize();
    dfree(h, dense, dn); dfree(h, s1, per); dfree(h, s2, per);
    if (st != IMF_OK) return bail(st);
    if (e != cudaSuccess) return bail(fail(h, IMF_ERR_CUDA, "tool spectrum: %s", cudaGetErrorString(e)));
    t.has_spec = true;
    t.set = true;
    if (tool_id == h->n_tools) h->n_tools++;
    return IMF_OK;
}

// near-threshold re-check, sweep and minimum over sharp points for one orientation batch
imf_status tail_batch(imf_handle h, const Tool &t, const float *rho, const uint8_t *fix, int o0, int nb, cudaStream_t s)
{
    const imf_options &op = h->opt;
    int *fcount = h->dev_small + 1;
    const long gso = (long)t.win[2] * t.win[1] * t.gpx;
    const long bso = (long)t.win[2] * t.win[1] * t.wpr;
    if (op.recheck) {
        RecheckArgs a{};
        a.flags = h->flags; a.count = fcount; a.cap = h->flag_cap; a.rho = rho; a.fix = fix;
        a.nx = op.nx; a.ny = op.ny; a.nz = op.nz; a.rt_off = t.rt_off; a.rt_start = t.rt_start;
        a.wx = t.win[0]; a.wy = t.win[1]; a.kx = t.kmax[0]; a.ky = t.kmax[1]; a.kz = t.kmax[2];
        a.g = h->g; a.g_sy = t.gpx; a.g_sz = (long)t.win[1] * t.gpx; a.g_so = gso;
        a.bits = h->bits; a.b_sy = t.wpr; a.b_sz = (long)t.win[1] * t.wpr; a.b_so = bso;
        a.theta = t.theta; a.orient_base = o0;
        Launch L(h, KID_RECHECK, s);
        launch_recheck_blocks(a, 152 * 64, s);     // up to 64 points (warps) in flight per SM
    }
    if (h->run_sweep) {
        const long lstride = (long)h->bits_n * h->slots;
        {
            SweepLevelsArgs a{};
            a.bits = h->bits; a.lstride = lstride; a.n = bso * nb; a.wpr = t.wpr;
            Launch L(h, KID_SWEEP_LEVELS, s);
            launch_sweep_levels(a, s);
        }
        SweepArgs a{};
        a.bits = h->bits; a.lstride = lstride; a.b_sy = t.wpr; a.b_sz = (long)t.win[1] * t.wpr; a.b_so = bso;
        a.pairs = t.sw_pairs; a.pair_start = t.sw_start; a.nx = op.nx; a.ny = op.ny; a.nz = op.nz;
        a.awords = h->awords; a.orient_base = o0; a.nb = nb; a.A = h->A;
        if (h->aset) {
            long base = 0;
            for (int i = 0; i < h->n_tools && &h->tools[i] != &t; ++i) base += h->tools[i].n_orient;
            a.A_per = h->aset + base * h->aset_so;
            a.a_per_so = h->aset_so;
            a.perm = t.perm_dev;
        }
        Launch L(h, KID_SWEEP, s);
        // per-orientation sets need every orientation's own sweep (no early exit); the loop form
        // (early exit per word) measured slower: 9.5 against 5.1 ms at 256^3 x 128
        if (h->opt.sweep_loop && !h->aset) launch_sweep_loop(a, h->nsm, s);
        else launch_sweep(a, s);
    }
    {
        Erode2Args a{};
        a.g = h->g; a.g_so = gso; a.gpx = t.gpx; a.gpy = t.win[1];
        a.wx = t.win[0]; a.wy = t.win[1]; a.wz = t.win[2];
        a.chunks = t.er_chunks; a.chunk_start = t.er_chunk_start; a.runs = t.er_runs;
        a.nx = op.nx; a.ny = op.ny; a.nz = op.nz; a.orient_base = o0; a.nb = nb; a.f = h->f;
        // (tile, orientation group) units: at least about twelve waves of resident blocks and
        // at most 16 orientations per block (measured optimum: 8 groups of 8 orientations at
        // 128^3 x 64, 4 groups of 16 at 256^3 with 64 orientations per launch)
        const long tiles = (long)((op.nx + kErTX - 1) / kErTX) * ((op.ny + kErTY - 1) / kErTY) *
                           ((op.nz + kErTZ - 1) / kErTZ);
        const long slots = (long)t.erode_bps * h->nsm;
        int G = op.erode_groups > 0 ? op.erode_groups
                                    : (int)std::max((12 * slots + tiles - 1) / tiles, (long)(nb + 15) / 16);
        a.ngroups = std::max(1, std::min(G, nb));
        Launch L(h, KID_ERODE, s);
        if (t.erode_levels) launch_erode3(a, t.erode_smem, s);
        else launch_erode2(a, t.erode_smem, erode_xt(h->opt), s);
    }
    h->last_batch_base = o0;
    h->last_batch_n = nb;
    return IMF_OK;
}

static imf_status compute_impl(imf_handle h, const float *rho, const uint8_t *fix, float *fbar, uint8_t *sec,
                               float *raw, uint8_t *acc, cudaStream_t s)
{
    const imf_options &op = h->opt;
    const long N = (long)op.nx * op.ny * op.nz;
    TRY(ensure_work(h));
    if (!h->f || !h->A || !h->dev_small || !h->flags || !h->Y1 || !h->Y2 || !h->g || !h->bits || !h->rho_spec ||
        !h->X1 || !h->X2 || h->slots < 1)
        return fail(h, IMF_ERR_OOM, "work buffers are not allocated");
    for (int ti = 0; ti < h->n_tools; ++ti)
        if (h->tools[ti].path == IMF_BF16_DIRECT && (!h->rhohl || h->slots < std::min(h->tools[ti].dG, h->tools[ti].n_orient)))
            return fail(h, IMF_ERR_OOM, "direct-path buffers are not allocated");
    h->last_stream = s;
    h->used_stream = true;
    int *status = h->dev_small, *fcount = h->dev_small + 1;
    unsigned *maxbits = (unsigned *)(h->dev_small + 2);
    {
        Launch L(h, KID_INIT, s);
        launch_fill_f32(h->f, INFINITY, N, s);
    }
    // the accessible output: from the minimum when that is exact (one tool, sharp points = the
    // whole cutter), else by the sweep; neither when the caller does not ask for it
    const bool acc_from_f = acc && !op.accessible_by_sweep && h->n_tools == 1 && h->tools[0].sharp_is_cutter;
    h->run_sweep = (acc && !acc_from_f) || h->aset != nullptr;
    if (h->run_sweep) CU(cudaMemsetAsync(h->A, 0, sizeof(uint32_t) * (size_t)op.nz * op.ny * h->awords, s));
    CU(cudaMemsetAsync(maxbits, 0, sizeof(unsigned), s));
    CU(cudaMemsetAsync(h->dev_small + 4, 0, sizeof(int), s));
    for (int ti = 0; ti < h->n_tools; ++ti) {
        const Tool &t = h->tools[ti];
        const long gso_ = (long)t.win[2] * t.win[1] * t.gpx;
        const long bso_ = (long)t.win[2] * t.win[1] * t.wpr;
        if (t.path == IMF_BF16_DIRECT) {
            {
                Launch L(h, KID_RHO_HL, s);
                launch_rho_hl(rho, fix, op.nx, op.ny, op.nz, t.dlo[0], t.dlo[1], t.dlo[2], t.dP[0], t.dP[1], t.dP[2],
                              h->rhohl, s);
            }
            for (size_t gi = 0; gi + 1 < t.grp_start.size(); ++gi) {
                const int o0 = t.grp_start[gi], nb = t.grp_start[gi + 1] - o0;
                if (op.recheck) CU(cudaMemsetAsync(fcount, 0, sizeof(int), s));
                {
                    DirectArgs a{};
                    a.rhohl = h->rhohl; a.PX = t.dP[0]; a.PY = t.dP[1]; a.PZ = t.dP[2];
                    a.lox = t.dlo[0]; a.loy = t.dlo[1]; a.loz = t.dlo[2];
                    a.tapoff = t.d_taps + t.grp_tap_off[gi]; a.kpad = t.grp_kpad[gi];
                    a.bmat = t.d_bmat + t.grp_b_off[gi]; a.N = t.grp_N[gi]; a.nb = nb;
                    const DirectGroup &gg = t.grp_geo[gi];
                    a.vlo[0] = gg.glo[0]; a.vlo[1] = gg.glo[1]; a.vlo[2] = gg.glo[2];
                    a.BX = gg.BX; a.BY = gg.BY; a.BZ = gg.BZ; a.sx = gg.sx;
                    a.nslab = gg.nslab;
                    for (int sl = 0; sl <= gg.nslab; ++sl) a.slab_c0[sl] = gg.c0[sl];
                    for (int sl = 0; sl < gg.nslab; ++sl) a.slab_z0[sl] = gg.z0[sl];
                    a.TY = t.dTY; a.TZ = t.dTZ;
                    a.wx = t.win[0]; a.wy = t.win[1]; a.wz = t.win[2];
                    a.kx = t.kmax[0]; a.ky = t.kmax[1]; a.kz = t.kmax[2];
                    a.ntx = (t.win[0] + 31) / 32; a.nty = (t.win[1] + t.dTY - 1) / t.dTY;
                    a.ntz = (t.win[2] + t.dTZ - 1) / t.dTZ;
                    a.g = h->g; a.g_sy = t.gpx; a.g_sz = (long)t.win[1] * t.gpx; a.g_so = gso_;
                    a.bits = h->bits; a.b_sy = t.wpr; a.b_sz = (long)t.win[1] * t.wpr; a.b_so = bso_;
                    a.theta = (float)t.theta; a.band = (float)t.band; a.flag = op.recheck;
                    a.flags = h->flags; a.flag_count = fcount; a.flag_total = h->dev_small + 4;
                    a.flag_cap = h->flag_cap; a.status = status; a.orient_base = o0;
                    Launch L(h, KID_DIRECT, s);
                    if (!launch_direct(a, h->nsm, s))
                        return fail(h, IMF_ERR_CUDA, "direct path: the rho_O box cannot be described by a tensor map");
                }
                TRY(tail_batch(h, t, rho, fix, o0, nb, s));
                h->last_tool = ti;
            }
            continue;
        }
        TRY(forward_real_3d(h, t, rho, fix, op.nx, op.ny, op.nz, h->X1, h->X2, h->rho_spec, 1.f, 0, s));
        const long y1so = (long)t.win[2] * t.P[1] * t.Hs;
        const long y2so = (long)t.win[2] * t.win[1] * t.Hs;
        const long gso = (long)t.win[2] * t.win[1] * t.gpx;
        const long bso = (long)t.win[2] * t.win[1] * t.wpr;
        const long spso = (long)t.P[2] * t.P[1] * t.Hs;
        for (int o0 = 0; o0 < t.n_orient; o0 += h->slots) {
            const int nb = std::min(h->slots, t.n_orient - o0);
            if (op.recheck) CU(cudaMemsetAsync(fcount, 0, sizeof(int), s));
            {
                AxisArgs a{};
                a.in = t.spec + spso * o0; a.in_so = spso; a.in_sb = t.Hs; a.in_sl = (long)t.P[1] * t.Hs;
                a.mul = h->rho_spec; a.mul_so = 0; a.mul_sb = t.Hs; a.mul_sl = (long)t.P[1] * t.Hs;
                a.out = h->Y1; a.out_so = y1so; a.out_sb = t.Hs; a.out_sl = (long)t.P[1] * t.Hs;
                a.nx = t.Hx; a.lin = t.P[2]; a.j0 = 0; a.lout = t.win[2]; a.scale = 1.f; a.tw = t.twz; a.plan = t.plz;
                set_split(h, a, t.sz); axis_opts(h, a);
                Launch L(h, KID_AXIS_INV_MUL, s);
                launch_axis_fft(1, a, t.P[1], nb, s);
            }
            AxisArgs ay{};
            ay.in = h->Y1; ay.in_so = y1so; ay.in_sb = (long)t.P[1] * t.Hs; ay.in_sl = t.Hs;
            ay.out = h->Y2; ay.out_so = y2so; ay.out_sb = (long)t.win[1] * t.Hs; ay.out_sl = t.Hs;
            ay.nx = t.Hx; ay.lin = t.P[1]; ay.j0 = 0; ay.lout = t.win[1]; ay.scale = 1.f; ay.tw = t.twy; ay.plan = t.ply;
            set_split(h, ay, t.sy); axis_opts(h, ay);
            IrfftArgs ax{};
            ax.in = h->Y2; ax.in_sy = t.Hs; ax.in_sz = (long)t.win[1] * t.Hs; ax.in_so = y2so;
            ax.rows_y = t.win[1]; ax.rows = t.win[1] * t.win[2]; ax.nout = t.win[0];
            ax.g = h->g; ax.g_sy = t.gpx; ax.g_sz = (long)t.win[1] * t.gpx; ax.g_so = gso;
            ax.bits = h->bits; ax.b_sy = t.wpr; ax.b_sz = (long)t.win[1] * t.wpr; ax.b_so = bso;
            ax.theta = (float)t.theta; ax.band = (float)t.band; ax.flag = op.recheck;
            ax.flags = h->flags; ax.flag_count = fcount; ax.flag_total = h->dev_small + 4; ax.flag_cap = h->flag_cap;
            ax.status = status;
            ax.orient_base = o0; ax.M = t.M; ax.twM = t.twM; ax.twP = t.twP; ax.plan = t.plM;
            set_split(h, ax, t.sM);
            ax.write_bits = h->run_sweep || h->keep_g;
            if (!op.separate_yx_passes && yx2_fits(ay, ax, t.Hs)) {
                Launch L(h, KID_YX, s);
                launch_yx2_threshold(ay, ax, t.Hs, t.win[2], nb, s);
            } else {
                {
                    Launch L(h, KID_AXIS_INV, s);
                    launch_axis_fft(1, ay, t.win[2], nb, s);
                }
                Launch L(h, KID_IRFFT_THRESH, s);
                const int tx = h->opt.fft_tma_x < 0 ? 1 : h->opt.fft_tma_x;
                if (!(tx && launch_irfft2_tma(ax, t.Hs, nb, s))) launch_irfft_threshold(ax, nb, s);
            }
            TRY(tail_batch(h, t, rho, fix, o0, nb, s));
            h->last_batch_base = o0;
            h->last_batch_n = nb;
            h->last_tool = ti;
        }
    }
    {
        Launch L(h, KID_MAX, s);
        launch_max_omega0(h->f, fix, N, maxbits, s);
    }
    {
        FinalizeArgs a{};
        a.f = h->f; a.rho = rho; a.fix = fix; a.A = h->A; a.nx = op.nx; a.ny = op.ny; a.nz = op.nz;
        a.awords = h->awords; a.maxbits = maxbits; a.lambda = op.lambda; a.tau = op.tau;
        a.fbar = fbar; a.secluded = sec; a.raw = raw; a.acc = acc;
        a.acc_from_f = acc_from_f; a.theta = (float)h->tools[0].theta;
        Launch L(h, KID_FINALIZE, s);
        launch_finalize(a, s);
    }
    CU(cudaGetLastError());
    h->computes++;
    return IMF_OK;
}

imf_status imf_compute(imf_handle h, const float *rho_omega, const uint8_t *fixture, float *imf_bar,
                       uint8_t *secluded, float *imf_raw, uint8_t *accessible, void *cuda_stream)
{
    if (!h) return IMF_ERR_INVALID_ARG;
    if (h->n_tools == 0) return fail(h, IMF_ERR_NOT_READY, "imf_compute before imf_set_tool");
    for (int i = 0; i < h->n_tools; ++i) {
        if (!h->tools[i].set) return fail(h, IMF_ERR_NOT_READY, "tool %d not set", i);
        if (h->tools[i].planned_only)
            return fail(h, IMF_ERR_NOT_READY, "tool %d was planned only (plan_only handle): nothing on the device", i);
    }
    if (!rho_omega || !imf_bar || !secluded) return fail(h, IMF_ERR_INVALID_ARG, "NULL required array");
    return compute_impl(h, rho_omega, fixture, imf_bar, secluded, imf_raw, accessible, (cudaStream_t)cuda_stream);
}

imf_status imf_compute_host(imf_handle h, const float *rho_omega, const uint8_t *fixture, float *imf_bar,
                            uint8_t *secluded, float *imf_raw, uint8_t *accessible, void *cuda_stream)
{
    if (!h) return IMF_ERR_INVALID_ARG;
    if (!rho_omega || !imf_bar || !secluded) return fail(h, IMF_ERR_INVALID_ARG, "NULL required array");
    const size_t N = (size_t)h->opt.nx * h->opt.ny * h->opt.nz;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!h->h_rho) {
        TRY(dalloc(h, &h->h_rho, N)); TRY(dalloc(h, &h->h_fbar, N)); TRY(dalloc(h, &h->h_raw, N));
        TRY(dalloc(h, &h->h_fix, N)); TRY(dalloc(h, &h->h_sec, N)); TRY(dalloc(h, &h->h_acc, N));
    }
    CU(cudaMemcpyAsync(h->h_rho, rho_omega, N * sizeof(float), cudaMemcpyHostToDevice, s));
    if (fixture) CU(cudaMemcpyAsync(h->h_fix, fixture, N, cudaMemcpyHostToDevice, s));
    TRY(imf_compute(h, h->h_rho, fixture ? h->h_fix : nullptr, h->h_fbar, h->h_sec, imf_raw ? h->h_raw : nullptr,
                    accessible ? h->h_acc : nullptr, cuda_stream));
    CU(cudaMemcpyAsync(imf_bar, h->h_fbar, N * sizeof(float), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(secluded, h->h_sec, N, cudaMemcpyDeviceToHost, s));
    if (imf_raw) CU(cudaMemcpyAsync(imf_raw, h->h_raw, N * sizeof(float), cudaMemcpyDeviceToHost, s));
    if (accessible) CU(cudaMemcpyAsync(accessible, h->h_acc, N, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return IMF_OK;
}

imf_status imf_penalize_sensitivity(imf_handle h, float *sens, const float *rho_omega, const float *imf_bar,
                                    const uint8_t *secluded, const uint8_t *fixture, double w_acc, void *cuda_stream)
{
    if (!h) return IMF_ERR_INVALID_ARG;
    if (!sens || !rho_omega || !imf_bar || !secluded) return fail(h, IMF_ERR_INVALID_ARG, "NULL required array");
    if (!(w_acc >= 0.0 && w_acc < 1.0)) return fail(h, IMF_ERR_INVALID_ARG, "w_acc %g outside [0, 1)", w_acc);
    const long N = (long)h->opt.nx * h->opt.ny * h->opt.nz;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!h->dev_small) {
        TRY(dalloc(h, &h->dev_small, (size_t)8));
        CU(cudaMemset(h->dev_small, 0, 8 * sizeof(int)));
    }
    unsigned *mb = (unsigned *)(h->dev_small + 3);
    h->last_stream = s;
    h->used_stream = true;
    CU(cudaMemsetAsync(mb, 0, sizeof(unsigned), s));
    {
        Launch L(h, KID_ABSMAX, s);
        launch_absmax_omega0(sens, fixture, N, mb, s);
    }
    {
        Launch L(h, KID_PENALIZE, s);
        launch_penalize(sens, rho_omega, imf_bar, secluded, N, mb, w_acc, h->opt.tau, s);
    }
    CU(cudaGetLastError());
    return IMF_OK;
}

imf_status imf_compute_accessible_sets(imf_handle h, const float *rho_omega, const uint8_t *fixture, float *imf_bar,
                                       uint8_t *secluded, uint32_t *sets, void *cuda_stream)
{
    if (!h) return IMF_ERR_INVALID_ARG;
    if (!sets) return fail(h, IMF_ERR_INVALID_ARG, "NULL sets");
    const long words = (long)h->opt.nz * h->opt.ny * ((h->opt.nx + 31) / 32);
    long n = 0;
    for (int i = 0; i < h->n_tools; ++i) n += h->tools[i].n_orient;
    h->aset = sets;
    h->aset_so = words;
    // every word of every set is written by the sweep; clearing first keeps orientations whose
    // cutter vanishes (no runs) empty
    cudaError_t e = cudaMemsetAsync(sets, 0, (size_t)std::max<long>(n, 1) * words * sizeof(uint32_t),
                                    (cudaStream_t)cuda_stream);
    imf_status st = e == cudaSuccess ? imf_compute(h, rho_omega, fixture, imf_bar, secluded, nullptr, nullptr, cuda_stream)
                                     : fail(h, IMF_ERR_CUDA, "clearing the sets: %s", cudaGetErrorString(e));
    h->aset = nullptr;
    h->aset_so = 0;
    return st;
}

imf_status imf_process_plan(imf_handle h, const uint32_t *sets, int n_sets, const float *rho_omega,
                            const uint8_t *fixture, int max_steps, int *order, long long *removed, int *n_steps,
                            long long *negative, long long *left, void *cuda_stream)
{
    if (!h) return IMF_ERR_INVALID_ARG;
    if (!sets || !rho_omega || !order || !removed || !n_steps) return fail(h, IMF_ERR_INVALID_ARG, "NULL argument");
    if (n_sets < 1 || max_steps < 0) return fail(h, IMF_ERR_INVALID_ARG, "n_sets %d / max_steps %d", n_sets, max_steps);
    const imf_options &op = h->opt;
    const long awords = (op.nx + 31) / 32;
    const long words = (long)op.nz * op.ny * awords;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if ((size_t)words > h->plan_rem_n) {
        dfree(h, h->plan_rem);
        h->plan_rem_n = 0;
        TRY(dalloc(h, &h->plan_rem, (size_t)words));
        h->plan_rem_n = (size_t)words;
    }
    if ((size_t)n_sets + 1 > h->plan_cnt_n) {
        dfree(h, h->plan_cnt);
        h->plan_cnt_n = 0;
        TRY(dalloc(h, &h->plan_cnt, (size_t)n_sets + 1));
        h->plan_cnt_n = (size_t)n_sets + 1;
    }
    h->last_stream = s;
    h->used_stream = true;
    {
        Launch L(h, KID_PLAN, s);
        launch_plan_init(rho_omega, fixture, op.nx, op.ny, op.nz, (int)awords, op.tau, h->plan_rem, s);
    }
    std::vector<unsigned long long> cnt(n_sets);
    auto counts = [&]() -> imf_status {
        CU(cudaMemsetAsync(h->plan_cnt, 0, sizeof(unsigned long long) * n_sets, s));
        {
            Launch L(h, KID_PLAN, s);
            launch_plan_count(sets, words, n_sets, h->plan_rem, h->plan_cnt, s);
        }
        CU(cudaMemcpyAsync(cnt.data(), h->plan_cnt, sizeof(unsigned long long) * n_sets, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        return IMF_OK;
    };
    // size of the negative space: popcount(remaining & remaining), in the counter after the sets'
    unsigned long long total = 0;
    CU(cudaMemsetAsync(h->plan_cnt + n_sets, 0, sizeof total, s));
    {
        Launch L(h, KID_PLAN, s);
        launch_plan_count(h->plan_rem, words, 1, h->plan_rem, h->plan_cnt + n_sets, s);
    }
    CU(cudaMemcpyAsync(&total, h->plan_cnt + n_sets, sizeof total, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    unsigned long long rest = total;
    int k = 0;
    while (k < max_steps && rest > 0) {
        TRY(counts());
        int best = 0;
        for (int i = 1; i < n_sets; ++i)
            if (cnt[i] > cnt[best]) best = i;
        if (cnt[best] == 0) break;
        order[k] = best;
        removed[k] = (long long)cnt[best];
        rest -= cnt[best];
        ++k;
        Launch L(h, KID_PLAN, s);
        launch_plan_remove(sets + (long)best * words, words, h->plan_rem, s);
    }
    CU(cudaStreamSynchronize(s));
    *n_steps = k;
    if (negative) *negative = (long long)total;
    if (left) *left = (long long)rest;
    return IMF_OK;
}

imf_status imf_capture_graph(imf_handle h, const float *rho_omega, const uint8_t *fixture, float *imf_bar,
                             uint8_t *secluded, float *imf_raw, uint8_t *accessible, void *cuda_stream)
{
    if (!h) return IMF_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!s) return fail(h, IMF_ERR_INVALID_ARG, "graph capture needs a non-default stream");
    TRY(imf_compute(h, rho_omega, fixture, imf_bar, secluded, imf_raw, accessible, cuda_stream));
    CU(cudaStreamSynchronize(s));
    if (h->graph_exec) { cudaGraphExecDestroy(h->graph_exec); h->graph_exec = nullptr; }
    if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
    const bool prof = h->prof;
    h->prof = false;
    CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const long launches = h->launches;
    imf_status st = compute_impl(h, rho_omega, fixture, imf_bar, secluded, imf_raw, accessible, s);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    h->prof = prof;
    h->launches = launches;
    h->computes--;
    if (st != IMF_OK) { if (g) cudaGraphDestroy(g); return st; }
    if (e != cudaSuccess) return fail(h, IMF_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    h->graph = g;
    CU(cudaGraphInstantiate(&h->graph_exec, g, 0));
    return IMF_OK;
}

imf_status imf_launch_graph(imf_handle h, void *cuda_stream)
{
    if (!h) return IMF_ERR_INVALID_ARG;
    if (!h->graph_exec) return fail(h, IMF_ERR_NOT_READY, "no captured graph");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    CU(cudaGraphLaunch(h->graph_exec, s));
    h->last_stream = s;
    h->used_stream = true;
    h->computes++;
    return IMF_OK;
}

imf_status imf_autotune(imf_handle h, const float *rho_omega, const uint8_t *fixture, float *imf_bar,
                        uint8_t *secluded, void *cuda_stream, int *best)
{
    if (!h) return IMF_ERR_INVALID_ARG;
    if (h->n_tools == 0) return fail(h, IMF_ERR_NOT_READY, "imf_autotune before imf_set_tool");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int maxo = 1;
    for (int i = 0; i < h->n_tools; ++i) maxo = std::max(maxo, h->tools[i].n_orient);
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    int best_nb = h->opt.orient_batch > 0 ? h->opt.orient_batch : 64;
    const int cands[6] = {4, 8, 16, 32, 64, 128};
    imf_status st = IMF_OK;
    for (int c = 0; c < 6 && st == IMF_OK; ++c) {
        const int nb = cands[c];
        if (nb > 4 && nb / 2 >= maxo) break;      // larger batches change nothing
        h->opt.orient_batch = nb;
        st = imf_compute(h, rho_omega, fixture, imf_bar, secluded, nullptr, nullptr, cuda_stream);
        if (st == IMF_ERR_BUDGET || st == IMF_ERR_OOM) { st = IMF_OK; cudaGetLastError(); break; }
        if (st != IMF_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < 2 && st == IMF_OK; ++r)
            st = imf_compute(h, rho_omega, fixture, imf_bar, secluded, nullptr, nullptr, cuda_stream);
        cudaEventRecord(e1, s);
        const cudaError_t es = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (es != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return fail(h, IMF_ERR_CUDA, "autotune: %s", cudaGetErrorString(es != cudaSuccess ? es : cudaGetLastError()));
        }
        if (st == IMF_OK && ms < best_ms) { best_ms = ms; best_nb = nb; }
    }
    if (st != IMF_OK) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return st;
    }
    h->opt.orient_batch = best_nb;
    TRY(ensure_work(h));
    // launch forms of the FFT passes and the work units of the minimum over sharp points:
    // coordinate descent from the current options, every candidate timed like the batches above
    // (same results whatever is chosen: each knob selects among equivalent kernels)
    auto time_now = [&](float *ms) -> imf_status {
        imf_status s1 = imf_compute(h, rho_omega, fixture, imf_bar, secluded, nullptr, nullptr, cuda_stream);
        if (s1 != IMF_OK) return s1;
        cudaEventRecord(e0, s);
        for (int r = 0; r < 2 && s1 == IMF_OK; ++r)
            s1 = imf_compute(h, rho_omega, fixture, imf_bar, secluded, nullptr, nullptr, cuda_stream);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
            return fail(h, IMF_ERR_CUDA, "autotune: %s", cudaGetErrorString(cudaGetLastError()));
        return s1;
    };
    {
        struct Knob {
            int *field;
            std::vector<int> values;
        };
        const Knob knobs[6] = {{&h->opt.fft_stages_only, {0, 1}},
                               {&h->opt.fft_tma, {-1, 1, 0, 10}},
                               {&h->opt.fft_wide_pencils, {-1, 0}},
                               {&h->opt.fft_tma_x, {-1, 0}},
                               {&h->opt.erode_groups, {0, 2, 4, 8, 16}},
                               {&h->opt.erode_xt, {0, 8}}};
        float cur = 1e30f;
        st = time_now(&cur);
        for (int k = 0; k < 6 && st == IMF_OK; ++k) {
            const int keep = *knobs[k].field;
            int best_v = keep;
            for (int v : knobs[k].values) {
                if (v == keep) continue;
                *knobs[k].field = v;
                float ms = 1e30f;
                st = time_now(&ms);
                if (st != IMF_OK) break;
                if (ms < 0.97f * cur) { cur = ms; best_v = v; }
            }
            *knobs[k].field = best_v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != IMF_OK) return st;
    // collision path: time the direct tensor-core path against the FFT path where both exist
    for (int ti = 0; ti < h->n_tools; ++ti) {
        Tool &t = h->tools[ti];
        if (!(t.dir_ok && t.has_spec) || h->opt.precision != IMF_AUTO) continue;
        float ms[2] = {1e30f, 1e30f};
        const int paths[2] = {IMF_FP32_FFT, IMF_BF16_DIRECT};
        for (int p = 0; p < 2; ++p) {
            t.path = paths[p];
            imf_status s2 = imf_compute(h, rho_omega, fixture, imf_bar, secluded, nullptr, nullptr, cuda_stream);
            if (s2 != IMF_OK) continue;
            cudaEvent_t a0, a1;
            cudaEventCreate(&a0);
            cudaEventCreate(&a1);
            cudaEventRecord(a0, s);
            s2 = imf_compute(h, rho_omega, fixture, imf_bar, secluded, nullptr, nullptr, cuda_stream);
            cudaEventRecord(a1, s);
            if (cudaEventSynchronize(a1) == cudaSuccess && s2 == IMF_OK) cudaEventElapsedTime(&ms[p], a0, a1);
            cudaEventDestroy(a0);
            cudaEventDestroy(a1);
        }
        t.path = ms[1] < ms[0] ? IMF_BF16_DIRECT : IMF_FP32_FFT;
        TRY(ensure_work(h));
    }
    if (h->graph_exec) { cudaGraphExecDestroy(h->graph_exec); h->graph_exec = nullptr; }
    if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
    if (best) *best = best_nb;
    return IMF_OK;
}

imf_status imf_set_path(imf_handle h, int tool_id, int path)
{
    if (!h || tool_id < 0 || tool_id >= h->n_tools || !h->tools[tool_id].set) return IMF_ERR_INVALID_ARG;
    Tool &t = h->tools[tool_id];
    if (path == IMF_BF16_DIRECT && !t.dir_ok)
        return fail(h, IMF_ERR_INVALID_ARG, "the direct path is not available for tool %d", tool_id);
    if (path == IMF_FP32_FFT && !t.has_spec)
        return fail(h, IMF_ERR_INVALID_ARG, "no FFT spectra for tool %d (created with IMF_BF16_DIRECT)", tool_id);
    if (path != IMF_BF16_DIRECT && path != IMF_FP32_FFT) return IMF_ERR_INVALID_ARG;
    if (h->used_stream) CU(cudaStreamSynchronize(h->last_stream));
    t.path = path;
    if (h->graph_exec) { cudaGraphExecDestroy(h->graph_exec); h->graph_exec = nullptr; }
    if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
    return IMF_OK;
}

imf_status imf_selftest_mma(int N, int K, const uint16_t *A, const uint16_t *B, float *D)
{
    if (!A || !B || !D) return IMF_ERR_INVALID_ARG;
    // the shapes the self-test kernel takes (checked again by its launcher), before any allocation
    if (N < 16 || N > 256 || N % 16 || K < 16 || K % 16 || (128L + N) * K * 2 + 64 > 200L * 1024)
        return IMF_ERR_INVALID_ARG;
    uint16_t *dA = nullptr, *dB = nullptr;
    float *dD = nullptr;
    int *dst = nullptr;
    int hst = 0;
    imf_status st = IMF_OK;
    if (cudaMalloc(&dA, (size_t)128 * K * 2) != cudaSuccess || cudaMalloc(&dB, (size_t)N * K * 2) != cudaSuccess ||
        cudaMalloc(&dD, (size_t)128 * N * 4) != cudaSuccess || cudaMalloc(&dst, sizeof(int)) != cudaSuccess) {
        st = IMF_ERR_OOM;
    } else {
        cudaMemcpy(dA, A, (size_t)128 * K * 2, cudaMemcpyHostToDevice);
        cudaMemcpy(dB, B, (size_t)N * K * 2, cudaMemcpyHostToDevice);
        cudaMemset(dst, 0, sizeof(int));
        if (run_mma_selftest(dA, dB, dD, N, K, dst, 0) != 0) st = IMF_ERR_INVALID_ARG;
        else if (cudaDeviceSynchronize() != cudaSuccess) st = IMF_ERR_CUDA;
        else {
            cudaMemcpy(D, dD, (size_t)128 * N * 4, cudaMemcpyDeviceToHost);
            cudaMemcpy(&hst, dst, sizeof(int), cudaMemcpyDeviceToHost);
            if (hst) st = (imf_status)hst;
        }
    }
    cudaFree(dA); cudaFree(dB); cudaFree(dD); cudaFree(dst);
    return st;
}

imf_status imf_sync_status(imf_handle h)
{
    if (!h) return IMF_ERR_INVALID_ARG;
    if (h->used_stream) CU(cudaStreamSynchronize(h->last_stream));
    CU(cudaGetLastError());
    if (!h->dev_small) return IMF_OK;
    int st[5] = {0, 0, 0, 0, 0};
    CU(cudaMemcpy(st, h->dev_small, sizeof st, cudaMemcpyDeviceToHost));
    h->flagged_last = st[4];
    h->flagged_total += st[4];
    if (st[0] != 0) {
        int z = 0;
        CU(cudaMemcpy(h->dev_small, &z, sizeof z, cudaMemcpyHostToDevice));
        return fail(h, (imf_status)st[0], "device status %d (near-threshold list capacity %d)", st[0], h->flag_cap);
    }
    return IMF_OK;
}

imf_status imf_get_tool_info(imf_handle h, int tool_id, imf_tool_info *out)
{
    if (!h || !out || tool_id < 0 || tool_id >= h->n_tools || !h->tools[tool_id].set) return IMF_ERR_INVALID_ARG;
    const Tool &t = h->tools[tool_id];
    out->n_orient = t.n_orient;
    for (int c = 0; c < 3; ++c) { out->P[c] = t.P[c]; out->kmax[c] = t.kmax[c]; out->win[c] = t.win[c]; }
    out->size_T = t.size_T;
    out->theta = t.theta;
    out->band = t.band;
    out->n_rt = t.n_rt;
    out->n_rk = t.n_rk;
    out->n_sharp = t.n_sh;
    out->path = t.path;
    out->spectra_bytes = t.spec_bytes;
    return IMF_OK;
}

imf_status imf_get_offsets(imf_handle h, int tool_id, int orient, int which, int32_t *out, long cap, long *n)
{
    if (!h || !n || tool_id < 0 || tool_id >= h->n_tools || !h->tools[tool_id].set) return IMF_ERR_INVALID_ARG;
    const Tool &t = h->tools[tool_id];
    if (orient < 0 || orient >= t.n_orient || which < 0 || which > 2) return IMF_ERR_INVALID_ARG;
    const int io = t.iperm[orient];
    const std::vector<int32_t> &v = which == 0 ? t.rt[io] : which == 1 ? t.rk[io] : t.sh[io];
    *n = (long)v.size() / 3;
    if (out) {
        if (cap < *n) return fail(h, IMF_ERR_INVALID_ARG, "capacity %ld < %ld", cap, *n);
        std::memcpy(out, v.data(), v.size() * sizeof(int32_t));
    }
    return IMF_OK;
}

imf_status imf_set_debug(imf_handle h, int keep_last_g)
{
    if (!h) return IMF_ERR_INVALID_ARG;
    h->keep_g = keep_last_g != 0;
    return IMF_OK;
}

imf_status imf_get_last_g(imf_handle h, int slot, float *g_out, long cap, int *orient_out)
{
    if (!h || h->last_tool < 0 || slot < 0 || slot >= h->last_batch_n) return IMF_ERR_INVALID_ARG;
    const Tool &t = h->tools[h->last_tool];
    const long n = (long)t.win[2] * t.win[1] * t.gpx;
    if (orient_out) *orient_out = t.perm[h->last_batch_base + slot];
    if (!g_out) return IMF_OK;
    if (cap < n) return fail(h, IMF_ERR_INVALID_ARG, "capacity %ld < %ld", cap, n);
    if (h->used_stream) CU(cudaStreamSynchronize(h->last_stream));
    CU(cudaMemcpy(g_out, h->g + (size_t)slot * h->g_n, n * sizeof(float), cudaMemcpyDeviceToHost));
    return IMF_OK;
}

imf_status imf_get_last_bits(imf_handle h, int slot, uint32_t *bits_out, long cap, int *orient_out)
{
    if (!h || h->last_tool < 0 || slot < 0 || slot >= h->last_batch_n) return IMF_ERR_INVALID_ARG;
    if (!h->keep_g && !h->run_sweep)
        return fail(h, IMF_ERR_NOT_READY, "free bits are kept only with imf_set_debug or on the sweep route");
    const Tool &t = h->tools[h->last_tool];
    const long n = (long)t.win[2] * t.win[1] * t.wpr;
    if (orient_out) *orient_out = t.perm[h->last_batch_base + slot];
    if (!bits_out) return IMF_OK;
    if (cap < n) return fail(h, IMF_ERR_INVALID_ARG, "capacity %ld < %ld", cap, n);
    if (h->used_stream) CU(cudaStreamSynchronize(h->last_stream));
    CU(cudaMemcpy(bits_out, h->bits + (size_t)slot * h->bits_n, n * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    return IMF_OK;
}

imf_status imf_get_options(imf_handle h, imf_options *out)
{
    if (!h || !out) return IMF_ERR_INVALID_ARG;
    *out = h->opt;
    return IMF_OK;
}

imf_status imf_get_stats(imf_handle h, imf_stats *out)
{
    if (!h || !out) return IMF_ERR_INVALID_ARG;
    out->launches = h->launches;
    out->computes = h->computes;
    out->flagged = h->flagged_last;
    out->flagged_total = h->flagged_total;
    out->n_kernels = KID_COUNT;
    out->owned_bytes = h->owned_bytes;
    return IMF_OK;
}

imf_status imf_footprint(imf_handle h, int slots, imf_footprint_info *out)
{
    if (!h || !out) return IMF_ERR_INVALID_ARG;
    if (h->n_tools == 0) return fail(h, IMF_ERR_NOT_READY, "imf_footprint before imf_set_tool");
    if (slots < 0) return fail(h, IMF_ERR_INVALID_ARG, "slots %d < 0", slots);
    const WorkSizes ws = work_sizes(h);
    const int s = slots > 0 ? std::max(slots, ws.min_slots) : default_slots(h, ws);
    size_t resident = 0, peak = 0;
    for (int i = 0; i < h->n_tools; ++i) {
        const Tool &t = h->tools[i];
        peak = std::max(peak, resident + t.setup_bytes);
        resident += t.spec_bytes + t.table_bytes;
    }
    out->resident = resident;
    out->work = work_bytes(h, ws, s);
    out->setup_peak = peak;
    out->total = std::max(resident + out->work, peak);
    out->slots = s;
    return IMF_OK;
}

imf_status imf_set_profiling(imf_handle h, int on)
{
    if (!h) return IMF_ERR_INVALID_ARG;
    h->prof = on != 0;
    return IMF_OK;
}

imf_status imf_get_kernel_time(imf_handle h, int i, const char **name, double *total_ms, long *count)
{
    if (!h || i < 0 || i >= KID_COUNT) return IMF_ERR_INVALID_ARG;
    drain_profile(h);
    if (name) *name = kKernelNames[i];
    if (total_ms) *total_ms = h->prof_ms[i];
    if (count) *count = h->prof_cnt[i];
    return IMF_OK;
}

imf_status imf_reset_kernel_times(imf_handle h)
{
    if (!h) return IMF_ERR_INVALID_ARG;
    drain_profile(h);
    for (int i = 0; i < KID_COUNT; ++i) { h->prof_ms[i] = 0; h->prof_cnt[i] = 0; }
    return IMF_OK;
}

} // extern "C"
