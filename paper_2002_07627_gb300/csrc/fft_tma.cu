// Host side of the TMA-fed persistent axis pass (fft_tma.cuh): tensor maps and the choice of
// the instance (compiled from fft_tma_inst.cu).
#include <algorithm>

#include "fft_tma.cuh"

namespace imf {
namespace tma_fft {

namespace {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda)
using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn()
{
    static EncodeFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// Tensor of complex64 elements (8-byte units) in memory order: kx (extent nx, contiguous),
// rows (stride rs), planes (stride ps), orientations (stride os; rank 4 only); box W kx x 1 row
// x box_j planes (axis_is_plane) or W x box_j rows x 1 plane, one orientation. Strides are in
// elements.
bool encode(CUtensorMap *m, const void *ptr, int rank, int nx, long rows, long rs, long planes, long ps, long norient,
            long os, int W, int box_j, bool axis_is_plane)
{
    EncodeFn fn = encode_fn();
    if (!fn) return false;
    if (reinterpret_cast<uint64_t>(ptr) & 15) return false;
    cuuint64_t dim[4] = {(cuuint64_t)nx, (cuuint64_t)rows, (cuuint64_t)planes, (cuuint64_t)norient};
    cuuint64_t stride[3] = {(cuuint64_t)rs * 8, (cuuint64_t)ps * 8, (cuuint64_t)os * 8};
    for (int i = 0; i < rank - 1; ++i)
        if (stride[i] == 0 || stride[i] % 16 || stride[i] >= (1ull << 40)) return false;
    cuuint32_t box[4] = {(cuuint32_t)W, axis_is_plane ? 1u : (cuuint32_t)box_j, axis_is_plane ? (cuuint32_t)box_j : 1u,
                         1u};
    cuuint32_t es[4] = {1, 1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, (cuuint32_t)rank, const_cast<void *>(ptr), dim, stride, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

} // namespace

namespace {

bool encode_tiled_es(CUtensorMap *m, const void *ptr, int rank, const uint64_t *dims, const uint64_t *strides_bytes,
                     const uint32_t *box, int es_bytes, CUtensorMapDataType dt)
{
    EncodeFn fn = encode_fn();
    if (!fn || rank < 1 || rank > 5 || (reinterpret_cast<uint64_t>(ptr) & 15)) return false;
    cuuint64_t dim[5], stride[4];
    cuuint32_t bx[5], es[5];
    for (int i = 0; i < rank; ++i) {
        dim[i] = dims[i];
        bx[i] = box[i];
        es[i] = 1;
        if (box[i] < 1 || box[i] > 256) return false;
    }
    for (int i = 0; i < rank - 1; ++i) {
        stride[i] = strides_bytes[i];
        if (stride[i] == 0 || stride[i] % 16 || stride[i] >= (1ull << 40)) return false;
    }
    if (((uint64_t)box[0] * es_bytes) % 16) return false;
    return fn(m, dt, (cuuint32_t)rank, const_cast<void *>(ptr), dim, stride, bx, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

} // namespace

bool encode_tiled(CUtensorMap *m, const void *ptr, int rank, const uint64_t *dims, const uint64_t *strides_bytes,
                  const uint32_t *box)
{
    return encode_tiled_es(m, ptr, rank, dims, strides_bytes, box, 8, CU_TENSOR_MAP_DATA_TYPE_UINT64);
}

bool encode_tiled_u32(CUtensorMap *m, const void *ptr, int rank, const uint64_t *dims, const uint64_t *strides_bytes,
                      const uint32_t *box)
{
    return encode_tiled_es(m, ptr, rank, dims, strides_bytes, box, 4, CU_TENSOR_MAP_DATA_TYPE_UINT32);
}

int sm_count()
{
    static int n[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!n[dev] && cudaDeviceGetAttribute(&n[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n[dev] = 152;
    return n[dev] > 0 ? n[dev] : 152;
}

} // namespace tma_fft

bool launch_axis2_tma(int sign, const AxisArgs &a, int nbatch, int norient, cudaStream_t s)
{
    using namespace tma_fft;
    if (a.A2 <= 0 || a.B2 <= 0) return false;
    const bool big = a.A2 > fft2::kMaxFactor;
    if (!fft2::is_split_choice(a.A2, a.B2, big ? fft2::kMaxFactorBig : fft2::kMaxFactor)) return false;
    const bool ws = a.tma == 2;            // warp-specialised: 8 pencils per item for both shapes
    // big factors: 16 pencils per item (128-byte rows per copy) where the option asks for it
    const bool wide = a.mul ? (a.wide & 1) != 0 : (a.wide & 2) != 0;
    const int W = ws ? 8 : big ? (wide ? 16 : 8) : 16;
    const int L = a.A2 * a.B2;
    if (!big && L < kMinLength) return false;
    Params P{};
    P.a = a;
    // which tensor dimension is the FFT axis: the smaller of the two strides is the row
    const bool plane = a.in_sl > a.in_sb;
    P.axis_is_plane = plane ? 1 : 0;
    P.nbox = (L + 255) / 256;
    P.box_j = ((L + P.nbox - 1) / P.nbox + 1) & ~1;      // even: 128-byte aligned boxes
    if (P.box_j > 256) return false;
    P.lrows = P.nbox * P.box_j;
    P.nchunks = (a.nx + W - 1) / W;
    P.norient = norient;
    P.nbatch = nbatch;
    P.items = (long)P.nchunks * norient * nbatch;
    if (P.items < 1) return true;
    const long rows = plane ? nbatch : a.lin, rs = plane ? a.in_sb : a.in_sl;
    const long planes = plane ? a.lin : nbatch, ps = plane ? a.in_sl : a.in_sb;
    const long os = a.in_so > 0 ? a.in_so : ps * planes;
    CUtensorMap in_map, mul_map;
    if (!encode(&in_map, a.in, 4, a.nx, rows, rs, planes, ps, norient, os, W, P.box_j, plane)) return false;
    const bool mul = a.mul != nullptr;
    if (mul) {
        if (a.mul_so != 0) return false;   // one factor shared by every orientation
        const long mrs = plane ? a.mul_sb : a.mul_sl, mps = plane ? a.mul_sl : a.mul_sb;
        if (!encode(&mul_map, a.mul, 3, a.nx, rows, mrs, planes, mps, 1, mps * planes, W, P.box_j, plane)) return false;
    } else {
        mul_map = in_map;
    }
    if (sign < 0 && mul) return false;
    const int v = sign < 0 ? 0 : mul ? 2 : 1;
    if (big) return v == 0 ? launch_tma_b0(in_map, mul_map, P, ws, W, s)
                  : v == 1 ? launch_tma_b1(in_map, mul_map, P, ws, W, s)
                           : launch_tma_b2(in_map, mul_map, P, ws, W, s);
    return v == 0 ? launch_tma_s0(in_map, mul_map, P, ws, W, s) : v == 1 ? launch_tma_s1(in_map, mul_map, P, ws, W, s)
                                                                         : launch_tma_s2(in_map, mul_map, P, ws, W, s);
}

} // namespace imf
