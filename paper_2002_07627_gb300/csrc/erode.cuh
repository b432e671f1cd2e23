// Declarations of the tiled minimum over sharp points (erode.cu; planned by erode_plan.h).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace imf {

// Tiled minimum over sharp points. A block owns kErTX x kErTY x kErTZ outputs (kErXT
// consecutive x per thread; 1024 threads, one block per SM); the sharp points of an
// orientation are runs along x, grouped in dz-chunks whose g tile fits the shared-memory
// budget. Larger blocks fill less halo per output and need fewer chunks per orientation
// (measured on 128^3 x 64 with 16 orientations per launch: 64 x 16 x 8 outputs in 1024
// threads 4.17 ms per step against 4.77 ms for 64 x 8 x 8 in 512 threads and 7.2 ms for
// 32 x 8 x 8 in 256 threads).
constexpr int kErTX = 64, kErTY = 16, kErTZ = 8, kErXT = 8, kErMaxL = 16;
// runs of the level kernel (erode3_kernel) are split at 31: any length up to 2^5 - 1 is two
// windows of one dyadic level
constexpr int kErMaxL3 = 31;
// longest tile row the level kernel builds levels for (four cells per lane of a warp)
constexpr int kErMaxRow3 = 128;
constexpr int kErThreads = (kErTX / kErXT) * kErTY * kErTZ;
// threads of a block with xt consecutive x outputs per thread
__host__ __device__ constexpr int er_threads(int xt) { return (kErTX / xt) * kErTY * kErTZ; }
constexpr int kErBlocksPerSM = 1024 / kErThreads;            // 64 registers per thread
// most run descriptors of one chunk (larger chunks are split)
constexpr int kErMaxRunsPerChunk = 2048;
// dynamic shared memory of one block (one per SM): a chunk's g tile followed by its run
// descriptors (8 bytes each), sized per chunk so that the tile takes what the runs leave
constexpr size_t kErodeBudget = 222 * 1024;
// float offset of a chunk's run descriptors behind its tile of tzh planes (8-byte aligned)
__host__ __device__ constexpr int er_runs_offset(int tzh, int pitch_z) { return (tzh * pitch_z + 1) & ~1; }
struct ErodeChunk {
    int run0, run1;              // runs of this chunk, sorted by length
    int lend[kErMaxL3 + 1];      // runs of length L are run0 + lend[L-1] .. run0 + lend[L] - 1
    int txh, tyh, tzh;           // tile extents
    int pitch_y, pitch_z;        // shared-memory row and plane pitch (floats)
    int ox, oy, oz;              // tile origin = block output origin + (ox, oy, oz) in window index
};
struct Erode2Args {
    const float *g;
    long g_so;
    int gpx, gpy;                // window pitch (x) and rows per z-plane
    int wx, wy, wz;              // window extents
    const ErodeChunk *chunks;
    const int *chunk_start;      // n_orient + 1
    const int2 *runs;            // (shared-memory offset, length)
    int nx, ny, nz;
    int orient_base, nb;
    int ngroups;                 // orientation groups per tile (blockIdx.z = group * tiles_z + tile z)
    float *f;
};
// xt = consecutive x outputs per thread: 8 (1024 threads, 64 registers each) or 16 (512 threads,
// 128 registers each); the plan does not depend on it
void launch_erode2(const Erode2Args &a, size_t smem, int xt, cudaStream_t s);
int erode2_blocks_per_sm(size_t smem, int xt);
// The same minimum with dyadic min levels built in place in the tile (runs up to kErMaxL3, tile
// rows up to kErMaxRow3); planned with plan_erode(..., kErMaxL3).
void launch_erode3(const Erode2Args &a, size_t smem, cudaStream_t s);
int erode3_blocks_per_sm(size_t smem);

} // namespace imf
