// FFT pass kernels of the collision convolution (Alg. 1 Convolve; App. B).
//
// The 3D real FFT of a padded grid [Pz][Py][Px] is split into one pass per axis. The x pass
// packs a real row of length P = 2M into M complex samples, transforms them and unpacks the
// half spectrum (M + 1 bins); the y and z passes transform columns of the half spectrum
// [z][y][kx] with W consecutive kx columns per block so that every global access is a
// 128-byte segment. Each pass stages its tile in shared memory and runs the Stockham stages
// of fft.cuh there. The inverse z pass multiplies the design spectrum by a tool spectrum as
// it loads (the pointwise product of App. B), and the inverse x pass writes the collision
// measure g together with the bit mask of collision-free translations (threshold of
// Eq. eq_conv_D) and the list of translations whose g lies within the re-check band.
#include "imf_internal.cuh"
#include "threshold_row.cuh"

namespace imf {

namespace {

// Stockham stages over a tile of W interleaved pencils (element (w, j) at w + j * sj);
// W is a power of two so q -> (w, jb) is a mask and a shift, and jb / Ns uses the plan's
// exact reciprocal.
template <int S, int R, int LOGW>
__device__ __forceinline__ void stage_loop(const float2 *src, float2 *dst, int L, int Ns, int sj, const float2 *tw,
                                           unsigned mul, int step)
{
    constexpr int W = 1 << LOGW;
    const int nb = (L / R) << LOGW;
    for (int q = threadIdx.x; q < nb; q += blockDim.x) {
        const int w = q & (W - 1), jb = q >> LOGW;
        stockham_bfly<S, R>(src, dst, w, jb, L, Ns, 1, sj, tw, (int)fast_div((unsigned)jb, mul), step);
    }
}

// Stockham stages over a tile of W interleaved pencils (element (w, j) at w + j * sj);
// W is a power of two so q -> (w, jb) is a mask and a shift, jb / Ns uses the plan's exact
// reciprocal, and the radix dispatch happens once per stage.
template <int S, int LOGW>
__device__ void run_stages(const FftPlan &plan, float2 *&src, float2 *&dst, int sj, const float2 *tw)
{
    const int L = plan.L;
    int Ns = 1;
    for (int s = 0; s < plan.nrad; ++s) {
        const int R = plan.rad[s];
        const unsigned mul = plan.mul[s];
        const int step = plan.step[s];
        switch (R) {
        case 2: stage_loop<S, 2, LOGW>(src, dst, L, Ns, sj, tw, mul, step); break;
        case 3: stage_loop<S, 3, LOGW>(src, dst, L, Ns, sj, tw, mul, step); break;
        case 4: stage_loop<S, 4, LOGW>(src, dst, L, Ns, sj, tw, mul, step); break;
        case 5: stage_loop<S, 5, LOGW>(src, dst, L, Ns, sj, tw, mul, step); break;
        case 7: stage_loop<S, 7, LOGW>(src, dst, L, Ns, sj, tw, mul, step); break;
        default: stage_loop<S, 8, LOGW>(src, dst, L, Ns, sj, tw, mul, step); break;
        }
        __syncthreads();
        float2 *t = src; src = dst; dst = t;
        Ns *= R;
    }
}

constexpr int kAxisW = 16;

template <int S>
__global__ void __launch_bounds__(kThreads) axis_fft_kernel(AxisArgs a)
{
    extern __shared__ float2 sm[];
    const int L = a.plan.L;
    float2 *buf0 = sm, *buf1 = sm + kAxisW * L, *tw = sm + 2 * kAxisW * L;
    for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = a.tw[i];
    const int kx0 = blockIdx.x * kAxisW;
    const long b = blockIdx.y, o = blockIdx.z;
    const float2 *in = a.in + o * a.in_so + b * a.in_sb + kx0;
    const float2 *mul = a.mul ? a.mul + o * a.mul_so + b * a.mul_sb + kx0 : nullptr;
    // loads are issued in groups of 8 per thread before any shared store (memory-level
    // parallelism); the optional pointwise factor is applied on the way in
    const int total = kAxisW * L;
    for (int base = 0; base < total; base += 8 * kThreads) {
        float2 v[8], m[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int idx = base + u * kThreads + threadIdx.x;
            const int w = idx % kAxisW, j = idx / kAxisW;
            v[u] = make_float2(0.f, 0.f);
            m[u] = make_float2(1.f, 0.f);
            if (idx < total && j < a.lin && kx0 + w < a.nx) {
                v[u] = in[(long)j * a.in_sl + w];
                if (mul) m[u] = mul[(long)j * a.mul_sl + w];
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int idx = base + u * kThreads + threadIdx.x;
            if (idx < total) buf0[idx] = mul ? c_mul(v[u], m[u]) : v[u];
        }
    }
    __syncthreads();
    float2 *src = buf0, *dst = buf1;
    run_stages<S, 4>(a.plan, src, dst, kAxisW, tw);
    float2 *out = a.out + o * a.out_so + b * a.out_sb + kx0;
    for (int idx = threadIdx.x; idx < kAxisW * a.lout; idx += blockDim.x) {
        const int w = idx % kAxisW, jj = idx / kAxisW;
        if (kx0 + w < a.nx) {
            float2 v = c_scale(src[(a.j0 + jj) * kAxisW + w], a.scale);
            if (a.conj_out) v.y = -v.y;
            out[(long)jj * a.out_sl + w] = v;
        }
    }
}

// x-pass tiles hold W rows interleaved: element (row w, sample j) at j * (W + 1) + w, so the
// Stockham stages and the row loads / stores touch consecutive or odd-strided banks.
template <int LOGW> __global__ void __launch_bounds__(kThreads) rfft_fwd_kernel(RfftArgs a)
{
    constexpr int W = 1 << LOGW;
    extern __shared__ float2 sm[];
    const int M = a.M, ld = W + 1;
    float2 *buf0 = sm, *buf1 = sm + (M + 1) * ld, *twM = sm + 2 * (M + 1) * ld, *twP = twM + M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) twM[i] = a.twM[i];
    for (int i = threadIdx.x; i <= M; i += blockDim.x) twP[i] = a.twP[i];
    const int r0 = blockIdx.x * W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // one warp per row (row -> (y, z) once), lanes over the packed samples
    for (int w = warp; w < W; w += kThreads / 32) {
        const int r = r0 + w;
        const bool rowok = r < a.rows;
        const int y = rowok ? r % a.rows_y : 0, z = rowok ? r / a.rows_y : 0;
        const float *row = a.src + z * a.src_sz + y * a.src_sy;
        const uint8_t *frow = a.fix ? a.fix + z * a.src_sz + y * a.src_sy : nullptr;
        for (int n0 = 0; n0 < M; n0 += 128) {
            float2 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int n = n0 + u * 32 + lane;
                v[u] = make_float2(0.f, 0.f);
                if (rowok && n < M) {
                    const int x0 = 2 * n, x1 = 2 * n + 1;
                    if (x0 < a.nin) v[u].x = frow ? fminf(1.f, row[x0] + (frow[x0] ? 1.f : 0.f)) : row[x0];
                    if (x1 < a.nin) v[u].y = frow ? fminf(1.f, row[x1] + (frow[x1] ? 1.f : 0.f)) : row[x1];
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int n = n0 + u * 32 + lane;
                if (n < M) buf0[n * ld + w] = v[u];
            }
        }
    }
    __syncthreads();
    float2 *src = buf0, *dst = buf1;
    run_stages<-1, LOGW>(a.plan, src, dst, ld, twM);
    // unpack: X[k] = (Z[k] + conj Z[M-k]) / 2 + exp(-2 pi i k / P) (Z[k] - conj Z[M-k]) / (2 i)
    for (int w = warp; w < W; w += kThreads / 32) {
        const int r = r0 + w;
        if (r >= a.rows) break;
        const int y = r % a.rows_y, z = r / a.rows_y;
        float2 *out = a.out + z * a.out_sz + y * a.out_sy;
        for (int k = lane; k <= M; k += 32) {
            const float2 zk = src[(k == M ? 0 : k) * ld + w];
            const float2 zc = c_conj(src[(k == 0 ? 0 : M - k) * ld + w]);
            const float2 e = c_scale(c_add(zk, zc), 0.5f);
            const float2 od = c_mul_si<-1>(c_scale(c_sub(zk, zc), 0.5f));
            out[k] = c_add(e, c_mul(twP[k], od));
        }
    }
}

template <int LOGW> __global__ void __launch_bounds__(kThreads) irfft_threshold_kernel(IrfftArgs a)
{
    constexpr int W = 1 << LOGW;
    extern __shared__ float2 sm[];
    const int M = a.M, ld = W + 1;
    float2 *buf0 = sm, *buf1 = sm + (M + 1) * ld, *twM = sm + 2 * (M + 1) * ld, *twP = twM + M;
    for (int i = threadIdx.x; i < M; i += blockDim.x) twM[i] = a.twM[i];
    for (int i = threadIdx.x; i <= M; i += blockDim.x) twP[i] = a.twP[i];
    const int r0 = blockIdx.x * W;
    const long o = blockIdx.z;
    const float2 *in = a.in + o * a.in_so;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int w = warp; w < W; w += kThreads / 32) {
        const int r = r0 + w;
        const bool rowok = r < a.rows;
        const int y = rowok ? r % a.rows_y : 0, z = rowok ? r / a.rows_y : 0;
        const float2 *row = in + z * a.in_sz + y * a.in_sy;
        for (int k0 = 0; k0 <= M; k0 += 128) {
            float2 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = k0 + u * 32 + lane;
                v[u] = (rowok && k <= M) ? row[k] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int k = k0 + u * 32 + lane;
                if (k <= M) buf1[k * ld + w] = v[u];
            }
        }
    }
    __syncthreads();
    // pack: Z[k] = (X[k] + conj X[M-k]) + i exp(+2 pi i k / P) (X[k] - conj X[M-k]), k < M
    for (int idx = threadIdx.x; idx < W * M; idx += blockDim.x) {
        const int w = idx % W, k = idx / W;
        const float2 xk = buf1[k * ld + w];
        const float2 xc = c_conj(buf1[(M - k) * ld + w]);
        const float2 e = c_add(xk, xc);
        const float2 od = c_mul(c_conj(twP[k]), c_sub(xk, xc));
        buf0[k * ld + w] = c_add(e, c_mul_si<1>(od));
    }
    __syncthreads();
    float2 *src = buf0, *dst = buf1;
    run_stages<1, LOGW>(a.plan, src, dst, ld, twM);
    for (int w = warp; w < W; w += nwarp) {
        const int r = r0 + w;
        if (r >= a.rows) break;  // warp-uniform
        threshold_row_any(a, src + w, ld, o, r, lane);
    }
}

template <typename K> void set_smem(K kernel, size_t bytes)
{
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// rows per x-pass block: 32 while the two staging buffers stay near 100 KB, else 16 or 8
int x_log_rows(int M)
{
    if ((size_t)(M + 1) * 33 * 16 <= 100 * 1024) return 5;
    if ((size_t)(M + 1) * 17 * 16 <= 100 * 1024) return 4;
    return 3;
}

size_t x_smem(int M, int W) { return (size_t)(2 * (M + 1) * (W + 1) + 2 * M + 1) * sizeof(float2); }

} // namespace

void launch_axis_fft(int sign, const AxisArgs &a, int nbatch, int norient, cudaStream_t s)
{
    if (a.A2 > 0) {
        launch_axis2(sign, a, nbatch, norient, s);
        return;
    }
    const size_t smem = (size_t)(2 * kAxisW * a.plan.L + a.plan.L) * sizeof(float2);
    dim3 grid((a.nx + kAxisW - 1) / kAxisW, nbatch, norient);
    if (sign < 0) {
        set_smem(axis_fft_kernel<-1>, smem);
        axis_fft_kernel<-1><<<grid, kThreads, smem, s>>>(a);
    } else {
        set_smem(axis_fft_kernel<1>, smem);
        axis_fft_kernel<1><<<grid, kThreads, smem, s>>>(a);
    }
}

void launch_rfft_fwd(const RfftArgs &a, cudaStream_t s)
{
    const int lw = x_log_rows(a.M), W = 1 << lw;
    const size_t smem = x_smem(a.M, W);
    dim3 grid((a.rows + W - 1) / W);
    if (lw == 5) { set_smem(rfft_fwd_kernel<5>, smem); rfft_fwd_kernel<5><<<grid, kThreads, smem, s>>>(a); }
    else if (lw == 4) { set_smem(rfft_fwd_kernel<4>, smem); rfft_fwd_kernel<4><<<grid, kThreads, smem, s>>>(a); }
    else { set_smem(rfft_fwd_kernel<3>, smem); rfft_fwd_kernel<3><<<grid, kThreads, smem, s>>>(a); }
}

void launch_irfft_threshold(const IrfftArgs &a, int norient, cudaStream_t s)
{
    if (a.A2 > 0) {
        launch_irfft2_threshold(a, norient, s);
        return;
    }
    const int lw = x_log_rows(a.M), W = 1 << lw;
    const size_t smem = x_smem(a.M, W);
    dim3 grid((a.rows + W - 1) / W, 1, norient);
    if (lw == 5) { set_smem(irfft_threshold_kernel<5>, smem); irfft_threshold_kernel<5><<<grid, kThreads, smem, s>>>(a); }
    else if (lw == 4) { set_smem(irfft_threshold_kernel<4>, smem); irfft_threshold_kernel<4><<<grid, kThreads, smem, s>>>(a); }
    else { set_smem(irfft_threshold_kernel<3>, smem); irfft_threshold_kernel<3><<<grid, kThreads, smem, s>>>(a); }
}

} // namespace imf
