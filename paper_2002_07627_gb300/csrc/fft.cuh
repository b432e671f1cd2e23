// Mixed-radix (2, 3, 4, 5, 7, 8) Stockham FFT building blocks, staged through shared memory.
//
// The collision convolution of Alg. 1 (Sec. 2.1.5 and App. B: two forward FFTs, a pointwise
// product and an inverse FFT) runs on padded grids whose extents are products of 2, 3, 5
// and 7, so every axis length factors into the radices below. Each stage is the self-sorting
// Stockham form: with Ns = product of the radices already applied, butterfly j of a stage of
// radix R reads x[j + r L/R] (r < R), multiplies by exp(S 2 pi i (j mod Ns) r / (Ns R)),
// applies an R-point DFT and writes to (j div Ns) Ns R + (j mod Ns) + s Ns. Output is in
// natural order with no digit reversal.
//
// Everything here is __host__ __device__ so that the host-side emulation used by the CPU
// tests runs the very same butterflies as the kernels.
#pragma once
#include <cuda_runtime.h>

#define FFT_HD __host__ __device__ __forceinline__

namespace imf {

FFT_HD float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
FFT_HD float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
FFT_HD float2 c_mul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
FFT_HD float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }
FFT_HD float2 c_scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * (S i), S = +1 or -1
template <int S> FFT_HD float2 c_mul_si(float2 a) { return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x); }

// DFT constants (cosines and sines of 2 pi k / R).
#define IMF_C5_1 0.30901699437494745f
#define IMF_C5_2 (-0.8090169943749473f)
#define IMF_S5_1 0.9510565162951535f
#define IMF_S5_2 0.5877852522924732f
#define IMF_S3 0.8660254037844386f
#define IMF_R2 0.7071067811865476f
#define IMF_C7_1 0.6234898018587336f
#define IMF_C7_2 (-0.22252093395631434f)
#define IMF_C7_3 (-0.900968867902419f)
#define IMF_S7_1 0.7818314824680298f
#define IMF_S7_2 0.9749279121818236f
#define IMF_S7_3 0.43388373911755823f

// R-point DFTs X[s] = sum_r v[r] exp(S 2 pi i r s / R), in place.
template <int S> FFT_HD void dft2(float2 *v)
{
    float2 a = v[0], b = v[1];
    v[0] = c_add(a, b);
    v[1] = c_sub(a, b);
}

template <int S> FFT_HD void dft3(float2 *v)
{
    float2 t = c_add(v[1], v[2]);
    float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
    float2 d = c_mul_si<S>(c_scale(c_sub(v[1], v[2]), IMF_S3));
    v[0] = c_add(v[0], t);
    v[1] = c_add(m, d);
    v[2] = c_sub(m, d);
}

template <int S> FFT_HD void dft4(float2 *v)
{
    float2 t0 = c_add(v[0], v[2]), t1 = c_sub(v[0], v[2]);
    float2 t2 = c_add(v[1], v[3]), t3 = c_mul_si<S>(c_sub(v[1], v[3]));
    v[0] = c_add(t0, t2);
    v[2] = c_sub(t0, t2);
    v[1] = c_add(t1, t3);
    v[3] = c_sub(t1, t3);
}

template <int S> FFT_HD void dft5(float2 *v)
{
    float2 a1 = c_add(v[1], v[4]), a2 = c_add(v[2], v[3]);
    float2 b1 = c_sub(v[1], v[4]), b2 = c_sub(v[2], v[3]);
    float2 x0 = v[0];
    float2 r1 = make_float2(x0.x + IMF_C5_1 * a1.x + IMF_C5_2 * a2.x, x0.y + IMF_C5_1 * a1.y + IMF_C5_2 * a2.y);
    float2 r2 = make_float2(x0.x + IMF_C5_2 * a1.x + IMF_C5_1 * a2.x, x0.y + IMF_C5_2 * a1.y + IMF_C5_1 * a2.y);
    float2 i1 = c_mul_si<S>(make_float2(IMF_S5_1 * b1.x + IMF_S5_2 * b2.x, IMF_S5_1 * b1.y + IMF_S5_2 * b2.y));
    float2 i2 = c_mul_si<S>(make_float2(IMF_S5_2 * b1.x - IMF_S5_1 * b2.x, IMF_S5_2 * b1.y - IMF_S5_1 * b2.y));
    v[0] = c_add(x0, c_add(a1, a2));
    v[1] = c_add(r1, i1);
    v[4] = c_sub(r1, i1);
    v[2] = c_add(r2, i2);
    v[3] = c_sub(r2, i2);
}

template <int S> FFT_HD void dft7(float2 *v)
{
    // X[s] = v0 + sum_{r=1..3} (v_r + v_{7-r}) cos(2 pi r s / 7) + S i (v_r - v_{7-r}) sin(2 pi r s / 7)
    float2 a1 = c_add(v[1], v[6]), a2 = c_add(v[2], v[5]), a3 = c_add(v[3], v[4]);
    float2 b1 = c_sub(v[1], v[6]), b2 = c_sub(v[2], v[5]), b3 = c_sub(v[3], v[4]);
    float2 x0 = v[0];
    // cos/sin of 2 pi (r s mod 7) / 7 for s = 1, 2, 3 and r = 1, 2, 3
    float2 r1 = make_float2(x0.x + IMF_C7_1 * a1.x + IMF_C7_2 * a2.x + IMF_C7_3 * a3.x,
                            x0.y + IMF_C7_1 * a1.y + IMF_C7_2 * a2.y + IMF_C7_3 * a3.y);
    float2 r2 = make_float2(x0.x + IMF_C7_2 * a1.x + IMF_C7_3 * a2.x + IMF_C7_1 * a3.x,
                            x0.y + IMF_C7_2 * a1.y + IMF_C7_3 * a2.y + IMF_C7_1 * a3.y);
    float2 r3 = make_float2(x0.x + IMF_C7_3 * a1.x + IMF_C7_1 * a2.x + IMF_C7_2 * a3.x,
                            x0.y + IMF_C7_3 * a1.y + IMF_C7_1 * a2.y + IMF_C7_2 * a3.y);
    // sin(2 pi r s / 7): s=1: (S1, S2, S3); s=2: (S2, -S3, -S1); s=3: (S3, -S1, S2)
    float2 i1 = c_mul_si<S>(make_float2(IMF_S7_1 * b1.x + IMF_S7_2 * b2.x + IMF_S7_3 * b3.x,
                                        IMF_S7_1 * b1.y + IMF_S7_2 * b2.y + IMF_S7_3 * b3.y));
    float2 i2 = c_mul_si<S>(make_float2(IMF_S7_2 * b1.x - IMF_S7_3 * b2.x - IMF_S7_1 * b3.x,
                                        IMF_S7_2 * b1.y - IMF_S7_3 * b2.y - IMF_S7_1 * b3.y));
    float2 i3 = c_mul_si<S>(make_float2(IMF_S7_3 * b1.x - IMF_S7_1 * b2.x + IMF_S7_2 * b3.x,
                                        IMF_S7_3 * b1.y - IMF_S7_1 * b2.y + IMF_S7_2 * b3.y));
    v[0] = c_add(x0, c_add(a1, c_add(a2, a3)));
    v[1] = c_add(r1, i1);
    v[6] = c_sub(r1, i1);
    v[2] = c_add(r2, i2);
    v[5] = c_sub(r2, i2);
    v[3] = c_add(r3, i3);
    v[4] = c_sub(r3, i3);
}

template <int S> FFT_HD void dft8(float2 *v)
{
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    dft4<S>(e);
    dft4<S>(o);
    // o[s] *= w8^s, w8 = exp(S 2 pi i / 8)
    float2 w1 = make_float2(IMF_R2, S * IMF_R2);
    float2 w3 = make_float2(-IMF_R2, S * IMF_R2);
    o[1] = c_mul(o[1], w1);
    o[2] = c_mul_si<S>(o[2]);
    o[3] = c_mul(o[3], w3);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        v[s] = c_add(e[s], o[s]);
        v[s + 4] = c_sub(e[s], o[s]);
    }
}

template <int S, int R> FFT_HD void dft(float2 *v)
{
    if constexpr (R == 2) dft2<S>(v);
    else if constexpr (R == 3) dft3<S>(v);
    else if constexpr (R == 4) dft4<S>(v);
    else if constexpr (R == 5) dft5<S>(v);
    else if constexpr (R == 7) dft7<S>(v);
    else if constexpr (R == 8) dft8<S>(v);
}

// Radix plan of one axis length. For every stage s, Ns = rad[0] * ... * rad[s-1];
// j / Ns = fast_div(j, mul[s]) exactly for 0 <= j < 2^20, and step[s] = L / (Ns rad[s]).
struct FftPlan {
    int L;          // transform length
    int nrad;       // number of stages
    int rad[16];    // radix of each stage
    unsigned mul[16];
    int step[16];
};

// j / d for j < 2^20 and 2 <= d <= 4096 with mul = ceil(2^32 / d): j mul / 2^32 exceeds j / d
// by less than j / 2^32 < 1 / d, which cannot carry past the next integer. mul = 0 means d = 1.
FFT_HD unsigned fast_div(unsigned j, unsigned mul)
{
    if (mul == 0) return j;
#ifdef __CUDA_ARCH__
    return __umulhi(j, mul);
#else
    return (unsigned)(((unsigned long long)j * mul) >> 32);
#endif
}

// One Stockham butterfly. Element (w, j) of the tile lives at w*sw + j*sj. `tw` holds
// exp(-2 pi i m / L), m < L.
template <int S, int R>
FFT_HD void stockham_bfly(const float2 *src, float2 *dst, int w, int jb, int L, int Ns, int sw, int sj,
                          const float2 *tw, int jdiv, int step)
{
    const int NR = L / R;
    const int k = jb - jdiv * Ns;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[w * sw + (jb + r * NR) * sj];
    if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
            float2 t = tw[k * r * step];
            if (S > 0) t.y = -t.y;
            v[r] = c_mul(v[r], t);
        }
    }
    dft<S, R>(v);
    const int base = jdiv * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[w * sw + (base + r * Ns) * sj] = v[r];
}

// jdiv = jb / Ns (passed in so the caller can use the plan's exact reciprocal)
template <int S>
FFT_HD void stockham_dispatch(int R, const float2 *src, float2 *dst, int w, int jb, int L, int Ns, int sw,
                              int sj, const float2 *tw, int jdiv, int step)
{
    switch (R) {
    case 2: stockham_bfly<S, 2>(src, dst, w, jb, L, Ns, sw, sj, tw, jdiv, step); break;
    case 3: stockham_bfly<S, 3>(src, dst, w, jb, L, Ns, sw, sj, tw, jdiv, step); break;
    case 4: stockham_bfly<S, 4>(src, dst, w, jb, L, Ns, sw, sj, tw, jdiv, step); break;
    case 5: stockham_bfly<S, 5>(src, dst, w, jb, L, Ns, sw, sj, tw, jdiv, step); break;
    case 7: stockham_bfly<S, 7>(src, dst, w, jb, L, Ns, sw, sj, tw, jdiv, step); break;
    case 8: stockham_bfly<S, 8>(src, dst, w, jb, L, Ns, sw, sj, tw, jdiv, step); break;
    default: break;
    }
}

inline unsigned div_magic(unsigned d)
{
    return d <= 1 ? 0u : (unsigned)(((1ull << 32) + d - 1) / d);
}

// Factor L into stages (largest radices first). Returns false if L has a prime factor > 7.
inline bool make_plan(int L, FftPlan *p)
{
    p->L = L;
    p->nrad = 0;
    int m = L;
    while (m % 8 == 0) { p->rad[p->nrad++] = 8; m /= 8; }
    while (m % 7 == 0) { p->rad[p->nrad++] = 7; m /= 7; }
    while (m % 5 == 0) { p->rad[p->nrad++] = 5; m /= 5; }
    while (m % 4 == 0) { p->rad[p->nrad++] = 4; m /= 4; }
    while (m % 3 == 0) { p->rad[p->nrad++] = 3; m /= 3; }
    while (m % 2 == 0) { p->rad[p->nrad++] = 2; m /= 2; }
    if (m != 1 || p->nrad > 16 || L > 4096) return false;
    int Ns = 1;
    for (int s = 0; s < p->nrad; ++s) {
        p->mul[s] = div_magic((unsigned)Ns);
        p->step[s] = L / (Ns * p->rad[s]);
        Ns *= p->rad[s];
    }
    return true;
}

// Host emulation of a whole 1D transform on one pencil (tests only): ping-pongs between
// `a` and `b` (each of length L) and returns the buffer holding the result.
template <int S> inline float2 *fft_pencil_host(const FftPlan &p, float2 *a, float2 *b, const float2 *tw)
{
    int Ns = 1;
    float2 *src = a, *dst = b;
    for (int s = 0; s < p.nrad; ++s) {
        int R = p.rad[s];
        for (int jb = 0; jb < p.L / R; ++jb)
            stockham_dispatch<S>(R, src, dst, 0, jb, p.L, Ns, 0, 1, tw, (int)fast_div((unsigned)jb, p.mul[s]), p.step[s]);
        float2 *t = src; src = dst; dst = t;
        Ns *= R;
    }
    return src;
}

} // namespace imf
