// Two-pass register FFT for lengths L = A * B with A, B in {2, ..., 16} (smooth).
//
// Cooley-Tukey with one split (the convolution of Alg. 1 / App. B needs forward and inverse
// DFTs along each axis of the padded grid): writing n = n1 + B n2 and k = k2 + A k1,
//   X[k2 + A k1] = sum_{n1 < B} w_B^{n1 k1} ( w_L^{n1 k2} sum_{n2 < A} x[n1 + B n2] w_A^{n2 k2} ),
// with w_N = exp(S 2 pi i / N). Pass 1: for each n1 an A-point DFT of the stride-B samples,
// times the twiddle w_L^{n1 k2}; pass 2: for each k2 a B-point DFT. In the kernels one thread
// holds one A-point (then one B-point) DFT in registers, so a pencil crosses shared memory
// once. The small DFTs are unrolled at compile time: composite sizes split again (same
// identity) with constant twiddles evaluated by constexpr Taylor series.
//
// All of it is __host__ __device__ so the CPU tests run the same arithmetic as the kernels.
#pragma once
#include <type_traits>

#include "fft.cuh"

namespace imf {
namespace fft2 {

constexpr int kMaxFactor = 16;      // factors of the kernels with 16 slots per pencil
constexpr int kMaxFactorBig = 24;   // factors of the axis kernel with 32 slots per pencil

__host__ __device__ constexpr bool supported(int n)
{
    return n == 2 || n == 3 || n == 4 || n == 5 || n == 6 || n == 7 || n == 8 || n == 9 || n == 10 || n == 12 ||
           n == 14 || n == 15 || n == 16;
}
// factors above 16 (only kernels built for them dispatch these)
__host__ __device__ constexpr bool supported_big(int n) { return n == 18 || n == 20 || n == 21 || n == 24; }

// cos and sin of 2 pi m / n from their Taylor series (argument reduced to [-pi, pi))
__host__ __device__ constexpr double taylor_cos(double x)
{
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 30; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double taylor_sin(double x)
{
    double term = x, sum = x;
    for (int k = 1; k < 30; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double turn_angle(int m, int n)
{
    const int r = ((m % n) + n) % n;
    const double pi = 3.14159265358979323846;
    const double a = 2.0 * pi * r / n;
    return a >= pi ? a - 2.0 * pi : a;
}

template <int I, int E> struct SFor {
    template <typename F> __host__ __device__ __forceinline__ static void run(F &&f)
    {
        if constexpr (I < E) {
            f(std::integral_constant<int, I>{});
            SFor<I + 1, E>::run(f);
        }
    }
};

// a * w_N^M with w_N = exp(S 2 pi i / N); exact for multiples of a quarter turn
template <int S, int M, int N> __host__ __device__ __forceinline__ float2 twiddle_const(float2 a)
{
    constexpr int m = ((M % N) + N) % N;
    if constexpr (m == 0) return a;
    else if constexpr (4 * m == N) return c_mul_si<S>(a);
    else if constexpr (2 * m == N) return make_float2(-a.x, -a.y);
    else if constexpr (4 * m == 3 * N) return c_mul_si<-S>(a);
    else {
        constexpr float c = (float)taylor_cos(turn_angle(m, N));
        constexpr float s = (float)(S * taylor_sin(turn_angle(m, N)));
        return c_mul(a, make_float2(c, s));
    }
}

__host__ __device__ constexpr int inner_factor(int n)
{
    return n % 4 == 0 ? 4 : n % 7 == 0 ? 7 : n % 5 == 0 ? 5 : n % 3 == 0 ? 3 : 2;
}

// In-place N-point DFT X[k] = sum_n v[n] w_N^{nk}, natural order in and out.
template <int S, int N> __host__ __device__ __forceinline__ void dft_reg(float2 *v)
{
    if constexpr (N == 1) {
    } else if constexpr (N == 2 || N == 3 || N == 4 || N == 5 || N == 7 || N == 8) {
        dft<S, N>(v);
    } else {
        constexpr int F = inner_factor(N), N2 = N / F;
        float2 t[N];
        SFor<0, N2>::run([&](auto I1) {
            constexpr int n1 = decltype(I1)::value;
            float2 u[F];
            SFor<0, F>::run([&](auto I2) { u[decltype(I2)::value] = v[n1 + N2 * decltype(I2)::value]; });
            dft<S, F>(u);
            SFor<0, F>::run([&](auto K2) {
                constexpr int k2 = decltype(K2)::value;
                t[n1 * F + k2] = twiddle_const<S, n1 * k2, N>(u[k2]);
            });
        });
        SFor<0, F>::run([&](auto K2) {
            constexpr int k2 = decltype(K2)::value;
            float2 u[N2];
            SFor<0, N2>::run([&](auto I1) { u[decltype(I1)::value] = t[decltype(I1)::value * F + k2]; });
            dft_reg<S, N2>(u);
            SFor<0, N2>::run([&](auto K1) { v[k2 + F * decltype(K1)::value] = u[decltype(K1)::value]; });
        });
    }
}

// Split of L for the two passes: A (pass-1 DFT size) >= B (pass-2 DFT size), both supported
// with factors up to maxA (kMaxFactor or kMaxFactorBig), as balanced as possible. Returns false
// when L has no such split.
__host__ __device__ constexpr bool choose_split(int L, int *A, int *B, int maxA = kMaxFactor)
{
    int bestA = 0, bestB = 0;
    for (int b = 2; b <= maxA; ++b) {
        if (L % b) continue;
        const int a = L / b;
        const bool oka = a <= maxA && (supported(a) || supported_big(a));
        const bool okb = b <= maxA && (supported(b) || supported_big(b));
        if (a < b || !oka || !okb) continue;
        if (!bestA || a < bestA) { bestA = a; bestB = b; }
    }
    if (!bestA) return false;
    *A = bestA;
    *B = bestB;
    return true;
}

// Whether (a, b) is the split choose_split returns for L = a b: the pairs the kernels that
// take both factors at compile time instantiate.
__host__ __device__ constexpr bool is_split_choice(int a, int b, int maxA)
{
    int A = 0, B = 0;
    return choose_split(a * b, &A, &B, maxA) && A == a && B == b;
}

// Pass-1 arithmetic of one thread: A-point DFT of v (the samples x[n1 + B n2], n2 < A), then
// v[k2] *= w_L^{S n1 k2} from tw[m] = exp(-2 pi i m / L) (n1 k2 < L needs no reduction).
template <int S, int A> __host__ __device__ __forceinline__ void twiddle(float2 *v, int n1, const float2 *tw)
{
    if (n1 == 0) return;
#pragma unroll
    for (int k2 = 1; k2 < A; ++k2) {
        float2 t = tw[n1 * k2];
        if (S > 0) t.y = -t.y;
        v[k2] = c_mul(v[k2], t);
    }
}
template <int S, int A> __host__ __device__ __forceinline__ void pass1(float2 *v, int n1, const float2 *tw)
{
    dft_reg<S, A>(v);
    twiddle<S, A>(v, n1, tw);
}

// Calls f(std::integral_constant<int, n>) for a supported size n (uniform branch).
template <typename F> __host__ __device__ __forceinline__ void with_size(int n, F &&f)
{
    switch (n) {
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    case 5: f(std::integral_constant<int, 5>{}); break;
    case 6: f(std::integral_constant<int, 6>{}); break;
    case 7: f(std::integral_constant<int, 7>{}); break;
    case 8: f(std::integral_constant<int, 8>{}); break;
    case 9: f(std::integral_constant<int, 9>{}); break;
    case 10: f(std::integral_constant<int, 10>{}); break;
    case 12: f(std::integral_constant<int, 12>{}); break;
    case 14: f(std::integral_constant<int, 14>{}); break;
    case 15: f(std::integral_constant<int, 15>{}); break;
    case 16: f(std::integral_constant<int, 16>{}); break;
    default: break;
    }
}

// with_size over the sizes above 16 as well (kernels with 32 slots per pencil).
template <typename F> __host__ __device__ __forceinline__ void with_size_big(int n, F &&f)
{
    switch (n) {
    case 18: f(std::integral_constant<int, 18>{}); break;
    case 20: f(std::integral_constant<int, 20>{}); break;
    case 21: f(std::integral_constant<int, 21>{}); break;
    case 24: f(std::integral_constant<int, 24>{}); break;
    default: with_size(n, f); break;
    }
}

// Host emulation of a whole transform of one pencil (tests): x (length L = A B) -> X with
// the kernels' pass structure and arithmetic; T is scratch of length L.
template <int S>
inline void fft2_pencil_host(int A, int B, const float2 *x, float2 *X, float2 *T, const float2 *tw)
{
    for (int n1 = 0; n1 < B; ++n1)
        with_size_big(A, [&](auto AA) {
            constexpr int a = decltype(AA)::value;
            float2 v[a];
            for (int n2 = 0; n2 < a; ++n2) v[n2] = x[n1 + B * n2];
            pass1<S, a>(v, n1, tw);
            for (int k2 = 0; k2 < a; ++k2) T[n1 * a + k2] = v[k2];
        });
    for (int k2 = 0; k2 < A; ++k2)
        with_size_big(B, [&](auto BB) {
            constexpr int b = decltype(BB)::value;
            float2 u[b];
            for (int n1 = 0; n1 < b; ++n1) u[n1] = T[n1 * A + k2];
            dft_reg<S, b>(u);
            for (int k1 = 0; k1 < b; ++k1) X[k2 + A * k1] = u[k1];
        });
}

} // namespace fft2
} // namespace imf
