// Host-only exports that run the kernels' FFT building blocks (fft.cuh, fft2.cuh) on the CPU,
// for the CPU unit tests. Not part of libimf and never loaded by the product path.
#include <cmath>
#include <vector>

#include "fft.cuh"
#include "fft2.cuh"

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
    if (L < 4 || !imf::fft2::choose_split(L, &A, &B)) return -1;
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
