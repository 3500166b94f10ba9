// Mono-exponential T2 maps of a recovered image series (Sec. IV-A: the paper's T2 maps are
// obtained by fitting a mono-exponential model to every pixel of the reconstructed series).
//
//   |x_n(r)| ~ A(r) exp(-t_n / T2(r))   over foreground pixels |x_0(r)| > frac * max_r |x_0(r)|,
//
// log-linear least squares for the initial (A, 1/T2), then Gauss-Newton steps on the un-logged
// residual (2 x 2 normal equations per pixel, columns scaled to unit norm before Cramer's rule),
// 1/T2 kept >= 1e-4 per ms. One thread per pixel, all in FP32. The foreground decision
// is taken in FP32 with separately rounded products and sums (no contraction), so a host that
// repeats it in FP32 reaches the same mask bit for bit.
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace recon {

namespace {

constexpr int kThreads = 256;

RECON_DEV float magnitude_rn(float2 v) {
    return __fsqrt_rn(__fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y)));
}

// max_r |x_0(r)| into *amax (non-negative floats order like their bit patterns: atomicMax on
// the bits is exact and independent of the order of arrival).
__global__ void __launch_bounds__(kThreads)
frame0_max_kernel(const float2* __restrict__ x, size_t npix, unsigned int* __restrict__ amax) {
    float m = 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix;
         i += (size_t)gridDim.x * blockDim.x)
        m = fmaxf(m, magnitude_rn(x[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(amax, __float_as_uint(m));
}

__global__ void __launch_bounds__(kThreads)
t2fit_kernel(const float2* __restrict__ x, int T, size_t npix, T2Times tm, float frac,
             const unsigned int* __restrict__ amax, int n_gn, float* __restrict__ t2,
             float* __restrict__ amp) {
    const size_t px = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (px >= npix) return;
    const float thr = __fmul_rn(frac, __uint_as_float(amax[0]));
    float y[kT2MaxT];
    for (int n = 0; n < T; ++n) y[n] = magnitude_rn(x[(size_t)n * npix + px]);
    if (!(y[0] > thr)) {
        t2[px] = __int_as_float(0x7fc00000);  // NaN: not foreground
        if (amp) amp[px] = __int_as_float(0x7fc00000);
        return;
    }
    constexpr float kRmin = 1e-4f;  // 1 / T2 >= 1e-4 per ms (T2 <= 1e4 ms)
    // log-linear initial guess: log y = log A - R t
    float tbar = 0.f, lbar = 0.f;
    for (int n = 0; n < T; ++n) {
        tbar += tm.t[n];
        lbar += logf(fmaxf(y[n], 1e-30f));
    }
    tbar /= T;
    lbar /= T;
    float sxy = 0.f, sxx = 0.f;
    for (int n = 0; n < T; ++n) {
        const float dt = tm.t[n] - tbar;
        sxy = fmaf(dt, logf(fmaxf(y[n], 1e-30f)) - lbar, sxy);
        sxx = fmaf(dt, dt, sxx);
    }
    float R = fmaxf(-sxy / sxx, kRmin);
    float A = expf(lbar + R * tbar);
    for (int it = 0; it < n_gn; ++it) {
        float a11 = 0.f, a12 = 0.f, a22 = 0.f, g1 = 0.f, g2 = 0.f;
        for (int n = 0; n < T; ++n) {
            const float e = expf(-tm.t[n] * R);
            const float model = A * e;
            const float res = model - y[n];
            const float jr = -tm.t[n] * model;
            a11 = fmaf(e, e, a11);
            a12 = fmaf(e, jr, a12);
            a22 = fmaf(jr, jr, a22);
            g1 = fmaf(e, res, g1);
            g2 = fmaf(jr, res, g2);
        }
        // the 2 x 2 system with both columns scaled to unit norm: [1 c; c 1], det (1-c)(1+c)
        if (a11 > 0.f && a22 > 0.f) {
            const float s1 = rsqrtf(a11), s2 = rsqrtf(a22);
            const float c = a12 * s1 * s2;
            const float det = (1.f - c) * (1.f + c);
            if (det > 1e-12f) {
                const float h1 = g1 * s1, h2 = g2 * s2;
                const float id = 1.f / det;
                A -= s1 * (h1 - c * h2) * id;
                R = fmaxf(R - s2 * (h2 - c * h1) * id, kRmin);
            }
        }
    }
    t2[px] = 1.0f / R;
    if (amp) amp[px] = A;
}

}  // namespace

cudaError_t launch_t2fit(const Dims& d, const float2* x, const T2Times& tm, float frac, int n_gn,
                         unsigned int* amax_scratch, float* t2, float* amp, cudaStream_t st) {
    if (d.T < 2 || d.T > kT2MaxT) return cudaErrorInvalidValue;
    const size_t npix = d.pixels();
    cudaError_t e = cudaMemsetAsync(amax_scratch, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    const int g0 = (int)((npix + kThreads - 1) / kThreads < 1024 ? (npix + kThreads - 1) / kThreads : 1024);
    frame0_max_kernel<<<g0, kThreads, 0, st>>>(x, npix, amax_scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int g1 = (int)((npix + kThreads - 1) / kThreads);
    t2fit_kernel<<<g1, kThreads, 0, st>>>(x, d.T, npix, tm, frac, amax_scratch, n_gn, t2, amp);
    return cudaGetLastError();
}

}  // namespace recon
