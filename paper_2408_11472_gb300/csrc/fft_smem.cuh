// fft_smem.cuh -- complex helpers and a radix-2 Stockham transform over rows held in
// shared memory, shared by the post-processing (synth.cu) and the delay-Doppler focusing
// (ddfocus.cu) kernels.
#pragma once

#include <cuda_runtime.h>

namespace rsim {
namespace fft {

template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

__device__ __forceinline__ void twiddle(int r, int N, float sign, float2& w) {
    float s, c;
    sincospif(2.0f * (float)r / (float)N, &s, &c);
    w = make_float2(c, sign * s);
}
__device__ __forceinline__ void twiddle(int r, int N, double sign, double2& w) {
    double s, c;
    sincospi(2.0 * (double)r / (double)N, &s, &c);
    w = make_double2(c, sign * s);
}

// Radix-2 Stockham autosort over `rows` independent N-point rows in shared memory.
// Input in a, returns the buffer holding the natural-order result.  tw[r] = exp(sign j 2 pi r/N).
template <typename T>
__device__ T* stockham(T* a, T* b, int rows, int N, int L, const T* __restrict__ tw) {
    const int half = N >> 1;
    for (int st = 0; st < L; ++st) {
        const int s = 1 << st;
        const int m = half >> st;
        for (int idx = threadIdx.x; idx < rows * half; idx += blockDim.x) {
            const int row = idx >> (L - 1);
            const int bi = idx & (half - 1);
            const int p = bi >> st, q = bi & (s - 1);
            const T w = tw[p << st];
            const T* ar = a + row * N;
            T* br = b + row * N;
            const T x0 = ar[q + s * p];
            const T x1 = ar[q + s * (p + m)];
            br[q + s * (2 * p)] = cadd(x0, x1);
            br[q + s * (2 * p + 1)] = cmul(csub(x0, x1), w);
        }
        __syncthreads();
        T* t = a; a = b; b = t;
    }
    return a;
}

}  // namespace fft
}  // namespace rsim
