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

// Radix-4 Stockham autosort (a final radix-2 stage when log2 N is odd) over `rows`
// independent N-point rows in shared memory: half the passes over the data of the radix-2
// version.  tw[n] = exp(sign j 2 pi n / N) for n < N/2 (the other half by W^{n+N/2} = -W^n);
// `sign` (+1 or -1) is the transform's.  Returns the buffer holding the natural-order result.
template <typename T>
__device__ __forceinline__ T tw_full(const T* tw, int e, int N) {
    const int h = N >> 1;
    if (e < h) return tw[e];
    const T w = tw[e - h];
    T r;
    r.x = -w.x;
    r.y = -w.y;
    return r;
}

template <typename T>
__device__ T* stockham4(T* a, T* b, int rows, int N, int L, const T* __restrict__ tw, int sign) {
    int s = 1, lg = 0;
    const int quarter = N >> 2;
    while (lg + 2 <= L) {                       // radix-4 stages: s = 4^(lg/2) = 2^lg
        const int m = quarter >> lg;
        for (int idx = threadIdx.x; idx < rows * quarter; idx += blockDim.x) {
            const int row = idx >> (L - 2);
            const int bi = idx & (quarter - 1);
            const int p = bi >> lg, q = bi & (s - 1);
            const T* ar = a + row * N;
            T* br = b + row * N;
            const T x0 = ar[q + s * p], x1 = ar[q + s * (p + m)];
            const T x2 = ar[q + s * (p + 2 * m)], x3 = ar[q + s * (p + 3 * m)];
            const T t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), d = csub(x1, x3);
            T t3;                               // sign j (x1 - x3)
            t3.x = -sign * d.y;
            t3.y = sign * d.x;
            const int e = p * s;
            br[q + s * (4 * p)] = cadd(t0, t2);
            br[q + s * (4 * p + 1)] = cmul(cadd(t1, t3), tw_full(tw, e, N));
            br[q + s * (4 * p + 2)] = cmul(csub(t0, t2), tw_full(tw, 2 * e, N));
            br[q + s * (4 * p + 3)] = cmul(csub(t1, t3), tw_full(tw, 3 * e, N));
        }
        __syncthreads();
        T* t = a; a = b; b = t;
        s <<= 2;
        lg += 2;
    }
    if (lg < L) {                               // last radix-2 stage: m = 1, unit twiddle
        const int half = N >> 1;
        for (int idx = threadIdx.x; idx < rows * half; idx += blockDim.x) {
            const int row = idx >> (L - 1);
            const int q = idx & (half - 1);
            const T* ar = a + row * N;
            T* br = b + row * N;
            const T x0 = ar[q], x1 = ar[q + half];
            br[q] = cadd(x0, x1);
            br[q + half] = csub(x0, x1);
        }
        __syncthreads();
        T* t = a; a = b; b = t;
    }
    return a;
}

// The same radix-4 Stockham transform with a single buffer: every pass reads all of a
// thread's butterfly inputs into registers, waits at a barrier, then writes the outputs to
// their Stockham positions in the same array.  Needs rows * N / 4 <= MAXB * blockDim.x
// (the caller checks); the result is in `a`, natural order.
template <typename T, int MAXB>
__device__ void stockham4_1buf(T* a, int rows, int N, int L, const T* __restrict__ tw, int sign) {
    const int quarter = N >> 2;
    const int total4 = rows * quarter;
    int s = 1, lg = 0;
    while (lg + 2 <= L) {
        const int m = quarter >> lg;
        T x[MAXB][4];
#pragma unroll
        for (int u = 0; u < MAXB; ++u) {
            const int idx = threadIdx.x + u * blockDim.x;
            if (idx < total4) {
                const int row = idx >> (L - 2), bi = idx & (quarter - 1);
                const int p = bi >> lg, q = bi & (s - 1);
                const T* ar = a + row * N;
#pragma unroll
                for (int k = 0; k < 4; ++k) x[u][k] = ar[q + s * (p + k * m)];
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < MAXB; ++u) {
            const int idx = threadIdx.x + u * blockDim.x;
            if (idx < total4) {
                const int row = idx >> (L - 2), bi = idx & (quarter - 1);
                const int p = bi >> lg, q = bi & (s - 1);
                T* ar = a + row * N;
                const T t0 = cadd(x[u][0], x[u][2]), t1 = csub(x[u][0], x[u][2]);
                const T t2 = cadd(x[u][1], x[u][3]), d = csub(x[u][1], x[u][3]);
                T t3;
                t3.x = -sign * d.y;
                t3.y = sign * d.x;
                const int e = p * s;
                ar[q + s * (4 * p)] = cadd(t0, t2);
                ar[q + s * (4 * p + 1)] = cmul(cadd(t1, t3), tw_full(tw, e, N));
                ar[q + s * (4 * p + 2)] = cmul(csub(t0, t2), tw_full(tw, 2 * e, N));
                ar[q + s * (4 * p + 3)] = cmul(csub(t1, t3), tw_full(tw, 3 * e, N));
            }
        }
        __syncthreads();
        s <<= 2;
        lg += 2;
    }
    if (lg < L) {                               // last radix-2 stage: pairs N/2 apart
        const int half = N >> 1;
        const int total2 = rows * half;
        T y[2 * MAXB][2];
#pragma unroll
        for (int u = 0; u < 2 * MAXB; ++u) {
            const int idx = threadIdx.x + u * blockDim.x;
            if (idx < total2) {
                const T* ar = a + (idx >> (L - 1)) * N;
                const int q = idx & (half - 1);
                y[u][0] = ar[q];
                y[u][1] = ar[q + half];
            }
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 2 * MAXB; ++u) {
            const int idx = threadIdx.x + u * blockDim.x;
            if (idx < total2) {
                T* ar = a + (idx >> (L - 1)) * N;
                const int q = idx & (half - 1);
                ar[q] = cadd(y[u][0], y[u][1]);
                ar[q + half] = csub(y[u][0], y[u][1]);
            }
        }
        __syncthreads();
    }
}

}  // namespace fft
}  // namespace rsim
