// alu_peaks.cu -- throughput microbenchmarks of the arithmetic pipes the scatterer pass uses,
// for the denominators of its roofline (measurement only; not part of the simulation).
//
// Each kernel runs CH independent dependency chains per thread of one instruction kind, on a
// grid of `blocks_per_sm` x SM-count CTAs of 256 threads, so every scheduler has many warps
// and many independent instructions in flight: the rate it sustains is the pipe's throughput.
//   kind 0: FFMA        fma.rn.f32            (1 FP32 lane-operation per thread instruction)
//   kind 1: FFMA2       fma.rn.f32x2          (2 FP32 lane-operations per thread instruction)
//   kind 2: MUFU.EX2    ex2.approx.ftz.f32
//   kind 3: MUFU.SIN    sin.approx.f32        (__sincosf issues a sine and a cosine)
//   kind 4: MUFU.COS    cos.approx.f32
//   kind 5: DFMA        fma.rn.f64
// One thread also reads clock64 and the global nanosecond timer at the start and the end of
// its CTA, which gives the SM clock the kernel ran at; the throughput per SM and clock is
// the lane-operation rate / (SMs x that clock).
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 16;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ float ex2f(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sinf_a(float x) {
    float y;
    asm volatile("sin.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float cosf_a(float x) {
    float y;
    asm volatile("cos.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct Timing {
    unsigned long long clk0, clk1, ns0, ns1;
};

template <int KIND, int CH>
__global__ void __launch_bounds__(kThreads) peak_kernel(int iters, float a, float b, float* sink,
                                                        Timing* tim) {
    unsigned long long c0 = 0, n0 = 0;
    if (threadIdx.x == 0) {
        c0 = clock64();
        n0 = global_ns();
    }
    float acc = 0.0f;
    if (KIND == 5) {
        double x[CH];
#pragma unroll
        for (int i = 0; i < CH; ++i) x[i] = 1e-3 * (threadIdx.x + i);
        const double ad = a, bd = b;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
                for (int i = 0; i < CH; ++i) x[i] = fma(x[i], ad, bd);
            }
        }
#pragma unroll
        for (int i = 0; i < CH; ++i) acc += (float)x[i];
    } else if (KIND == 1) {
        float2 x[CH];
#pragma unroll
        for (int i = 0; i < CH; ++i) x[i] = make_float2(1e-3f * threadIdx.x + i, 2e-3f * i);
        const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
                for (int i = 0; i < CH; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
            }
        }
#pragma unroll
        for (int i = 0; i < CH; ++i) acc += x[i].x + x[i].y;
    } else {
        float x[CH];
#pragma unroll
        for (int i = 0; i < CH; ++i) x[i] = 1e-3f * threadIdx.x + 0.01f * i;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
                for (int i = 0; i < CH; ++i) {
                    if (KIND == 0) x[i] = fmaf(x[i], a, b);
                    if (KIND == 2) x[i] = ex2f(-x[i]);   // stays in [0.5, 1] from [0, 1]
                    if (KIND == 3) x[i] = sinf_a(x[i]);
                    if (KIND == 4) x[i] = cosf_a(x[i]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < CH; ++i) acc += x[i];
    }
    if (acc == 1234.5678f) sink[blockIdx.x] = acc;  // never true; keeps the chains live
    __syncthreads();
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        tim->clk0 = c0;
        tim->ns0 = n0;
        tim->clk1 = clock64();
        tim->ns1 = global_ns();
    }
}

template <int KIND>
cudaError_t launch(int blocks, int iters, float* sink, Timing* tim, cudaStream_t s) {
    constexpr int CH = (KIND == 5) ? 4 : 8;
    peak_kernel<KIND, CH><<<blocks, kThreads, 0, s>>>(iters, 0.999999f, 1e-7f, sink, tim);
    return cudaGetLastError();
}

cudaError_t launch_kind(int kind, int blocks, int iters, float* sink, Timing* tim,
                        cudaStream_t s) {
    switch (kind) {
    case 0: return launch<0>(blocks, iters, sink, tim, s);
    case 1: return launch<1>(blocks, iters, sink, tim, s);
    case 2: return launch<2>(blocks, iters, sink, tim, s);
    case 3: return launch<3>(blocks, iters, sink, tim, s);
    case 4: return launch<4>(blocks, iters, sink, tim, s);
    case 5: return launch<5>(blocks, iters, sink, tim, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// Runs microbenchmark `kind` (0..5, above) on the current device: one warm-up launch, then
// `reps` timed launches (CUDA events on the legacy default stream).  Outputs: lane-operations
// per second over the whole GPU (best launch), the SM clock the kernel ran at (MHz, from
// clock64 against the global timer over CTA 0), lane-operations per SM per clock, and the
// SM count.  `sink` and `tim` are device buffers of >= blocks_per_sm * SMs floats and
// 32 bytes.  Returns 0, or a cudaError_t value.
extern "C" int alu_peak_run(int kind, int blocks_per_sm, int iters, int reps, float* sink,
                            void* tim, double* ops_per_s, double* sm_mhz, double* ops_per_clk_sm,
                            int* n_sms) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    const int blocks = blocks_per_sm * sms;
    Timing* t = static_cast<Timing*>(tim);
    cudaEvent_t a, b;
    if ((e = cudaEventCreate(&a)) != cudaSuccess) return (int)e;
    if ((e = cudaEventCreate(&b)) != cudaSuccess) return (int)e;
    e = launch_kind(kind, blocks, iters, sink, t, 0);
    float best = 1e30f;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        cudaEventRecord(a, 0);
        e = launch_kind(kind, blocks, iters, sink, t, 0);
        cudaEventRecord(b, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (ms < best) best = ms;
    }
    Timing h{};
    if (e == cudaSuccess) e = cudaMemcpy(&h, t, sizeof(h), cudaMemcpyDeviceToHost);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return (int)e;
    const int ch = (kind == 5) ? 4 : 8;
    const double lanes = (kind == 1) ? 2.0 : 1.0;
    const double ops = (double)blocks * kThreads * (double)iters * kUnroll * ch * lanes;
    *ops_per_s = ops / (best * 1e-3);
    const double mhz = (h.ns1 > h.ns0) ? (double)(h.clk1 - h.clk0) / (double)(h.ns1 - h.ns0) * 1e3
                                       : 0.0;
    *sm_mhz = mhz;
    *ops_per_clk_sm = (mhz > 0) ? *ops_per_s / ((double)sms * mhz * 1e6) : 0.0;
    *n_sms = sms;
    return 0;
}
