// synth.cu -- fast-mode post-processing (Section III.B, steps 2-4, with Eq. (1)) and
// its adjoint, for sm_103a.
//
// Forward: one CTA per (segment i, block of gates).  It stages the spectra of updates i
// and i+1 for its gates in shared memory, runs the n_doppler-point inverse transforms
// there (radix-4 Stockham autosort, unnormalised, twiddles exp(+j 2 pi r / N)), and
// writes the blended pulses x in [p_i, p_{i+1}) directly:
//   Y[x, g] = W(u) s_i[g, (x - p_i) mod N] + W(1 - u) s_{i+1}[g, (x - p_{i+1}) mod N],
//   u = (x - p_i) / n_fast.
// Each spectrum is transformed by the two CTAs that use it; the transforms are tiny next to
// the scatterer pass and this keeps every CTA independent (no inter-CTA traffic).
// Adjoint: one CTA per (spectrum, block of gates): fold dL/dY of the pulses within
// n_fast of p_s onto the N periodic offsets (windowed, fixed x order), then the forward
// transform (twiddles exp(-j 2 pi r / N)).
#include "rsim_internal.cuh"
#include "rsim_kernels.h"
#include "fft_smem.cuh"

namespace rsim {

namespace {

using namespace fft;

// Blend window W(d), d in [0, 1]: 0 sqrt(1 - d) (Eq. 1), 1 cos(pi d / 2), 2 1 - d.
__device__ __forceinline__ float window_w(int w, float d) {
    if (d >= 1.0f) return 0.0f;
    if (w == 0) return sqrtf(1.0f - d);
    if (w == 1) return cospif(0.5f * d);
    return 1.0f - d;
}
__device__ __forceinline__ double window_w(int w, double d) {
    if (d >= 1.0) return 0.0;
    if (w == 0) return sqrt(1.0 - d);
    if (w == 1) return cospi(0.5 * d);
    return 1.0 - d;
}

// Window table size: W(d / n_fast) for d = 0 .. n_fast is tabulated per CTA when
// n_fast < kWinTable (the blend then reads both weights of a pulse from shared memory).
constexpr int kWinTable = 1024;
// Forward synthesis CTA: kSynthThreads threads stage at most 2048 complex elements
// (2 spectra x gates per CTA x n_doppler), kSynthStage per thread.
constexpr int kSynthThreads = 256;
constexpr int kSynthStage = 8;

template <typename R>
__global__ void __launch_bounds__(kSynthThreads) synth_kernel(SynthArgs a, int64_t seg0, int lg_gpc,
                                                    const typename Cplx<R>::T* __restrict__ spec,
                                                    typename Cplx<R>::T* __restrict__ iq) {
    using T = typename Cplx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.n_doppler, L = a.log2_nd;
    const int gpc = 1 << lg_gpc;                    // gates per CTA (a power of two <= 32)
    const int NS = N + 1;                           // odd row stride: the blend reads columns
    T* tw = reinterpret_cast<T*>(smem_raw);
    T* buf0 = tw + (N >> 1);
    T* buf1 = buf0 + 2 * gpc * NS;
    R* wt = reinterpret_cast<R*>(buf1 + 2 * gpc * NS);
    const int64_t i = seg0 + blockIdx.x;            // segment between updates i and i + 1
    const int g0 = blockIdx.y * gpc;
    // Rows of buf0: [spectrum i | spectrum i + 1] x [gate g0 .. g0 + gpc), N bins each:
    // at most kSynthStage elements per thread (the launch guarantees it), all loaded into
    // registers before any is stored so that the loads are in flight together.
    const int total = (2 * gpc) << L;
    T v[kSynthStage];
#pragma unroll
    for (int u = 0; u < kSynthStage; ++u) {
        const int idx = threadIdx.x + u * kSynthThreads;
        const int row = idx >> L, k = idx & (N - 1);
        const int g = g0 + (row & (gpc - 1));
        const int64_t si = i + (row >> lg_gpc) - a.update0;
        v[u].x = R(0); v[u].y = R(0);
        if (idx < total && g < a.n_gates && si >= 0 && si < a.n_spectra)
            v[u] = spec[(si * a.n_gates + g) * N + k];
    }
    const R inv_nf = R(1) / R(a.n_fast);
    const bool table = a.n_fast < kWinTable;
    for (int r = threadIdx.x; r < (N >> 1); r += blockDim.x) twiddle(r, N, R(1), tw[r]);
    if (table)
        for (int d = threadIdx.x; d <= a.n_fast; d += blockDim.x) wt[d] = window_w(a.window, R(d) * inv_nf);
#pragma unroll
    for (int u = 0; u < kSynthStage; ++u) {
        const int idx = threadIdx.x + u * kSynthThreads;
        if (idx < total) buf0[(idx >> L) * NS + (idx & (N - 1))] = v[u];
    }
    __syncthreads();
    const T* res = stockham4(buf0, buf1, 2 * gpc, N, L, tw, 1, NS);
    const int64_t p_i = i * a.n_fast;
    const int64_t x_lo = max(p_i, a.pulse0);
    const int64_t x_hi = min(p_i + a.n_fast, a.pulse0 + a.n_pulses);
    // Thread -> (gate gg, pulse offset): gpc consecutive threads write one pulse's gates.
    const int gg = threadIdx.x & (gpc - 1);
    const int g = g0 + gg;
    if (g >= a.n_gates) return;
    const T* r0 = res + gg * NS;
    const T* r1 = res + (gpc + gg) * NS;
    const int xs = blockDim.x >> lg_gpc;
    for (int64_t x = x_lo + (threadIdx.x >> lg_gpc); x < x_hi; x += xs) {
        const int d = (int)(x - p_i);               // 0 <= d < n_fast
        const R w0 = table ? wt[d] : window_w(a.window, R(d) * inv_nf);
        const R w1 = table ? wt[a.n_fast - d] : window_w(a.window, R(a.n_fast - d) * inv_nf);
        const T y = cadd(cscale(r0[d & (N - 1)], w0), cscale(r1[(d - a.n_fast) & (N - 1)], w1));
        iq[(x - a.pulse0) * a.n_gates + g] = y;
    }
}

template <typename R>
__global__ void __launch_bounds__(256) synth_backward_kernel(
    SynthArgs a, int gpc, const typename Cplx<R>::T* __restrict__ gy,
    typename Cplx<R>::T* __restrict__ gspec) {
    using T = typename Cplx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.n_doppler;
    T* tw = reinterpret_cast<T*>(smem_raw);
    T* buf0 = tw + (N >> 1);
    T* buf1 = buf0 + gpc * N;
    const int s = blockIdx.x;
    const int64_t p_s = (a.update0 + s) * (int64_t)a.n_fast;
    const int g0 = blockIdx.y * gpc;
    for (int r = threadIdx.x; r < (N >> 1); r += blockDim.x) twiddle(r, N, R(-1), tw[r]);
    const int64_t x_lo = max(p_s - a.n_fast + 1, a.pulse0);
    const int64_t x_hi = min(p_s + a.n_fast - 1, a.pulse0 + a.n_pulses - 1);
    const R inv_nf = R(1) / R(a.n_fast);
    for (int idx = threadIdx.x; idx < gpc * N; idx += blockDim.x) {
        const int m = idx / gpc, gg = idx - m * gpc;
        const int g = g0 + gg;
        T acc;
        acc.x = R(0); acc.y = R(0);
        if (g < a.n_gates && x_lo <= x_hi) {
            int64_t x = x_lo + ((m - (x_lo - p_s)) & (N - 1));
            for (; x <= x_hi; x += N) {
                const int64_t dist = x >= p_s ? x - p_s : p_s - x;
                const R w = window_w(a.window, R(dist) * inv_nf);
                acc = cadd(acc, cscale(gy[(x - a.pulse0) * a.n_gates + g], w));
            }
        }
        buf0[gg * N + m] = acc;
    }
    __syncthreads();
    const T* res = stockham4(buf0, buf1, gpc, N, a.log2_nd, tw, -1);
    for (int idx = threadIdx.x; idx < gpc * N; idx += blockDim.x) {
        const int gg = idx / N, k = idx - gg * N;
        const int g = g0 + gg;
        if (g < a.n_gates) gspec[((int64_t)s * a.n_gates + g) * N + k] = res[idx];
    }
}

// Gates per CTA: a power of two (so it divides the 256 threads), at most 32, about
// 1024 (FP32) or 512 (FP64) staged complex elements per spectrum, and no more than the
// smallest power of two >= n_gates.
int lg_gates_per_cta(int n_gates, int N, bool fp64) {
    const int elems = fp64 ? 512 : 1024;  // complex elements per staged spectrum tile
    int lg = 0;
    while (lg < 5 && (2 << lg) * N <= elems && (1 << lg) < n_gates) ++lg;
    return lg;
}

}  // namespace

cudaError_t launch_synth(const SynthArgs& a, bool fp64, const void* spectra, void* iq,
                         cudaStream_t stream) {
    const int N = a.n_doppler;
    const int lg_gpc = lg_gates_per_cta(a.n_gates, N, fp64);
    const int gpc = 1 << lg_gpc;
    const int64_t seg0 = a.pulse0 / a.n_fast;
    const int64_t seg1 = (a.pulse0 + a.n_pulses - 1) / a.n_fast;
    const dim3 grid((unsigned)(seg1 - seg0 + 1), (unsigned)((a.n_gates + gpc - 1) / gpc));
    const size_t esz = fp64 ? sizeof(double2) : sizeof(float2);
    const size_t win = a.n_fast < kWinTable ? (size_t)(a.n_fast + 1) * (esz / 2) : 0;
    const size_t smem = esz * ((size_t)(N >> 1) + 4 * (size_t)gpc * (N + 1)) + win;
    if (smem > 48 * 1024) {
        const cudaError_t e = fp64
            ? cudaFuncSetAttribute(synth_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
            : cudaFuncSetAttribute(synth_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (((2 * gpc) << a.log2_nd) > kSynthThreads * kSynthStage) return cudaErrorInvalidValue;
    if (fp64) synth_kernel<double><<<grid, kSynthThreads, smem, stream>>>(
        a, seg0, lg_gpc, static_cast<const double2*>(spectra), static_cast<double2*>(iq));
    else synth_kernel<float><<<grid, kSynthThreads, smem, stream>>>(
        a, seg0, lg_gpc, static_cast<const float2*>(spectra), static_cast<float2*>(iq));
    return cudaGetLastError();
}

cudaError_t launch_synth_backward(const SynthArgs& a, bool fp64, const void* grad_iq,
                                  void* grad_spectra, cudaStream_t stream) {
    const int N = a.n_doppler;
    const int gpc = 1 << lg_gates_per_cta(a.n_gates, N, fp64);
    const dim3 grid((unsigned)a.n_spectra, (unsigned)((a.n_gates + gpc - 1) / gpc));
    const size_t esz = fp64 ? sizeof(double2) : sizeof(float2);
    const size_t smem = esz * ((size_t)(N >> 1) + 2 * (size_t)gpc * N);
    if (smem > 48 * 1024) {
        const cudaError_t e = fp64
            ? cudaFuncSetAttribute(synth_backward_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
            : cudaFuncSetAttribute(synth_backward_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (fp64) synth_backward_kernel<double><<<grid, 256, smem, stream>>>(
        a, gpc, static_cast<const double2*>(grad_iq), static_cast<double2*>(grad_spectra));
    else synth_backward_kernel<float><<<grid, 256, smem, stream>>>(
        a, gpc, static_cast<const float2*>(grad_iq), static_cast<float2*>(grad_spectra));
    return cudaGetLastError();
}

}  // namespace rsim
