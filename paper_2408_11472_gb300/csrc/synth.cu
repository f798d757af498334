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

template <typename R>
__global__ void __launch_bounds__(256) synth_kernel(SynthArgs a, int64_t seg0, int gpc,
                                                    const typename Cplx<R>::T* __restrict__ spec,
                                                    typename Cplx<R>::T* __restrict__ iq) {
    using T = typename Cplx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = a.n_doppler;
    T* tw = reinterpret_cast<T*>(smem_raw);
    T* buf0 = tw + (N >> 1);
    T* buf1 = buf0 + 2 * gpc * N;
    const int64_t i = seg0 + blockIdx.x;            // segment between updates i and i + 1
    const int g0 = blockIdx.y * gpc;
    for (int r = threadIdx.x; r < (N >> 1); r += blockDim.x) twiddle(r, N, R(1), tw[r]);
    for (int idx = threadIdx.x; idx < 2 * gpc * N; idx += blockDim.x) {
        const int row = idx / N, k = idx - row * N;
        const int sp = row / gpc, gg = row - sp * gpc;
        const int g = g0 + gg;
        const int64_t si = i + sp - a.update0;
        T v;
        v.x = R(0); v.y = R(0);
        if (g < a.n_gates && si >= 0 && si < a.n_spectra) v = spec[(si * a.n_gates + g) * N + k];
        buf0[idx] = v;
    }
    __syncthreads();
    const T* res = stockham4(buf0, buf1, 2 * gpc, N, a.log2_nd, tw, 1);
    const int64_t p_i = i * a.n_fast;
    const int64_t x_lo = max(p_i, a.pulse0);
    const int64_t x_hi = min(p_i + a.n_fast, a.pulse0 + a.n_pulses);
    const int64_t count = (x_hi - x_lo) * gpc;
    const R inv_nf = R(1) / R(a.n_fast);
    for (int64_t idx = threadIdx.x; idx < count; idx += blockDim.x) {
        const int gg = (int)(idx % gpc);
        const int64_t x = x_lo + idx / gpc;
        const int g = g0 + gg;
        if (g >= a.n_gates) continue;
        const R w0 = window_w(a.window, R(x - p_i) * inv_nf);
        const R w1 = window_w(a.window, R(p_i + a.n_fast - x) * inv_nf);
        const int m0 = (int)((x - p_i) & (N - 1));
        const int m1 = (int)((x - p_i - a.n_fast) & (N - 1));
        const T y = cadd(cscale(res[gg * N + m0], w0), cscale(res[(gpc + gg) * N + m1], w1));
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

int gates_per_cta(int n_gates, int N, bool fp64) {
    const int elems = fp64 ? 512 : 1024;  // complex elements per staged spectrum tile
    int gpc = elems / N;
    if (gpc < 1) gpc = 1;
    if (gpc > 32) gpc = 32;
    if (gpc > n_gates) gpc = n_gates;
    return gpc;
}

}  // namespace

cudaError_t launch_synth(const SynthArgs& a, bool fp64, const void* spectra, void* iq,
                         cudaStream_t stream) {
    const int N = a.n_doppler;
    const int gpc = gates_per_cta(a.n_gates, N, fp64);
    const int64_t seg0 = a.pulse0 / a.n_fast;
    const int64_t seg1 = (a.pulse0 + a.n_pulses - 1) / a.n_fast;
    const dim3 grid((unsigned)(seg1 - seg0 + 1), (unsigned)((a.n_gates + gpc - 1) / gpc));
    const size_t esz = fp64 ? sizeof(double2) : sizeof(float2);
    const size_t smem = esz * ((size_t)(N >> 1) + 4 * (size_t)gpc * N);
    if (smem > 48 * 1024) {
        const cudaError_t e = fp64
            ? cudaFuncSetAttribute(synth_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
            : cudaFuncSetAttribute(synth_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (fp64) synth_kernel<double><<<grid, 256, smem, stream>>>(
        a, seg0, gpc, static_cast<const double2*>(spectra), static_cast<double2*>(iq));
    else synth_kernel<float><<<grid, 256, smem, stream>>>(
        a, seg0, gpc, static_cast<const float2*>(spectra), static_cast<float2*>(iq));
    return cudaGetLastError();
}

cudaError_t launch_synth_backward(const SynthArgs& a, bool fp64, const void* grad_iq,
                                  void* grad_spectra, cudaStream_t stream) {
    const int N = a.n_doppler;
    const int gpc = gates_per_cta(a.n_gates, N, fp64);
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
