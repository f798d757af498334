// ddfocus.cu -- delay-Doppler focusing of the simulated IQ (Section IV.C), for sm_103a.
//
// One CTA per burst of `burst` consecutive pulses, the whole burst held in shared memory
// (burst x n_gates complex, two buffers):
//   1. Doppler centroid correction  y_k *= exp(-j 2 pi nu_c k), and the factor (-1)^k that
//      centres the beams (beam f <-> nu_f = (f - burst/2) / burst);
//   2. along-track transform per gate (radix-4 Stockham, twiddles exp(-j 2 pi r / N));
//   3. range transform per beam, the delay phase coefficients exp(+j 2 pi q' s_f / n_gates)
//      (signed range frequency q', range migration s_f of the beam in gates), inverse range
//      transform scaled by 1 / n_gates;
//   4. output of the focused beams (optional) and the multi-looked waveform
//      W[g] = (1 / burst) sum_f |Y_f[g]|^2, summed over f in order (deterministic).
// Beam geometry (flat earth, constant velocity V, reference range R_0 of the burst's centre
// pulse): beam f sees the along-track offset x_f = nu_f lambda R_0 PRF / (2 |V_xy|), whose
// range exceeds the nadir's by x_f^2 / (2 R_0): s_f = x_f^2 / (2 R_0 gate_width).
#include "rsim_internal.cuh"
#include "rsim_kernels.h"
#include "fft_smem.cuh"

namespace rsim {

namespace {

using namespace fft;

__global__ void __launch_bounds__(512) dd_focus_kernel(DdArgs a, const float2* __restrict__ iq,
                                                      float2* __restrict__ focused,
                                                      float* __restrict__ multilook) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Nb = a.burst, G = a.n_gates;
    float2* tw_b = reinterpret_cast<float2*>(smem_raw);   // exp(-j 2 pi r / Nb), r < Nb/2
    float2* tw_gf = tw_b + (Nb >> 1);                      // exp(-j 2 pi r / G)
    float2* tw_gi = tw_gf + (G >> 1);                      // exp(+j 2 pi r / G)
    float2* cent = tw_gi + (G >> 1);                       // per pulse: centroid factor
    float2* shift = cent + Nb;                              // per beam: s_f / G (hi, lo)
    float2* buf0 = shift + Nb;
    float2* buf1 = buf0 + Nb * G;
    const int64_t b = blockIdx.x;
    for (int r = threadIdx.x; r < (Nb >> 1); r += blockDim.x) twiddle(r, Nb, -1.0f, tw_b[r]);
    for (int r = threadIdx.x; r < (G >> 1); r += blockDim.x) {
        twiddle(r, G, -1.0f, tw_gf[r]);
        twiddle(r, G, 1.0f, tw_gi[r]);
    }
    // per pulse: exp(-j 2 pi nu_c k) (-1)^k (centroid correction and beam centring);
    // per beam: the migration in range-transform cycles s_f / G as hi + lo floats
    const double r0 = fma(a.r_ref_rate, (double)(a.pulse0 + b * Nb + Nb / 2) * a.inv_prf, a.r_ref0);
    for (int k = threadIdx.x; k < Nb; k += blockDim.x) {
        double ph = a.nu_c * (double)k;                    // cycles
        ph -= rint(ph);
        double s, c;
        sincospi(-2.0 * ph, &s, &c);
        const float sg = (k & 1) ? -1.0f : 1.0f;
        cent[k] = make_float2(sg * (float)c, sg * (float)s);
        const double nu = (double)(k - Nb / 2) / (double)Nb;
        const double x = a.vh > 0.0 ? nu * a.lambda * r0 * a.prf / (2.0 * a.vh) : 0.0;
        const double sfg = x * x / (2.0 * r0 * a.gate_width) / (double)G;
        const float hi = (float)sfg;
        shift[k] = make_float2(hi, (float)(sfg - (double)hi));
    }
    __syncthreads();
    // 1. load the burst (pulse-major rows), apply the per-pulse factor, store gate-major
    //    ([g][k]) for the along-track transforms
    const float2* src = iq + b * (int64_t)Nb * G;
    for (int idx = threadIdx.x; idx < Nb * G; idx += blockDim.x) {
        const int k = idx / G, g = idx - k * G;
        buf0[g * Nb + k] = cmul(__ldg(src + idx), cent[k]);
    }
    __syncthreads();
    // 2. along-track transforms: rows = gates
    float2* res = stockham4(buf0, buf1, G, Nb, a.log2_b, tw_b, -1);
    float2* other = (res == buf0) ? buf1 : buf0;
    // 3. beams as rows ([f][g]) for the range transforms
    for (int idx = threadIdx.x; idx < Nb * G; idx += blockDim.x) {
        const int f = idx / G, g = idx - f * G;
        other[idx] = res[g * Nb + f];
    }
    __syncthreads();
    res = stockham4(other, res, Nb, G, a.log2_g, tw_gf, -1);
    other = (res == buf0) ? buf1 : buf0;
    for (int idx = threadIdx.x; idx < Nb * G; idx += blockDim.x) {
        const int f = idx / G, q = idx - f * G;
        const float qs = (float)(q < G / 2 ? q : q - G);   // signed range frequency
        const float2 sh = shift[f];
        // q' s_f / G in cycles: the product with the hi part is split error-free
        const float p = qs * sh.x;
        const float pe = fmaf(qs, sh.x, -p);
        const float ph = (p - rintf(p)) + fmaf(qs, sh.y, pe);
        float s, c;
        sincospif(2.0f * ph, &s, &c);
        res[idx] = cmul(res[idx], make_float2(c, s));
    }
    __syncthreads();
    res = stockham4(res, other, Nb, G, a.log2_g, tw_gi, 1);
    const float inv_g = 1.0f / (float)G;
    // 4. outputs
    if (focused) {
        float2* dst = focused + b * (int64_t)Nb * G;
        for (int idx = threadIdx.x; idx < Nb * G; idx += blockDim.x) dst[idx] = cscale(res[idx], inv_g);
    }
    const float norm = inv_g * inv_g / (float)Nb;
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
        float acc = 0.0f;
        for (int f = 0; f < Nb; ++f) {
            const float2 v = res[f * G + g];
            acc = fmaf(v.x, v.x, fmaf(v.y, v.y, acc));
        }
        multilook[b * G + g] = acc * norm;
    }
}

}  // namespace

size_t dd_focus_smem_bytes(int burst, int n_gates) {
    return sizeof(float2) * ((size_t)(burst / 2) + (size_t)n_gates + 2 * (size_t)burst +
                             2 * (size_t)burst * n_gates);
}

cudaError_t launch_dd_focus(const DdArgs& a, int64_t n_bursts, const void* iq, void* focused,
                            float* multilook, cudaStream_t stream) {
    const size_t smem = dd_focus_smem_bytes(a.burst, a.n_gates);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(dd_focus_kernel,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem);
        if (e != cudaSuccess) return e;
    }
    dd_focus_kernel<<<(unsigned)n_bursts, 512, smem, stream>>>(
        a, static_cast<const float2*>(iq), static_cast<float2*>(focused), multilook);
    return cudaGetLastError();
}

}  // namespace rsim
