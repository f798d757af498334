// ddfocus.cu -- delay-Doppler focusing of the simulated IQ (Section IV.C), for sm_103a.
//
// One thread-block cluster of `cl` CTAs per burst of `burst` consecutive pulses (cl = 8, or
// fewer when the burst or the gate count is below 8); the burst (burst x n_gates complex) is
// spread over the cluster's shared memory and exchanged through distributed shared memory:
//   1. each CTA loads its n_gates / cl gates of every pulse, applies the Doppler centroid
//      correction y_k *= exp(-j 2 pi nu_c k) and the factor (-1)^k that centres the beams
//      (beam f <-> nu_f = (f - burst/2) / burst), and runs the along-track transforms of its
//      gates (radix-4 Stockham, twiddles exp(-j 2 pi r / N));
//   2. after a cluster barrier each CTA gathers its burst / cl beams over all gates from the
//      gates' owners (distributed shared memory), then runs per beam the range transform, the
//      delay phase coefficients exp(+j 2 pi q' s_f / n_gates) (signed range frequency q',
//      range migration s_f of the beam in gates) and the inverse range transform (1 / n_gates);
//   3. output of the focused beams (optional); each CTA sums |Y_f[g]|^2 over its beams (in
//      beam order), and after a barrier the multi-looked waveform
//      W[g] = (1 / burst) sum_f |Y_f[g]|^2 of its gates adds the cl partial sums in rank order
//      (deterministic).
// Beam geometry (flat earth, constant velocity V, reference range R_0 of the burst's centre
// pulse): beam f sees the along-track offset x_f = nu_f lambda R_0 PRF / (2 |V_xy|), whose
// range exceeds the nadir's by x_f^2 / (2 R_0): s_f = x_f^2 / (2 R_0 gate_width).
#include <cooperative_groups.h>

#include "rsim_internal.cuh"
#include "rsim_kernels.h"
#include "fft_smem.cuh"

namespace rsim {

namespace {

using namespace fft;

namespace cg = cooperative_groups;

constexpr int kDdThreads = 256;

__global__ void __launch_bounds__(kDdThreads) dd_focus_kernel(DdArgs a, int lcl, int64_t burst0,
                                                             const float2* __restrict__ iq,
                                                             float2* __restrict__ focused,
                                                             float* __restrict__ multilook) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cluster = cg::this_cluster();
    const int cl = 1 << lcl;
    const int r = (int)cluster.block_rank();                // this CTA's part of the burst
    const int64_t b = burst0 + (int64_t)(blockIdx.x >> lcl);
    const int Nb = a.burst, G = a.n_gates;
    const int lgl = a.log2_g - lcl, lnl = a.log2_b - lcl;
    const int Gl = 1 << lgl, Nl = 1 << lnl;                 // gates, beams per CTA
    float2* tw_b = reinterpret_cast<float2*>(smem_raw);   // exp(-j 2 pi r / Nb), r < Nb/2
    float2* tw_gf = tw_b + (Nb >> 1);                      // exp(-j 2 pi r / G)
    float2* tw_gi = tw_gf + (G >> 1);                      // exp(+j 2 pi r / G)
    float2* cent = tw_gi + (G >> 1);                       // per pulse: centroid factor
    float2* shift = cent + Nb;                              // per beam: s_f / G (hi, lo)
    float* part = reinterpret_cast<float*>(shift + Nb);     // per gate: this CTA's beam sum
    float2* buf0 = reinterpret_cast<float2*>(part + G);
    float2* buf1 = buf0 + Nb * Gl;
    for (int t = threadIdx.x; t < (Nb >> 1); t += blockDim.x) twiddle(t, Nb, -1.0f, tw_b[t]);
    for (int t = threadIdx.x; t < (G >> 1); t += blockDim.x) {
        twiddle(t, G, -1.0f, tw_gf[t]);
        twiddle(t, G, 1.0f, tw_gi[t]);
    }
    // per pulse: exp(-j 2 pi nu_c k) (-1)^k (centroid correction and beam centring);
    // per beam: the migration in range-transform cycles s_f / G as hi + lo floats
    const double r0 = fma(a.r_ref_rate, (double)(a.pulse0 + b * Nb + Nb / 2) * a.inv_prf, a.r_ref0);
    for (int k = threadIdx.x; k < Nb; k += blockDim.x) {
        // nu_c k reduced to [-1/2, 1/2] cycles in FP64, its sine and cosine in FP32 (a few
        // 1e-8 of error; the FP64 pipe runs 1/64 of the FP32 rate)
        double ph = a.nu_c * (double)k;                    // cycles
        ph -= rint(ph);
        float sn, cs;
        sincospif(-2.0f * (float)ph, &sn, &cs);
        const float sg = (k & 1) ? -1.0f : 1.0f;
        cent[k] = make_float2(sg * cs, sg * sn);
        if ((k >> lnl) == r) {       // the migration of this CTA's beams only
            // s_f / G = x_f^2 / (2 R_0 gate_width G) = nu_f^2 R_0 (lambda PRF / (2 V))^2
            // / (2 gate_width G): the constant factor comes from the host (no FP64 divide)
            const double nu = (double)(k - Nb / 2) * (1.0 / (double)Nb);
            const double sfg = nu * nu * r0 * a.mig_c;
            const float hi = (float)sfg;
            shift[k] = make_float2(hi, (float)(sfg - (double)hi));
        }
    }
    __syncthreads();
    // 1. this CTA's gates of every pulse (pulse-major rows), gate-major ([gl][k]) for the
    //    along-track transforms
    const float2* src = iq + b * (int64_t)Nb * G + r * Gl;
    for (int idx = threadIdx.x; idx < Nb * Gl; idx += blockDim.x) {
        const int k = idx >> lgl, gl = idx & (Gl - 1);
        buf0[gl * Nb + k] = cmul(__ldg(src + (int64_t)k * G + gl), cent[k]);
    }
    __syncthreads();
    float2* res = stockham4(buf0, buf1, Gl, Nb, a.log2_b, tw_b, -1);
    float2* other = (res == buf0) ? buf1 : buf0;
    cluster.sync();                  // every CTA's along-track results are in place
    // 2. this CTA's beams as rows ([fl][g]), gathered from the gates' owners (every CTA runs
    //    the same passes, so the result sits in the same buffer in each)
    for (int idx = threadIdx.x; idx < Nl * G; idx += blockDim.x) {
        const int fl = idx >> a.log2_g, g = idx & (G - 1);
        const float2* owner = cluster.map_shared_rank(res, (unsigned)(g >> lgl));
        other[idx] = owner[(g & (Gl - 1)) * Nb + (r << lnl) + fl];
    }
    cluster.sync();                  // all reads of the along-track results are done
    res = stockham4(other, res, Nl, G, a.log2_g, tw_gf, -1);
    other = (res == buf0) ? buf1 : buf0;
    for (int idx = threadIdx.x; idx < Nl * G; idx += blockDim.x) {
        const int fl = idx >> a.log2_g, q = idx & (G - 1);
        const float qs = (float)(q < G / 2 ? q : q - G);   // signed range frequency
        const float2 sh = shift[(r << lnl) + fl];
        // q' s_f / G in cycles: the product with the hi part is split error-free
        const float p = qs * sh.x;
        const float pe = fmaf(qs, sh.x, -p);
        const float ph = (p - rintf(p)) + fmaf(qs, sh.y, pe);
        float sn, cs;
        sincospif(2.0f * ph, &sn, &cs);
        res[idx] = cmul(res[idx], make_float2(cs, sn));
    }
    __syncthreads();
    res = stockham4(res, other, Nl, G, a.log2_g, tw_gi, 1);
    const float inv_g = 1.0f / (float)G;
    // 3. outputs: the focused beams, then the multi-look
    if (focused) {
        float2* dst = focused + b * (int64_t)Nb * G + (int64_t)(r << lnl) * G;
        for (int idx = threadIdx.x; idx < Nl * G; idx += blockDim.x) dst[idx] = cscale(res[idx], inv_g);
    }
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
        float acc = 0.0f;
        for (int fl = 0; fl < Nl; ++fl) {
            const float2 v = res[fl * G + g];
            acc = fmaf(v.x, v.x, fmaf(v.y, v.y, acc));
        }
        part[g] = acc;
    }
    cluster.sync();                  // every CTA's partial sums are in place
    const float norm = inv_g * inv_g / (float)Nb;
    for (int gl = threadIdx.x; gl < Gl; gl += blockDim.x) {
        const int g = (r << lgl) + gl;
        float acc = 0.0f;
        for (int o = 0; o < cl; ++o) acc += cluster.map_shared_rank(part, (unsigned)o)[g];
        multilook[b * G + g] = acc * norm;
    }
    cluster.sync();                  // no CTA leaves while another still reads its memory
}

}  // namespace

// Cluster size (log2) for a burst: up to 8 CTAs (the portable cluster size), as many as both
// the gates and the beams split into
int dd_cluster_log2(int burst, int n_gates) {
    int l = 0;
    while (l < 3 && (burst >> (l + 1)) >= 1 && (n_gates >> (l + 1)) >= 1) ++l;
    return l;
}

size_t dd_focus_smem_bytes(int burst, int n_gates) {
    const int cl = 1 << dd_cluster_log2(burst, n_gates);
    return sizeof(float2) * ((size_t)(burst / 2) + (size_t)n_gates + 2 * (size_t)burst +
                             2 * (size_t)burst * n_gates / cl) +
           sizeof(float) * (size_t)n_gates;
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
    const int lcl = dd_cluster_log2(a.burst, a.n_gates);
    const int64_t per_launch = (int64_t)1 << 28;           // bursts per launch (grid limit)
    for (int64_t b0 = 0; b0 < n_bursts; b0 += per_launch) {
        const int64_t nb = n_bursts - b0 < per_launch ? n_bursts - b0 : per_launch;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(nb << lcl));
        cfg.blockDim = dim3(kDdThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 1u << lcl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        const cudaError_t e = cudaLaunchKernelEx(&cfg, dd_focus_kernel, a, lcl, b0,
                                                 static_cast<const float2*>(iq),
                                                 static_cast<float2*>(focused), multilook);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace rsim
