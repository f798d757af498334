// accumulate.cu -- scatterer-streaming summation kernels for sm_103a.
//
//  * accumulate_*: regular mode (Section II.A, one sample per pulse, cells = gates) and
//    the fast-mode Doppler pass (Algorithm 1 of Section III.B, one sample per update,
//    cells = gate x Doppler bin).  Each CTA owns 512 consecutive scatterers (128 threads x 4) held in
//    registers for ALL of its samples, so the 28 B of input per scatterer are read from
//    HBM once per launch however many samples there are.  Per (CTA, sample) FP64 constants
//    of a CTA reference point are computed by one thread per sample into shared memory.
//    Contributions leave a warp as merged runs and are added with 64-bit integer atomics
//    into a fixed-point workspace (exact, order-independent sums).
//  * finalize: fixed-point workspace -> complex output (+=).
//  * cells: per-scatterer gate / bin decisions (same arithmetic as accumulate).
//  * backward_*: adjoint gather -- per scatterer, recompute C and its z-derivative at every
//    sample and gather dL/dT of its cell; no atomics (one thread owns each scatterer).
#include "rsim_internal.cuh"
#include "rsim_kernels.h"

namespace rsim {

namespace {

// Load kItems consecutive floats starting at base (vectorised when all arrays are 16-byte
// aligned and the items are in range; base is a multiple of kItems).
__device__ __forceinline__ void load_items(const float* __restrict__ p, int64_t base, int64_t n,
                                           bool vec, float (&v)[kItems]) {
    if (vec && base + kItems <= n) {
        if (kItems % 4 == 0) {
#pragma unroll
            for (int j = 0; j < kItems / 4; ++j) {
                const float4 q = __ldcs(reinterpret_cast<const float4*>(p + base) + j);
                v[4 * j + 0] = q.x; v[4 * j + 1] = q.y; v[4 * j + 2] = q.z; v[4 * j + 3] = q.w;
            }
        } else if (kItems == 2) {
            const float2 q = __ldcs(reinterpret_cast<const float2*>(p + base));
            v[0] = q.x; v[kItems - 1] = q.y;
        } else {
            v[0] = __ldcs(p + base);
        }
    } else {
#pragma unroll
        for (int q = 0; q < kItems; ++q) v[q] = (base + q < n) ? __ldcs(p + base + q) : 0.0f;
    }
}

struct Raw {
    float x[kItems], y[kItems], z[kItems], vx[kItems], vy[kItems], vz[kItems], s[kItems];
};

__device__ __forceinline__ void load_raw(const Scat& sc, int64_t base, Raw& r) {
    const bool vec = sc.vec4 != 0;
    load_items(sc.x, base, sc.n, vec, r.x);
    load_items(sc.y, base, sc.n, vec, r.y);
    load_items(sc.z, base, sc.n, vec, r.z);
    load_items(sc.vx, base, sc.n, vec, r.vx);
    load_items(sc.vy, base, sc.n, vec, r.vy);
    load_items(sc.vz, base, sc.n, vec, r.vz);
    load_items(sc.nrcs, base, sc.n, vec, r.s);
}

// Reference point of the CTA's chunk: the (x, y) of its middle scatterer.
__device__ __forceinline__ void chunk_ref(const Scat& sc, int64_t chunk0, float& cx, float& cy) {
    const int64_t mid = min(chunk0 + (int64_t)(kChunk / 2), sc.n - 1);
    cx = __ldg(sc.x + mid);
    cy = __ldg(sc.y + mid);
}

__device__ __forceinline__ void items_split(const Model& m, const Raw& r, float cx, float cy,
                                            int64_t base, int64_t n, ItemF (&it)[kItems]) {
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        it[q].lx0 = r.x[q] - cx;
        it[q].ly0 = r.y[q] - cy;
        it[q].z = r.z[q];
        it[q].vx = r.vx[q];
        it[q].vy = r.vy[q];
        it[q].vz = r.vz[q];
        it[q].amp0 = sqrtf(r.s[q] * (float)m.area);
        const float epv = fmaf(m.ep[0], r.vx[q], fmaf(m.ep[1], r.vy[q], m.ep[2] * r.vz[q]));
        const float vv = fmaf(r.vx[q], r.vx[q], fmaf(r.vy[q], r.vy[q], r.vz[q] * r.vz[q]));
        it[q].c1 = m.dt_f * fmaf(-m.hdt_f, vv, epv);
        it[q].ok = (base + q < n) ? 1 : 0;
    }
}

__device__ __forceinline__ void items_fp64(const Model& m, const Raw& r, ItemD (&it)[kItems]) {
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        it[q].x = r.x[q];
        it[q].y = r.y[q];
        it[q].z = r.z[q];
        it[q].vx = r.vx[q];
        it[q].vy = r.vy[q];
        it[q].vz = r.vz[q];
        it[q].amp0 = sqrt((double)r.s[q] * m.area);
    }
}

__device__ __forceinline__ int64_t sample_pulse(const Schedule& sch, int s) {
    return sch.pulse_base + (int64_t)s * sch.pulse_stride;
}

}  // namespace

// ------------------------------------------------------------------------------- forward
template <bool DOPPLER>
__global__ void __launch_bounds__(kThreads, kMinBlocks) accumulate_split_kernel(
    Model m, Schedule sch, Scat sc, unsigned long long* __restrict__ ws) {
    __shared__ SplitConst tab[kTab];
    __shared__ Fp64Const tab64[kTab];
    constexpr unsigned kFull = 0xffffffffu;
    const int64_t chunk0 = (int64_t)blockIdx.x * kChunk;
    const int64_t base = chunk0 + (int64_t)threadIdx.x * kItems;
    float cx, cy;
    chunk_ref(sc, chunk0, cx, cy);
    ItemF it[kItems];
    {
        Raw r;
        load_raw(sc, base, r);
        items_split(m, r, cx, cy, base, sc.n, it);
    }
    const int cells = m.n_gates * m.n_doppler;
    const int s_begin = blockIdx.y * sch.samples_per_group;
    const int s_end = min(sch.n_samples, s_begin + sch.samples_per_group);
    for (int sb = s_begin; sb < s_end; sb += kTab) {
        const int nb = min(kTab, s_end - sb);
        __syncthreads();
        if (threadIdx.x < nb) {
            const int64_t pulse = sample_pulse(sch, sb + threadIdx.x);
            tab[threadIdx.x] = make_split_const(m, pulse, cx, cy);
            tab64[threadIdx.x] = make_fp64_const(m, pulse);
        }
        __syncthreads();
        for (int j = 0; j < nb; ++j) {
            const int s = sb + j;
            const SampleF k = load_sample(tab[j]);
            int key[kItems];
            float re[kItems], im[kItems];
            int fl = 0;
#pragma unroll
            for (int q = 0; q < kItems; ++q) {
                int f;
                key[q] = eval_split<DOPPLER, false, false>(m, k, it[q], re[q], im[q], f);
                fl |= f << (2 * q);
            }
            // rare: items near a cell edge or far off nadir, re-evaluated exactly
            if (__any_sync(kFull, fl != 0)) {
#pragma unroll
                for (int q = 0; q < kItems; ++q) {
                    if ((fl >> (2 * q)) & 3) {
                        int f;
                        const bool in = it[q].ok != 0;  // padding items read nothing
                        key[q] = eval_split<DOPPLER, true, false>(
                            m, k, it[q], re[q], im[q], f, &tab64[j],
                            in ? __ldg(sc.x + base + q) : 0.0f, in ? __ldg(sc.y + base + q) : 0.0f);
                    }
                }
            }
            warp_reduce_emit<float, kItems>(key, re, im, ws + (int64_t)s * cells * 2);
        }
    }
}

template <bool DOPPLER>
__global__ void __launch_bounds__(kThreads) accumulate_fp64_kernel(
    Model m, Schedule sch, Scat sc, unsigned long long* __restrict__ ws) {
    __shared__ Fp64Const tab[kTab];
    const int64_t chunk0 = (int64_t)blockIdx.x * kChunk;
    const int64_t base = chunk0 + (int64_t)threadIdx.x * kItems;
    ItemD it[kItems];
    {
        Raw r;
        load_raw(sc, base, r);
        items_fp64(m, r, it);
    }
    const int cells = m.n_gates * m.n_doppler;
    const int s_begin = blockIdx.y * sch.samples_per_group;
    const int s_end = min(sch.n_samples, s_begin + sch.samples_per_group);
    for (int sb = s_begin; sb < s_end; sb += kTab) {
        const int nb = min(kTab, s_end - sb);
        __syncthreads();
        if (threadIdx.x < nb) tab[threadIdx.x] = make_fp64_const(m, sample_pulse(sch, sb + threadIdx.x));
        __syncthreads();
        for (int j = 0; j < nb; ++j) {
            const int s = sb + j;
            const Fp64Const& k = tab[j];
            int key[kItems];
            double re[kItems], im[kItems];
#pragma unroll
            for (int q = 0; q < kItems; ++q)
                key[q] = eval_fp64<DOPPLER, false>(m, k, it[q], base + q, sc.n, re[q], im[q], nullptr);
            warp_reduce_emit<double, kItems>(key, re, im, ws + (int64_t)s * cells * 2);
        }
    }
}

// Fixed point (q 2^-32) to float without the FP64 pipe: |q| = hi 2^32 + lo, both unsigned
// 32-bit, so small values keep their full relative precision.
__device__ __forceinline__ float fixed_to_f32(long long q) {
    const unsigned long long a = (unsigned long long)(q < 0 ? -q : q);
    const unsigned hi = (unsigned)(a >> 32);
    const unsigned lo = (unsigned)(a & 0xffffffffull);
    const float v = fmaf(__uint2float_rn(lo), 2.3283064365386963e-10f, __uint2float_rn(hi));
    return q < 0 ? -v : v;
}

template <typename T>
__device__ __forceinline__ T fixed_to(long long q);
template <>
__device__ __forceinline__ float fixed_to<float>(long long q) { return fixed_to_f32(q); }
template <>
__device__ __forceinline__ double fixed_to<double>(long long q) { return (double)q * (1.0 / kFixScale); }

template <typename T>
__global__ void finalize_kernel(const long long* __restrict__ ws, T* __restrict__ out,
                                int64_t n_vals) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_vals; i += stride) {
        out[i] += fixed_to<T>(__ldcs(ws + i));
    }
}

// ------------------------------------------------------------------------------- cells
__global__ void __launch_bounds__(kThreads) cells_kernel(Model m, int64_t pulse, int fp64,
                                                         int doppler, Scat sc, int32_t* gate,
                                                         int32_t* bin, double* gcoord,
                                                         double* bcoord) {
    const int64_t chunk0 = (int64_t)blockIdx.x * kChunk;
    const int64_t base = chunk0 + (int64_t)threadIdx.x * kItems;
    Raw r;
    load_raw(sc, base, r);
    int key[kItems], g[kItems];
    double gc[kItems], bc[kItems];
    if (!fp64) {
        float cx, cy;
        chunk_ref(sc, chunk0, cx, cy);
        ItemF it[kItems];
        items_split(m, r, cx, cy, base, sc.n, it);
        const SampleF k = load_sample(make_split_const(m, pulse, cx, cy));
        const Fp64Const k64 = make_fp64_const(m, pulse);
#pragma unroll
        for (int q = 0; q < kItems; ++q) {
            float re, im;
            int f;
            key[q] = doppler
                ? eval_split<true, true, false>(m, k, it[q], re, im, f, &k64, r.x[q], r.y[q], nullptr, &g[q], &gc[q], &bc[q])
                : eval_split<false, true, false>(m, k, it[q], re, im, f, &k64, r.x[q], r.y[q], nullptr, &g[q], &gc[q], &bc[q]);
        }
    } else {
        ItemD it[kItems];
        items_fp64(m, r, it);
        const Fp64Const k = make_fp64_const(m, pulse);
#pragma unroll
        for (int q = 0; q < kItems; ++q) {
            double re, im;
            key[q] = doppler ? eval_fp64<true, false>(m, k, it[q], base + q, sc.n, re, im, nullptr, &g[q], &gc[q], &bc[q])
                             : eval_fp64<false, false>(m, k, it[q], base + q, sc.n, re, im, nullptr, &g[q], &gc[q], &bc[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        const int64_t n = base + q;
        if (n >= sc.n) continue;
        if (gate) gate[n] = g[q];
        if (bin) bin[n] = doppler ? ((int)floor(bc[q]) & (m.n_doppler - 1)) : 0;
        if (gcoord) gcoord[n] = gc[q];
        if (bcoord) bcoord[n] = bc[q];
        (void)key[q];
    }
}

// ------------------------------------------------------------------------------- backward
template <bool DOPPLER>
__global__ void __launch_bounds__(kThreads) backward_split_kernel(
    Model m, Schedule sch, Scat sc, const float2* __restrict__ G, float* __restrict__ grad_z,
    float* __restrict__ grad_nrcs) {
    __shared__ SplitConst tab[kTab];
    __shared__ Fp64Const tab64[kTab];
    const int64_t chunk0 = (int64_t)blockIdx.x * kChunk;
    const int64_t base = chunk0 + (int64_t)threadIdx.x * kItems;
    float cx, cy;
    chunk_ref(sc, chunk0, cx, cy);
    ItemF it[kItems];
    float sig[kItems], xo[kItems], yo[kItems];
    {
        Raw r;
        load_raw(sc, base, r);
        items_split(m, r, cx, cy, base, sc.n, it);
#pragma unroll
        for (int q = 0; q < kItems; ++q) { sig[q] = r.s[q]; xo[q] = r.x[q]; yo[q] = r.y[q]; }
    }
    float gz[kItems], gs[kItems];
#pragma unroll
    for (int q = 0; q < kItems; ++q) { gz[q] = 0.f; gs[q] = 0.f; }
    const int cells = m.n_gates * m.n_doppler;
    for (int sb = 0; sb < sch.n_samples; sb += kTab) {
        const int nb = min(kTab, sch.n_samples - sb);
        __syncthreads();
        if (threadIdx.x < nb) {
            const int64_t pulse = sample_pulse(sch, sb + threadIdx.x);
            tab[threadIdx.x] = make_split_const(m, pulse, cx, cy);
            tab64[threadIdx.x] = make_fp64_const(m, pulse);
        }
        __syncthreads();
        for (int j = 0; j < nb; ++j) {
            const int s = sb + j;
            const SampleF k = load_sample(tab[j]);
#pragma unroll
            for (int q = 0; q < kItems; ++q) {
                float re, im;
                int f;
                DerivF dv;
                const int key = eval_split<DOPPLER, true, true>(m, k, it[q], re, im, f, &tab64[j],
                                                                 xo[q], yo[q], &dv);
                if (key >= 0) {
                    const float2 g = __ldg(G + (int64_t)s * cells + key);
                    const float cr = fmaf(g.x, re, g.y * im);   // Re(conj(G) C)
                    const float ci = fmaf(g.x, im, -g.y * re);  // Im(conj(G) C)
                    gz[q] = fmaf(cr, dv.dlna, fmaf(-ci, dv.dphi, gz[q]));
                    gs[q] += cr;
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        const int64_t n = base + q;
        if (n >= sc.n) continue;
        if (grad_z) grad_z[n] += gz[q];
        if (grad_nrcs && sig[q] > 0.f) grad_nrcs[n] += gs[q] / (2.0f * sig[q]);
    }
}

template <bool DOPPLER>
__global__ void __launch_bounds__(kThreads) backward_fp64_kernel(
    Model m, Schedule sch, Scat sc, const double2* __restrict__ G, float* __restrict__ grad_z,
    float* __restrict__ grad_nrcs) {
    __shared__ Fp64Const tab[kTab];
    const int64_t chunk0 = (int64_t)blockIdx.x * kChunk;
    const int64_t base = chunk0 + (int64_t)threadIdx.x * kItems;
    ItemD it[kItems];
    float sig[kItems];
    {
        Raw r;
        load_raw(sc, base, r);
        items_fp64(m, r, it);
#pragma unroll
        for (int q = 0; q < kItems; ++q) sig[q] = r.s[q];
    }
    double gz[kItems], gs[kItems];
#pragma unroll
    for (int q = 0; q < kItems; ++q) { gz[q] = 0.0; gs[q] = 0.0; }
    const int cells = m.n_gates * m.n_doppler;
    for (int sb = 0; sb < sch.n_samples; sb += kTab) {
        const int nb = min(kTab, sch.n_samples - sb);
        __syncthreads();
        if (threadIdx.x < nb) tab[threadIdx.x] = make_fp64_const(m, sample_pulse(sch, sb + threadIdx.x));
        __syncthreads();
        for (int j = 0; j < nb; ++j) {
            const int s = sb + j;
            const Fp64Const& k = tab[j];
#pragma unroll
            for (int q = 0; q < kItems; ++q) {
                double re, im;
                DerivD dv;
                const int key = eval_fp64<DOPPLER, true>(m, k, it[q], base + q, sc.n, re, im, &dv);
                if (key >= 0) {
                    const double2 g = G[(int64_t)s * cells + key];
                    const double cr = g.x * re + g.y * im;
                    const double ci = g.x * im - g.y * re;
                    gz[q] += cr * dv.dlna - ci * dv.dphi;
                    gs[q] += cr;
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        const int64_t n = base + q;
        if (n >= sc.n) continue;
        if (grad_z) grad_z[n] += (float)gz[q];
        if (grad_nrcs && sig[q] > 0.f) grad_nrcs[n] += (float)(gs[q] / (2.0 * (double)sig[q]));
    }
}

// ------------------------------------------------------------------------------- launchers
cudaError_t launch_accumulate(const Model& m, const Schedule& sch, const Scat& sc, bool fp64,
                              bool doppler, unsigned long long* ws, dim3 grid,
                              cudaStream_t stream) {
    if (fp64) {
        if (doppler) accumulate_fp64_kernel<true><<<grid, kThreads, 0, stream>>>(m, sch, sc, ws);
        else accumulate_fp64_kernel<false><<<grid, kThreads, 0, stream>>>(m, sch, sc, ws);
    } else {
        if (doppler) accumulate_split_kernel<true><<<grid, kThreads, 0, stream>>>(m, sch, sc, ws);
        else accumulate_split_kernel<false><<<grid, kThreads, 0, stream>>>(m, sch, sc, ws);
    }
    return cudaGetLastError();
}

cudaError_t launch_finalize(const void* ws, void* out, int64_t n_vals, bool fp64,
                            int n_sms, cudaStream_t stream) {
    const int threads = 256;
    int64_t blocks = (n_vals + threads - 1) / threads;
    const int64_t cap = (int64_t)n_sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (fp64) finalize_kernel<double><<<(unsigned)blocks, threads, 0, stream>>>(
        static_cast<const long long*>(ws), static_cast<double*>(out), n_vals);
    else finalize_kernel<float><<<(unsigned)blocks, threads, 0, stream>>>(
        static_cast<const long long*>(ws), static_cast<float*>(out), n_vals);
    return cudaGetLastError();
}

cudaError_t launch_cells(const Model& m, int64_t pulse, bool fp64, bool doppler, const Scat& sc,
                         int32_t* gate, int32_t* bin, double* gc, double* bc,
                         cudaStream_t stream) {
    const unsigned blocks = (unsigned)((sc.n + kChunk - 1) / kChunk);
    cells_kernel<<<blocks, kThreads, 0, stream>>>(m, pulse, fp64 ? 1 : 0, doppler ? 1 : 0, sc, gate,
                                                  bin, gc, bc);
    return cudaGetLastError();
}

cudaError_t launch_backward(const Model& m, const Schedule& sch, const Scat& sc, bool fp64,
                            bool doppler, const void* G, float* grad_z, float* grad_nrcs,
                            cudaStream_t stream) {
    const unsigned blocks = (unsigned)((sc.n + kChunk - 1) / kChunk);
    if (fp64) {
        const double2* g = static_cast<const double2*>(G);
        if (doppler) backward_fp64_kernel<true><<<blocks, kThreads, 0, stream>>>(m, sch, sc, g, grad_z, grad_nrcs);
        else backward_fp64_kernel<false><<<blocks, kThreads, 0, stream>>>(m, sch, sc, g, grad_z, grad_nrcs);
    } else {
        const float2* g = static_cast<const float2*>(G);
        if (doppler) backward_split_kernel<true><<<blocks, kThreads, 0, stream>>>(m, sch, sc, g, grad_z, grad_nrcs);
        else backward_split_kernel<false><<<blocks, kThreads, 0, stream>>>(m, sch, sc, g, grad_z, grad_nrcs);
    }
    return cudaGetLastError();
}

}  // namespace rsim
