// surface.cu -- spectral update of the sea surface at an update time (Algorithm 1's
// update_simulation: the surface is regenerated at every update), for sm_103a.
//
// Linear deep-water waves from one-sided coefficients A(k) on the L x L wave-number grid
// (index [iy][ix], k = 2 pi fftfreq(L, spacing)), omega = sqrt(g |k|):
//   eta = s Re IFFT2[A e^{-j omega t}],  v_z = s Re IFFT2[-j omega A e^{-j omega t}],
//   v_x = s Re IFFT2[omega k_x/|k| A e^{-j omega t}],  v_y likewise with k_y,
// IFFT2 normalised by 1/L^2.  Each real field is the inverse transform of the Hermitian part
// H(k) = (X(k) + conj(X(-k))) / 2 of its spectrum X, so two real fields share one complex
// transform: IFFT2[H_a + j H_b] = a + j b.  Two packed transforms (eta + j v_z,
// v_x + j v_y) per update:
//   rows pass    : one CTA per pair of rows iy, -iy builds the packed rows of both from
//                  A(k), A(-k) and the phase e^{-j omega t} (read straight from global
//                  memory; H(-k) = conj(H(k))) and transforms them along x (shared memory);
//   columns pass : one CTA per block of columns (32 bytes of every row) transforms along y
//                  and writes the fields.
// Both passes use the register mixed-radix transform (radix-16 passes, one shared-memory
// copy of the data in a padded layout: three passes over shared memory for L = 2048).
// omega / (2 pi) is tabulated once per spectrum (FP64, stored as hi + lo floats) so that
// the phase omega t stays accurate to ~1e-7 cycles for t of hours.
#include "rsim_internal.cuh"
#include "rsim_kernels.h"
#include "fft_smem.cuh"

namespace rsim {

namespace {

using namespace fft;

__device__ __forceinline__ double wave_number(int i, int L, double dk) {
    return (double)(i < L / 2 ? i : i - L) * dk;      // 2 pi fftfreq(L, spacing)[i]
}

// Asynchronous global -> shared copies (cp.async, 8 bytes; both addresses 8-byte aligned).
__device__ __forceinline__ void cp_async8(float2* smem_dst, const float2* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;"
                 :: "r"(d), "l"((unsigned long long)__cvta_generic_to_global(gmem_src)) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// L2 eviction priorities (createpolicy + .L2::cache_hint): the row pass writes the packed
// intermediate (64 MB at L = 2048) as evict_last so that the column pass finds it in L2, and
// the data read or written once (coefficients, omega table, the intermediate's second read,
// the fields) go as evict_first.
__device__ __forceinline__ unsigned long long l2_evict_last() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned long long l2_evict_first() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ float2 ld_l2hint(const float2* p, unsigned long long pol) {
    float2 v;
    asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
        : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_l2hint(float2* p, float2 v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;"
                 :: "l"(p), "f"(v.x), "f"(v.y), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_l2hint(float* p, float v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" :: "l"(p), "f"(v), "l"(pol) : "memory");
}

// The spectrum's tables: omega / (2 pi) as hi + lo floats for every grid point, the wave
// numbers 2 pi fftfreq(L, spacing) as floats, and the full inverse-transform twiddle table
// (so that the per-update kernels run no FP64 and no sine per CTA).
__global__ void surf_prepare_kernel(SurfArgs a, float2* __restrict__ omega, float* __restrict__ kf,
                                    float2* __restrict__ twf) {
    const int64_t n = (int64_t)a.L * a.L;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int iy = (int)(idx / a.L), ix = (int)(idx - (int64_t)iy * a.L);
        const double kx = wave_number(ix, a.L, a.dk), ky = wave_number(iy, a.L, a.dk);
        const double w = sqrt(a.g * sqrt(kx * kx + ky * ky)) / 6.283185307179586476925;
        const float hi = (float)w;
        omega[idx] = make_float2(hi, (float)(w - (double)hi));
        if (idx < a.L) {
            kf[idx] = (float)wave_number((int)idx, a.L, a.dk);
            twiddle_full((int)idx, a.L, 1.0f, twf[idx]);
        }
    }
}

constexpr int kRowsThreads = 512;    // rows k and -k, two packed transforms: 4 rows of <= 2048
constexpr int kRowsThreadsBig = 1024; // 4 rows of 4096 points
constexpr int kColsMaxThreads = 1024; // at most 16384 points (C columns of L): 16 per thread

// Rows pass: one CTA per pair of rows iy and -iy (rows 0 and L/2 are their own partners).
// The coefficients of both rows and the omega row of iy are read straight from global memory
// (coalesced; the row of -k in reverse order).  Each grid point k gives the Hermitian parts
// H(k) of the four spectra, and H(-k) = conj(H(k)) exactly, so one evaluation fills both
// rows' entries: half the coefficient reads and half the phase work of a CTA per row.  The
// packed rows (eta + j v_z, v_x + j v_y of row iy, then of row -iy) hold the only
// shared-memory copy.
template <int TH>
__global__ void __launch_bounds__(TH) surf_rows_kernel(SurfArgs a, const float2* __restrict__ coef,
                                                       const float2* __restrict__ omega,
                                                       const float* __restrict__ kf,
                                                       const float2* __restrict__ twf_g,
                                                       float2* __restrict__ tmp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = a.L, NP = padded_len(L);
    float2* tw = reinterpret_cast<float2*>(smem_raw);     // exp(+j 2 pi r / L), r < L
    float2* buf0 = tw + L;
    const int iy = blockIdx.x;                              // 0 .. L / 2
    const int iyn = (L - iy) & (L - 1);                     // row of -k
    const bool pair = iyn != iy;
    for (int r = threadIdx.x; r < L; r += TH) tw[r] = __ldg(twf_g + r);
    const float ky = __ldg(kf + iy);
    const float2* rowA = coef + (int64_t)iy * L;
    const float2* rowB = coef + (int64_t)iyn * L;
    const float2* rowW = omega + (int64_t)iy * L;
    const unsigned long long first = l2_evict_first(), last = l2_evict_last();
#pragma unroll 4
    for (int ix = threadIdx.x; ix < L; ix += TH) {
        const int ixn = (L - ix) & (L - 1);
        const float kx = __ldg(kf + ix);
        const float2 A1 = ld_l2hint(rowA + ix, first);
        const float2 A2 = ld_l2hint(rowB + ixn, first);
        // e^{-j omega t}: omega t / 2 pi = w t with w = hi + lo, t = t_hi + t_lo
        const float2 w = ld_l2hint(rowW + ix, first);
        const float p = w.x * a.t_hi;
        const float pe = fmaf(w.x, a.t_hi, -p);
        float f = (p - rintf(p)) + (pe + fmaf(w.x, a.t_lo, w.y * a.t_hi));
        f -= rintf(f);
        float sn, cs;
        __sincosf(6.283185307179586f * f, &sn, &cs);       // |2 pi f| <= pi
        const float2 E = make_float2(cs, -sn);
        const float2 F1 = cmul(A1, E), F2 = cmul(A2, E);    // F(k), F(-k)
        const float om = 6.283185307179586f * (w.x + w.y);   // the same |k| at n and -n
        const float k2 = fmaf(kx, kx, ky * ky);
        const float ik = k2 > 0.f ? rsqrtf(k2) : 0.f;
        const float ux = kx * ik, uy = ky * ik;
        // direction at the grid point -n: -k_hat, except on the Nyquist row / column, which
        // the grid maps onto itself with the same wave number
        const float uxn = ixn == ix ? ux : -ux, uyn = iyn == iy ? uy : -uy;
        // Hermitian parts (X(n) + conj(X(-n))) / 2 of the four spectra
        const float2 he = make_float2(0.5f * (F1.x + F2.x), 0.5f * (F1.y - F2.y));       // X = F
        // X = -j omega F (the same factor at -n): (-j omega F1 + conj(-j omega F2)) / 2
        const float2 hz = make_float2(0.5f * om * (F1.y + F2.y), 0.5f * om * (F2.x - F1.x));
        // X = omega u F
        const float2 hx = make_float2(0.5f * om * fmaf(ux, F1.x, uxn * F2.x),
                                      0.5f * om * fmaf(ux, F1.y, -uxn * F2.y));
        const float2 hy = make_float2(0.5f * om * fmaf(uy, F1.x, uyn * F2.x),
                                      0.5f * om * fmaf(uy, F1.y, -uyn * F2.y));
        buf0[pad16(ix)] = make_float2(he.x - hz.y, he.y + hz.x);       // H_eta + j H_vz
        buf0[NP + pad16(ix)] = make_float2(hx.x - hy.y, hx.y + hy.x);  // H_vx + j H_vy
        if (pair) {  // at -n: conj(H_eta) + j conj(H_vz), conj(H_vx) + j conj(H_vy)
            buf0[2 * NP + pad16(ixn)] = make_float2(he.x + hz.y, hz.x - he.y);
            buf0[3 * NP + pad16(ixn)] = make_float2(hx.x + hy.y, hy.x - hx.y);
        }
    }
    __syncthreads();
    const int rows = pair ? 4 : 2;
    // rows L <= 16 x TH; the last pass writes the transformed rows straight to global memory
    // (consecutive threads: consecutive points of a row)
    const int log2s = fft_rows_reg_but_last<16>(buf0, rows, L, a.log2L, tw, 1.0f, NP);
    fft_last_pass_store<16, false>(buf0, rows, 0, a.log2L, log2s, NP, 1.0f,
                                   [&](int row, int n, float2 v) {
        const int y = (row & 2) ? iyn : iy;                 // rows: iy, iy, -iy, -iy
        st_l2hint(tmp + (int64_t)(row & 1) * L * L + (int64_t)y * L + n, v, last);
    });
}

// Column stride in shared memory: padded_len(L) + 4 elements, so that the C columns of one
// row (32 bytes apart per column) fall in different bank groups when a row is stored or read.
__host__ __device__ constexpr int cols_stride(int L) { return padded_len(L) + 4; }

// Columns pass: one CTA per block of C columns of one packed transform (gridDim.y), one
// radix-16 butterfly per thread (C L / 16 threads).  For L >= 256 the first pass reads its
// butterflies straight from global memory (the C columns of a row side by side: 64 bytes for
// C = 8) and the last pass writes the fields straight back; the passes between run in shared
// memory.
__global__ void __launch_bounds__(kColsMaxThreads) surf_cols_kernel(SurfArgs a, const float2* __restrict__ tmp,
                                                           const float2* __restrict__ twf_g,
                                                           float* __restrict__ z, float* __restrict__ vx,
                                                           float* __restrict__ vy, float* __restrict__ vz) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int L = a.L, C = a.cols, NP = cols_stride(L);
    float2* tw = reinterpret_cast<float2*>(smem_raw);
    float2* buf0 = tw + L;
    const int ix0 = blockIdx.x * C;
    const int pair = blockIdx.y;
    const float2* src = tmp + (int64_t)pair * L * L + ix0;
    const int lc = __ffs(C) - 1;                          // C is a power of two
    for (int r = threadIdx.x; r < L; r += blockDim.x) cp_async8(tw + r, twf_g + r);
    cp_async_commit();
    int log2s0 = 0;
    if (C * (L >> 4) == (int)blockDim.x && a.log2L >= 8) {
        // first radix-16 pass straight from global memory: butterfly p of column c takes rows
        // p + k L / 16 (the C columns of a row are adjacent in memory and in the warp);
        // written to the padded columns in shared memory
        const int nb = L >> 4;
        const int c = threadIdx.x & (C - 1), p = threadIdx.x >> lc;   // one butterfly each
        float2 x[16];
        const unsigned long long first = l2_evict_first();
#pragma unroll
        for (int k = 0; k < 16; ++k) x[k] = ld_l2hint(src + (int64_t)(p + k * nb) * L + c, first);
        cp_async_wait<0>();
        __syncthreads();                                  // the twiddle table is in place
        dft_reg<16>(x, 1.0f);
        twiddle16(x, tw, p);
        float2* ab = buf0 + c * NP + pad16(16 * p);
#pragma unroll
        for (int j = 0; j < 16; ++j) ab[j] = x[j];
        __syncthreads();
        log2s0 = 4;
    } else {
        for (int idx = threadIdx.x; idx < C * L; idx += blockDim.x) {
            const int iy = idx >> lc, cc = idx & (C - 1);
            cp_async8(buf0 + cc * NP + pad16(iy), src + (int64_t)iy * L + cc);
        }
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
    }
    float* fa = pair == 0 ? z : vx;
    float* fb = pair == 0 ? vz : vy;
    // C L <= 16 x blockDim.x; the last pass writes the fields straight to global memory, the
    // C columns of one row from adjacent threads (32 bytes per row and field for C = 8)
    const int log2s = fft_rows_reg_but_last<16>(buf0, C, L, a.log2L, tw, 1.0f, NP, log2s0);
    const float sc = a.scale_over_L2;
    const unsigned long long out_pol = l2_evict_first();
    fft_last_pass_store<16, true>(buf0, C, lc, a.log2L, log2s, NP, 1.0f,
                                  [&](int c, int iy, float2 v) {
        const int64_t o = (int64_t)iy * L + ix0 + c;
        st_l2hint(fa + o, v.x * sc, out_pol);
        st_l2hint(fb + o, v.y * sc, out_pol);
    });
}

}  // namespace

size_t surf_rows_smem(int L) {
    return sizeof(float2) * ((size_t)L + 4 * (size_t)padded_len(L));
}
size_t surf_cols_smem(int L, int cols) {
    return sizeof(float2) * ((size_t)L + (size_t)cols * cols_stride(L));
}

SurfTables surf_tables(int L, void* workspace) {
    SurfTables t;
    char* base = static_cast<char*>(workspace);
    const size_t n = (size_t)L * L;
    t.omega = reinterpret_cast<float2*>(base);
    t.tmp = reinterpret_cast<float2*>(base + 8 * n);
    t.twf = reinterpret_cast<float2*>(base + 24 * n);
    t.kf = reinterpret_cast<float*>(base + 24 * n + 8 * (size_t)L);
    return t;
}

cudaError_t launch_surf_prepare(const SurfArgs& a, const SurfTables& t, int n_sms,
                                cudaStream_t stream) {
    const int64_t n = (int64_t)a.L * a.L;
    const int64_t want = (n + 255) / 256;
    const unsigned blocks = (unsigned)(want < (int64_t)n_sms * 8 ? want : (int64_t)n_sms * 8);
    surf_prepare_kernel<<<blocks, 256, 0, stream>>>(a, t.omega, t.kf, t.twf);
    return cudaGetLastError();
}

cudaError_t launch_surf_at(const SurfArgs& a, const void* coef, const SurfTables& t,
                           float* z, float* vx, float* vy, float* vz, cudaStream_t stream) {
    const size_t s1 = surf_rows_smem(a.L), s2 = surf_cols_smem(a.L, a.cols);
    cudaError_t e;
    const bool big = a.L > 2048;
    if (s1 > 48 * 1024 &&
        (e = big ? cudaFuncSetAttribute(surf_rows_kernel<kRowsThreadsBig>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1)
                 : cudaFuncSetAttribute(surf_rows_kernel<kRowsThreads>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1)) !=
            cudaSuccess)
        return e;
    if (s2 > 48 * 1024 &&
        (e = cudaFuncSetAttribute(surf_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)s2)) != cudaSuccess)
        return e;
    const unsigned row_pairs = (unsigned)(a.L / 2 + 1);   // rows 0 .. L/2 with their partners
    if (big)
        surf_rows_kernel<kRowsThreadsBig><<<row_pairs, kRowsThreadsBig, s1, stream>>>(
            a, static_cast<const float2*>(coef), t.omega, t.kf, t.twf, t.tmp);
    else
        surf_rows_kernel<kRowsThreads><<<row_pairs, kRowsThreads, s1, stream>>>(
            a, static_cast<const float2*>(coef), t.omega, t.kf, t.twf, t.tmp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int cols_threads = a.cols * a.L / 16;                 // one radix-16 butterfly per thread
    cols_threads = cols_threads < 32 ? 32 : (cols_threads + 31) / 32 * 32;
    if (cols_threads > kColsMaxThreads) return cudaErrorInvalidValue;
    surf_cols_kernel<<<dim3((unsigned)(a.L / a.cols), 2), cols_threads, s2, stream>>>(
        a, t.tmp, t.twf, z, vx, vy, vz);
    return cudaGetLastError();
}

}  // namespace rsim
