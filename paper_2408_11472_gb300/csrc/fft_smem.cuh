// fft_smem.cuh -- complex helpers and Stockham transforms over rows held in shared memory:
// radix-4 passes between two buffers (post-processing in synth.cu, delay-Doppler focusing
// in ddfocus.cu) and mixed-radix passes held in registers over a padded layout (surface
// synthesis in surface.cu).
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
// Entry n < N of the full table: twiddle(n) for n < N / 2, and -twiddle(n - N / 2) above
// (W^(n + N/2) = -W^n, exact), so a butterfly reads any power with one look-up.
__device__ __forceinline__ void twiddle_full(int n, int N, float sign, float2& w) {
    const int h = N >> 1;
    twiddle(n < h ? n : n - h, N, sign, w);
    if (n >= h) w = make_float2(-w.x, -w.y);
}

// Radix-4 Stockham autosort (a final radix-2 stage when log2 N is odd) over `rows`
// independent N-point rows in shared memory: half the passes over the data that radix-2
// stages need.  tw[n] = exp(sign j 2 pi n / N) for n < N/2 (the other half by W^{n+N/2} = -W^n);
// `sign` (+1 or -1) is the transform's.  Row r starts at element r * stride of each buffer
// (stride 0 means N; an odd stride lets a later pass read down a column without bank
// conflicts).  Returns the buffer holding the natural-order result.
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
__device__ T* stockham4(T* a, T* b, int rows, int N, int L, const T* __restrict__ tw, int sign,
                        int stride = 0) {
    int s = 1, lg = 0;
    const int quarter = N >> 2;
    const int rs = stride > 0 ? stride : N;
    while (lg + 2 <= L) {                       // radix-4 stages: s = 4^(lg/2) = 2^lg
        const int m = quarter >> lg;
        for (int idx = threadIdx.x; idx < rows * quarter; idx += blockDim.x) {
            const int row = idx >> (L - 2);
            const int bi = idx & (quarter - 1);
            const int p = bi >> lg, q = bi & (s - 1);
            const T* ar = a + row * rs;
            T* br = b + row * rs;
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
            const T* ar = a + row * rs;
            T* br = b + row * rs;
            const T x0 = ar[q], x1 = ar[q + half];
            br[q] = cadd(x0, x1);
            br[q + half] = csub(x0, x1);
        }
        __syncthreads();
        T* t = a; a = b; b = t;
    }
    return a;
}

// ---------------------------------------------------------------------------------------
// Mixed-radix Stockham passes held in registers: radix-16 passes while at least four
// bits of the length remain, then one radix-8, 4 or 2 pass (2048 = 16 x 16 x 8: three
// passes over shared memory instead of six radix-4 ones).  Each pass is the radix-R
// Stockham step (stride s = product of the previous radices, m = N / (R s)):
//     y[q + s (R p + j)] = w_N^{j p s} sum_k x[q + s (p + k m)] w_R^{j k},
// with w_M = exp(sign j 2 pi / M); a thread reads its R inputs into registers, the block
// waits, then each thread writes its outputs in place (one buffer).  The rows sit in shared
// memory with one spare element after every 16 (index pad16), which puts the strided
// accesses of every pass in distinct banks.  Row r starts at r * padded_len(N).

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> 4); }

// exp(sign j 2 pi m / 16) for the m the radix-16 and radix-8 steps use
__device__ __forceinline__ float2 w16(int m, float sign) {
    constexpr float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f;  // cos, sin pi/8
    constexpr float h = 0.70710678118654752f;                                // sqrt(1/2)
    float c, s;
    switch (m) {
        case 1: c = c1; s = s1; break;
        case 2: c = h; s = h; break;
        case 3: c = s1; s = c1; break;
        case 4: c = 0.0f; s = 1.0f; break;
        case 6: c = -h; s = h; break;
        case 9: c = -c1; s = -s1; break;
        default: c = 1.0f; s = 0.0f; break;
    }
    return make_float2(c, sign * s);
}

__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3, float sign) {
    const float2 t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), d = csub(x1, x3);
    const float2 t3 = make_float2(-sign * d.y, sign * d.x);  // sign j (x1 - x3)
    x0 = cadd(t0, t2);
    x1 = cadd(t1, t3);
    x2 = csub(t0, t2);
    x3 = csub(t1, t3);
}

// In-register DFTs, natural order in and out.  16 = 4 x 4 (n = 4 n1 + n2, k = k1 + 4 k2):
// 4-point DFTs over n1, twiddles w_16^{n2 k1}, 4-point DFTs over n2.  8 = 4 x 2 likewise.
template <int R> __device__ __forceinline__ void dft_reg(float2 (&x)[R], float sign);

template <> __device__ __forceinline__ void dft_reg<16>(float2 (&x)[16], float sign) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4(x[n2], x[4 + n2], x[8 + n2], x[12 + n2], sign);
    // x[4 k1 + n2] now holds the k1-th output of the n2-th transform
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1)
#pragma unroll
        for (int n2 = 1; n2 < 4; ++n2) x[4 * k1 + n2] = cmul(x[4 * k1 + n2], w16(n2 * k1, sign));
    float2 y[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 a0 = x[4 * k1], a1 = x[4 * k1 + 1], a2 = x[4 * k1 + 2], a3 = x[4 * k1 + 3];
        dft4(a0, a1, a2, a3, sign);
        y[k1] = a0;
        y[k1 + 4] = a1;
        y[k1 + 8] = a2;
        y[k1 + 12] = a3;
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = y[j];
}

template <> __device__ __forceinline__ void dft_reg<8>(float2 (&x)[8], float sign) {
    dft4(x[0], x[2], x[4], x[6], sign);
    dft4(x[1], x[3], x[5], x[7], sign);
    // x[2 k1 + n2]: k1-th output of the n2-th transform; w_8^{k1} on the odd one
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) x[2 * k1 + 1] = cmul(x[2 * k1 + 1], w16(2 * k1, sign));
    float2 y[8];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        y[k1] = cadd(x[2 * k1], x[2 * k1 + 1]);
        y[k1 + 4] = csub(x[2 * k1], x[2 * k1 + 1]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = y[j];
}

template <> __device__ __forceinline__ void dft_reg<4>(float2 (&x)[4], float sign) {
    dft4(x[0], x[1], x[2], x[3], sign);
}

template <> __device__ __forceinline__ void dft_reg<2>(float2 (&x)[2], float) {
    const float2 t = x[0];
    x[0] = cadd(t, x[1]);
    x[1] = csub(t, x[1]);
}

// x[j] *= w^(j e), j = 1..15, with w^(j e) from the four table entries twf[e], twf[2e],
// twf[4e], twf[8e] (at most three products each): four shared-memory reads per radix-16
// butterfly instead of fifteen.
__device__ __forceinline__ void twiddle16(float2 (&x)[16], const float2* __restrict__ twf, int e) {
    float2 w[16];
    w[1] = twf[e];
    w[2] = twf[2 * e];
    w[4] = twf[4 * e];
    w[8] = twf[8 * e];
    w[3] = cmul(w[1], w[2]);
    w[5] = cmul(w[1], w[4]);
    w[6] = cmul(w[2], w[4]);
    w[7] = cmul(w[3], w[4]);
#pragma unroll
    for (int j = 9; j < 16; ++j) w[j] = cmul(w[j - 8], w[8]);
#pragma unroll
    for (int j = 1; j < 16; ++j) x[j] = cmul(x[j], w[j]);
}

// One pass of radix R over `rows` padded rows, row r at element r * NP; U = work units per
// thread (the caller guarantees rows * N / R <= U * blockDim.x).  twf: the full table
// twf[n] = exp(sign j 2 pi n / N), n < N (see twiddle_full).
template <int R, int U>
__device__ __forceinline__ void stockham_pass_reg(float2* a, int rows, int N, int log2N, int log2s,
                                                  const float2* __restrict__ twf, float sign,
                                                  int NP) {
    constexpr int log2R = R == 16 ? 4 : R == 8 ? 3 : R == 4 ? 2 : 1;
    const int log2nb = log2N - log2R;           // butterflies per row: N / R
    const int nb = 1 << log2nb;
    const int s = 1 << log2s;
    const int m = nb >> log2s;                  // N / (R s)
    const int total = rows << log2nb;
    // Padded offsets: pad16(i + 16 t) = pad16(i) + 17 t, so when a butterfly's elements are a
    // multiple of 16 apart their padded offsets are one base plus a fixed stride (no per-element
    // index arithmetic).  Loads are N / R apart; stores s apart, or consecutive within one
    // aligned group of 16 when R s = 16.
    const int ld = nb;                                  // s m = N / R
    const bool ld_fast = (ld & 15) == 0;
    const bool st_fast = (s & 15) == 0 || R * s == 16;
    const int ld_step = ld + (ld >> 4);
    const int st_step = (s & 15) == 0 ? s + (s >> 4) : s;
    const bool last = log2s + log2R == log2N;
    float2 x[U][R];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int idx = threadIdx.x + u * blockDim.x;
        if (idx < total) {
            const int bi = idx & (nb - 1);
            const int p = bi >> log2s, q = bi & (s - 1);
            const float2* ar = a + (idx >> log2nb) * NP;
            if (ld_fast) {
                const float2* ab = ar + pad16(q + s * p);
#pragma unroll
                for (int k = 0; k < R; ++k) x[u][k] = ab[k * ld_step];
            } else {
#pragma unroll
                for (int k = 0; k < R; ++k) x[u][k] = ar[pad16(q + s * (p + k * m))];
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int idx = threadIdx.x + u * blockDim.x;
        if (idx < total) {
            const int bi = idx & (nb - 1);
            const int p = bi >> log2s, q = bi & (s - 1);
            float2* ar = a + (idx >> log2nb) * NP;
            dft_reg<R>(x[u], sign);
            const int e = p * s;
            const int o = q + s * (R * p);
            // the last pass (s = N / R, so p = 0) has unit twiddles
            if (!last) {
                if constexpr (R == 16) {
                    twiddle16(x[u], twf, e);
                } else {
#pragma unroll
                    for (int j = 1; j < R; ++j) x[u][j] = cmul(x[u][j], twf[j * e]);
                }
            }
            if (st_fast) {
                float2* ab = ar + pad16(o);
#pragma unroll
                for (int j = 0; j < R; ++j) ab[j * st_step] = x[u][j];
            } else {
#pragma unroll
                for (int j = 0; j < R; ++j) ar[pad16(o + s * j)] = x[u][j];
            }
        }
    }
    __syncthreads();
}

// The register-radix transform of `rows` padded rows of N = 2^log2N points (N >= 2), row r at
// element r * NP (NP >= padded_len(N)): radix-16 passes, then one last pass of radix 2, 4, 8
// or 16.  This runs every pass but the last (from log2s0: the caller may have done the
// first ones) and returns the log2 stride of the last pass, whose radix is
// 2^(log2N - returned value); fft_last_pass_store runs it.  MAXE bounds the elements per
// thread: rows * N <= MAXE * blockDim.x (MAXE a multiple of 16).  twf: the full twiddle
// table (twiddle_full).
template <int MAXE>
__device__ int fft_rows_reg_but_last(float2* a, int rows, int N, int log2N,
                                     const float2* __restrict__ twf, float sign, int NP,
                                     int log2s0 = 0) {
    int log2s = log2s0;
    while (log2N - log2s > 4) {
        stockham_pass_reg<16, MAXE / 16>(a, rows, N, log2N, log2s, twf, sign, NP);
        log2s += 4;
    }
    return log2s;
}

// The last pass (radix R, stride s = N / R, unit twiddles) of `rows` padded rows that went
// through the others, handing output element n = q + s j of row `row` to store(row, n, value)
// instead of writing it back to shared memory: butterfly (row, q) reads elements q + s k.
// ROW_FAST: consecutive threads take consecutive rows (rows = 2^lr), so that one output index
// of several rows is stored by adjacent threads; otherwise consecutive q.  U: rows * s <= U *
// blockDim.x.  The caller's last barrier is stockham_pass_reg's.
template <int R, int U, bool ROW_FAST, typename Store>
__device__ __forceinline__ void last_pass_store(const float2* a, int rows, int lr, int log2N,
                                                int NP, float sign, Store store) {
    constexpr int log2R = R == 16 ? 4 : R == 8 ? 3 : R == 4 ? 2 : 1;
    const int log2s = log2N - log2R, sd = 1 << log2s;
    const int total = rows << log2s;
    const bool fast = (sd & 15) == 0;
    const int ld_step = sd + (sd >> 4);
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int idx = threadIdx.x + u * blockDim.x;
        if (idx < total) {
            const int row = ROW_FAST ? (idx & (rows - 1)) : (idx >> log2s);
            const int q = ROW_FAST ? (idx >> lr) : (idx & (sd - 1));
            const float2* ar = a + row * NP;
            float2 x[R];
            if (fast) {
                const float2* ab = ar + pad16(q);
#pragma unroll
                for (int k = 0; k < R; ++k) x[k] = ab[k * ld_step];
            } else {
#pragma unroll
                for (int k = 0; k < R; ++k) x[k] = ar[pad16(q + sd * k)];
            }
            dft_reg<R>(x, sign);
#pragma unroll
            for (int j = 0; j < R; ++j) store(row, q + sd * j, x[j]);
        }
    }
}

// The last pass of fft_rows_reg_but_last's rows with its outputs sent to store (see
// last_pass_store); MAXE as for fft_rows_reg_but_last.
template <int MAXE, bool ROW_FAST, typename Store>
__device__ __forceinline__ void fft_last_pass_store(const float2* a, int rows, int lr, int log2N,
                                                    int log2s, int NP, float sign, Store store) {
    switch (log2N - log2s) {
        case 4: last_pass_store<16, MAXE / 16, ROW_FAST>(a, rows, lr, log2N, NP, sign, store); break;
        case 3: last_pass_store<8, MAXE / 8, ROW_FAST>(a, rows, lr, log2N, NP, sign, store); break;
        case 2: last_pass_store<4, MAXE / 4, ROW_FAST>(a, rows, lr, log2N, NP, sign, store); break;
        default: last_pass_store<2, MAXE / 2, ROW_FAST>(a, rows, lr, log2N, NP, sign, store); break;
    }
}

}  // namespace fft
}  // namespace rsim
