// accumulate.cu -- scatterer-streaming summation kernels for sm_103a.
//
//  * accumulate_*: regular mode (Section II.A, one sample per pulse, cells = gates) and
//    the fast-mode Doppler pass (Algorithm 1 of Section III.B, one sample per update,
//    cells = gate x Doppler bin).  Each CTA owns kChunk consecutive scatterers (kThreads x
//    kItems) held in registers for ALL of its samples, so the 28 B of input per scatterer
//    are read from HBM once per launch however many samples there are.  Per (CTA, sample)
//    FP64 constants of a CTA reference point are computed by one thread per sample into
//    shared memory, together with a culling flag: a sample none of whose scatterers can
//    reach the range window is skipped by the whole CTA.  Contributions leave a warp as
//    merged runs and are added with 64-bit integer atomics into a fixed-point workspace
//    (exact, order-independent sums).
//    The batched variants run many independent scatterer sets (realizations of the same
//    track) in one launch; every realization keeps its own chunking, so its result is
//    bit-identical to a launch of its own.
//  * finalize: fixed-point workspace -> complex output (+=).
//  * cells: per-scatterer gate / bin decisions (same arithmetic as accumulate).
//  * backward_*: adjoint gather -- per scatterer, recompute C and its z-derivative at every
//    sample and gather dL/dT of its cell; no atomics (one thread owns each scatterer).
#include "rsim_internal.cuh"
#include "rsim_kernels.h"

namespace rsim {

namespace {

// Load IT consecutive floats starting at base (vectorised when all arrays are 16-byte
// aligned and the items are in range; base is a multiple of IT).
template <int IT>
__device__ __forceinline__ void load_items(const float* __restrict__ p, int64_t base, int64_t n,
                                           bool vec, float (&v)[IT]) {
    if (vec && base + IT <= n) {
        if (IT % 4 == 0) {
#pragma unroll
            for (int j = 0; j < IT / 4; ++j) {
                const float4 q = __ldcs(reinterpret_cast<const float4*>(p + base) + j);
                v[4 * j + 0] = q.x; v[4 * j + 1] = q.y; v[4 * j + 2] = q.z; v[4 * j + 3] = q.w;
            }
        } else if (IT == 2) {
            const float2 q = __ldcs(reinterpret_cast<const float2*>(p + base));
            v[0] = q.x; v[IT - 1] = q.y;
        } else {
            v[0] = __ldcs(p + base);
        }
    } else {
#pragma unroll
        for (int q = 0; q < IT; ++q) v[q] = (base + q < n) ? __ldcs(p + base + q) : 0.0f;
    }
}

template <int IT>
struct RawT {
    float x[IT], y[IT], z[IT], vx[IT], vy[IT], vz[IT], s[IT];
};
using Raw = RawT<kItems>;

template <int IT>
__device__ __forceinline__ void load_raw(const Scat& sc, int64_t base, RawT<IT>& r) {
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

// dt Q, Q = P(t0) - c: the platform at the set's epoch t0 relative to the CTA reference point
// (cx, cy, 0), times the PRI (the constant part of dt D(t) in the pulse-pair range change).
__device__ __forceinline__ float3 chunk_dq(const Model& m, const double* p0, double t0, float cx,
                                           float cy) {
    const double dt = m.inv_prf;
    return make_float3((float)(dt * (platform_coord(m, p0, 0, t0) - (double)cx)),
                       (float)(dt * (platform_coord(m, p0, 1, t0) - (double)cy)),
                       (float)(dt * platform_coord(m, p0, 2, t0)));
}

// The item's part of the pulse-pair range change (gam, beta; see ItemF) from its position
// and velocity (the same arithmetic as item_split).
__device__ __forceinline__ void item_motion(const Model& m, ItemF& it, float3 dq) {
    const float vx = it.vx, vy = it.vy, vz = it.vz, z = it.z;
    const float epv = fmaf(m.ep[0], vx, fmaf(m.ep[1], vy, m.ep[2] * vz));
    const float vv = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
    const float c1 = m.dt_f * fmaf(-m.hdt_f, vv, epv);
    const float ex = fmaf(-vx, m.dt_f, m.ep[0]), ey = fmaf(-vy, m.dt_f, m.ep[1]);
    const float ez = fmaf(-vz, m.dt_f, m.ep[2]);
    // gam = l0.e + c1 + dt (Q.v), beta = v.e + e_p.v  (see ItemF)
    it.gam = fmaf(it.lx0, ex, fmaf(it.ly0, ey, fmaf(z, ez, c1))) +
             fmaf(dq.x, vx, fmaf(dq.y, vy, dq.z * vz));
    it.beta = fmaf(vx, ex, fmaf(vy, ey, vz * ez)) + epv;
}

// item_motion for two items as the lanes of packed FP32 pairs: the same operations in the
// same order, each lane rounded as the scalar operation (negations moved onto the constants
// are exact), so each lane's gam and beta equal item_motion's, which the deferred exact
// re-evaluation uses.
__device__ __forceinline__ void item_motion2(const Model& m, ItemF2& it, float3 dq) {
    const float2 vx = it.vx, vy = it.vy, vz = it.vz, z = it.z;
    const float2 epv = __ffma2_rn(f2(m.ep[0]), vx,
                                  __ffma2_rn(f2(m.ep[1]), vy, __fmul2_rn(f2(m.ep[2]), vz)));
    const float2 vv = __ffma2_rn(vx, vx, __ffma2_rn(vy, vy, __fmul2_rn(vz, vz)));
    const float2 c1 = __fmul2_rn(f2(m.dt_f), __ffma2_rn(f2(-m.hdt_f), vv, epv));
    const float2 ex = __ffma2_rn(vx, f2(-m.dt_f), f2(m.ep[0]));
    const float2 ey = __ffma2_rn(vy, f2(-m.dt_f), f2(m.ep[1]));
    const float2 ez = __ffma2_rn(vz, f2(-m.dt_f), f2(m.ep[2]));
    it.gam = __fadd2_rn(
        __ffma2_rn(it.lx0, ex, __ffma2_rn(it.ly0, ey, __ffma2_rn(z, ez, c1))),
        __ffma2_rn(f2(dq.x), vx, __ffma2_rn(f2(dq.y), vy, __fmul2_rn(f2(dq.z), vz))));
    it.beta = __fadd2_rn(__ffma2_rn(vx, ex, __ffma2_rn(vy, ey, __fmul2_rn(vz, ez))), epv);
}

__device__ __forceinline__ ItemF item_split(const Model& m, float x, float y, float z, float vx,
                                            float vy, float vz, float nrcs, float cx, float cy,
                                            float area, float3 dq) {
    ItemF it;
    it.lx0 = x - cx;
    it.ly0 = y - cy;
    it.z = z;
    it.vx = vx;
    it.vy = vy;
    it.vz = vz;
    it.amp0 = sqrtf(nrcs * area);
    const float epv = fmaf(m.ep[0], vx, fmaf(m.ep[1], vy, m.ep[2] * vz));
    const float vv = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
    const float c1 = m.dt_f * fmaf(-m.hdt_f, vv, epv);
    const float ex = fmaf(-vx, m.dt_f, m.ep[0]), ey = fmaf(-vy, m.dt_f, m.ep[1]);
    const float ez = fmaf(-vz, m.dt_f, m.ep[2]);
    // gam = l0.e + c1 + dt (Q.v), beta = v.e + e_p.v  (see ItemF)
    it.gam = fmaf(it.lx0, ex, fmaf(it.ly0, ey, fmaf(z, ez, c1))) +
             fmaf(dq.x, vx, fmaf(dq.y, vy, dq.z * vz));
    it.beta = fmaf(vx, ex, fmaf(vy, ey, vz * ez)) + epv;
    return it;
}

template <int IT>
__device__ __forceinline__ void items_split(const Model& m, const RawT<IT>& r, float cx, float cy,
                                            float area, float3 dq, ItemF (&it)[IT]) {
#pragma unroll
    for (int q = 0; q < IT; ++q)
        it[q] = item_split(m, r.x[q], r.y[q], r.z[q], r.vx[q], r.vy[q], r.vz[q], r.s[q], cx, cy,
                           area, dq);
}

__device__ __forceinline__ void items_fp64(const Raw& r, double area, ItemD (&it)[kItems]) {
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
        it[q].x = r.x[q];
        it[q].y = r.y[q];
        it[q].z = r.z[q];
        it[q].vx = r.vx[q];
        it[q].vy = r.vy[q];
        it[q].vz = r.vz[q];
        it[q].amp0 = sqrt((double)r.s[q] * area);
    }
}

// Culling bounds of the CTA's scatterers around its reference point (cx, cy, 0):
// lmax >= max |r - c|, vmax >= max |v| over the real (non-padding) items, enlarged so that
// FP32 rounding of the norms cannot make the bound too tight.
template <int IT>
__device__ __forceinline__ void chunk_bounds(const RawT<IT>& r, float cx, float cy, int64_t base,
                                             int64_t n, float* s_red) {
    float l = 0.f, v = 0.f;
#pragma unroll
    for (int q = 0; q < IT; ++q) {
        if (base + q < n) {
            const float dx = r.x[q] - cx, dy = r.y[q] - cy;
            l = fmaxf(l, sqrtf(fmaf(dx, dx, fmaf(dy, dy, r.z[q] * r.z[q]))));
            v = fmaxf(v, sqrtf(fmaf(r.vx[q], r.vx[q], fmaf(r.vy[q], r.vy[q], r.vz[q] * r.vz[q]))));
        }
    }
    // non-negative floats order like their bit patterns
    const unsigned lb = __reduce_max_sync(0xffffffffu, __float_as_uint(l));
    const unsigned vb = __reduce_max_sync(0xffffffffu, __float_as_uint(v));
    if (threadIdx.x == 0) { s_red[0] = 0.f; s_red[1] = 0.f; }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        atomicMax(reinterpret_cast<unsigned*>(s_red), lb);
        atomicMax(reinterpret_cast<unsigned*>(s_red + 1), vb);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        s_red[0] = s_red[0] * (1.0f + 1e-6f) + 1e-3f;
        s_red[1] = s_red[1] * (1.0f + 1e-6f);
    }
    // the table builders read s_red after the next barrier
}

__device__ __forceinline__ int64_t sample_pulse(const Schedule& sch, int s) {
    return sch.pulse_base + (int64_t)s * sch.pulse_stride;
}

// Compaction of one block of samples: thread j < nb holds sample j and whether the CTA's
// scatterers can reach the range window there.  Returns how many can (CTA-uniform) and sets
// slot to this thread's place among them, in sample order.  s_cnt: one int per warp.
// Every thread of the CTA calls this (it holds a barrier).
template <int TH = kThreads>
__device__ __forceinline__ int compact_samples(bool act, int* s_cnt, int& slot) {
    constexpr int kWarps = TH / 32;
    const unsigned bal = __ballot_sync(0xffffffffu, act);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) s_cnt[w] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
#pragma unroll
    for (int i = 0; i < kWarps; ++i) {
        const int c = s_cnt[i];
        before += (i < w) ? c : 0;
        total += c;
    }
    slot = before + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u));
    return total;
}

// One CTA's work on one scatterer set: chunk starting at chunk0, samples [s_begin, s_end).
// sc points into kernel-parameter space (a single set's parameter, or a batch entry), so the
// set's pointers are read from the constant bank where needed instead of held in registers.
struct ChunkCtx {
    const Scat* sc;
    const double* p0;   // platform at t = 0 relative to this set's origin
    float area;
    int64_t chunk0;
    unsigned long long* ws;
};

// Deferred exact evaluations.  An item whose fast evaluation is flagged (coordinate within
// rounding of a cell edge, or far off nadir) leaves the warp's merged sum and is queued
// (chunk item index | table slot << 16) in its warp's shared-memory queue; the warp later
// re-evaluates each queued item exactly and adds it to the workspace on its own.  Keeping
// that rare, register-hungry path out of the per-sample loop keeps the loop within the
// register budget.  Every contribution is added in fixed point, so the split between
// merged and single additions does not change the result's determinism.
__host__ __device__ constexpr int queue_len(int items) { return 64 * items; }  // entries per warp; flushed before it can overflow

// The FP64 constants of the exact re-decision are made here, per queued item, from the
// entry's sample index: the queue is rare, so they are not tabulated for every sample.
template <bool DOPPLER, bool ANT>
__device__ __noinline__ void flush_queue(const Model& m, const Schedule& sch, const Scat& sc,
                                         const double* p0, int64_t chunk0, float cx, float cy,
                                         float area, float3 dq, const SplitConst* tab,
                                         const int* queue, int n) {
    for (int e = threadIdx.x & 31; e < n; e += 32) {
        const int code = queue[e];
        const int i = code & 0xffff, j = code >> 16;
        const int64_t idx = chunk0 + i;
        if (idx >= sc.n) continue;  // padding items carry no amplitude
        const float x = __ldg(sc.x + idx), y = __ldg(sc.y + idx);
        const ItemF it = item_split(m, x, y, __ldg(sc.z + idx), __ldg(sc.vx + idx),
                                    __ldg(sc.vy + idx), __ldg(sc.vz + idx), __ldg(sc.nrcs + idx),
                                    cx, cy, area, dq);
        const SampleF k = load_sample(tab[j]);
        const Fp64Const k64 = make_fp64_const(m, p0, sc.t0, sample_pulse(sch, sample_index(tab[j])));
        float re, im;
        int f;
        const int key = eval_split<DOPPLER, true, false, ANT>(m, k, it, re, im, f, &k64, x, y);
        if (key >= 0) emit_cell(sample_out(tab[j]), key, re, im);
    }
    __syncwarp();
}

// dt (P(t0) - c) = dt D(t) - e_p (t - t0): the per-sample dq of a sample whose state has its
// own epoch t0, from the sample's entry.
__device__ __forceinline__ float3 state_dq(const Model& m, const SampleF& k) {
    return make_float3(fmaf(-m.ep[0], k.t, k.Dx * m.dt_f), fmaf(-m.ep[1], k.t, k.Dy * m.dt_f),
                       fmaf(-m.ep[2], k.t, k.Dz * m.dt_f));
}

// flush_queue for samples with their own surface states: the item's height, velocity and
// epoch are those of its sample's state.
template <bool DOPPLER, bool ANT>
__device__ __noinline__ void flush_states_queue(const Model& m, const Schedule& sch,
                                                const Scat& sc, const StatesParams& sp,
                                                const double* p0, int64_t chunk0, float cx,
                                                float cy, float area, const SplitConst* tab,
                                                const int* queue, int n) {
    for (int e = threadIdx.x & 31; e < n; e += 32) {
        const int code = queue[e];
        const int i = code & 0xffff, j = code >> 16;
        const int64_t idx = chunk0 + i;
        if (idx >= sc.n) continue;  // padding items carry no amplitude
        const SampleF k = load_sample(tab[j]);
        const int s = sample_index(tab[j]);
        const StateEntry& st = sp.s[s];
        const float x = __ldg(sc.x + idx), y = __ldg(sc.y + idx);
        ItemF it;
        it.lx0 = x - cx;
        it.ly0 = y - cy;
        it.z = __ldg(st.z + idx);
        it.vx = __ldg(st.vx + idx);
        it.vy = __ldg(st.vy + idx);
        it.vz = __ldg(st.vz + idx);
        it.amp0 = sqrtf(__ldg(sc.nrcs + idx) * area);
        item_motion(m, it, state_dq(m, k));
        const Fp64Const k64 = make_fp64_const(m, p0, st.t0, sample_pulse(sch, s));
        float re, im;
        int f;
        const int key = eval_split<DOPPLER, true, false, ANT>(m, k, it, re, im, f, &k64, x, y);
        if (key >= 0) emit_cell(sample_out(tab[j]), key, re, im);
    }
    __syncwarp();
}

template <bool DOPPLER, bool ANT, int IT>
__device__ __forceinline__ void accumulate_split_chunk(const Model& m, const Schedule& sch,
                                                       const ChunkCtx& cx_, int s_begin,
                                                       int s_end) {
    constexpr int TH = kChunk / IT;       // threads of the CTA
    constexpr int kQueue = queue_len(IT);
    static_assert(TH >= kTab && TH % 32 == 0, "CTA shape");
    __shared__ SplitConst tab[kTab];
    __shared__ float s_red[2];
    __shared__ int s_cnt[TH / 32];
    __shared__ int s_queue[TH / 32][kQueue];
    // amplitude and pulse-pair constants of the thread's item pairs: read once per sample, so
    // they wait in shared memory (thread-private slots) rather than in registers
    __shared__ float2 s_ext[3][IT / 2][TH];
    constexpr unsigned kFull = 0xffffffffu;
    const Scat& sc = *cx_.sc;
    const int lane = threadIdx.x & 31;
    int* const queue = s_queue[threadIdx.x >> 5];
    float cx, cy;
    chunk_ref(sc, cx_.chunk0, cx, cy);
    const float3 dq = chunk_dq(m, cx_.p0, sc.t0, cx, cy);
    static_assert(IT % 2 == 0, "items are evaluated in pairs");
    ItemF2 it2[IT / 2];  // the thread's scatterers, paired for the .f32x2 evaluation
    {
        const int64_t base = cx_.chunk0 + (int64_t)threadIdx.x * IT;
        RawT<IT> r;
        load_raw(sc, base, r);
        ItemF it[IT];
        items_split(m, r, cx, cy, cx_.area, dq, it);
#pragma unroll
        for (int p = 0; p < IT / 2; ++p) {
            it2[p] = pack_items(it[2 * p], it[2 * p + 1]);
            s_ext[0][p][threadIdx.x] = it2[p].amp0;
            s_ext[1][p][threadIdx.x] = it2[p].gam;
            s_ext[2][p][threadIdx.x] = it2[p].beta;
        }
        chunk_bounds(r, cx, cy, base, sc.n, s_red);
    }
    const int cells = m.n_gates * m.n_doppler;
    for (int sb = s_begin; sb < s_end; sb += kTab) {
        const int nb = min(kTab, s_end - sb);
        __syncthreads();
        // the table keeps only the samples the CTA can contribute to
        const int s = sb + threadIdx.x;
        const int64_t pulse = sample_pulse(sch, s);
        const bool act = threadIdx.x < nb &&
                         cta_reaches_window(m, cx_.p0, sc.t0, pulse, cx, cy, s_red[0], s_red[1]) &&
                         RSIM_CHECK_OK(s < sch.n_samples, kChkSample, s);
        int slot;
        const int na = compact_samples<TH>(act, s_cnt, slot);
        if (act) {
            SplitConst kc = make_split_const(m, cx_.p0, sc.t0, pulse, cx, cy, s_red[0], s_red[1]);
            set_sample_slot(kc, s, cx_.ws + (int64_t)s * cells * 2);
            tab[slot] = kc;
        }
        __syncthreads();
        int nq = 0;  // entries in this warp's queue (warp-uniform)
        for (int j = 0; j < na; ++j) {
            const SampleF k = load_sample(tab[j]);
            int key[IT];
            float re[IT], im[IT];
            bool deferred = false;
#pragma unroll
            for (int q = 0; q < IT; q += 2) {
                float2 r2, i2;
                bool d;
                ItemF2 itq = it2[q / 2];
                itq.amp0 = s_ext[0][q / 2][threadIdx.x];
                itq.gam = s_ext[1][q / 2][threadIdx.x];
                itq.beta = s_ext[2][q / 2][threadIdx.x];
                eval_split_pair<DOPPLER, ANT>(m, k, itq, key[q], key[q + 1], r2, i2, d);
                re[q] = r2.x; re[q + 1] = r2.y;
                im[q] = i2.x; im[q + 1] = i2.y;
                deferred |= d;
            }
            if (__any_sync(kFull, deferred)) {  // rare: queue the flagged items
#pragma unroll
                for (int q = 0; q < IT; ++q) {
                    const bool mine = key[q] == kKeyDeferred;
                    const unsigned b = __ballot_sync(kFull, mine);
                    if (mine)
                        queue[nq + __popc(b & ((1u << lane) - 1u))] =
                            (threadIdx.x * IT + q) | (j << 16);
                    nq += __popc(b);
                }
            }
            warp_reduce_emit<float, IT>(key, re, im, sample_out(tab[j]), (unsigned)cells);
            if (nq > kQueue - 32 * IT) {  // room for one more sample's worth
                __syncwarp();
                flush_queue<DOPPLER, ANT>(m, sch, sc, cx_.p0, cx_.chunk0, cx, cy, cx_.area, dq, tab,
                                          queue, nq);
                nq = 0;
            }
        }
        if (nq > 0) {  // before the table is rebuilt
            __syncwarp();
            flush_queue<DOPPLER, ANT>(m, sch, sc, cx_.p0, cx_.chunk0, cx, cy, cx_.area, dq, tab,
                                      queue, nq);
        }
    }
}

template <bool DOPPLER, bool ANT>
__device__ __forceinline__ void accumulate_fp64_chunk(const Model& m, const Schedule& sch,
                                                      const ChunkCtx& cx_, int s_begin,
                                                      int s_end) {
    __shared__ Fp64Const tab[kTab];
    __shared__ float s_red[2];
    __shared__ int s_cnt[kThreads / 32];
    const Scat& sc = *cx_.sc;
    const int64_t base = cx_.chunk0 + (int64_t)threadIdx.x * kItems;
    float cx, cy;
    chunk_ref(sc, cx_.chunk0, cx, cy);
    ItemD it[kItems];
    {
        Raw r;
        load_raw(sc, base, r);
        items_fp64(r, (double)cx_.area, it);
        chunk_bounds(r, cx, cy, base, sc.n, s_red);
    }
    const int cells = m.n_gates * m.n_doppler;
    for (int sb = s_begin; sb < s_end; sb += kTab) {
        const int nb = min(kTab, s_end - sb);
        __syncthreads();
        const int64_t pulse = sample_pulse(sch, sb + threadIdx.x);
        const bool act = threadIdx.x < nb &&
                         cta_reaches_window(m, cx_.p0, sc.t0, pulse, cx, cy, s_red[0], s_red[1]) &&
                         RSIM_CHECK_OK(sb + (int)threadIdx.x < sch.n_samples, kChkSample,
                                       sb + (int)threadIdx.x);
        int slot;
        const int na = compact_samples(act, s_cnt, slot);
        if (act) {
            Fp64Const kd = make_fp64_const(m, cx_.p0, sc.t0, pulse);
            kd.index = sb + threadIdx.x;
            tab[slot] = kd;
        }
        __syncthreads();
        for (int j = 0; j < na; ++j) {
            const Fp64Const& k = tab[j];
            const int s = k.index;
            int key[kItems];
            double re[kItems], im[kItems];
#pragma unroll
            for (int q = 0; q < kItems; ++q)
                key[q] = eval_fp64<DOPPLER, false, ANT>(m, k, it[q], base + q, sc.n, re[q], im[q], nullptr);
            warp_reduce_emit<double, kItems>(key, re, im, cx_.ws + (int64_t)s * cells * 2,
                                             (unsigned)cells);
        }
    }
}

// ---------------------------------------------------------------------------------------
// Updates with their own surface states (Algorithm 1 regenerates the surface at every
// update): sample s of the launch takes the CTA's horizontal positions and NRCS with the
// heights, velocities and epoch of state s.  The horizontal part of every item stays in
// registers; each sample's heights and velocities are loaded straight into registers as
// float4 groups while the CTA's block of the next sample's fields is prefetched into L2.
// (Copying them into shared memory with cp.async one sample ahead, two buffers, took 14 %
// longer.)  No culling: every (CTA, sample) pair is evaluated (the states' heights are not
// known when the CTA starts).

// Four consecutive items of one state field (16-byte aligned arrays), zero past the end of
// the set: one vector load unless the group straddles the end.
__device__ __forceinline__ float4 load_state4(const float* __restrict__ f, int64_t i, int64_t n,
                                              bool full) {
    if (full || i + 4 <= n) return __ldg(reinterpret_cast<const float4*>(f + i));
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < n) r.x = __ldg(f + i);
    if (i + 1 < n) r.y = __ldg(f + i + 1);
    if (i + 2 < n) r.z = __ldg(f + i + 2);
    if (i + 3 < n) r.w = __ldg(f + i + 3);
    return r;
}

// Hint: the block's kChunk items of one field of a later state into L2 (one bulk prefetch,
// no completion to wait for; the block lies inside the set, 16-byte aligned).
__device__ __forceinline__ void prefetch_state_l2(const float* f) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;"
                 :: "l"((unsigned long long)__cvta_generic_to_global(f)),
                    "r"((unsigned)(kChunk * sizeof(float)))
                 : "memory");
}

template <bool DOPPLER, bool ANT, int IT>
__device__ __forceinline__ void accumulate_split_states_chunk(const Model& m, const Schedule& sch,
                                                              const StatesParams& sp,
                                                              const ChunkCtx& cx_, int s_begin,
                                                              int s_end) {
    constexpr int TH = kChunk / IT;
    constexpr int kQueue = 32 * IT;        // flushed after any sample that deferred an item
    static_assert(IT % 4 == 0, "items are fetched as float4 groups");
    __shared__ SplitConst tab[kMaxStates];
    __shared__ int s_queue[TH / 32][kQueue];
    constexpr unsigned kFull = 0xffffffffu;
    const Scat& sc = *cx_.sc;
    const int lane = threadIdx.x & 31;
    int* const queue = s_queue[threadIdx.x >> 5];
    float cx, cy;
    chunk_ref(sc, cx_.chunk0, cx, cy);
    const int64_t base = cx_.chunk0 + (int64_t)threadIdx.x * IT;
    float lx0[IT], ly0[IT], amp0[IT];
    {
        float xv[IT], yv[IT], sv[IT];
        const bool vec = sc.vec4 != 0;
        load_items(sc.x, base, sc.n, vec, xv);
        load_items(sc.y, base, sc.n, vec, yv);
        load_items(sc.nrcs, base, sc.n, vec, sv);
#pragma unroll
        for (int q = 0; q < IT; ++q) {
            lx0[q] = xv[q] - cx;
            ly0[q] = yv[q] - cy;
            amp0[q] = sqrtf(sv[q] * cx_.area);
        }
    }
    const int cells = m.n_gates * m.n_doppler;
    const int nb = s_end - s_begin;        // <= kMaxStates
    if (threadIdx.x < nb) {
        const int s = s_begin + threadIdx.x;
        SplitConst kc = make_split_const(m, cx_.p0, sp.s[s].t0, sample_pulse(sch, s), cx, cy,
                                         0.f, 0.f);
        set_sample_slot(kc, s, cx_.ws + (int64_t)s * cells * 2);
        tab[threadIdx.x] = kc;
    }
    __syncthreads();
    const bool full = cx_.chunk0 + kChunk <= sc.n;  // the block lies inside the set
    int nq = 0;
    for (int j = 0; j < nb; ++j) {
        const StateEntry& stj = sp.s[s_begin + j];
        if (threadIdx.x < 4 && j + 1 < nb && full) {
            const StateEntry& stn = sp.s[s_begin + j + 1];
            const float* f = threadIdx.x == 0 ? stn.z
                           : threadIdx.x == 1 ? stn.vx
                           : threadIdx.x == 2 ? stn.vy : stn.vz;
            prefetch_state_l2(f + cx_.chunk0);
        }
        const SampleF k = load_sample(tab[j]);
        const float3 dq = state_dq(m, k);
        ItemF2 it2[IT / 2];
#pragma unroll
        for (int h = 0; h < IT / 4; ++h) {
            const int64_t i4 = base + 4 * h;
            const float4 z4 = load_state4(stj.z, i4, sc.n, full);
            const float4 vx4 = load_state4(stj.vx, i4, sc.n, full);
            const float4 vy4 = load_state4(stj.vy, i4, sc.n, full);
            const float4 vz4 = load_state4(stj.vz, i4, sc.n, full);
#pragma unroll
            for (int u = 0; u < 2; ++u) {      // the pairs (4h, 4h + 1) and (4h + 2, 4h + 3)
                const int q = 4 * h + 2 * u;
                ItemF2& t = it2[q / 2];
                t.lx0 = make_float2(lx0[q], lx0[q + 1]);
                t.ly0 = make_float2(ly0[q], ly0[q + 1]);
                t.z = u ? make_float2(z4.z, z4.w) : make_float2(z4.x, z4.y);
                t.vx = u ? make_float2(vx4.z, vx4.w) : make_float2(vx4.x, vx4.y);
                t.vy = u ? make_float2(vy4.z, vy4.w) : make_float2(vy4.x, vy4.y);
                t.vz = u ? make_float2(vz4.z, vz4.w) : make_float2(vz4.x, vz4.y);
                t.amp0 = make_float2(amp0[q], amp0[q + 1]);
                item_motion2(m, t, dq);
            }
        }
        int key[IT];
        float re[IT], im[IT];
        bool deferred = false;
#pragma unroll
        for (int q = 0; q < IT; q += 2) {
            float2 r2, i2;
            bool d;
            eval_split_pair<DOPPLER, ANT>(m, k, it2[q / 2], key[q], key[q + 1], r2, i2, d);
            re[q] = r2.x; re[q + 1] = r2.y;
            im[q] = i2.x; im[q + 1] = i2.y;
            deferred |= d;
        }
        if (__any_sync(kFull, deferred)) {  // rare: queue the flagged items
#pragma unroll
            for (int q = 0; q < IT; ++q) {
                const bool mine = key[q] == kKeyDeferred;
                const unsigned b = __ballot_sync(kFull, mine);
                if (mine)
                    queue[nq + __popc(b & ((1u << lane) - 1u))] = (threadIdx.x * IT + q) | (j << 16);
                nq += __popc(b);
            }
        }
        warp_reduce_emit<float, IT>(key, re, im, sample_out(tab[j]), (unsigned)cells);
        if (nq > 0) {
            __syncwarp();
            flush_states_queue<DOPPLER, ANT>(m, sch, sc, sp, cx_.p0, cx_.chunk0, cx, cy,
                                             cx_.area, tab, queue, nq);
            nq = 0;
        }
    }
}

template <bool DOPPLER, bool ANT>
__device__ __forceinline__ void accumulate_fp64_states_chunk(const Model& m, const Schedule& sch,
                                                             const StatesParams& sp,
                                                             const ChunkCtx& cx_, int s_begin,
                                                             int s_end) {
    __shared__ Fp64Const tab[kMaxStates];
    const Scat& sc = *cx_.sc;
    const int64_t base = cx_.chunk0 + (int64_t)threadIdx.x * kItems;
    ItemD it[kItems];
    {
        Raw r;
        load_raw(sc, base, r);       // z, vx, vy, vz replaced per sample below
        items_fp64(r, (double)cx_.area, it);
    }
    const int cells = m.n_gates * m.n_doppler;
    const int nb = s_end - s_begin;
    if (threadIdx.x < nb) {
        const int s = s_begin + threadIdx.x;
        Fp64Const kd = make_fp64_const(m, cx_.p0, sp.s[s].t0, sample_pulse(sch, s));
        kd.index = s;
        tab[threadIdx.x] = kd;
    }
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        const Fp64Const& k = tab[j];
        const StateEntry& st = sp.s[k.index];
#pragma unroll
        for (int q = 0; q < kItems; ++q) {
            const int64_t i = base + q;
            const bool in = i < sc.n;
            it[q].z = in ? __ldg(st.z + i) : 0.f;
            it[q].vx = in ? __ldg(st.vx + i) : 0.f;
            it[q].vy = in ? __ldg(st.vy + i) : 0.f;
            it[q].vz = in ? __ldg(st.vz + i) : 0.f;
        }
        int key[kItems];
        double re[kItems], im[kItems];
#pragma unroll
        for (int q = 0; q < kItems; ++q)
            key[q] = eval_fp64<DOPPLER, false, ANT>(m, k, it[q], base + q, sc.n, re[q], im[q], nullptr);
        warp_reduce_emit<double, kItems>(key, re, im, cx_.ws + (int64_t)k.index * cells * 2,
                                         (unsigned)cells);
    }
}

__device__ __forceinline__ void sample_range(const Schedule& sch, int& s_begin, int& s_end) {
    s_begin = blockIdx.y * sch.samples_per_group;
    s_end = min(sch.n_samples, s_begin + sch.samples_per_group);
}

// Realization of a global chunk index in a batch (binary search over chunk_begin).
__device__ __forceinline__ int batch_find(const BatchParams& bp, int64_t chunk) {
    int lo = 0, hi = bp.n_real - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bp.e[mid].chunk_begin <= chunk) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ ChunkCtx batch_ctx(const BatchParams& bp, int r, int64_t chunk) {
    const BatchEntry& e = bp.e[r];
    ChunkCtx c;
    c.sc = &e.sc;
    c.p0 = e.p0;
    c.area = e.area;
    c.chunk0 = (chunk - e.chunk_begin) * kChunk;
    c.ws = e.ws;
    return c;
}

}  // namespace

// ------------------------------------------------------------------------------- forward
template <bool DOPPLER, bool ANT>
__global__ void __launch_bounds__(kChunk / split_items(ANT), ANT ? kMinBlocksAnt : kMinBlocks) accumulate_split_kernel(
    const __grid_constant__ Model m, const Schedule sch, const __grid_constant__ Scat sc,
    unsigned long long* __restrict__ ws) {
    ChunkCtx c;
    c.sc = &sc;
    c.p0 = m.p0;
    c.area = (float)m.area;
    c.chunk0 = (int64_t)blockIdx.x * kChunk;
    c.ws = ws;
    int s0, s1;
    sample_range(sch, s0, s1);
    accumulate_split_chunk<DOPPLER, ANT, split_items(ANT)>(m, sch, c, s0, s1);
}

template <bool DOPPLER, bool ANT>
__global__ void __launch_bounds__(kChunk / split_items(ANT), ANT ? kMinBlocksAnt : kMinBlocks) accumulate_split_batched_kernel(
    const __grid_constant__ Model m, const Schedule sch, const __grid_constant__ BatchParams bp) {
    const int r = batch_find(bp, blockIdx.x);
    const ChunkCtx c = batch_ctx(bp, r, blockIdx.x);
    int s0, s1;
    sample_range(sch, s0, s1);
    accumulate_split_chunk<DOPPLER, ANT, split_items(ANT)>(m, sch, c, s0, s1);
}

// Persistent form of the batched pass: one wave of CTAs; each takes work items
// (block of scatterers, group of updates) in order from `counter` (zeroed before the launch)
// until the n_chunks x groups items are gone.  Item i is chunk i / groups, update group
// i % groups, so consecutive items share a block's scatterers.  A plain atomic increment per
// item: no CTA waits on another.
template <bool DOPPLER, bool ANT>
__global__ void __launch_bounds__(kChunk / split_items(ANT), ANT ? kMinBlocksAnt : kMinBlocks) accumulate_split_batched_persistent_kernel(
    const __grid_constant__ Model m, const Schedule sch, const __grid_constant__ BatchParams bp,
    unsigned* __restrict__ counter, int64_t n_chunks, int groups) {
    __shared__ unsigned s_item;
    const int64_t total = n_chunks * groups;
    for (;;) {
        __syncthreads();                   // the last item's shared tables are no longer read
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1u);
        __syncthreads();
        const int64_t i = s_item;
        if (i >= total) break;
        const int64_t chunk = i / groups;
        const int g = (int)(i - chunk * groups);
        const int r = batch_find(bp, chunk);
        const ChunkCtx c = batch_ctx(bp, r, chunk);
        const int s0 = g * sch.samples_per_group;
        const int s1 = min(sch.n_samples, s0 + sch.samples_per_group);
        accumulate_split_chunk<DOPPLER, ANT, split_items(ANT)>(m, sch, c, s0, s1);
    }
}

template <bool DOPPLER, bool ANT>
__global__ void __launch_bounds__(kThreads) accumulate_fp64_kernel(
    const __grid_constant__ Model m, const Schedule sch, const __grid_constant__ Scat sc,
    unsigned long long* __restrict__ ws) {
    ChunkCtx c;
    c.sc = &sc;
    c.p0 = m.p0;
    c.area = (float)m.area;
    c.chunk0 = (int64_t)blockIdx.x * kChunk;
    c.ws = ws;
    int s0, s1;
    sample_range(sch, s0, s1);
    accumulate_fp64_chunk<DOPPLER, ANT>(m, sch, c, s0, s1);
}

template <bool DOPPLER, bool ANT>
__global__ void __launch_bounds__(kThreads) accumulate_fp64_batched_kernel(
    const __grid_constant__ Model m, const Schedule sch, const __grid_constant__ BatchParams bp) {
    const int r = batch_find(bp, blockIdx.x);
    const ChunkCtx c = batch_ctx(bp, r, blockIdx.x);
    int s0, s1;
    sample_range(sch, s0, s1);
    accumulate_fp64_chunk<DOPPLER, ANT>(m, sch, c, s0, s1);
}

template <bool DOPPLER, bool ANT>
__global__ void __launch_bounds__(kChunk / split_items(ANT), ANT ? kMinBlocksAnt : kMinBlocks) accumulate_split_states_kernel(
    const __grid_constant__ Model m, const Schedule sch, const __grid_constant__ Scat sc,
    const __grid_constant__ StatesParams sp, unsigned long long* __restrict__ ws) {
    ChunkCtx c;
    c.sc = &sc;
    c.p0 = m.p0;
    c.area = (float)m.area;
    c.chunk0 = (int64_t)blockIdx.x * kChunk;
    c.ws = ws;
    accumulate_split_states_chunk<DOPPLER, ANT, split_items(ANT)>(m, sch, sp, c, 0, sch.n_samples);
}

template <bool DOPPLER, bool ANT>
__global__ void __launch_bounds__(kThreads) accumulate_fp64_states_kernel(
    const __grid_constant__ Model m, const Schedule sch, const __grid_constant__ Scat sc,
    const __grid_constant__ StatesParams sp, unsigned long long* __restrict__ ws) {
    ChunkCtx c;
    c.sc = &sc;
    c.p0 = m.p0;
    c.area = (float)m.area;
    c.chunk0 = (int64_t)blockIdx.x * kChunk;
    c.ws = ws;
    accumulate_fp64_states_chunk<DOPPLER, ANT>(m, sch, sp, c, 0, sch.n_samples);
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

// Batched finalize: gridDim.y indexes the realization.
template <typename T>
__global__ void finalize_batched_kernel(FinalizeBatch fb, int64_t n_vals) {
    const long long* __restrict__ ws = static_cast<const long long*>(fb.ws[blockIdx.y]);
    T* __restrict__ out = static_cast<T*>(fb.out[blockIdx.y]);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_vals; i += stride) {
        out[i] += fixed_to<T>(__ldcs(ws + i));
    }
}

// ------------------------------------------------------------------------------- cells
template <bool ANT>
__global__ void __launch_bounds__(kThreads) cells_kernel(Model m, int64_t pulse, int fp64,
                                                         int doppler, Scat sc, int32_t* gate,
                                                         int32_t* bin, double* gcoord,
                                                         double* bcoord, void* contrib) {
    const int64_t chunk0 = (int64_t)blockIdx.x * kChunk;
    const int64_t base = chunk0 + (int64_t)threadIdx.x * kItems;
    Raw r;
    load_raw(sc, base, r);
    int key[kItems], g[kItems];
    double gc[kItems], bc[kItems], cre[kItems], cim[kItems];
    if (!fp64) {
        float cx, cy;
        chunk_ref(sc, chunk0, cx, cy);
        ItemF it[kItems];
        items_split(m, r, cx, cy, (float)m.area, chunk_dq(m, m.p0, sc.t0, cx, cy), it);
        const SampleF k = load_sample(make_split_const(m, m.p0, sc.t0, pulse, cx, cy, 0.f, 0.f));
        const Fp64Const k64 = make_fp64_const(m, m.p0, sc.t0, pulse);
#pragma unroll
        for (int q = 0; q < kItems; ++q) {
            float re, im;
            int f;
            key[q] = doppler
                ? eval_split<true, true, false, ANT>(m, k, it[q], re, im, f, &k64, r.x[q], r.y[q], nullptr, &g[q], &gc[q], &bc[q])
                : eval_split<false, true, false, ANT>(m, k, it[q], re, im, f, &k64, r.x[q], r.y[q], nullptr, &g[q], &gc[q], &bc[q]);
            cre[q] = re;
            cim[q] = im;
        }
    } else {
        ItemD it[kItems];
        items_fp64(r, m.area, it);
        const Fp64Const k = make_fp64_const(m, m.p0, sc.t0, pulse);
#pragma unroll
        for (int q = 0; q < kItems; ++q) {
            double re, im;
            key[q] = doppler ? eval_fp64<true, false, ANT>(m, k, it[q], base + q, sc.n, re, im, nullptr, &g[q], &gc[q], &bc[q])
                             : eval_fp64<false, false, ANT>(m, k, it[q], base + q, sc.n, re, im, nullptr, &g[q], &gc[q], &bc[q]);
            cre[q] = re;
            cim[q] = im;
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
        if (contrib) {
            if (fp64) static_cast<double2*>(contrib)[n] = make_double2(cre[q], cim[q]);
            else static_cast<float2*>(contrib)[n] = make_float2((float)cre[q], (float)cim[q]);
        }
        (void)key[q];
    }
}

// ------------------------------------------------------------------------- window counts
// Scatterers outside the range window (Section II.A: only facets whose range falls in one of
// the n_gates gates contribute), per sample of a summation call.  The decisions are the
// summation's own: the same culling test per (block, sample) -- a block that cannot reach the
// window counts all its scatterers -- and, for the others, the split path's FP32 gate with the
// FP64 re-decision near a cell edge (the scalar evaluation with the re-decision inline takes
// the same decisions as the paired evaluation and its deferred queue), or the FP64 path's.
// Grid: (block of scatterers, group of kCountSamples samples); one atomic add per warp and
// sample into counts[s].
constexpr int kCountSamples = 32;

template <bool DOPPLER, bool ANT>
__global__ void __launch_bounds__(kThreads) window_count_kernel(
    const __grid_constant__ Model m, const Schedule sch, const __grid_constant__ Scat sc,
    int fp64, unsigned long long* __restrict__ counts) {
    __shared__ SplitConst tab[kCountSamples];
    __shared__ Fp64Const tab64[kCountSamples];
    __shared__ float s_red[2];
    __shared__ int s_reach[kCountSamples];
    const int64_t chunk0 = (int64_t)blockIdx.x * kChunk;
    const int64_t base = chunk0 + (int64_t)threadIdx.x * kItems;
    const int s0 = (int)blockIdx.y * kCountSamples;
    const int ns = min(kCountSamples, sch.n_samples - s0);
    Raw r;
    load_raw(sc, base, r);
    float cx, cy;
    chunk_ref(sc, chunk0, cx, cy);
    chunk_bounds(r, cx, cy, base, sc.n, s_red);
    __syncthreads();
    if (threadIdx.x < ns) {
        const int64_t pulse = sample_pulse(sch, s0 + threadIdx.x);
        s_reach[threadIdx.x] = cta_reaches_window(m, m.p0, sc.t0, pulse, cx, cy, s_red[0], s_red[1]);
        tab64[threadIdx.x] = make_fp64_const(m, m.p0, sc.t0, pulse);
        if (!fp64)
            tab[threadIdx.x] = make_split_const(m, m.p0, sc.t0, pulse, cx, cy, s_red[0], s_red[1]);
    }
    __syncthreads();
    int valid = 0;
#pragma unroll
    for (int q = 0; q < kItems; ++q) valid += (base + q < sc.n) ? 1 : 0;
    ItemF itf[kItems];
    ItemD itd[kItems];
    if (!fp64) items_split(m, r, cx, cy, (float)m.area, chunk_dq(m, m.p0, sc.t0, cx, cy), itf);
    else items_fp64(r, m.area, itd);
    for (int j = 0; j < ns; ++j) {
        int n_out = valid;  // culled: every scatterer of the block is outside
        if (s_reach[j]) {
            n_out = 0;
            if (!fp64) {
                const SampleF k = load_sample(tab[j]);
#pragma unroll
                for (int q = 0; q < kItems; ++q) {
                    float re, im;
                    int f, g;
                    eval_split<DOPPLER, true, false, ANT>(m, k, itf[q], re, im, f, &tab64[j],
                                                          r.x[q], r.y[q], nullptr, &g);
                    n_out += (base + q < sc.n && (unsigned)g >= (unsigned)m.n_gates) ? 1 : 0;
                }
            } else {
#pragma unroll
                for (int q = 0; q < kItems; ++q) {
                    double re, im;
                    int g;
                    eval_fp64<DOPPLER, false, ANT>(m, tab64[j], itd[q], base + q, sc.n, re, im,
                                                   nullptr, &g);
                    n_out += (base + q < sc.n && (unsigned)g >= (unsigned)m.n_gates) ? 1 : 0;
                }
            }
        }
        const unsigned w = __reduce_add_sync(0xffffffffu, (unsigned)n_out);
        if ((threadIdx.x & 31) == 0 && w != 0)
            atomicAdd(counts + s0 + j, (unsigned long long)w);
    }
}

// ------------------------------------------------------------------------------- backward
template <bool DOPPLER, bool ANT>
__global__ void __launch_bounds__(kThreads) backward_split_kernel(
    Model m, Schedule sch, Scat sc, const float2* __restrict__ G, float* __restrict__ grad_z,
    float* __restrict__ grad_nrcs) {
    __shared__ SplitConst tab[kTab];
    __shared__ Fp64Const tab64[kTab];
    __shared__ float s_red[2];
    __shared__ int s_cnt[kThreads / 32];
    const int64_t chunk0 = (int64_t)blockIdx.x * kChunk;
    const int64_t base = chunk0 + (int64_t)threadIdx.x * kItems;
    float cx, cy;
    chunk_ref(sc, chunk0, cx, cy);
    ItemF it[kItems];
    float sig[kItems], xo[kItems], yo[kItems];
    {
        Raw r;
        load_raw(sc, base, r);
        items_split(m, r, cx, cy, (float)m.area, chunk_dq(m, m.p0, sc.t0, cx, cy), it);
        chunk_bounds(r, cx, cy, base, sc.n, s_red);
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
        const int s = sb + threadIdx.x;
        const int64_t pulse = sample_pulse(sch, s);
        const bool act = threadIdx.x < nb &&
                         cta_reaches_window(m, m.p0, sc.t0, pulse, cx, cy, s_red[0], s_red[1]);
        int slot;
        const int na = compact_samples(act, s_cnt, slot);
        if (act) {
            SplitConst kc = make_split_const(m, m.p0, sc.t0, pulse, cx, cy, s_red[0], s_red[1]);
            set_sample_slot(kc, s, nullptr);
            tab[slot] = kc;
            tab64[slot] = make_fp64_const(m, m.p0, sc.t0, pulse);
        }
        __syncthreads();
        for (int j = 0; j < na; ++j) {
            const int s = sample_index(tab[j]);
            const SampleF k = load_sample(tab[j]);
#pragma unroll
            for (int q = 0; q < kItems; ++q) {
                float re, im;
                int f;
                DerivF dv;
                const int key = eval_split<DOPPLER, true, true, ANT>(m, k, it[q], re, im, f, &tab64[j],
                                                                 xo[q], yo[q], &dv);
                if (key >= 0 && RSIM_CHECK_OK(key < cells, kChkGather, key)) {
                    const float2 g = __ldg(G + (int64_t)s * cells + key);
                    const float cr = fmaf(g.x, re, g.y * im);   // Re(conj(G) C)
                    const float ci = fmaf(g.x, im, -g.y * re);  // Im(conj(G) C)
                    gz[q] = fmaf(cr, dv.dlna, fmaf(-ci, dv.dphi, gz[q]));
                    if (ANT) gz[q] = fmaf(g.x, dv.pat.x, fmaf(g.y, dv.pat.y, gz[q]));  // Re(conj(G) dC_pat)
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

template <bool DOPPLER, bool ANT>
__global__ void __launch_bounds__(kThreads) backward_fp64_kernel(
    Model m, Schedule sch, Scat sc, const double2* __restrict__ G, float* __restrict__ grad_z,
    float* __restrict__ grad_nrcs) {
    __shared__ Fp64Const tab[kTab];
    __shared__ float s_red[2];
    __shared__ int s_cnt[kThreads / 32];
    const int64_t chunk0 = (int64_t)blockIdx.x * kChunk;
    const int64_t base = chunk0 + (int64_t)threadIdx.x * kItems;
    float cx, cy;
    chunk_ref(sc, chunk0, cx, cy);
    ItemD it[kItems];
    float sig[kItems];
    {
        Raw r;
        load_raw(sc, base, r);
        items_fp64(r, m.area, it);
        chunk_bounds(r, cx, cy, base, sc.n, s_red);
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
        const int64_t pulse = sample_pulse(sch, sb + threadIdx.x);
        const bool act = threadIdx.x < nb &&
                         cta_reaches_window(m, m.p0, sc.t0, pulse, cx, cy, s_red[0], s_red[1]);
        int slot;
        const int na = compact_samples(act, s_cnt, slot);
        if (act) {
            Fp64Const kd = make_fp64_const(m, m.p0, sc.t0, pulse);
            kd.index = sb + threadIdx.x;
            tab[slot] = kd;
        }
        __syncthreads();
        for (int j = 0; j < na; ++j) {
            const Fp64Const& k = tab[j];
            const int s = k.index;
#pragma unroll
            for (int q = 0; q < kItems; ++q) {
                double re, im;
                DerivD dv;
                const int key = eval_fp64<DOPPLER, true, ANT>(m, k, it[q], base + q, sc.n, re, im, &dv);
                if (key >= 0 && RSIM_CHECK_OK(key < cells, kChkGather, key)) {
                    const double2 g = G[(int64_t)s * cells + key];
                    const double cr = g.x * re + g.y * im;
                    const double ci = g.x * im - g.y * re;
                    gz[q] += cr * dv.dlna - ci * dv.dphi;
                    if (ANT) gz[q] += g.x * dv.pat.x + g.y * dv.pat.y;
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
    const bool ant = m.ant != nullptr;
    if (fp64) {
        if (ant) {
            if (doppler) accumulate_fp64_kernel<true, true><<<grid, kThreads, 0, stream>>>(m, sch, sc, ws);
            else accumulate_fp64_kernel<false, true><<<grid, kThreads, 0, stream>>>(m, sch, sc, ws);
        } else {
            if (doppler) accumulate_fp64_kernel<true, false><<<grid, kThreads, 0, stream>>>(m, sch, sc, ws);
            else accumulate_fp64_kernel<false, false><<<grid, kThreads, 0, stream>>>(m, sch, sc, ws);
        }
    } else {
        if (ant) {
            if (doppler) accumulate_split_kernel<true, true><<<grid, kChunk / split_items(true), 0, stream>>>(m, sch, sc, ws);
            else accumulate_split_kernel<false, true><<<grid, kChunk / split_items(true), 0, stream>>>(m, sch, sc, ws);
        } else {
            if (doppler) accumulate_split_kernel<true, false><<<grid, kChunk / split_items(false), 0, stream>>>(m, sch, sc, ws);
            else accumulate_split_kernel<false, false><<<grid, kChunk / split_items(false), 0, stream>>>(m, sch, sc, ws);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_accumulate_batched(const Model& m, const Schedule& sch, const BatchParams& bp,
                                      bool fp64, bool doppler, dim3 grid, cudaStream_t stream) {
    const bool ant = m.ant != nullptr;
    if (fp64) {
        if (ant) {
            if (doppler) accumulate_fp64_batched_kernel<true, true><<<grid, kThreads, 0, stream>>>(m, sch, bp);
            else accumulate_fp64_batched_kernel<false, true><<<grid, kThreads, 0, stream>>>(m, sch, bp);
        } else {
            if (doppler) accumulate_fp64_batched_kernel<true, false><<<grid, kThreads, 0, stream>>>(m, sch, bp);
            else accumulate_fp64_batched_kernel<false, false><<<grid, kThreads, 0, stream>>>(m, sch, bp);
        }
    } else {
        if (ant) {
            if (doppler) accumulate_split_batched_kernel<true, true><<<grid, kChunk / split_items(true), 0, stream>>>(m, sch, bp);
            else accumulate_split_batched_kernel<false, true><<<grid, kChunk / split_items(true), 0, stream>>>(m, sch, bp);
        } else {
            if (doppler) accumulate_split_batched_kernel<true, false><<<grid, kChunk / split_items(false), 0, stream>>>(m, sch, bp);
            else accumulate_split_batched_kernel<false, false><<<grid, kChunk / split_items(false), 0, stream>>>(m, sch, bp);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_accumulate_states(const Model& m, const Schedule& sch, const Scat& sc,
                                     const StatesParams& sp, bool fp64, bool doppler,
                                     unsigned long long* ws, unsigned n_chunks,
                                     cudaStream_t stream) {
    const bool ant = m.ant != nullptr;
    if (fp64) {
        if (ant) {
            if (doppler) accumulate_fp64_states_kernel<true, true><<<n_chunks, kThreads, 0, stream>>>(m, sch, sc, sp, ws);
            else accumulate_fp64_states_kernel<false, true><<<n_chunks, kThreads, 0, stream>>>(m, sch, sc, sp, ws);
        } else {
            if (doppler) accumulate_fp64_states_kernel<true, false><<<n_chunks, kThreads, 0, stream>>>(m, sch, sc, sp, ws);
            else accumulate_fp64_states_kernel<false, false><<<n_chunks, kThreads, 0, stream>>>(m, sch, sc, sp, ws);
        }
    } else {
        if (ant) {
            if (doppler) accumulate_split_states_kernel<true, true><<<n_chunks, kChunk / split_items(true), 0, stream>>>(m, sch, sc, sp, ws);
            else accumulate_split_states_kernel<false, true><<<n_chunks, kChunk / split_items(true), 0, stream>>>(m, sch, sc, sp, ws);
        } else {
            if (doppler) accumulate_split_states_kernel<true, false><<<n_chunks, kChunk / split_items(false), 0, stream>>>(m, sch, sc, sp, ws);
            else accumulate_split_states_kernel<false, false><<<n_chunks, kChunk / split_items(false), 0, stream>>>(m, sch, sc, sp, ws);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_accumulate_batched_persistent(const Model& m, const Schedule& sch,
                                                 const BatchParams& bp, bool doppler,
                                                 unsigned* counter, int64_t n_chunks, int groups,
                                                 unsigned n_ctas, cudaStream_t stream) {
    if (m.ant) {
        if (doppler) accumulate_split_batched_persistent_kernel<true, true><<<n_ctas, kChunk / split_items(true), 0, stream>>>(m, sch, bp, counter, n_chunks, groups);
        else accumulate_split_batched_persistent_kernel<false, true><<<n_ctas, kChunk / split_items(true), 0, stream>>>(m, sch, bp, counter, n_chunks, groups);
    } else {
        if (doppler) accumulate_split_batched_persistent_kernel<true, false><<<n_ctas, kChunk / split_items(false), 0, stream>>>(m, sch, bp, counter, n_chunks, groups);
        else accumulate_split_batched_persistent_kernel<false, false><<<n_ctas, kChunk / split_items(false), 0, stream>>>(m, sch, bp, counter, n_chunks, groups);
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

cudaError_t launch_finalize_batched(const FinalizeBatch& fb, int n_real, int64_t n_vals, bool fp64,
                                    int n_sms, cudaStream_t stream) {
    const int threads = 256;
    int64_t blocks = (n_vals + threads - 1) / threads;
    int64_t cap = ((int64_t)n_sms * 8 + n_real - 1) / n_real;
    if (cap < 1) cap = 1;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    const dim3 grid((unsigned)blocks, (unsigned)n_real);
    if (fp64) finalize_batched_kernel<double><<<grid, threads, 0, stream>>>(fb, n_vals);
    else finalize_batched_kernel<float><<<grid, threads, 0, stream>>>(fb, n_vals);
    return cudaGetLastError();
}

#ifdef RSIM_CHECK
cudaError_t check_take(cudaStream_t stream, unsigned long long* word) {
    *word = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(word, g_check_word, sizeof(*word), 0,
                                              cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess && *word != 0) {
        static const unsigned long long zero = 0;
        e = cudaMemcpyToSymbolAsync(g_check_word, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice,
                                    stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    }
    return e;
}
#endif

cudaError_t launch_window_count(const Model& m, const Schedule& sch, const Scat& sc, bool fp64,
                                bool doppler, unsigned long long* counts, cudaStream_t stream) {
    const int64_t chunks = (sc.n + kChunk - 1) / kChunk;
    const dim3 grid((unsigned)chunks, (unsigned)((sch.n_samples + kCountSamples - 1) / kCountSamples));
    const int f = fp64 ? 1 : 0;
    if (m.ant) {
        if (doppler) window_count_kernel<true, true><<<grid, kThreads, 0, stream>>>(m, sch, sc, f, counts);
        else window_count_kernel<false, true><<<grid, kThreads, 0, stream>>>(m, sch, sc, f, counts);
    } else {
        if (doppler) window_count_kernel<true, false><<<grid, kThreads, 0, stream>>>(m, sch, sc, f, counts);
        else window_count_kernel<false, false><<<grid, kThreads, 0, stream>>>(m, sch, sc, f, counts);
    }
    return cudaGetLastError();
}

cudaError_t launch_cells(const Model& m, int64_t pulse, bool fp64, bool doppler, const Scat& sc,
                         int32_t* gate, int32_t* bin, double* gc, double* bc, void* contrib,
                         cudaStream_t stream) {
    const unsigned blocks = (unsigned)((sc.n + kChunk - 1) / kChunk);
    if (m.ant)
        cells_kernel<true><<<blocks, kThreads, 0, stream>>>(m, pulse, fp64 ? 1 : 0, doppler ? 1 : 0,
                                                            sc, gate, bin, gc, bc, contrib);
    else
        cells_kernel<false><<<blocks, kThreads, 0, stream>>>(m, pulse, fp64 ? 1 : 0, doppler ? 1 : 0,
                                                             sc, gate, bin, gc, bc, contrib);
    return cudaGetLastError();
}

cudaError_t launch_backward(const Model& m, const Schedule& sch, const Scat& sc, bool fp64,
                            bool doppler, const void* G, float* grad_z, float* grad_nrcs,
                            cudaStream_t stream) {
    const unsigned blocks = (unsigned)((sc.n + kChunk - 1) / kChunk);
    if (fp64) {
        const double2* g = static_cast<const double2*>(G);
        if (m.ant) {
            if (doppler) backward_fp64_kernel<true, true><<<blocks, kThreads, 0, stream>>>(m, sch, sc, g, grad_z, grad_nrcs);
            else backward_fp64_kernel<false, true><<<blocks, kThreads, 0, stream>>>(m, sch, sc, g, grad_z, grad_nrcs);
        } else {
            if (doppler) backward_fp64_kernel<true, false><<<blocks, kThreads, 0, stream>>>(m, sch, sc, g, grad_z, grad_nrcs);
            else backward_fp64_kernel<false, false><<<blocks, kThreads, 0, stream>>>(m, sch, sc, g, grad_z, grad_nrcs);
        }
    } else {
        const float2* g = static_cast<const float2*>(G);
        if (m.ant) {
            if (doppler) backward_split_kernel<true, true><<<blocks, kThreads, 0, stream>>>(m, sch, sc, g, grad_z, grad_nrcs);
            else backward_split_kernel<false, true><<<blocks, kThreads, 0, stream>>>(m, sch, sc, g, grad_z, grad_nrcs);
        } else {
            if (doppler) backward_split_kernel<true, false><<<blocks, kThreads, 0, stream>>>(m, sch, sc, g, grad_z, grad_nrcs);
            else backward_split_kernel<false, false><<<blocks, kThreads, 0, stream>>>(m, sch, sc, g, grad_z, grad_nrcs);
        }
    }
    return cudaGetLastError();
}

}  // namespace rsim
