// rsim_internal.cuh -- device-side model, per-scatterer evaluation and the
// deterministic warp-level scatter-add shared by the summation kernels.
//
// Method: arXiv 2408.11472.  Regular mode: complex sum of every scatterer into its
// range gate at each pulse (Section II.A, Fig. 1 step 4).  Fast mode: Algorithm 1 of
// Section III.B -- at each update pulse p_i the scatterer's complex amplitude C_i,
// range R_i and pulse-pair Doppler D_i = arg(conj(C_{i+1}) C_i) PRF are rasterised
// into a (gate, Doppler bin) spectrum.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rsim {

// Launch shape of the summation kernels (compile-time; the defaults are the tuned values).
#ifndef RSIM_THREADS
#define RSIM_THREADS 128
#endif
#ifndef RSIM_ITEMS
#define RSIM_ITEMS 8
#endif
#ifndef RSIM_MIN_BLOCKS
#define RSIM_MIN_BLOCKS 4
#endif
#ifndef RSIM_ITEMS_ANT
#define RSIM_ITEMS_ANT 4
#endif
#ifndef RSIM_MIN_BLOCKS_ANT
#define RSIM_MIN_BLOCKS_ANT 2
#endif
constexpr int kThreads = RSIM_THREADS;        // summation CTA size
constexpr int kItems = RSIM_ITEMS;            // consecutive scatterers per thread (2, 4, 8)
constexpr int kMinBlocks = RSIM_MIN_BLOCKS;   // resident CTAs per SM the register budget targets
constexpr int kChunk = kThreads * kItems;     // scatterers sharing one FP64 reference point
// The split summation kernels with a tabulated antenna pattern hold more per item, so they
// run the same chunk with fewer items per thread (and more threads).
constexpr int kItemsAnt = RSIM_ITEMS_ANT;
constexpr int kMinBlocksAnt = RSIM_MIN_BLOCKS_ANT;
__host__ __device__ constexpr int split_items(bool ant) { return ant ? kItemsAnt : kItems; }
constexpr int kTab = kThreads < 128 ? kThreads : 128;  // samples per block of reference constants
constexpr double kFixScale = 4294967296.0;    // fixed point: value = q * 2^-32
static_assert(kItems == 2 || kItems == 4 || kItems == 8, "items per thread");
static_assert(kChunk % kItemsAnt == 0 && (kChunk / kItemsAnt) % 32 == 0 && kChunk / kItemsAnt <= 1024,
              "antenna CTA shape");
static_assert(kThreads >= 64 && kThreads >= kTab && kThreads % 32 == 0, "CTA size");
// Split path: an FP32 gate / bin coordinate this close to an integer edge is re-decided
// in FP64.  The FP32 coordinate error grows with the coordinate's distance from the
// CTA reference point (about 3e-7 of it) on top of a few 1e-7 absolute, so the band is
// base + 4e-7 |coordinate| -- ten times the worst error seen.
constexpr float kGateEps = 2e-5f;
constexpr float kBinEps = 5e-6f;
constexpr float kEpsSlope = 4e-7f;
// 1.5 2^23: for |x| < 2^22, x + kRoundMagic is an integer-valued float whose bit pattern is
// that of kRoundMagic plus rint(x)
constexpr float kRoundMagic = 12582912.0f;
constexpr float kTwoPiF = 6.28318530717958647692f;
constexpr float kInvLn2F = 1.44269504088896340736f;

// Debug-build checks (compiled with -DRSIM_CHECK).  A failed check records its code and the
// offending value in the translation unit's check word (the first failure wins) and skips
// the access or addition it guards; the entry point reads the word once the call's kernels
// have run and returns RSIM_ERR_CHECK.  Without RSIM_CHECK every check is the constant true
// and costs nothing.
enum CheckCode : unsigned {
    kChkBin = 1,     // Doppler bin outside [0, n_doppler) when the cell key is formed
    kChkFixed = 2,   // a contribution sum at or beyond 2^30 (outside the fixed-point range)
    kChkSample = 3,  // sample slot outside the call's samples
    kChkGather = 4,  // adjoint gather cell outside [0, n_gates n_doppler)
};
#ifdef RSIM_CHECK
static __device__ unsigned long long g_check_word;
static __device__ __noinline__ void check_record(unsigned code, long long value) {
    const unsigned long long w = ((unsigned long long)code << 56) |
                                 ((unsigned long long)value & ((1ull << 56) - 1ull));
    atomicCAS(&g_check_word, 0ull, w);
}
#define RSIM_CHECK_OK(cond, code, value) \
    ((cond) || (::rsim::check_record((code), (long long)(value)), false))
#else
#define RSIM_CHECK_OK(cond, code, value) (true)
#endif

// Host-prepared constants of the model (kernel parameter).
struct Model {
    double prf, inv_prf;
    double p0[3];           // platform position at t = 0, relative to the scene origin
    double v[3];            // platform velocity
    double r_ref0, r_ref_rate;
    double two_over_lambda; // cycles of two-way phase per metre of range
    double inv_gw;          // 1 / gate width
    double half_gates;      // n_gates / 2
    double beam_k;          // exponent of 2 in the pattern: -2 / beamwidth^2
    double area;            // facet area
    int n_gates;
    int n_doppler;          // 1 in regular mode
    // FP32 copies for the split path
    float inv_gw_f, beam_k_f, chi_hi, chi_lo, dt_f, hdt_f, ep[3], inv_nd;
    float chi_lo_rad;       // -2 pi chi_lo: radians of phase per metre carried by chi_lo
    // off-nadir series in qb = beam_k rho^2 / D_z^2: beam_k atan(q)^2 = qb (1 + qb (s1 + qb s2))
    float s1, s2, qb_wide, inv_beam_k;
    // tabulated two-way pattern on a u-v grid (nullptr: the analytic Gaussian pattern)
    const float2* ant;      // [ant_nv][ant_nu] complex
    int ant_nu, ant_nv;
    double ant_u0, ant_v0, ant_idu, ant_idv;
    float ant_u0_f, ant_v0_f, ant_idu_f, ant_idv_f;
    float nd_over_2pi_f;    // n_doppler / (2 pi): radians of phase advance to bins
};

// Tabulated two-way pattern at the facet's direction cosines (u, v) = (s - P)_{x,y} / R
// (Section II.A: patterns recorded on a u-v grid, interpolated per facet): bilinear in the
// real and imaginary parts, 0 outside the grid.  Optionally the partial derivatives of the
// interpolant dG/du, dG/dv.  FP32 (split path) and FP64 versions.
__device__ __forceinline__ float2 pattern_f(const Model& m, float u, float v,
                                            float2* gu = nullptr, float2* gv = nullptr) {
    const float fu = __fmul_rn(u - m.ant_u0_f, m.ant_idu_f);  // not contracted into tu below
    const float fv = __fmul_rn(v - m.ant_v0_f, m.ant_idv_f);
    const float iu = floorf(fu), iv = floorf(fv);
    if (!(iu >= 0.0f && iu <= (float)(m.ant_nu - 2) && iv >= 0.0f && iv <= (float)(m.ant_nv - 2))) {
        if (gu) *gu = make_float2(0.f, 0.f);
        if (gv) *gv = make_float2(0.f, 0.f);
        return make_float2(0.f, 0.f);
    }
    const float tu = fu - iu, tv = fv - iv;
    const float2* p = m.ant + (int64_t)iv * m.ant_nu + (int64_t)iu;
    const float2 g00 = __ldg(p), g10 = __ldg(p + 1);
    const float2 g01 = __ldg(p + m.ant_nu), g11 = __ldg(p + m.ant_nu + 1);
    const float ax = fmaf(tu, g10.x - g00.x, g00.x), ay = fmaf(tu, g10.y - g00.y, g00.y);
    const float bx = fmaf(tu, g11.x - g01.x, g01.x), by = fmaf(tu, g11.y - g01.y, g01.y);
    if (gu) {
        const float cx = fmaf(tv, (g11.x - g01.x) - (g10.x - g00.x), g10.x - g00.x);
        const float cy = fmaf(tv, (g11.y - g01.y) - (g10.y - g00.y), g10.y - g00.y);
        *gu = make_float2(cx * m.ant_idu_f, cy * m.ant_idu_f);
        *gv = make_float2((bx - ax) * m.ant_idv_f, (by - ay) * m.ant_idv_f);
    }
    return make_float2(fmaf(tv, bx - ax, ax), fmaf(tv, by - ay, ay));
}

// The facet's cell of the grid and its bilinear weights, kept to evaluate the pattern at a
// nearby direction (the second pulse of the pair) without reloading the corners when that
// direction falls in the same cell.
struct PatCellF {
    float2 g00, g10, g01, g11;
    float iu, iv;
};

__device__ __forceinline__ float2 pattern_cell_f(const Model& m, float u, float v, PatCellF& c) {
    const float fu = __fmul_rn(u - m.ant_u0_f, m.ant_idu_f);  // not contracted into tu below
    const float fv = __fmul_rn(v - m.ant_v0_f, m.ant_idv_f);
    c.iu = floorf(fu);
    c.iv = floorf(fv);
    if (!(c.iu >= 0.0f && c.iu <= (float)(m.ant_nu - 2) && c.iv >= 0.0f &&
          c.iv <= (float)(m.ant_nv - 2))) {
        c.iu = -1.0f;  // outside: no cell
        return make_float2(0.f, 0.f);
    }
    const float2* p = m.ant + (int64_t)c.iv * m.ant_nu + (int64_t)c.iu;
    c.g00 = __ldg(p);
    c.g10 = __ldg(p + 1);
    c.g01 = __ldg(p + m.ant_nu);
    c.g11 = __ldg(p + m.ant_nu + 1);
    const float tu = fu - c.iu, tv = fv - c.iv;
    const float ax = fmaf(tu, c.g10.x - c.g00.x, c.g00.x), ay = fmaf(tu, c.g10.y - c.g00.y, c.g00.y);
    const float bx = fmaf(tu, c.g11.x - c.g01.x, c.g01.x), by = fmaf(tu, c.g11.y - c.g01.y, c.g01.y);
    return make_float2(fmaf(tv, bx - ax, ax), fmaf(tv, by - ay, ay));
}

// The pattern at (u, v), reusing cell c's corners when (u, v) lies in it (the same values
// pattern_f would load).
__device__ __forceinline__ float2 pattern_near_f(const Model& m, float u, float v,
                                                 const PatCellF& c) {
    const float fu = __fmul_rn(u - m.ant_u0_f, m.ant_idu_f);  // not contracted into tu below
    const float fv = __fmul_rn(v - m.ant_v0_f, m.ant_idv_f);
    const float iu = floorf(fu), iv = floorf(fv);
    // (a first point outside the table has no corners to reuse: c.iu = -1)
    if (c.iu < 0.0f || iu != c.iu || iv != c.iv) return pattern_f(m, u, v);
    const float tu = fu - iu, tv = fv - iv;
    const float ax = fmaf(tu, c.g10.x - c.g00.x, c.g00.x), ay = fmaf(tu, c.g10.y - c.g00.y, c.g00.y);
    const float bx = fmaf(tu, c.g11.x - c.g01.x, c.g01.x), by = fmaf(tu, c.g11.y - c.g01.y, c.g01.y);
    return make_float2(fmaf(tv, bx - ax, ax), fmaf(tv, by - ay, ay));
}

// arg(z) for the small phase steps of the pattern over one pulse: atan(t) = t (1 - t^2/3)
// to 1e-11 for |t| < 0.01 (t = Im z / Re z, Re z > 0), else the full atan2.
__device__ __forceinline__ float small_arg_f(float im, float re) {
    if (re > 0.0f && fabsf(im) < 0.01f * re) {
        const float t = __fdividef(im, re);
        return t * fmaf(t * t, -1.0f / 3.0f, 1.0f);
    }
    return atan2f(im, re);
}

__device__ __forceinline__ double2 pattern_d(const Model& m, double u, double v,
                                             double2* gu = nullptr, double2* gv = nullptr) {
    const double fu = (u - m.ant_u0) * m.ant_idu;
    const double fv = (v - m.ant_v0) * m.ant_idv;
    const double iu = floor(fu), iv = floor(fv);
    if (!(iu >= 0.0 && iu <= (double)(m.ant_nu - 2) && iv >= 0.0 && iv <= (double)(m.ant_nv - 2))) {
        if (gu) *gu = make_double2(0.0, 0.0);
        if (gv) *gv = make_double2(0.0, 0.0);
        return make_double2(0.0, 0.0);
    }
    const double tu = fu - iu, tv = fv - iv;
    const float2* p = m.ant + (int64_t)iv * m.ant_nu + (int64_t)iu;
    const float2 f00 = __ldg(p), f10 = __ldg(p + 1);
    const float2 f01 = __ldg(p + m.ant_nu), f11 = __ldg(p + m.ant_nu + 1);
    const double2 g00 = make_double2(f00.x, f00.y), g10 = make_double2(f10.x, f10.y);
    const double2 g01 = make_double2(f01.x, f01.y), g11 = make_double2(f11.x, f11.y);
    const double ax = fma(tu, g10.x - g00.x, g00.x), ay = fma(tu, g10.y - g00.y, g00.y);
    const double bx = fma(tu, g11.x - g01.x, g01.x), by = fma(tu, g11.y - g01.y, g01.y);
    if (gu) {
        const double cx = fma(tv, (g11.x - g01.x) - (g10.x - g00.x), g10.x - g00.x);
        const double cy = fma(tv, (g11.y - g01.y) - (g10.y - g00.y), g10.y - g00.y);
        *gu = make_double2(cx * m.ant_idu, cy * m.ant_idu);
        *gv = make_double2((bx - ax) * m.ant_idv, (by - ay) * m.ant_idv);
    }
    return make_double2(fma(tv, bx - ax, ax), fma(tv, by - ay, ay));
}

// Bins added to the pulse-pair Doppler coordinate by the tabulated pattern: Algorithm 1
// takes D_i from arg(conj(C_{i+1}) C_i), and C carries the pattern, so the pattern's own
// phase change between the facet's directions at the two pulses joins the geometric one.
// g1 = the pattern at the first pulse; d = P - s there; the second pulse sees
// d + (V - v) / PRF.
__device__ __forceinline__ double pattern_bin_shift_d(const Model& m, double dx, double dy,
                                                      double dz, double vx, double vy,
                                                      double vz, double2 g1) {
    const double dt = m.inv_prf;
    const double x2 = fma(m.v[0] - vx, dt, dx), y2 = fma(m.v[1] - vy, dt, dy);
    const double z2 = fma(m.v[2] - vz, dt, dz);
    const double R2 = sqrt(fma(x2, x2, fma(y2, y2, z2 * z2)));
    const double2 g2 = pattern_d(m, -x2 / R2, -y2 / R2);
    const double re = fma(g2.x, g1.x, g2.y * g1.y), im = fma(g2.y, g1.x, -g2.x * g1.y);
    return atan2(im, re) * ((double)m.n_doppler / 6.283185307179586476925);
}

// Sample schedule: sample s is pulse pulse_base + s * pulse_stride.
struct Schedule {
    int64_t pulse_base;
    int32_t pulse_stride;
    int32_t n_samples;
    int32_t samples_per_group;  // gridDim.y splits the samples into groups of this size
    int32_t pad;
};

struct Scat {
    const float *x, *y, *z, *vx, *vy, *vz, *nrcs;
    int64_t n;
    double t0;  // epoch of the state: s(t) = origin + r + v (t - t0)
    int vec4;   // all arrays 16-byte aligned: load 4 consecutive scatterers as float4
    int pad;
};

// Many scatterer sets (realizations of the same track) in one launch.  Per-set data ride
// in the kernel parameters (up to kMaxBatch sets per launch, 11.5 KB).
constexpr int kMaxBatch = 96;

struct BatchEntry {
    Scat sc;
    double p0[3];              // platform at t = 0 relative to this set's origin
    int64_t chunk_begin;       // first global chunk (CTA) index of this set
    unsigned long long* ws;    // this set's fixed-point workspace
    float area;                // facet area
    int pad;
};

struct BatchParams {
    int n_real;
    int pad;
    BatchEntry e[kMaxBatch];
};

// Surface states of a block of updates (Algorithm 1 regenerates the surface at every
// update): per update the heights and velocities of the set and their epoch; the horizontal
// positions and NRCS are the scatterer set's own.
constexpr int kMaxStates = 64;

struct StateEntry {
    const float *z, *vx, *vy, *vz;
    double t0;
};

struct StatesParams {
    int n;
    int pad;
    StateEntry s[kMaxStates];
};

struct FinalizeBatch {
    const void* ws[kMaxBatch];
    void* out[kMaxBatch];
};

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ int clamp_floor(double v) {
    return (int)floor(fmax(fmin(v, 1.0e9), -1.0e9));
}

// Platform coordinate i at time t, p0 = platform at t = 0 relative to the scatterers' origin.
__device__ __forceinline__ double platform_coord(const Model& m, const double* p0, int i, double t) {
    return fma(m.v[i], t, p0[i]);
}

// ---------------------------------------------------------------------------------------
// FP64 geometry of one scatterer at time t, platform at (Px, Py, Pz) relative to the
// origin, reference range rref.  Range excess in the cancellation-free form
// dR = (rho^2 + (dz - r_ref)(dz + r_ref)) / (R + r_ref).
struct GeomD {
    double dx, dy, dz, rho2, R, dR;
};

__device__ __forceinline__ GeomD geom_fp64(double t, double Px, double Py, double Pz, double rref,
                                           double x, double y, double z, double vx, double vy,
                                           double vz) {
    GeomD g;
    g.dx = Px - fma(vx, t, x);
    g.dy = Py - fma(vy, t, y);
    g.dz = Pz - fma(vz, t, z);
    g.rho2 = fma(g.dx, g.dx, g.dy * g.dy);
    g.R = sqrt(fma(g.dz, g.dz, g.rho2));
    g.dR = fma(g.dz - rref, g.dz + rref, g.rho2) / (g.R + rref);
    return g;
}

// Pre-floor pulse-pair Doppler bin coordinate nu n_doppler + 1/2 in FP64, with the range
// change over one PRI D = (2 d.e + |e|^2) / (R + R'), e = (V - v) dt, and
// nu = -2 D / lambda wrapped to [-1/2, 1/2) (phase advance of C per pulse, cycles).
__device__ __forceinline__ double bin_coord_fp64(const Model& m, const GeomD& g, double vx,
                                                 double vy, double vz) {
    const double dt = m.inv_prf;
    const double ex = (m.v[0] - vx) * dt, ey = (m.v[1] - vy) * dt, ez = (m.v[2] - vz) * dt;
    const double n2 = fma(2.0, fma(g.dx, ex, fma(g.dy, ey, g.dz * ez)),
                          fma(ex, ex, fma(ey, ey, ez * ez)));
    const double D0 = n2 / (2.0 * g.R);
    const double D = n2 / fma(2.0, g.R, D0);
    double nu = -D * m.two_over_lambda;
    nu -= rint(nu);
    return fma(nu, (double)m.n_doppler, 0.5);
}

// Per-sample constants of the FP64 path.
struct Fp64Const {
    double t;                // scatterer time since the set's epoch, t_pulse - t0
    double Px, Py, Pz;       // platform at t_pulse relative to the origin
    double rref;             // r_ref(t_pulse)
    double psiref;           // 2 r_ref / lambda - rint(.)  [cycles]
    int active;              // 0: no scatterer of the CTA can fall in the range window
    int index;               // sample index (set when the table is compacted)
};

__device__ __forceinline__ Fp64Const make_fp64_const(const Model& m, const double* p0, double t0,
                                                     int64_t pulse) {
    Fp64Const k;
    const double tp = (double)pulse * m.inv_prf;
    k.t = tp - t0;
    k.Px = platform_coord(m, p0, 0, tp);
    k.Py = platform_coord(m, p0, 1, tp);
    k.Pz = platform_coord(m, p0, 2, tp);
    k.rref = fma(m.r_ref_rate, tp, m.r_ref0);
    const double psi = k.rref * m.two_over_lambda;
    k.psiref = psi - rint(psi);
    k.active = 1;
    k.index = 0;
    return k;
}

// Culling bound of a CTA: every scatterer of the chunk lies within |l(t)| <= lmax + vmax |t|
// (t counted from the set's epoch)
// of the reference point c, and |R - R_c| <= |l(t)| (triangle inequality), so its gate
// coordinate lies within that distance / gate width of c's.  A sample whose band misses
// the window [0, n_gates) has no contribution from the CTA.  G = gate coordinate of c.
__device__ __forceinline__ int window_reachable(const Model& m, double G, double t, float lmax,
                                                float vmax) {
    const double B = ((double)lmax + (double)vmax * fabs(t)) * m.inv_gw + 2.0;
    return (G + B >= 0.0 && G - B < (double)m.n_gates) ? 1 : 0;
}

// Window test of a CTA at one pulse: G is the gate coordinate of its reference point
// (cx, cy, 0) (the same value make_split_const computes).
__device__ __forceinline__ int cta_reaches_window(const Model& m, const double* p0, double t0,
                                                  int64_t pulse, float cx, float cy, float lmax,
                                                  float vmax) {
    const double t = (double)pulse * m.inv_prf;
    const double Dx = platform_coord(m, p0, 0, t) - (double)cx;
    const double Dy = platform_coord(m, p0, 1, t) - (double)cy;
    const double Dz = platform_coord(m, p0, 2, t);
    const double rref = fma(m.r_ref_rate, t, m.r_ref0);
    // R_c - r_ref = (D_x^2 + D_y^2 + (D_z - r_ref)(D_z + r_ref)) / (R_c + r_ref), the
    // cancelling difference taken in FP64, the rest in FP32 (no FP64 square root); with
    // R_c + r_ref from one refinement the relative error is ~1e-7 + (dR / 2 r_ref)^2, far
    // inside the 2-gate margin of the bound
    const float num = fmaf((float)Dx, (float)Dx,
                           fmaf((float)Dy, (float)Dy, (float)(Dz - rref) * (float)(Dz + rref)));
    const float two_r = 2.0f * (float)rref;
    const float d1 = num / two_r;
    const float dR = num / (two_r + d1);
    const double G = (double)dR * m.inv_gw + m.half_gates;
    return window_reachable(m, G, t - t0, lmax, vmax);
}

// ---------------------------------------------------------------------------------------
// Per (reference point c, sample) constants of the split path, computed in FP64 once per
// CTA and sample, rounded to FP32 and packed for 128-bit shared-memory loads.
// D = P(t) - origin - c, R_c = |D|, e_p = platform displacement over one PRI.
struct __align__(16) SplitConst {
    float4 a;   // t - t0 (scatterer time since the set's epoch), D_x, D_y, D_z
    float4 b;   // D / R_c (x, y, z), 1 / (2 R_c)
    float4 c;   // 1 / R_c, frac of the gate coordinate of c less 1/2,
                // -2 pi (2 R_c / lambda - rint(.)) [rad], log2 (r_ref/R_c)^2
    float4 d;   // beam_k / D_z^2, K0 = M . e_p as hi + lo (M = D + e_p/2), -n_doppler 2 / (lambda R_c)
    float4 e;   // floor of the gate coordinate of c (int bits); active flag, then the sample
                // index (int bits); the sample's workspace slice (pointer bits, lo + hi)
    float4 f;   // beam series offsets qA0 = (D_x^2 + D_y^2) beam_k / D_z^2 and
                // qA1 = 2 R_c beam_k / D_z^2; unused; band of the FP32 gate decision
};

// Register copy of one table entry.
struct SampleF {
    float t, Dx, Dy, Dz, ux, uy, uz, h, invRc, gfrac_h, psic, l2kappa, kq, K0hi, K0lo, kbin;
    float qA0, qA1, gthr;
    int gint;
};

__device__ __forceinline__ int sample_index(const SplitConst& s) { return __float_as_int(s.e.y); }

// After the activity test: the entry carries its sample index and output slice instead.
__device__ __forceinline__ void set_sample_slot(SplitConst& s, int index,
                                                unsigned long long* out) {
    const unsigned long long u = reinterpret_cast<unsigned long long>(out);
    s.e.y = __int_as_float(index);
    s.e.z = __uint_as_float((unsigned)(u & 0xffffffffull));
    s.e.w = __uint_as_float((unsigned)(u >> 32));
}

// Workspace slice of a table entry (read where it is used, so no register holds it
// across the evaluation).
__device__ __forceinline__ unsigned long long* sample_out(const SplitConst& s) {
    const float2 p = *reinterpret_cast<const float2*>(&s.e.z);
    return reinterpret_cast<unsigned long long*>(
        ((unsigned long long)__float_as_uint(p.y) << 32) | __float_as_uint(p.x));
}

__device__ __forceinline__ SampleF load_sample(const SplitConst& s) {
    const float4 a = s.a, b = s.b, c = s.c, d = s.d, f = s.f;
    SampleF k;
    k.t = a.x; k.Dx = a.y; k.Dy = a.z; k.Dz = a.w;
    k.ux = b.x; k.uy = b.y; k.uz = b.z; k.h = b.w;
    k.invRc = c.x; k.gfrac_h = c.y; k.psic = c.z; k.l2kappa = c.w;
    k.kq = d.x; k.K0hi = d.y; k.K0lo = d.z; k.kbin = d.w;
    k.qA0 = f.x; k.qA1 = f.y; k.gthr = f.w;
    k.gint = __float_as_int(s.e.x);
    return k;
}

__device__ __forceinline__ SplitConst make_split_const(const Model& m, const double* p0,
                                                       double t0, int64_t pulse, float cx,
                                                       float cy, float lmax, float vmax) {
    const double t = (double)pulse * m.inv_prf;
    const double ts = t - t0;
    const double Dx = platform_coord(m, p0, 0, t) - (double)cx;
    const double Dy = platform_coord(m, p0, 1, t) - (double)cy;
    const double Dz = platform_coord(m, p0, 2, t);
    const double Rc = sqrt(Dx * Dx + Dy * Dy + Dz * Dz);
    const double rref = fma(m.r_ref_rate, t, m.r_ref0);
    const double G = (Rc - rref) * m.inv_gw + m.half_gates;
    const double Gi = floor(G);
    double psi = Rc * m.two_over_lambda;
    psi -= rint(psi);
    // 1 / R_c from the FP32 reciprocal and one Newton step (FP64 accurate, no FP64 divide:
    // the FP64 pipe is 1/64 of FP32 and this runs once per CTA and sample)
    const double inv0 = (double)(1.0f / (float)Rc);
    const double inv = fma(inv0, fma(-Rc, inv0, 1.0), inv0);
    const double dt = m.inv_prf;
    const double epx = m.v[0] * dt, epy = m.v[1] * dt, epz = m.v[2] * dt;
    const double K0 = (Dx + 0.5 * epx) * epx + (Dy + 0.5 * epy) * epy + (Dz + 0.5 * epz) * epz;
    const float K0hi = (float)K0;
    // log2 (r_ref / R_c)^2 = 2 log2(1 + x), x = (r_ref - R_c) / R_c tiny: FP32 log1p of the
    // FP64 difference; beam_k / D_z^2 in FP32 (a float constant either way)
    const float xref = (float)((rref - Rc) * inv);
    const float invDz = 1.0f / (float)Dz;
    const float kq = m.beam_k_f * invDz * invDz;
    SplitConst k;
    k.a = make_float4((float)ts, (float)Dx, (float)Dy, (float)Dz);
    k.b = make_float4((float)(Dx * inv), (float)(Dy * inv), (float)(Dz * inv), (float)(0.5 * inv));
    k.c = make_float4((float)inv, (float)(G - Gi - 0.5), (float)(-6.283185307179586476925 * psi),
                      2.0f * kInvLn2F * log1pf(xref));
    k.d = make_float4(kq, K0hi, (float)(K0 - (double)K0hi),
                      (float)(-(double)m.n_doppler * m.two_over_lambda * inv));
    const double gi = fmax(fmin(Gi, 1.0e9), -1.0e9);
    k.e = make_float4(__int_as_float((int)gi),
                      __int_as_float(window_reachable(m, G, ts, lmax, vmax)), 0.f, 0.f);
    // an item inside the window has |gate coordinate - gi| <= max(|gi|, |n_gates - gi|): the
    // FP32 error of its coordinate grows with that bound (out-of-window items need no band)
    const double gspan = fmax(fabs(gi), fabs((double)m.n_gates - gi)) + 2.0;
    k.f = make_float4((float)((Dx * Dx + Dy * Dy) * (double)kq), (float)(2.0 * Rc * (double)kq),
                      0.f, (float)(0.5 - (double)kGateEps - (double)kEpsSlope * gspan));
    return k;
}

// Scatterer registers of the split path (positions relative to the CTA reference point).
// The pulse-pair range change needs (d + e/2).e with d = D - l, e = e_p - v dt the
// scatterer's displacement relative to the platform over one PRI and D = P(t) - c linear in
// t: (d + e/2).e = K0 - [dt (D.v) + l.e_p + c1], and with l = l0 + v t, D = Q + V t
// (Q = P(t0) - c, t counted from the set's epoch) the bracket is gam + t beta, where
// gam = l0.e + c1 + dt (Q.v) and beta = v.e + e_p.v carry the item's part
// (c1 = dt e_p.v - dt^2 |v|^2 / 2, l0 = (lx0, ly0, z) the position at the epoch).
struct ItemF {
    float lx0, ly0, z, vx, vy, vz, amp0, gam, beta;  // padding past the end of a set: amp0 = 0
};

// Quantities the adjoint needs besides C.
struct DerivF {
    float dlna;  // d ln|C| / dz, without the tabulated pattern's own variation
    float dphi;  // d arg C / dz  [rad / m]
    float2 pat;  // tabulated pattern only: a e^{-j 2 pi f} dG/dz (0 otherwise)
};

// Result flags of the fast evaluation.
constexpr int kFlagRefine = 1;  // gate or bin coordinate within rounding of a cell edge
constexpr int kFlagWide = 2;    // off-nadir angle beyond the series' range (q^2 >= 0.01)
// Key of an item the fast evaluation defers to the exact one (distinct from -1, out of the
// window; both are below every cell key).
constexpr int kKeyDeferred = -2;

// FP64 re-decision of the gate and bin of one scatterer (kept out of line so that none of
// its FP64 work is hoisted into the common path).
template <bool ANT>
static __device__ __noinline__ void refine_fp64(const Model& m, const Fp64Const& k64, double x, double y,
                                         double z, double vx, double vy, double vz, bool doppler,
                                         int* g, int* kb, double* gc, double* bc) {
    const GeomD gd = geom_fp64(k64.t, k64.Px, k64.Py, k64.Pz, k64.rref, x, y, z, vx, vy, vz);
    *gc = fma(gd.dR, m.inv_gw, m.half_gates);
    *g = clamp_floor(*gc);
    *kb = 0;
    *bc = 0.5;
    if (doppler) {
        *bc = bin_coord_fp64(m, gd, vx, vy, vz);
        if (ANT) {
            const double2 g1 = pattern_d(m, -gd.dx / gd.R, -gd.dy / gd.R);
            *bc += pattern_bin_shift_d(m, gd.dx, gd.dy, gd.dz, vx, vy, vz, g1);
        }
        *kb = clamp_floor(*bc) & (m.n_doppler - 1);
    }
}

// Split-path evaluation of one scatterer at one sample.  Returns the cell key
// g * n_doppler + bin, or -1 when out of the range window or not a scatterer.
// GENERAL = false: straight-line code; items that need the FP64 re-decision or the exact
//   off-nadir angle are only flagged, and their key is kKeyDeferred (the caller
//   re-evaluates them with GENERAL = true).
// GENERAL = true: takes those branches (tab64 and the scatterer's original x, y needed).
// For unflagged items both give bit-identical results.
template <bool DOPPLER, bool GENERAL, bool DERIV, bool ANT = false>
__device__ __forceinline__ int eval_split(const Model& m, const SampleF& k, const ItemF& it,
                                          float& re, float& im, int& flags,
                                          const Fp64Const* k64 = nullptr, float x_orig = 0.f,
                                          float y_orig = 0.f, DerivF* dv = nullptr,
                                          int* g_out = nullptr, double* gc_out = nullptr,
                                          double* bc_out = nullptr) {
    const float lx = fmaf(it.vx, k.t, it.lx0);
    const float ly = fmaf(it.vy, k.t, it.ly0);
    const float lz = fmaf(it.vz, k.t, it.z);
    // R - R_c = (|l|^2 - 2 D.l) / (R + R_c); -u.l and |l|^2 built from their horizontal
    // parts, which the beam angle below reuses
    const float nuxy = fmaf(-k.ux, lx, __fmul_rn(-k.uy, ly));
    const float nul = fmaf(-k.uz, lz, nuxy);
    const float lxy2 = fmaf(lx, lx, __fmul_rn(ly, ly));
    const float ll = fmaf(lz, lz, lxy2);
    const float dR0 = fmaf(ll, k.h, nul);
    const float dR = __fmul_rn(dR0, fmaf(-dR0, k.h, 1.0f));
    // gate: the coordinate less 1/2 (gch), rounded to the nearest integer, is the offset from
    // the reference gate, read from the low mantissa bits of gch + 1.5 2^23 (|gch| < 2^22; a
    // larger |gch| lands outside the window, or the sample's band flags every item); cell
    // edges sit at half-integers of gch, and items within the band of one are re-decided in
    // FP64
    const float gch = fmaf(dR, m.inv_gw_f, k.gfrac_h);
    const float gr = gch + kRoundMagic;
    int g = k.gint + (__float_as_int(gr) - __float_as_int(kRoundMagic));
    const bool gflag = fabsf(fmaf(gr - kRoundMagic, -1.0f, gch)) > k.gthr;
    bool wide = false, bflag = false;
    // |C| = sqrt(sigma A) 2^E, E = beam_k atan(q)^2 + log2 (r_ref/R_c)^2 - 2 log2(1 + dR/R_c),
    // q = rho / d_z (series in qb = beam_k q^2 below 0.01 q^2; the exact angle beyond), with
    // qb = beam_k rho^2 / D_z^2 and rho^2 = |D_xy - l_xy|^2 = |D_xy|^2 - 2 R_c u_xy.l + |l_xy|^2
    const float dx = k.Dx - lx, dy = k.Dy - ly;
    const float qb = fmaf(k.qA1, nuxy, fmaf(lxy2, k.kq, k.qA0));
    float T = k.l2kappa;  // tabulated pattern: applied to C below
    if (!ANT) {
        T = fmaf(qb, fmaf(qb, fmaf(qb, m.s2, m.s1), 1.0f), k.l2kappa);
        wide = qb < m.qb_wide;
        if (wide) {
            if (GENERAL) {
                const float th = atan2f(sqrtf(fmaf(dx, dx, dy * dy)), k.Dz - lz);
                T = fmaf(th * th, m.beam_k_f, k.l2kappa);
            }
        }
    }
    // products that later meet an addition are rounded on their own (__fmul_rn is never
    // contracted into an FMA), as in the paired evaluation
    const float xr = __fmul_rn(dR, k.invRc);
    const float E = fmaf(xr, fmaf(xr, kInvLn2F, -2.0f * kInvLn2F), T);
    const float a = it.amp0 * ex2_approx(E);
    // phase psi_c + dR 2/lambda in cycles, reduced to [-1/2, 1/2] (2/lambda as hi + lo: the
    // integer part leaves dR chi_hi exactly in one FMA), taken as the argument -2 pi f in
    // radians so that C = a (cos, sin) of it; psi_c and the chi_lo term are carried in
    // radians (|arg| <= 2 pi: the hardware sine and cosine take their arguments modulo one turn)
    const float nk = rintf(__fmul_rn(dR, -m.chi_hi));
    const float fr = fmaf(dR, m.chi_hi, nk);
    const float arg = fmaf(dR, m.chi_lo_rad, fmaf(fr, -kTwoPiF, k.psic));
    float sn, cs;
    __sincosf(arg, &sn, &cs);
    float2 gu, gv, G;
    PatCellF cell;
    float pu = 0.f, pv = 0.f, pat_bins = 0.f;
    if (ANT) {
        // C = a G(u, v) e^{-j 2 pi f}, (u, v) = -(d_x, d_y) / R, 1 / R = (1 / R_c)(1 - dR / R_c)
        // (the bracket one FMA, as the paired evaluation forms it)
        const float invR = k.invRc * fmaf(dR, -k.invRc, 1.0f);
        pu = __fmul_rn(-dx, invR);  // rounded before the table look-up subtracts u0
        pv = __fmul_rn(-dy, invR);
        if (DERIV) G = pattern_f(m, pu, pv, &gu, &gv);
        else G = pattern_cell_f(m, pu, pv, cell);
        if (DOPPLER) {
            // the pattern's phase change over the pulse pair joins the Doppler
            // (Algorithm 1 takes it from arg(conj(C2) C1)); d at the second pulse is
            // d + e_p - v dt
            const float ex = fmaf(-it.vx, m.dt_f, m.ep[0]), ey = fmaf(-it.vy, m.dt_f, m.ep[1]);
            const float u2 = __fmul_rn(-(dx + ex), invR), v2 = __fmul_rn(-(dy + ey), invR);
            const float2 G2 = DERIV ? pattern_f(m, u2, v2) : pattern_near_f(m, u2, v2, cell);
            const float pr = fmaf(G2.x, G.x, G2.y * G.y), pi = fmaf(G2.y, G.x, -G2.x * G.y);
            pat_bins = __fmul_rn(small_arg_f(pi, pr), m.nd_over_2pi_f);
        }
        // e^{-j 2 pi f} = cs + j sn
        re = a * fmaf(G.x, cs, -G.y * sn);
        im = a * fmaf(G.y, cs, G.x * sn);
    } else {
        re = a * cs;
        im = a * sn;
    }
    int kb = 0;
    float b = 0.0f;
    if (DOPPLER) {
        // pulse-pair range change D = 2 (d + e/2).e / (R + R'), (d + e/2).e = K0 - (gam + t beta);
        // b = nu n_doppler = -n_doppler 2 D / lambda (unwrapped: the bin is taken mod
        // n_doppler); bin = nearest integer to b
        const float item = fmaf(k.t, it.beta, it.gam);
        b = ((k.K0hi - item) + k.K0lo) * k.kbin;
        b = fmaf(b, -xr, b);                       // 1 / (R_c + dR) = (1 / R_c)(1 - dR / R_c)
        if (ANT) b += pat_bins;
        // nearest integer mod n_doppler (a power of two <= 2^22) from the low mantissa bits;
        // beyond |b| ~ 1e6 the band below flags every item
        const float bm = b + kRoundMagic;
        kb = __float_as_int(bm) & (m.n_doppler - 1);
        bflag = fabsf(fmaf(bm - kRoundMagic, -1.0f, b)) > fmaf(-fabsf(b), kEpsSlope, 0.5f - kBinEps);
    }
    if (DERIV) {
        // dR/dz = -d_z / R, dtheta/dz = rho / R^2,
        // d ln a / dz = 2 d_z / R^2 - 4 ln2 theta rho / (theta_b^2 R^2), d phi / dz = 4 pi d_z / (lambda R)
        const float dz = k.Dz - lz;
        const float invR = k.invRc * fmaf(dR, -k.invRc, 1.0f);
        const float invR2 = invR * invR;
        dv->dphi = kTwoPiF * (m.chi_hi + m.chi_lo) * dz * invR;  // chi = 2 / lambda
        if (ANT) {
            // d/dz of the pattern: dG/du du/dz + dG/dv dv/dz, du/dz = u d_z / R^2 (same for v)
            dv->dlna = 2.0f * dz * invR2;
            const float su = pu * dz * invR2, svv = pv * dz * invR2;
            const float dgx = fmaf(gu.x, su, gv.x * svv), dgy = fmaf(gu.y, su, gv.y * svv);
            dv->pat = make_float2(a * fmaf(dgx, cs, -dgy * sn), a * fmaf(dgy, cs, dgx * sn));
        } else {
            const float rho2 = fmaf(dx, dx, dy * dy);
            const float q2 = qb * m.inv_beam_k;
            float rho_theta;
            if (q2 < 1e-2f) {
                rho_theta = rho2 / dz * fmaf(q2, fmaf(q2, 0.2f, -1.0f / 3.0f), 1.0f);
            } else {
                rho_theta = sqrtf(rho2) * atan2f(sqrtf(rho2), dz);
            }
            // beam_k = -2 / theta_b^2 (base 2), so -4 ln2 / theta_b^2 = 2 ln2 beam_k
            dv->dlna = (2.0f * dz + 1.38629436111989061883f * m.beam_k_f * rho_theta) * invR2;
            dv->pat = make_float2(0.f, 0.f);
        }
    }
    double gcd = (double)k.gint + (double)gch + 0.5;
    double bcd = (double)b - (double)m.n_doppler * rint((double)b / (double)m.n_doppler) + 0.5;
    const bool refine = gflag || bflag;
    if (GENERAL && refine) {
        int g2, kb2;
        refine_fp64<ANT>(m, *k64, (double)x_orig, (double)y_orig, (double)it.z, (double)it.vx,
                    (double)it.vy, (double)it.vz, DOPPLER, &g2, &kb2, &gcd, &bcd);
        g = g2;
        kb = kb2;
    }
    flags = (refine ? kFlagRefine : 0) | (wide ? kFlagWide : 0);
    if (g_out) *g_out = g;
    if (gc_out) *gc_out = gcd;
    if (bc_out) *bc_out = bcd;
    // padding items (past the end of the set) carry zero amplitude: harmless in any cell
    int key = ((unsigned)g < (unsigned)m.n_gates) ? g * m.n_doppler + kb : -1;
    if (!RSIM_CHECK_OK((unsigned)kb < (unsigned)m.n_doppler, kChkBin, kb)) key = -1;
    return (!GENERAL && (refine || wide)) ? kKeyDeferred : key;
}

// Two scatterers (items 2p and 2p + 1 of a thread) as lanes of packed FP32 pairs.
struct ItemF2 {
    float2 lx0, ly0, z, vx, vy, vz, amp0, gam, beta;
};

__device__ __forceinline__ ItemF2 pack_items(const ItemF& a, const ItemF& b) {
    ItemF2 r;
    r.lx0 = make_float2(a.lx0, b.lx0);
    r.ly0 = make_float2(a.ly0, b.ly0);
    r.z = make_float2(a.z, b.z);
    r.vx = make_float2(a.vx, b.vx);
    r.vy = make_float2(a.vy, b.vy);
    r.vz = make_float2(a.vz, b.vz);
    r.amp0 = make_float2(a.amp0, b.amp0);
    r.gam = make_float2(a.gam, b.gam);
    r.beta = make_float2(a.beta, b.beta);
    return r;
}

__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }

// Bilinear interpolation of the corners of cells c0 and c1 at (tu, tv) for two points as
// the lanes of pairs (real parts in gx, imaginary parts in gy): each lane's operations are
// those of pattern_cell_f's interpolation (b - a as fma(a, -1, b), exact).
__device__ __forceinline__ void pattern_interp_f2(const PatCellF& c0, const PatCellF& c1,
                                                  float2 tu, float2 tv, float2& gx,
                                                  float2& gy) {
    const float2 neg1 = f2(-1.0f);
    const float2 g00x = make_float2(c0.g00.x, c1.g00.x), g00y = make_float2(c0.g00.y, c1.g00.y);
    const float2 g10x = make_float2(c0.g10.x, c1.g10.x), g10y = make_float2(c0.g10.y, c1.g10.y);
    const float2 g01x = make_float2(c0.g01.x, c1.g01.x), g01y = make_float2(c0.g01.y, c1.g01.y);
    const float2 g11x = make_float2(c0.g11.x, c1.g11.x), g11y = make_float2(c0.g11.y, c1.g11.y);
    const float2 ax = __ffma2_rn(tu, __ffma2_rn(g00x, neg1, g10x), g00x);
    const float2 ay = __ffma2_rn(tu, __ffma2_rn(g00y, neg1, g10y), g00y);
    const float2 bx = __ffma2_rn(tu, __ffma2_rn(g01x, neg1, g11x), g01x);
    const float2 by = __ffma2_rn(tu, __ffma2_rn(g01y, neg1, g11y), g01y);
    gx = __ffma2_rn(tv, __ffma2_rn(ax, neg1, bx), ax);
    gy = __ffma2_rn(tv, __ffma2_rn(ay, neg1, by), ay);
}

// pattern_cell_f for two points as the lanes of pairs, without a branch: a point outside
// the table loads the table's first cell and gives 0 (and c.iu = -1), as pattern_cell_f.
// Per lane the same values as two pattern_cell_f calls.  The grid coordinates
// (u - u0) / du are formed lane by lane in scalar FP32: u is a paired product, and a paired
// product that feeds a paired addition can come out of code generation as one paired FMA
// (one rounding where the scalar form rounds twice), even from the _rn intrinsics.
__device__ __forceinline__ void pattern_cell_f2(const Model& m, float2 u, float2 v, float2& gx,
                                                float2& gy, PatCellF& c0, PatCellF& c1) {
    const float2 fu = make_float2(__fmul_rn(u.x - m.ant_u0_f, m.ant_idu_f),
                                  __fmul_rn(u.y - m.ant_u0_f, m.ant_idu_f));
    const float2 fv = make_float2(__fmul_rn(v.x - m.ant_v0_f, m.ant_idv_f),
                                  __fmul_rn(v.y - m.ant_v0_f, m.ant_idv_f));
    const float2 iu = make_float2(floorf(fu.x), floorf(fu.y));
    const float2 iv = make_float2(floorf(fv.x), floorf(fv.y));
    const float umax = (float)(m.ant_nu - 2), vmax = (float)(m.ant_nv - 2);
    const bool in0 = iu.x >= 0.0f && iu.x <= umax && iv.x >= 0.0f && iv.x <= vmax;
    const bool in1 = iu.y >= 0.0f && iu.y <= umax && iv.y >= 0.0f && iv.y <= vmax;
    const int o0 = in0 ? (int)iv.x * m.ant_nu + (int)iu.x : 0;
    const int o1 = in1 ? (int)iv.y * m.ant_nu + (int)iu.y : 0;
    c0.g00 = __ldg(m.ant + o0);
    c0.g10 = __ldg(m.ant + o0 + 1);
    c0.g01 = __ldg(m.ant + o0 + m.ant_nu);
    c0.g11 = __ldg(m.ant + o0 + m.ant_nu + 1);
    c1.g00 = __ldg(m.ant + o1);
    c1.g10 = __ldg(m.ant + o1 + 1);
    c1.g01 = __ldg(m.ant + o1 + m.ant_nu);
    c1.g11 = __ldg(m.ant + o1 + m.ant_nu + 1);
    c0.iu = in0 ? iu.x : -1.0f;
    c0.iv = iv.x;
    c1.iu = in1 ? iu.y : -1.0f;
    c1.iv = iv.y;
    const float2 neg1 = f2(-1.0f);
    pattern_interp_f2(c0, c1, __ffma2_rn(iu, neg1, fu), __ffma2_rn(iv, neg1, fv), gx, gy);
    if (!in0) { gx.x = 0.0f; gy.x = 0.0f; }
    if (!in1) { gx.y = 0.0f; gy.y = 0.0f; }
}

// pattern_near_f for two points as the lanes of pairs: both in their first point's cell
// (the usual case over one pulse), the corners are reused as pairs; otherwise each lane
// takes pattern_near_f.  Per lane the same values as two pattern_near_f calls (the grid
// coordinates lane by lane, as pattern_cell_f2).
__device__ __forceinline__ void pattern_near_f2(const Model& m, float2 u, float2 v,
                                                const PatCellF& c0, const PatCellF& c1,
                                                float2& gx, float2& gy) {
    const float2 fu = make_float2(__fmul_rn(u.x - m.ant_u0_f, m.ant_idu_f),
                                  __fmul_rn(u.y - m.ant_u0_f, m.ant_idu_f));
    const float2 fv = make_float2(__fmul_rn(v.x - m.ant_v0_f, m.ant_idv_f),
                                  __fmul_rn(v.y - m.ant_v0_f, m.ant_idv_f));
    const float2 iu = make_float2(floorf(fu.x), floorf(fu.y));
    const float2 iv = make_float2(floorf(fv.x), floorf(fv.y));
    const bool same = c0.iu >= 0.0f && iu.x == c0.iu && iv.x == c0.iv &&
                      c1.iu >= 0.0f && iu.y == c1.iu && iv.y == c1.iv;
    if (same) {
        const float2 neg1 = f2(-1.0f);
        pattern_interp_f2(c0, c1, __ffma2_rn(iu, neg1, fu), __ffma2_rn(iv, neg1, fv), gx, gy);
    } else {
        const float2 h0 = pattern_near_f(m, u.x, v.x, c0), h1 = pattern_near_f(m, u.y, v.y, c1);
        gx = make_float2(h0.x, h1.x);
        gy = make_float2(h0.y, h1.y);
    }
}

// eval_split<DOPPLER, GENERAL = false, DERIV = false, ANT> for two scatterers at once on
// the paired FP32 instructions (fma / add / mul .f32x2: one issue slot for both); the
// tabulated pattern's look-ups run per lane.
// Every pair operation rounds each lane as the scalar operation it replaces, and the
// negations the pair forms cannot take as operand modifiers are exact rewrites
// (fma(x, -1, y) = y - x, products with negated constants), so each lane's key, re and im
// are bit-identical to the scalar evaluation's.  No paired product is an operand of a
// paired addition (code generation may fuse the two into one FFMA2): such a sum is written
// as an FMA on both sides, or taken per lane in scalar FP32.
// Keys: g n_doppler + bin inside the range window; every item outside it gets the one key
// n_gates n_doppler (an unsigned minimum: negative gates wrap to large unsigned values), which
// the emission drops; items the exact evaluation must take get kKeyDeferred, and `defer`
// reports whether either of the two did.
template <bool DOPPLER, bool ANT>
__device__ __forceinline__ void eval_split_pair(const Model& m, const SampleF& k, const ItemF2& it,
                                                int& key0, int& key1, float2& re, float2& im,
                                                bool& defer) {
    const float2 one = f2(1.0f), neg1 = f2(-1.0f);
    const float2 t2 = f2(k.t);
    const float2 lx = __ffma2_rn(it.vx, t2, it.lx0);
    const float2 ly = __ffma2_rn(it.vy, t2, it.ly0);
    const float2 lz = __ffma2_rn(it.vz, t2, it.z);
    // -u.l and |l|^2 from their horizontal parts (as eval_split; the signs ride on constants)
    const float2 nuxy = __ffma2_rn(f2(-k.ux), lx, __fmul2_rn(f2(-k.uy), ly));
    const float2 nul = __ffma2_rn(f2(-k.uz), lz, nuxy);
    const float2 lxy2 = __ffma2_rn(lx, lx, __fmul2_rn(ly, ly));
    const float2 ll = __ffma2_rn(lz, lz, lxy2);
    const float2 dR0 = __ffma2_rn(ll, f2(k.h), nul);
    const float2 dR = __fmul2_rn(dR0, __ffma2_rn(dR0, f2(-k.h), one));
    // gate (as eval_split)
    const float2 gch = __ffma2_rn(dR, f2(m.inv_gw_f), f2(k.gfrac_h));
    const float2 gr = __fadd2_rn(gch, f2(kRoundMagic));
    const float2 gd = __ffma2_rn(__fadd2_rn(gr, f2(-kRoundMagic)), neg1, gch);
    const int g0 = k.gint + (__float_as_int(gr.x) - __float_as_int(kRoundMagic));
    const int g1 = k.gint + (__float_as_int(gr.y) - __float_as_int(kRoundMagic));
    // amplitude (the tabulated pattern multiplies C below)
    float2 T = f2(k.l2kappa), qb = f2(0.0f), ndx, ndy;
    if (!ANT) {
        qb = __ffma2_rn(f2(k.qA1), nuxy, __ffma2_rn(lxy2, f2(k.kq), f2(k.qA0)));
        T = __ffma2_rn(qb, __ffma2_rn(qb, __ffma2_rn(qb, f2(m.s2), f2(m.s1)), one), T);
    } else {
        ndx = __ffma2_rn(f2(k.Dx), neg1, lx);   // -d_x = l_x - D_x (exact negation)
        ndy = __ffma2_rn(f2(k.Dy), neg1, ly);
    }
    // -x_r = -dR / R_c; E = x_r (x_r c - 2c) + T = (-x_r)((-x_r) c + 2c) + T
    const float2 nxr = __fmul2_rn(dR, f2(-k.invRc));
    const float2 E = __ffma2_rn(nxr, __ffma2_rn(nxr, f2(kInvLn2F), f2(2.0f * kInvLn2F)), T);
    const float2 a = __fmul2_rn(it.amp0, make_float2(ex2_approx(E.x), ex2_approx(E.y)));
    // phase (as eval_split): -k = rint(-dR chi_hi), fr = dR chi_hi - k,
    // arg = dR (-2 pi chi_lo) + (fr (-2 pi) + psi_c [rad])
    const float2 np = __fmul2_rn(dR, f2(-m.chi_hi));
    const float2 fr = __ffma2_rn(dR, f2(m.chi_hi), make_float2(rintf(np.x), rintf(np.y)));
    const float2 arg = __ffma2_rn(dR, f2(m.chi_lo_rad), __ffma2_rn(fr, f2(-kTwoPiF), f2(k.psic)));
    float2 sn, cs;
    __sincosf(arg.x, &sn.x, &cs.x);
    __sincosf(arg.y, &sn.y, &cs.y);
    float2 pat_bins = f2(0.0f);
    if (!ANT) {
        re = __fmul2_rn(a, cs);
        im = __fmul2_rn(a, sn);
    } else {
        // (u, v) = -(d_x, d_y) / R with 1 / R = (1 / R_c)(1 - dR / R_c), the bracket one FMA,
        // as eval_split
        const float2 invR = __fmul2_rn(f2(k.invRc), __ffma2_rn(dR, f2(-k.invRc), one));
        const float2 pu = __fmul2_rn(ndx, invR), pv = __fmul2_rn(ndy, invR);
        // the two look-ups as pairs (per lane the operations of pattern_cell_f /
        // pattern_near_f); products negated exactly as -(x y) = x (-y)
        PatCellF c0, c1;
        float2 gx, gy;
        pattern_cell_f2(m, pu, pv, gx, gy, c0, c1);
        if (DOPPLER) {
            // -(d + e) at the second pulse, e = e_p - v dt carried as -e (exact)
            const float2 nex = __ffma2_rn(it.vx, f2(m.dt_f), f2(-m.ep[0]));
            const float2 ney = __ffma2_rn(it.vy, f2(m.dt_f), f2(-m.ep[1]));
            const float2 u2 = __fmul2_rn(__fadd2_rn(ndx, nex), invR);
            const float2 v2 = __fmul2_rn(__fadd2_rn(ndy, ney), invR);
            float2 hx, hy;
            pattern_near_f2(m, u2, v2, c0, c1, hx, hy);
            const float2 pi = __ffma2_rn(hy, gx, __fmul2_rn(hx, __fmul2_rn(gy, neg1)));
            const float2 pr = __ffma2_rn(hx, gx, __fmul2_rn(hy, gy));
            pat_bins = make_float2(__fmul_rn(small_arg_f(pi.x, pr.x), m.nd_over_2pi_f),
                                   __fmul_rn(small_arg_f(pi.y, pr.y), m.nd_over_2pi_f));
        }
        re = __fmul2_rn(a, __ffma2_rn(gx, cs, __fmul2_rn(gy, __fmul2_rn(sn, neg1))));
        im = __fmul2_rn(a, __ffma2_rn(gy, cs, __fmul2_rn(gx, sn)));
    }
    bool refine0 = fabsf(gd.x) > k.gthr, refine1 = fabsf(gd.y) > k.gthr;
    int kb0 = 0, kb1 = 0;
    if (DOPPLER) {
        const float2 item = __ffma2_rn(t2, it.beta, it.gam);
        float2 b = __fmul2_rn(__fadd2_rn(__ffma2_rn(item, neg1, f2(k.K0hi)), f2(k.K0lo)), f2(k.kbin));
        b = __ffma2_rn(b, nxr, b);
        if (ANT) b = __fadd2_rn(b, pat_bins);
        const float2 bm = __fadd2_rn(b, f2(kRoundMagic));
        const float2 bd = __ffma2_rn(__fadd2_rn(bm, f2(-kRoundMagic)), neg1, b);
        kb0 = __float_as_int(bm.x) & (m.n_doppler - 1);
        kb1 = __float_as_int(bm.y) & (m.n_doppler - 1);
        refine0 |= fabsf(bd.x) > fmaf(-fabsf(b.x), kEpsSlope, 0.5f - kBinEps);
        refine1 |= fabsf(bd.y) > fmaf(-fabsf(b.y), kEpsSlope, 0.5f - kBinEps);
    }
    const unsigned cells = (unsigned)(m.n_gates * m.n_doppler);
    // (without DOPPLER there is one bin: n_doppler = 1, key = gate)
    int c0 = (int)min((unsigned)(DOPPLER ? g0 * m.n_doppler + kb0 : g0), cells);
    int c1 = (int)min((unsigned)(DOPPLER ? g1 * m.n_doppler + kb1 : g1), cells);
    if (!RSIM_CHECK_OK((unsigned)kb0 < (unsigned)m.n_doppler, kChkBin, kb0)) c0 = (int)cells;
    if (!RSIM_CHECK_OK((unsigned)kb1 < (unsigned)m.n_doppler, kChkBin, kb1)) c1 = (int)cells;
    const bool d0 = refine0 || (!ANT && qb.x < m.qb_wide);
    const bool d1 = refine1 || (!ANT && qb.y < m.qb_wide);
    key0 = d0 ? kKeyDeferred : c0;
    key1 = d1 ? kKeyDeferred : c1;
    defer = d0 || d1;
}

// Squared off-nadir angle atan(rho / d_z)^2 in FP64 (series for small angles).
__device__ __forceinline__ double theta2_d(double rho2, double dz) {
    const double q2 = rho2 / (dz * dz);
    if (q2 < 1e-3) {
        return q2 * fma(q2, fma(q2, fma(q2, -44.0 / 105.0, 23.0 / 45.0), -2.0 / 3.0), 1.0);
    }
    const double th = atan2(sqrt(rho2), dz);
    return th * th;
}

// Scatterer registers of the FP64 path (positions relative to the origin).
struct ItemD {
    float x, y, z, vx, vy, vz;
    double amp0;
};

struct DerivD {
    double dlna, dphi;
    double2 pat;  // tabulated pattern only: a e^{-j 2 pi f} dG/dz
};

template <bool DOPPLER, bool DERIV, bool ANT = false>
__device__ __forceinline__ int eval_fp64(const Model& m, const Fp64Const& k, const ItemD& it,
                                         int64_t n, int64_t n_total, double& re, double& im,
                                         DerivD* dv, int* g_out = nullptr,
                                         double* gc_out = nullptr, double* bc_out = nullptr) {
    const double vx = it.vx, vy = it.vy, vz = it.vz;
    const GeomD gd = geom_fp64(k.t, k.Px, k.Py, k.Pz, k.rref, (double)it.x, (double)it.y,
                               (double)it.z, vx, vy, vz);
    const double gc = fma(gd.dR, m.inv_gw, m.half_gates);
    const int g = clamp_floor(gc);
    const double rr = k.rref / gd.R;
    const double a = ANT ? it.amp0 * rr * rr
                         : it.amp0 * exp2(m.beam_k * theta2_d(gd.rho2, gd.dz)) * rr * rr;
    double f = k.psiref + gd.dR * m.two_over_lambda;
    f -= rint(f);
    double sn, cs;
    sincospi(2.0 * f, &sn, &cs);
    double2 gu, gv, G;
    double pu = 0.0, pv = 0.0;
    if (ANT) {
        pu = -gd.dx / gd.R;
        pv = -gd.dy / gd.R;
        G = pattern_d(m, pu, pv, DERIV ? &gu : nullptr, DERIV ? &gv : nullptr);
        re = a * fma(G.x, cs, G.y * sn);
        im = a * fma(G.y, cs, -G.x * sn);
    } else {
        re = a * cs;
        im = -a * sn;
    }
    int kb = 0;
    double bc = 0.5;
    if (DOPPLER) {
        bc = bin_coord_fp64(m, gd, vx, vy, vz);
        if (ANT) bc += pattern_bin_shift_d(m, gd.dx, gd.dy, gd.dz, vx, vy, vz, G);
        kb = clamp_floor(bc) & (m.n_doppler - 1);
    }
    if (DERIV) {
        const double R2 = gd.R * gd.R;
        dv->dphi = 2.0 * 3.14159265358979323846 * m.two_over_lambda * gd.dz / gd.R;
        if (ANT) {
            dv->dlna = 2.0 * gd.dz / R2;
            const double su = pu * gd.dz / R2, svv = pv * gd.dz / R2;
            const double dgx = fma(gu.x, su, gv.x * svv), dgy = fma(gu.y, su, gv.y * svv);
            dv->pat = make_double2(a * fma(dgx, cs, dgy * sn), a * fma(dgy, cs, -dgx * sn));
        } else {
            double rho_theta;
            const double q2 = gd.rho2 / (gd.dz * gd.dz);
            if (q2 < 1e-3) {
                rho_theta = gd.rho2 / gd.dz * fma(q2, fma(q2, fma(q2, -1.0 / 7.0, 0.2), -1.0 / 3.0), 1.0);
            } else {
                rho_theta = sqrt(gd.rho2) * atan2(sqrt(gd.rho2), gd.dz);
            }
            dv->dlna = (2.0 * gd.dz + 2.0 * 0.69314718055994530942 * m.beam_k * rho_theta) / R2;
            dv->pat = make_double2(0.0, 0.0);
        }
    }
    if (g_out) *g_out = g;
    if (gc_out) *gc_out = gc;
    if (bc_out) *bc_out = bc;
    if (!RSIM_CHECK_OK((unsigned)kb < (unsigned)m.n_doppler, kChkBin, kb)) return -1;
    return (n < n_total && g >= 0 && g < m.n_gates) ? g * m.n_doppler + kb : -1;
}

// ---------------------------------------------------------------------------------------
// Deterministic scatter-add.  Contributions are summed in 64-bit fixed point
// (q = rint(v * 2^32)); integer addition is associative, so the result does not depend
// on the order in which atomics land.  Before touching memory, each warp merges runs of
// equal keys: in-lane over the thread's consecutive scatterers, then across lanes with a
// segmented Hillis-Steele scan (fixed order), so only run tails are emitted.
// v * 2^32 as a 64-bit integer (2^-31 resolution, |v| < 2^30), branch-free.  The hardware
// float -> int64 conversion issues on the FP64 pipe, which runs at 1/64 of the FP32 rate
// on this GPU; one per emitted run made that pipe the bottleneck of the whole summation.
// Here v = t + r with t = trunc(v) and |r| < 1 (both exact in FP32), and only 32-bit
// conversions are used.
__device__ __forceinline__ long long fixed_from_f32(float v) {
    const float t = truncf(v);
    const float r = v - t;
    const long long hi = (long long)__float2int_rz(v);  // = (int) t, without waiting for t
    const long long lo = (long long)__float2int_rn(r * 2147483648.0f);
    return (long long)((unsigned long long)hi << 32) + lo * 2;
}

// v * 2^32 rounded, with integer operations only (the FP64 path's values carry more bits
// than two FP32 conversions keep).  Valid for |v| < 2^30.
__device__ __forceinline__ long long fixed_from_f64(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ffull);
    const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
    const int sh = e - 1043;                                      // v 2^32 = m 2^(e - 1043)
    unsigned long long q;
    if (sh >= 0) {
        q = m << (sh > 10 ? 10 : sh);
    } else {
        const int r = -sh;
        q = r > 54 ? 0ull : ((m >> (r - 1)) + 1ull) >> 1;
    }
    if (e == 0) q = 0ull;
    return (b >> 63) ? -(long long)q : (long long)q;
}

template <typename T>
__device__ __forceinline__ long long to_fixed(T v);
template <>
__device__ __forceinline__ long long to_fixed<float>(float v) { return fixed_from_f32(v); }
template <>
__device__ __forceinline__ long long to_fixed<double>(double v) { return fixed_from_f64(v); }

// Fire-and-forget global reduction (no return value, so the warp does not wait for it).
// The workspace is global memory; the address space is stated explicitly because the
// pointer may come out of a shared-memory table, where the compiler cannot infer it.
__device__ __forceinline__ void red_add_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("red.global.add.u64 [%0], %1;"
                 :
                 : "l"((unsigned long long)__cvta_generic_to_global(p)), "l"(v)
                 : "memory");
}

template <typename T>
__device__ __forceinline__ void emit_cell(unsigned long long* __restrict__ base, int key, T re,
                                          T im) {
    if (!RSIM_CHECK_OK(fabs((double)re) < 1073741824.0 && fabs((double)im) < 1073741824.0,
                       kChkFixed, key))
        return;
    const long long qr = to_fixed(re), qi = to_fixed(im);
    // a zero addend (padding items) is a no-op: not worth a test per emission
    red_add_u64(base + 2 * (int64_t)key, (unsigned long long)qr);
    red_add_u64(base + 2 * (int64_t)key + 1, (unsigned long long)qi);
}

// In-lane inclusive run sum: prev + v where the run continues, v where it starts, as one
// (paired) FMA with a 0 / 1 factor -- the same values either way.
__device__ __forceinline__ void run_sum(bool same, float& sr, float& si, float pr, float pi,
                                        float vr, float vi) {
    const float s = same ? 1.0f : 0.0f;
    const float2 r = __ffma2_rn(make_float2(s, s), make_float2(pr, pi), make_float2(vr, vi));
    sr = r.x;
    si = r.y;
}
__device__ __forceinline__ void run_sum(bool same, double& sr, double& si, double pr, double pi,
                                        double vr, double vi) {
    sr = same ? pr + vr : vr;
    si = same ? pi + vi : vi;
}

// Keys at or above `cells` (out of the window, deferred, or -1) are merged like any other and
// dropped at emission.
template <typename T, int J>
__device__ __forceinline__ void warp_reduce_emit(const int (&key)[J], const T (&re)[J],
                                               const T (&im)[J],
                                               unsigned long long* __restrict__ base,
                                               unsigned cells) {
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    // in-lane inclusive run sums; bit q of tails: a run ends at item q
    T sr[J], si[J];
    sr[0] = re[0];
    si[0] = im[0];
    unsigned tails = 0u;
#pragma unroll
    for (int q = 1; q < J; ++q) {
        const bool same = key[q] == key[q - 1];
        run_sum(same, sr[q], si[q], sr[q - 1], si[q - 1], re[q], im[q]);
        if (!same) tails |= 1u << (q - 1);
    }
    const bool uniform = tails == 0u;
    const int first_end = __ffs(tails | (1u << (J - 1))) - 1;  // end of the lane's first run
    const int prev_last = __shfl_up_sync(kFull, key[J - 1], 1);
    const bool link = lane > 0 && prev_last == key[0];  // first run continues lane-1's last run
    // segmented inclusive scan (fixed order) of the lanes' last-run sums; a lane heads a
    // segment unless all its items continue lane-1's last run, and a lane at distance dist
    // from its segment's head takes the partial of lane - d while d <= dist
    T cr = sr[J - 1], ci = si[J - 1];
    const unsigned heads = __ballot_sync(kFull, !uniform || !link);  // bit 0 always set
    const int dist = lane - (31 - __clz(heads & (kFull >> (31 - lane))));
    // FP32: segments of more than 8 lanes are rare (a lane continues its left neighbour's
    // last run and has no run end of its own), so the last two steps run only when the warp
    // has one; the FP64 path (bound by its FP64 evaluation) keeps all five
    constexpr int kFirstSteps = sizeof(T) == sizeof(float) ? 8 : 32;
#pragma unroll
    for (int d = 1; d < kFirstSteps; d <<= 1) {
        const T ur = __shfl_up_sync(kFull, cr, d);
        const T ui = __shfl_up_sync(kFull, ci, d);
        if (dist >= d) {
            cr = ur + cr;
            ci = ui + ci;
        }
    }
    if (kFirstSteps < 32 && __any_sync(kFull, dist >= 8)) {
#pragma unroll
        for (int d = 8; d < 32; d <<= 1) {
            const T ur = __shfl_up_sync(kFull, cr, d);
            const T ui = __shfl_up_sync(kFull, ci, d);
            if (dist >= d) {
                cr = ur + cr;
                ci = ui + ci;
            }
        }
    }
    T in_r = __shfl_up_sync(kFull, cr, 1), in_i = __shfl_up_sync(kFull, ci, 1);
    if (!link) {
        in_r = T(0);
        in_i = T(0);
    }
    const int next_link = __shfl_down_sync(kFull, link ? 1 : 0, 1);
    if (lane == 31 || !next_link) tails |= 1u << (J - 1);
    // emit the pending run tails, one per lane per round
    while (__any_sync(kFull, tails != 0u)) {
        if (tails) {
            const int q = __ffs(tails) - 1;
            tails &= tails - 1u;
            // binary selection by the bits of q
            int kk[J];
            T rr[J], ii[J];
#pragma unroll
            for (int j = 0; j < J; ++j) { kk[j] = key[j]; rr[j] = sr[j]; ii[j] = si[j]; }
#pragma unroll
            for (int w = 1; w < J; w <<= 1) {
                const bool bit = (q & w) != 0;
#pragma unroll
                for (int j = 0; j < J; j += 2 * w) {
                    kk[j] = bit ? kk[j + w] : kk[j];
                    rr[j] = bit ? rr[j + w] : rr[j];
                    ii[j] = bit ? ii[j + w] : ii[j];
                }
            }
            const int k = kk[0];
            T vr = rr[0], vi = ii[0];
            if (q <= first_end) {  // the lane's first run: add the carry from the left
                vr += in_r;
                vi += in_i;
            }
            if ((unsigned)k < cells) emit_cell(base, k, vr, vi);  // out-of-window runs dropped
        }
    }
}


}  // namespace rsim
