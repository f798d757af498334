// abi.cu -- the C ABI of librsim (declared in include/rsim.h): argument validation,
// workspace checks, model constants, kernel launches and the batched-pass autotuner.  No
// device memory is allocated here; every device buffer, including scratch, belongs to the
// caller.
#include <algorithm>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <string>
#include <vector>

#include "rsim.h"
#include "rsim_internal.cuh"
#include "rsim_kernels.h"

namespace {

thread_local std::string g_last_error;

rsim_status fail(rsim_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

rsim_status cuda_fail(cudaError_t e, const char* what) {
    return fail(RSIM_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// Return value of an entry point whose kernels were all launched: RSIM_OK, or, in a
// -DRSIM_CHECK build, RSIM_ERR_CHECK if one of them failed a check (the build reads the
// summation unit's check word here, which synchronises the stream).
rsim_status checked_ok(cudaStream_t stream) {
#ifdef RSIM_CHECK
    static const char* const names[] = {"?", "Doppler bin range", "fixed-point range",
                                        "sample slot", "adjoint gather cell"};
    unsigned long long w = 0;
    const cudaError_t e = rsim::check_take(stream, &w);
    if (e != cudaSuccess) return cuda_fail(e, "check word read");
    if (w != 0) {
        const unsigned code = (unsigned)(w >> 56);
        long long v = (long long)(w & ((1ull << 56) - 1ull));
        if (v & (1ll << 55)) v -= (1ll << 56);  // sign of the recorded value
        return fail(RSIM_ERR_CHECK, "bounds check failed: %s (value %lld)",
                    names[code < 5 ? code : 0], v);
    }
#else
    (void)stream;
#endif
    return RSIM_OK;
}

int device_sms() {
    static int cache[256] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return 132;
    if (cache[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 132;
        cache[dev] = v;
    }
    return cache[dev];
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }
bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

rsim_status check_radar(const rsim_radar* r) {
    if (!r) return fail(RSIM_ERR_INVALID_ARG, "radar is NULL");
    if (!finite_pos(r->carrier_hz) || !finite_pos(r->prf_hz) || !finite_pos(r->c_mps) ||
        !finite_pos(r->gate_width_m) || !finite_pos(r->beamwidth_rad))
        return fail(RSIM_ERR_INVALID_ARG, "radar constants must be finite and > 0");
    if (r->n_gates < 1 || r->n_gates > 4096)
        return fail(RSIM_ERR_INVALID_ARG, "n_gates=%d outside [1, 4096]", r->n_gates);
    if (r->reserved != 0) return fail(RSIM_ERR_INVALID_ARG, "radar.reserved must be 0");
    if (const rsim_antenna* a = r->antenna) {
        if (!a->gain || !aligned(a->gain, 8))
            return fail(RSIM_ERR_INVALID_ARG, "antenna.gain is NULL or not 8-byte aligned");
        if (a->nu < 2 || a->nv < 2 || (int64_t)a->nu * a->nv >= ((int64_t)1 << 31))
            return fail(RSIM_ERR_INVALID_ARG, "antenna grid %d x %d: need nu, nv >= 2, nu*nv < 2^31",
                        a->nu, a->nv);
        if (!finite_pos(a->du) || !finite_pos(a->dv) || !std::isfinite(a->u0) || !std::isfinite(a->v0))
            return fail(RSIM_ERR_INVALID_ARG, "antenna grid origin must be finite, steps finite and > 0");
    }
    return RSIM_OK;
}

rsim_status check_platform(const rsim_platform* p) {
    if (!p) return fail(RSIM_ERR_INVALID_ARG, "platform is NULL");
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(p->p0[i]) || !std::isfinite(p->v[i]))
            return fail(RSIM_ERR_INVALID_ARG, "platform position/velocity must be finite");
    if (!finite_pos(p->r_ref0) || !std::isfinite(p->r_ref_rate))
        return fail(RSIM_ERR_INVALID_ARG, "r_ref0 must be finite and > 0, r_ref_rate finite");
    return RSIM_OK;
}

rsim_status check_scat(const rsim_scatterers* s) {
    if (!s) return fail(RSIM_ERR_INVALID_ARG, "scatterers is NULL");
    if (s->n < 0) return fail(RSIM_ERR_INVALID_ARG, "scatterer count %lld < 0", (long long)s->n);
    if (s->n > ((int64_t)1 << 40)) return fail(RSIM_ERR_INVALID_ARG, "scatterer count too large");
    if (s->n > 0) {
        const float* p[7] = {s->x, s->y, s->z, s->vx, s->vy, s->vz, s->nrcs};
        for (int i = 0; i < 7; ++i) {
            if (!p[i]) return fail(RSIM_ERR_INVALID_ARG, "scatterer array %d is NULL", i);
            if (!aligned(p[i], 4)) return fail(RSIM_ERR_INVALID_ARG, "scatterer array %d misaligned", i);
        }
    }
    if (!finite_pos(s->facet_area_m2)) return fail(RSIM_ERR_INVALID_ARG, "facet_area_m2 must be > 0");
    if (!std::isfinite(s->t0)) return fail(RSIM_ERR_INVALID_ARG, "t0 must be finite");
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(s->origin[i])) return fail(RSIM_ERR_INVALID_ARG, "origin must be finite");
    return RSIM_OK;
}

rsim_status check_precision(rsim_precision p) {
    if (p != RSIM_FP64 && p != RSIM_SPLIT) return fail(RSIM_ERR_INVALID_ARG, "unknown precision %d", (int)p);
    return RSIM_OK;
}

rsim::Model make_model(const rsim_radar* r, const rsim_platform* p, const rsim_scatterers* s,
                       int n_doppler) {
    rsim::Model m;
    std::memset(&m, 0, sizeof(m));
    m.prf = r->prf_hz;
    m.inv_prf = 1.0 / r->prf_hz;
    for (int i = 0; i < 3; ++i) {
        m.p0[i] = p->p0[i] - s->origin[i];
        m.v[i] = p->v[i];
    }
    m.r_ref0 = p->r_ref0;
    m.r_ref_rate = p->r_ref_rate;
    m.two_over_lambda = 2.0 * r->carrier_hz / r->c_mps;
    m.inv_gw = 1.0 / r->gate_width_m;
    m.half_gates = 0.5 * (double)r->n_gates;
    m.beam_k = -2.0 / (r->beamwidth_rad * r->beamwidth_rad);
    m.area = s->facet_area_m2;
    m.n_gates = r->n_gates;
    m.n_doppler = n_doppler;
    m.inv_gw_f = (float)m.inv_gw;
    m.beam_k_f = (float)m.beam_k;
    m.chi_hi = (float)m.two_over_lambda;
    m.chi_lo = (float)(m.two_over_lambda - (double)m.chi_hi);
    m.chi_lo_rad = (float)(-6.283185307179586476925 * (m.two_over_lambda - (double)m.chi_hi));
    m.dt_f = (float)m.inv_prf;
    m.hdt_f = (float)(0.5 * m.inv_prf);
    for (int i = 0; i < 3; ++i) m.ep[i] = (float)(p->v[i] * m.inv_prf);
    m.inv_nd = (float)(1.0 / (double)n_doppler);
    m.s1 = (float)(-2.0 / (3.0 * m.beam_k));
    m.s2 = (float)(23.0 / (45.0 * m.beam_k * m.beam_k));
    m.qb_wide = (float)(1e-2 * m.beam_k);
    m.inv_beam_k = (float)(1.0 / m.beam_k);
    m.nd_over_2pi_f = (float)((double)n_doppler / 6.283185307179586476925);
    if (const rsim_antenna* a = r->antenna) {
        m.ant = static_cast<const float2*>(a->gain);
        m.ant_nu = a->nu;
        m.ant_nv = a->nv;
        m.ant_u0 = a->u0;
        m.ant_v0 = a->v0;
        m.ant_idu = 1.0 / a->du;
        m.ant_idv = 1.0 / a->dv;
        m.ant_u0_f = (float)a->u0;
        m.ant_v0_f = (float)a->v0;
        m.ant_idu_f = (float)m.ant_idu;
        m.ant_idv_f = (float)m.ant_idv;
    }
    return m;
}

rsim::Scat make_scat(const rsim_scatterers* s) {
    rsim::Scat sc;
    sc.x = s->x; sc.y = s->y; sc.z = s->z;
    sc.vx = s->vx; sc.vy = s->vy; sc.vz = s->vz; sc.nrcs = s->nrcs;
    sc.n = s->n;
    sc.t0 = s->t0;
    const float* p[7] = {s->x, s->y, s->z, s->vx, s->vy, s->vz, s->nrcs};
    int vec = 1;
    for (int i = 0; i < 7; ++i) vec &= aligned(p[i], 16) ? 1 : 0;
    sc.vec4 = vec;
    sc.pad = 0;
    return sc;
}

size_t ws_bytes(int64_t n_samples, int n_gates, int n_doppler) {
    return (size_t)n_samples * (size_t)n_gates * (size_t)n_doppler * 16u;
}

// Sample schedule of a summation launch.  The samples are split over gridDim.y only when the
// scatterer chunks alone cannot fill the GPU (about 8 resident CTAs' worth per SM).
// Returns the number of sample groups (gridDim.y).
// Samples per CTA: spg_req > 0 forces it (clamped to what the grid allows), 0 = enough
// groups for about 8 CTAs per SM.
int64_t plan_samples(int64_t chunks, int64_t pulse_base, int32_t stride, int32_t n_samples,
                     rsim::Schedule* sch, int32_t spg_req = 0) {
    const int64_t target = (int64_t)device_sms() * 8;
    int64_t groups = (target + chunks - 1) / chunks;
    if (groups < 1) groups = 1;
    if (groups > n_samples) groups = n_samples;
    int64_t spg = (n_samples + groups - 1) / groups;
    if (spg_req > 0) spg = spg_req < n_samples ? spg_req : n_samples;
    if (spg < (n_samples + 65534) / 65535) spg = (n_samples + 65534) / 65535;
    groups = (n_samples + spg - 1) / spg;
    sch->pulse_base = pulse_base;
    sch->pulse_stride = stride;
    sch->n_samples = n_samples;
    sch->samples_per_group = (int32_t)spg;
    sch->pad = 0;
    return groups;
}

size_t batch_stride(int32_t n_samples, int32_t n_gates, int32_t n_doppler) {
    const size_t b = ws_bytes(n_samples, n_gates, n_doppler);
    return (b + 255u) & ~(size_t)255u;
}

// Shared body of rsim_direct_sum and rsim_doppler_accumulate; with partial = true (the
// blockwise entry point) only the summation kernel runs: no clear, no finalize, out unused.
rsim_status run_accumulate(const rsim_radar* radar, const rsim_platform* platform,
                           const rsim_scatterers* scat, int64_t pulse_base, int32_t stride,
                           int32_t n_samples, int32_t n_doppler, bool doppler,
                           rsim_precision precision, void* out, void* workspace,
                           size_t workspace_bytes, cudaStream_t stream, bool partial = false,
                           unsigned long long* out_of_window = nullptr) {
    rsim_status st;
    if ((st = check_radar(radar)) != RSIM_OK) return st;
    if ((st = check_platform(platform)) != RSIM_OK) return st;
    if ((st = check_scat(scat)) != RSIM_OK) return st;
    if ((st = check_precision(precision)) != RSIM_OK) return st;
    if (n_samples < 0) return fail(RSIM_ERR_INVALID_ARG, "sample count %d < 0", n_samples);
    if (pulse_base < 0) return fail(RSIM_ERR_INVALID_ARG, "first pulse/update index < 0");
    if (pulse_base + (int64_t)n_samples * stride > ((int64_t)1 << 52))
        return fail(RSIM_ERR_INVALID_ARG, "pulse index out of range");
    if (n_samples == 0 || scat->n == 0) return RSIM_OK;  // nothing to add
    const bool fp64 = precision == RSIM_FP64;
    if (!partial) {
        if (!out) return fail(RSIM_ERR_INVALID_ARG, "output is NULL");
        if (!aligned(out, fp64 ? 16 : 8)) return fail(RSIM_ERR_INVALID_ARG, "output misaligned");
    }
    if (out_of_window && !aligned(out_of_window, 8))
        return fail(RSIM_ERR_INVALID_ARG, "out_of_window not 8-byte aligned");
    const size_t need = ws_bytes(n_samples, radar->n_gates, n_doppler);
    if (!workspace) return fail(RSIM_ERR_WORKSPACE, "workspace is NULL (need %zu bytes)", need);
    if (!aligned(workspace, 16)) return fail(RSIM_ERR_WORKSPACE, "workspace not 16-byte aligned");
    if (workspace_bytes < need)
        return fail(RSIM_ERR_WORKSPACE, "workspace of %zu bytes < %zu required", workspace_bytes, need);

    const rsim::Model m = make_model(radar, platform, scat, n_doppler);
    const rsim::Scat sc = make_scat(scat);
    const int64_t chunks = (scat->n + rsim::kChunk - 1) / rsim::kChunk;
    if (chunks > 0x7fffffff) return fail(RSIM_ERR_INVALID_ARG, "too many scatterers");
    rsim::Schedule sch;
    const int64_t groups = plan_samples(chunks, pulse_base, stride, n_samples, &sch);

    cudaError_t e = cudaSuccess;
    if (!partial && (e = cudaMemsetAsync(workspace, 0, need, stream)) != cudaSuccess)
        return cuda_fail(e, "workspace clear");
    e = rsim::launch_accumulate(m, sch, sc, fp64, doppler,
                                static_cast<unsigned long long*>(workspace),
                                dim3((unsigned)chunks, (unsigned)groups), stream);
    if (partial) {
        if (e != cudaSuccess) return cuda_fail(e, "summation kernel launch");
        return checked_ok(stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "summation kernel launch");
    if (out_of_window &&
        (e = rsim::launch_window_count(m, sch, sc, fp64, doppler, out_of_window, stream)) != cudaSuccess)
        return cuda_fail(e, "window count kernel launch");
    e = rsim::launch_finalize(workspace, out, (int64_t)(need / 8), fp64, device_sms(), stream);
    if (e != cudaSuccess) return cuda_fail(e, "finalize kernel launch");
    return checked_ok(stream);
}

rsim_status check_synth_args(const rsim_radar* radar, int32_t n_spectra, int64_t update0,
                             int32_t n_fast, int32_t n_doppler, int64_t pulse0, int32_t n_pulses,
                             int window, rsim_precision precision) {
    rsim_status st;
    if ((st = check_radar(radar)) != RSIM_OK) return st;
    if ((st = check_precision(precision)) != RSIM_OK) return st;
    if (window < 0 || window > 2) return fail(RSIM_ERR_INVALID_ARG, "unknown window %d", window);
    if (n_fast < 1) return fail(RSIM_ERR_INVALID_ARG, "n_fast=%d < 1 (regular mode is rsim_direct_sum)", n_fast);
    if (!is_pow2(n_doppler) || n_doppler < 2 || n_doppler > 1024)
        return fail(RSIM_ERR_INVALID_ARG, "n_doppler=%d must be a power of two in [2, 1024]", n_doppler);
    if ((int64_t)radar->n_gates * n_doppler > (1 << 20))
        return fail(RSIM_ERR_INVALID_ARG, "n_gates * n_doppler > 2^20");
    if (n_spectra < 0 || n_pulses < 0 || update0 < 0 || pulse0 < 0)
        return fail(RSIM_ERR_INVALID_ARG, "negative count or index");
    if (pulse0 + (int64_t)n_pulses > ((int64_t)1 << 52))
        return fail(RSIM_ERR_INVALID_ARG, "pulse index out of range");
    if (n_pulses == 0) return RSIM_OK;
    const int64_t first = pulse0 / n_fast;
    const int64_t x_last = pulse0 + n_pulses - 1;
    const int64_t need_last = (x_last % n_fast == 0) ? x_last / n_fast : x_last / n_fast + 1;
    if (first < update0 || need_last > update0 + (int64_t)n_spectra - 1)
        return fail(RSIM_ERR_INVALID_ARG,
                    "pulses [%lld, %lld] need spectra of updates [%lld, %lld], given [%lld, %lld]",
                    (long long)pulse0, (long long)x_last, (long long)first, (long long)need_last,
                    (long long)update0, (long long)(update0 + n_spectra - 1));
    return RSIM_OK;
}

rsim::SynthArgs make_synth_args(const rsim_radar* radar, int32_t n_spectra, int64_t update0,
                                int32_t n_fast, int32_t n_doppler, int64_t pulse0,
                                int32_t n_pulses, int window) {
    rsim::SynthArgs a;
    a.n_gates = radar->n_gates;
    a.n_doppler = n_doppler;
    int L = 0;
    while ((1 << L) < n_doppler) ++L;
    a.log2_nd = L;
    a.n_fast = n_fast;
    a.n_spectra = n_spectra;
    a.n_pulses = n_pulses;
    a.update0 = update0;
    a.pulse0 = pulse0;
    a.window = window;
    return a;
}

}  // namespace

namespace rsim {

// Sets the calling thread's rsim_last_error() message (for entry points in other
// translation units).
void set_last_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

}  // namespace rsim

extern "C" {

int rsim_version(void) { return RSIM_ABI_VERSION; }

int rsim_check_build(void) {
#ifdef RSIM_CHECK
    return 1;
#else
    return 0;
#endif
}

const char* rsim_last_error(void) { return g_last_error.c_str(); }

int rsim_block_scatterers(void) { return rsim::kChunk; }

size_t rsim_workspace_size(int32_t n_samples, int32_t n_gates, int32_t n_doppler) {
    if (n_samples < 0 || n_gates < 1 || n_gates > 4096 || !is_pow2(n_doppler) || n_doppler > 4096)
        return 0;
    return ws_bytes(n_samples, n_gates, n_doppler);
}

rsim_status rsim_direct_sum(const rsim_radar* radar, const rsim_platform* platform,
                            const rsim_scatterers* scat, int64_t pulse0, int32_t n_pulses,
                            rsim_precision precision, void* iq, void* workspace,
                            size_t workspace_bytes, unsigned long long* out_of_window,
                            cudaStream_t stream) {
    return run_accumulate(radar, platform, scat, pulse0, 1, n_pulses, 1, false, precision, iq,
                          workspace, workspace_bytes, stream, false, out_of_window);
}

rsim_status rsim_doppler_accumulate(const rsim_radar* radar, const rsim_platform* platform,
                                    const rsim_scatterers* scat, int64_t update0,
                                    int32_t n_updates, int32_t n_fast, int32_t n_doppler,
                                    rsim_precision precision, void* spectra, void* workspace,
                                    size_t workspace_bytes, unsigned long long* out_of_window,
                                    cudaStream_t stream) {
    if (n_fast < 1) return fail(RSIM_ERR_INVALID_ARG, "n_fast=%d < 1 (regular mode is rsim_direct_sum)", n_fast);
    if (!is_pow2(n_doppler) || n_doppler > 4096)
        return fail(RSIM_ERR_INVALID_ARG, "n_doppler=%d must be a power of two in [1, 4096]", n_doppler);
    if (radar && (int64_t)radar->n_gates * n_doppler > ((int64_t)1 << 24))
        return fail(RSIM_ERR_INVALID_ARG, "n_gates * n_doppler > 2^24");
    if (update0 < 0) return fail(RSIM_ERR_INVALID_ARG, "update0 < 0");
    if (update0 > (((int64_t)1 << 52) / n_fast)) return fail(RSIM_ERR_INVALID_ARG, "update0 too large");
    return run_accumulate(radar, platform, scat, update0 * (int64_t)n_fast, n_fast, n_updates,
                          n_doppler, true, precision, spectra, workspace, workspace_bytes, stream,
                          false, out_of_window);
}

rsim_status rsim_synth_pulses(const rsim_radar* radar, const void* spectra, int32_t n_spectra,
                              int64_t update0, int32_t n_fast, int32_t n_doppler,
                              int64_t pulse0, int32_t n_pulses, rsim_window window,
                              rsim_precision precision, void* iq, cudaStream_t stream) {
    rsim_status st = check_synth_args(radar, n_spectra, update0, n_fast, n_doppler, pulse0,
                                      n_pulses, (int)window, precision);
    if (st != RSIM_OK) return st;
    if (n_pulses == 0) return RSIM_OK;
    const bool fp64 = precision == RSIM_FP64;
    if (!spectra || !iq) return fail(RSIM_ERR_INVALID_ARG, "spectra / iq is NULL");
    if (!aligned(spectra, fp64 ? 16 : 8) || !aligned(iq, fp64 ? 16 : 8))
        return fail(RSIM_ERR_INVALID_ARG, "spectra / iq misaligned");
    const rsim::SynthArgs a = make_synth_args(radar, n_spectra, update0, n_fast, n_doppler, pulse0,
                                              n_pulses, (int)window);
    const cudaError_t e = rsim::launch_synth(a, fp64, spectra, iq, stream);
    if (e != cudaSuccess) return cuda_fail(e, "synth kernel launch");
    return RSIM_OK;
}

rsim_status rsim_scatterer_cells(const rsim_radar* radar, const rsim_platform* platform,
                                 const rsim_scatterers* scat, int64_t pulse, int32_t n_doppler,
                                 rsim_precision precision, int32_t* gate, int32_t* bin,
                                 double* gate_coord, double* bin_coord, cudaStream_t stream) {
    rsim_status st;
    if ((st = check_radar(radar)) != RSIM_OK) return st;
    if ((st = check_platform(platform)) != RSIM_OK) return st;
    if ((st = check_scat(scat)) != RSIM_OK) return st;
    if ((st = check_precision(precision)) != RSIM_OK) return st;
    if (!is_pow2(n_doppler) || n_doppler > 4096)
        return fail(RSIM_ERR_INVALID_ARG, "n_doppler=%d must be a power of two in [1, 4096]", n_doppler);
    if (pulse < 0 || pulse > ((int64_t)1 << 52)) return fail(RSIM_ERR_INVALID_ARG, "pulse out of range");
    if (scat->n == 0) return RSIM_OK;
    const rsim::Model m = make_model(radar, platform, scat, n_doppler);
    const rsim::Scat sc = make_scat(scat);
    const cudaError_t e = rsim::launch_cells(m, pulse, precision == RSIM_FP64, n_doppler > 1, sc,
                                             gate, bin, gate_coord, bin_coord, nullptr, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cells kernel launch");
    return checked_ok(stream);
}

static_assert(RSIM_MAX_STATES == rsim::kMaxStates, "states per launch");

rsim_status rsim_doppler_accumulate_states(const rsim_radar* radar, const rsim_platform* platform,
                                           const rsim_scatterers* scat, int64_t update0,
                                           int32_t n_updates, const rsim_surface_state* states,
                                           int32_t n_fast, int32_t n_doppler,
                                           rsim_precision precision, void* workspace,
                                           size_t workspace_bytes, cudaStream_t stream) {
    rsim_status st;
    if ((st = check_radar(radar)) != RSIM_OK) return st;
    if ((st = check_platform(platform)) != RSIM_OK) return st;
    if ((st = check_precision(precision)) != RSIM_OK) return st;
    if (n_fast < 1) return fail(RSIM_ERR_INVALID_ARG, "n_fast=%d < 1", n_fast);
    if (!is_pow2(n_doppler) || n_doppler > 4096)
        return fail(RSIM_ERR_INVALID_ARG, "n_doppler=%d must be a power of two in [1, 4096]", n_doppler);
    if ((int64_t)radar->n_gates * n_doppler > ((int64_t)1 << 24))
        return fail(RSIM_ERR_INVALID_ARG, "n_gates * n_doppler > 2^24");
    if (update0 < 0 || update0 > (((int64_t)1 << 52) / n_fast) - RSIM_MAX_STATES)
        return fail(RSIM_ERR_INVALID_ARG, "update index out of range");
    if (n_updates < 0 || n_updates > RSIM_MAX_STATES)
        return fail(RSIM_ERR_INVALID_ARG, "n_updates=%d outside [0, %d]", n_updates, RSIM_MAX_STATES);
    if (!scat) return fail(RSIM_ERR_INVALID_ARG, "scatterers is NULL");
    if (scat->n < 0 || scat->n > ((int64_t)1 << 40))
        return fail(RSIM_ERR_INVALID_ARG, "scatterer count out of range");
    if (scat->n > 0 && (!scat->x || !scat->y || !scat->nrcs || !aligned(scat->x, 4) ||
                        !aligned(scat->y, 4) || !aligned(scat->nrcs, 4)))
        return fail(RSIM_ERR_INVALID_ARG, "scatterer x, y or nrcs NULL or misaligned");
    if (!finite_pos(scat->facet_area_m2)) return fail(RSIM_ERR_INVALID_ARG, "facet_area_m2 must be > 0");
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(scat->origin[i])) return fail(RSIM_ERR_INVALID_ARG, "origin must be finite");
    if (n_updates > 0 && !states) return fail(RSIM_ERR_INVALID_ARG, "states is NULL");
    rsim::StatesParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.n = n_updates;
    for (int i = 0; i < n_updates; ++i) {
        const rsim_surface_state& q = states[i];
        const float* f[4] = {q.z, q.vx, q.vy, q.vz};
        for (int c = 0; c < 4; ++c)
            if (scat->n > 0 && (!f[c] || !aligned(f[c], 16)))
                return fail(RSIM_ERR_INVALID_ARG, "state %d array %d NULL or not 16-byte aligned", i, c);
        if (!std::isfinite(q.t0)) return fail(RSIM_ERR_INVALID_ARG, "state %d epoch not finite", i);
        sp.s[i].z = q.z;
        sp.s[i].vx = q.vx;
        sp.s[i].vy = q.vy;
        sp.s[i].vz = q.vz;
        sp.s[i].t0 = q.t0;
    }
    const size_t need = ws_bytes(n_updates, radar->n_gates, n_doppler);
    if (!workspace) return fail(RSIM_ERR_WORKSPACE, "workspace is NULL (need %zu bytes)", need);
    if (!aligned(workspace, 16)) return fail(RSIM_ERR_WORKSPACE, "workspace not 16-byte aligned");
    if (workspace_bytes < need)
        return fail(RSIM_ERR_WORKSPACE, "workspace of %zu bytes < %zu required", workspace_bytes, need);
    if (n_updates == 0 || scat->n == 0) return RSIM_OK;
    const rsim::Model m = make_model(radar, platform, scat, n_doppler);
    const rsim::Scat sc = make_scat(scat);
    const int64_t chunks = (scat->n + rsim::kChunk - 1) / rsim::kChunk;
    if (chunks > 0x7fffffff) return fail(RSIM_ERR_INVALID_ARG, "too many scatterers");
    rsim::Schedule sch;
    sch.pulse_base = update0 * (int64_t)n_fast;
    sch.pulse_stride = n_fast;
    sch.n_samples = n_updates;
    sch.samples_per_group = n_updates;
    sch.pad = 0;
    const cudaError_t e = rsim::launch_accumulate_states(
        m, sch, sc, sp, precision == RSIM_FP64, true, static_cast<unsigned long long*>(workspace),
        (unsigned)chunks, stream);
    if (e != cudaSuccess) return cuda_fail(e, "summation kernel launch");
    return checked_ok(stream);
}

rsim_status rsim_doppler_accumulate_partial(const rsim_radar* radar, const rsim_platform* platform,
                                            const rsim_scatterers* scat, int64_t update0,
                                            int32_t n_updates, int32_t n_fast, int32_t n_doppler,
                                            rsim_precision precision, void* workspace,
                                            size_t workspace_bytes, cudaStream_t stream) {
    if (n_fast < 1) return fail(RSIM_ERR_INVALID_ARG, "n_fast=%d < 1", n_fast);
    if (!is_pow2(n_doppler) || n_doppler > 4096)
        return fail(RSIM_ERR_INVALID_ARG, "n_doppler=%d must be a power of two in [1, 4096]", n_doppler);
    if (update0 < 0 || update0 > (((int64_t)1 << 52) / n_fast))
        return fail(RSIM_ERR_INVALID_ARG, "update index out of range");
    return run_accumulate(radar, platform, scat, update0 * (int64_t)n_fast, n_fast, n_updates,
                          n_doppler, true, precision, nullptr, workspace, workspace_bytes, stream,
                          true);
}

rsim_status rsim_workspace_clear(int32_t n_updates, int32_t n_gates, int32_t n_doppler,
                                 void* workspace, size_t workspace_bytes, cudaStream_t stream) {
    if (n_updates < 0 || n_gates < 1 || n_doppler < 1)
        return fail(RSIM_ERR_INVALID_ARG, "bad workspace shape");
    const size_t need = ws_bytes(n_updates, n_gates, n_doppler);
    if (need == 0) return RSIM_OK;
    if (!workspace || !aligned(workspace, 16) || workspace_bytes < need)
        return fail(RSIM_ERR_WORKSPACE, "workspace: need %zu bytes, 16-byte aligned", need);
    const cudaError_t e = cudaMemsetAsync(workspace, 0, need, stream);
    if (e != cudaSuccess) return cuda_fail(e, "workspace clear");
    return RSIM_OK;
}

rsim_status rsim_workspace_finalize(int32_t n_updates, int32_t n_gates, int32_t n_doppler,
                                    rsim_precision precision, const void* workspace,
                                    size_t workspace_bytes, void* out, cudaStream_t stream) {
    rsim_status st;
    if ((st = check_precision(precision)) != RSIM_OK) return st;
    if (n_updates < 0 || n_gates < 1 || n_doppler < 1)
        return fail(RSIM_ERR_INVALID_ARG, "bad workspace shape");
    const size_t need = ws_bytes(n_updates, n_gates, n_doppler);
    if (need == 0) return RSIM_OK;
    const bool fp64 = precision == RSIM_FP64;
    if (!workspace || !aligned(workspace, 16) || workspace_bytes < need)
        return fail(RSIM_ERR_WORKSPACE, "workspace: need %zu bytes, 16-byte aligned", need);
    if (!out || !aligned(out, fp64 ? 16 : 8)) return fail(RSIM_ERR_INVALID_ARG, "output NULL or misaligned");
    const cudaError_t e = rsim::launch_finalize(workspace, out, (int64_t)(need / 8), fp64,
                                                device_sms(), stream);
    if (e != cudaSuccess) return cuda_fail(e, "finalize kernel launch");
    return RSIM_OK;
}

rsim_status rsim_delay_doppler(const rsim_radar* radar, const rsim_platform* platform,
                               const void* iq, int64_t pulse0, int32_t n_pulses, int32_t burst,
                               void* focused, float* multilook, cudaStream_t stream) {
    rsim_status st;
    if ((st = check_radar(radar)) != RSIM_OK) return st;
    if ((st = check_platform(platform)) != RSIM_OK) return st;
    if (pulse0 < 0 || n_pulses < 0) return fail(RSIM_ERR_INVALID_ARG, "negative pulse index or count");
    if (!is_pow2(burst) || burst < 2 || burst > 1024 || !is_pow2(radar->n_gates) ||
        radar->n_gates < 2 || (int64_t)burst * radar->n_gates > 12288)
        return fail(RSIM_ERR_UNSUPPORTED, "burst=%d, n_gates=%d: need powers of two >= 2, "
                    "burst <= 1024, burst * n_gates <= 12288", burst, radar->n_gates);
    const int64_t n_bursts = n_pulses / burst;
    if (n_bursts == 0) return RSIM_OK;
    if (!iq || !multilook) return fail(RSIM_ERR_INVALID_ARG, "iq / multilook is NULL");
    if (!aligned(iq, 8) || !aligned(multilook, 4) || (focused && !aligned(focused, 8)))
        return fail(RSIM_ERR_INVALID_ARG, "iq / focused / multilook misaligned");
    rsim::DdArgs a;
    a.n_gates = radar->n_gates;
    a.burst = burst;
    a.log2_g = 0;
    while ((1 << a.log2_g) < radar->n_gates) ++a.log2_g;
    a.log2_b = 0;
    while ((1 << a.log2_b) < burst) ++a.log2_b;
    a.pulse0 = pulse0;
    a.lambda = radar->c_mps / radar->carrier_hz;
    a.prf = radar->prf_hz;
    a.inv_prf = 1.0 / radar->prf_hz;
    a.nu_c = -2.0 * platform->v[2] / (a.lambda * radar->prf_hz);
    a.vh = std::hypot(platform->v[0], platform->v[1]);
    a.gate_width = radar->gate_width_m;
    a.r_ref0 = platform->r_ref0;
    a.r_ref_rate = platform->r_ref_rate;
    {
        const double q = a.vh > 0.0 ? a.lambda * a.prf / (2.0 * a.vh) : 0.0;
        a.mig_c = q * q / (2.0 * a.gate_width * (double)a.n_gates);
    }
    const cudaError_t e = rsim::launch_dd_focus(a, n_bursts, iq, focused, multilook, stream);
    if (e != cudaSuccess) return cuda_fail(e, "delay-Doppler kernel launch");
    return RSIM_OK;
}

static rsim_status surface_args(const rsim_wave_spectrum* sp, rsim::SurfArgs* a) {
    if (!sp) return fail(RSIM_ERR_INVALID_ARG, "spectrum is NULL");
    if (!is_pow2(sp->L) || sp->L < 2 || sp->L > 4096)
        return fail(RSIM_ERR_INVALID_ARG, "spectrum L=%d must be a power of two in [2, 4096]", sp->L);
    if (!sp->coef || !aligned(sp->coef, 8))
        return fail(RSIM_ERR_INVALID_ARG, "spectrum coef is NULL or not 8-byte aligned");
    if (sp->reserved != 0) return fail(RSIM_ERR_INVALID_ARG, "spectrum.reserved must be 0");
    if (!finite_pos(sp->spacing) || !finite_pos(sp->g) || !std::isfinite(sp->scale))
        return fail(RSIM_ERR_INVALID_ARG, "spectrum spacing, g must be finite and > 0, scale finite");
    a->L = sp->L;
    a->log2L = 0;
    while ((1 << a->log2L) < sp->L) ++a->log2L;
    int c = 8;
    while (c > 1 && ((int64_t)c * sp->L > 16384 || c > sp->L)) c >>= 1;  // <= 16384 points per CTA
    a->cols = c;
    a->dk = 6.283185307179586476925 / ((double)sp->L * sp->spacing);
    a->g = sp->g;
    a->t_hi = 0.f;
    a->t_lo = 0.f;
    a->scale_over_L2 = (float)(sp->scale / ((double)sp->L * (double)sp->L));
    return RSIM_OK;
}

size_t rsim_surface_workspace_size(int32_t L) {
    if (L < 1) return 0;
    const size_t b = (size_t)24 * (size_t)L * (size_t)L + (size_t)12 * (size_t)L;
    return (b + 255u) & ~(size_t)255u;
}

rsim_status rsim_surface_prepare(const rsim_wave_spectrum* spectrum, void* workspace,
                                 size_t workspace_bytes, cudaStream_t stream) {
    rsim::SurfArgs a;
    rsim_status st = surface_args(spectrum, &a);
    if (st != RSIM_OK) return st;
    const size_t need = rsim_surface_workspace_size(a.L);
    if (!workspace || !aligned(workspace, 256) || workspace_bytes < need)
        return fail(RSIM_ERR_WORKSPACE, "surface workspace: need %zu bytes, 256-byte aligned", need);
    const cudaError_t e = rsim::launch_surf_prepare(a, rsim::surf_tables(a.L, workspace),
                                                    device_sms(), stream);
    if (e != cudaSuccess) return cuda_fail(e, "surface prepare kernel launch");
    return RSIM_OK;
}

rsim_status rsim_surface_at(const rsim_wave_spectrum* spectrum, double t, float* z, float* vx,
                            float* vy, float* vz, void* workspace, size_t workspace_bytes,
                            cudaStream_t stream) {
    rsim::SurfArgs a;
    rsim_status st = surface_args(spectrum, &a);
    if (st != RSIM_OK) return st;
    if (!std::isfinite(t)) return fail(RSIM_ERR_INVALID_ARG, "t must be finite");
    const size_t need = rsim_surface_workspace_size(a.L);
    if (!workspace || !aligned(workspace, 256) || workspace_bytes < need)
        return fail(RSIM_ERR_WORKSPACE, "surface workspace: need %zu bytes, 256-byte aligned", need);
    float* outs[4] = {z, vx, vy, vz};
    for (int i = 0; i < 4; ++i)
        if (!outs[i] || !aligned(outs[i], 4)) return fail(RSIM_ERR_INVALID_ARG, "output field NULL or misaligned");
    a.t_hi = (float)t;
    a.t_lo = (float)(t - (double)a.t_hi);
    const cudaError_t e = rsim::launch_surf_at(a, spectrum->coef, rsim::surf_tables(a.L, workspace),
                                               z, vx, vy, vz, stream);
    if (e != cudaSuccess) return cuda_fail(e, "surface kernels launch");
    return RSIM_OK;
}

rsim_status rsim_scatterer_echo(const rsim_radar* radar, const rsim_platform* platform,
                                const rsim_scatterers* scat, int64_t pulse,
                                rsim_precision precision, void* contrib, cudaStream_t stream) {
    rsim_status st;
    if ((st = check_radar(radar)) != RSIM_OK) return st;
    if ((st = check_platform(platform)) != RSIM_OK) return st;
    if ((st = check_scat(scat)) != RSIM_OK) return st;
    if ((st = check_precision(precision)) != RSIM_OK) return st;
    if (pulse < 0 || pulse > ((int64_t)1 << 52)) return fail(RSIM_ERR_INVALID_ARG, "pulse out of range");
    if (scat->n == 0) return RSIM_OK;
    const bool fp64 = precision == RSIM_FP64;
    if (!contrib || !aligned(contrib, fp64 ? 16 : 8))
        return fail(RSIM_ERR_INVALID_ARG, "contrib is NULL or misaligned");
    const rsim::Model m = make_model(radar, platform, scat, 1);
    const rsim::Scat sc = make_scat(scat);
    const cudaError_t e = rsim::launch_cells(m, pulse, fp64, false, sc, nullptr, nullptr, nullptr,
                                             nullptr, contrib, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cells kernel launch");
    return checked_ok(stream);
}

rsim_status rsim_synth_pulses_backward(const rsim_radar* radar, const void* grad_iq,
                                       int32_t n_spectra, int64_t update0, int32_t n_fast,
                                       int32_t n_doppler, int64_t pulse0, int32_t n_pulses,
                                       rsim_window window, rsim_precision precision,
                                       void* grad_spectra, cudaStream_t stream) {
    rsim_status st = check_synth_args(radar, n_spectra, update0, n_fast, n_doppler, pulse0,
                                      n_pulses, (int)window, precision);
    if (st != RSIM_OK) return st;
    if (n_spectra == 0) return RSIM_OK;
    const bool fp64 = precision == RSIM_FP64;
    if (!grad_spectra || (n_pulses > 0 && !grad_iq))
        return fail(RSIM_ERR_INVALID_ARG, "grad_iq / grad_spectra is NULL");
    if (!aligned(grad_spectra, fp64 ? 16 : 8) || (grad_iq && !aligned(grad_iq, fp64 ? 16 : 8)))
        return fail(RSIM_ERR_INVALID_ARG, "grad_iq / grad_spectra misaligned");
    const rsim::SynthArgs a = make_synth_args(radar, n_spectra, update0, n_fast, n_doppler, pulse0,
                                              n_pulses, (int)window);
    const cudaError_t e = rsim::launch_synth_backward(a, fp64, grad_iq, grad_spectra, stream);
    if (e != cudaSuccess) return cuda_fail(e, "synth backward kernel launch");
    return RSIM_OK;
}

static rsim_status run_backward(const rsim_radar* radar, const rsim_platform* platform,
                                const rsim_scatterers* scat, int64_t pulse_base, int32_t stride,
                                int32_t n_samples, int32_t n_doppler, bool doppler,
                                rsim_precision precision, const void* G, float* grad_z,
                                float* grad_nrcs, cudaStream_t stream) {
    rsim_status st;
    if ((st = check_radar(radar)) != RSIM_OK) return st;
    if ((st = check_platform(platform)) != RSIM_OK) return st;
    if ((st = check_scat(scat)) != RSIM_OK) return st;
    if ((st = check_precision(precision)) != RSIM_OK) return st;
    if (n_samples < 0 || pulse_base < 0) return fail(RSIM_ERR_INVALID_ARG, "negative count or index");
    if (pulse_base + (int64_t)n_samples * stride > ((int64_t)1 << 52))
        return fail(RSIM_ERR_INVALID_ARG, "pulse index out of range");
    if (n_samples == 0 || scat->n == 0 || (!grad_z && !grad_nrcs)) return RSIM_OK;
    const bool fp64 = precision == RSIM_FP64;
    if (!G) return fail(RSIM_ERR_INVALID_ARG, "incoming gradient is NULL");
    if (!aligned(G, fp64 ? 16 : 8)) return fail(RSIM_ERR_INVALID_ARG, "incoming gradient misaligned");
    const rsim::Model m = make_model(radar, platform, scat, n_doppler);
    const rsim::Scat sc = make_scat(scat);
    rsim::Schedule sch;
    sch.pulse_base = pulse_base;
    sch.pulse_stride = stride;
    sch.n_samples = n_samples;
    sch.samples_per_group = n_samples;
    sch.pad = 0;
    const cudaError_t e = rsim::launch_backward(m, sch, sc, fp64, doppler, G, grad_z, grad_nrcs, stream);
    if (e != cudaSuccess) return cuda_fail(e, "backward kernel launch");
    return checked_ok(stream);
}

rsim_status rsim_doppler_accumulate_backward(const rsim_radar* radar,
                                             const rsim_platform* platform,
                                             const rsim_scatterers* scat, int64_t update0,
                                             int32_t n_updates, int32_t n_fast,
                                             int32_t n_doppler, rsim_precision precision,
                                             const void* grad_spectra, float* grad_z,
                                             float* grad_nrcs, cudaStream_t stream) {
    if (n_fast < 1) return fail(RSIM_ERR_INVALID_ARG, "n_fast=%d < 1", n_fast);
    if (!is_pow2(n_doppler) || n_doppler > 4096)
        return fail(RSIM_ERR_INVALID_ARG, "n_doppler=%d must be a power of two in [1, 4096]", n_doppler);
    if (update0 < 0 || update0 > (((int64_t)1 << 52) / n_fast))
        return fail(RSIM_ERR_INVALID_ARG, "update0 out of range");
    return run_backward(radar, platform, scat, update0 * (int64_t)n_fast, n_fast, n_updates,
                        n_doppler, true, precision, grad_spectra, grad_z, grad_nrcs, stream);
}

// Work counters of the persistent batched launches, one per launch, after the sets' regions.
size_t batch_counters_bytes(int32_t n_real) {
    return ((size_t)4 * (size_t)(n_real > 0 ? n_real : 0) + 255u) & ~(size_t)255u;
}

size_t rsim_batched_workspace_size(int32_t n_real, int32_t n_samples, int32_t n_gates,
                                   int32_t n_doppler) {
    if (n_real < 0 || rsim_workspace_size(n_samples, n_gates, n_doppler) == 0) return 0;
    return (size_t)n_real * batch_stride(n_samples, n_gates, n_doppler) + batch_counters_bytes(n_real);
}

rsim_status rsim_doppler_accumulate_batched(const rsim_radar* radar, const rsim_platform* platform,
                                            int32_t n_real, const rsim_scatterers* scats,
                                            int64_t update0, int32_t n_updates, int32_t n_fast,
                                            int32_t n_doppler, rsim_precision precision,
                                            void* const* spectra, const rsim_tuning* tuning,
                                            void* workspace, size_t workspace_bytes,
                                            cudaStream_t stream) {
    rsim_status st;
    int sets_per_launch = rsim::kMaxBatch;
    int32_t spg_req = 0;
    int persistent = 0;
    if (tuning) {
        for (int i = 0; i < 5; ++i)
            if (tuning->reserved[i] != 0) return fail(RSIM_ERR_INVALID_ARG, "tuning.reserved must be 0");
        if (tuning->persistent < 0 || tuning->persistent > 8)
            return fail(RSIM_ERR_INVALID_ARG, "tuning.persistent=%d not in [0, 8]", tuning->persistent);
        persistent = tuning->persistent;
        if (tuning->sets_per_launch < 0 || tuning->sets_per_launch > rsim::kMaxBatch)
            return fail(RSIM_ERR_INVALID_ARG, "tuning.sets_per_launch=%d not in [0, %d]",
                        tuning->sets_per_launch, rsim::kMaxBatch);
        if (tuning->samples_per_group < 0)
            return fail(RSIM_ERR_INVALID_ARG, "tuning.samples_per_group < 0");
        if (tuning->sets_per_launch > 0) sets_per_launch = tuning->sets_per_launch;
        spg_req = tuning->samples_per_group;
    }
    if ((st = check_radar(radar)) != RSIM_OK) return st;
    if ((st = check_platform(platform)) != RSIM_OK) return st;
    if ((st = check_precision(precision)) != RSIM_OK) return st;
    if (n_fast < 1) return fail(RSIM_ERR_INVALID_ARG, "n_fast=%d < 1", n_fast);
    if (!is_pow2(n_doppler) || n_doppler > 4096)
        return fail(RSIM_ERR_INVALID_ARG, "n_doppler=%d must be a power of two in [1, 4096]", n_doppler);
    if ((int64_t)radar->n_gates * n_doppler > ((int64_t)1 << 24))
        return fail(RSIM_ERR_INVALID_ARG, "n_gates * n_doppler > 2^24");
    if (n_real < 0 || n_updates < 0 || update0 < 0)
        return fail(RSIM_ERR_INVALID_ARG, "negative count or index");
    if (update0 > (((int64_t)1 << 52) / n_fast) - n_updates)
        return fail(RSIM_ERR_INVALID_ARG, "update index out of range");
    if (n_real == 0 || n_updates == 0) return RSIM_OK;
    if (!scats || !spectra) return fail(RSIM_ERR_INVALID_ARG, "scatterer / spectra arrays are NULL");
    const bool fp64 = precision == RSIM_FP64;
    for (int r = 0; r < n_real; ++r) {
        if ((st = check_scat(&scats[r])) != RSIM_OK)
            return fail(st, "realization %d: %s", r, g_last_error.c_str());
        if (scats[r].n > 0 && (!spectra[r] || !aligned(spectra[r], fp64 ? 16 : 8)))
            return fail(RSIM_ERR_INVALID_ARG, "realization %d: spectra NULL or misaligned", r);
    }
    const size_t stride_b = batch_stride(n_updates, radar->n_gates, n_doppler);
    const size_t need = (size_t)n_real * stride_b + batch_counters_bytes(n_real);
    if (fp64) persistent = 0;                       // the persistent form is the split path's
    if (!workspace) return fail(RSIM_ERR_WORKSPACE, "workspace is NULL (need %zu bytes)", need);
    if (!aligned(workspace, 256)) return fail(RSIM_ERR_WORKSPACE, "workspace not 256-byte aligned");
    if (workspace_bytes < need)
        return fail(RSIM_ERR_WORKSPACE, "workspace of %zu bytes < %zu required", workspace_bytes, need);

    const rsim::Model m = make_model(radar, platform, &scats[0], n_doppler);
    cudaError_t e = cudaMemsetAsync(workspace, 0, need, stream);
    if (e != cudaSuccess) return cuda_fail(e, "workspace clear");
    const int64_t n_vals = (int64_t)(ws_bytes(n_updates, radar->n_gates, n_doppler) / 8);
    static thread_local rsim::BatchParams bp;       // 11.5 KB: kept off the host stack
    static thread_local rsim::FinalizeBatch fb;
    unsigned* counters = reinterpret_cast<unsigned*>(static_cast<char*>(workspace) +
                                                     (size_t)n_real * stride_b);
    int n_launch = 0;
    int r = 0;
    while (r < n_real) {
        int k = 0;
        int64_t chunks = 0;
        for (; r < n_real && k < sets_per_launch; ++r) {
            if (scats[r].n == 0) continue;
            rsim::BatchEntry& be = bp.e[k];
            be.sc = make_scat(&scats[r]);
            for (int i = 0; i < 3; ++i) be.p0[i] = platform->p0[i] - scats[r].origin[i];
            be.chunk_begin = chunks;
            be.ws = reinterpret_cast<unsigned long long*>(static_cast<char*>(workspace) + (size_t)r * stride_b);
            be.area = (float)scats[r].facet_area_m2;
            be.pad = 0;
            fb.ws[k] = be.ws;
            fb.out[k] = spectra[r];
            chunks += (scats[r].n + rsim::kChunk - 1) / rsim::kChunk;
            ++k;
        }
        if (k == 0) break;
        if (chunks > 0x7fffffff) return fail(RSIM_ERR_INVALID_ARG, "too many scatterers in one batch");
        bp.n_real = k;
        bp.pad = 0;
        rsim::Schedule sch;
        const int64_t groups = plan_samples(chunks, update0 * (int64_t)n_fast, n_fast, n_updates, &sch,
                                            spg_req);
        if (persistent > 0) {
            const int64_t items = chunks * groups;
            if (items > 0x7fffffff) return fail(RSIM_ERR_INVALID_ARG, "too many work items in one batch");
            int64_t ctas = (int64_t)device_sms() * persistent;
            if (ctas > items) ctas = items;
            e = rsim::launch_accumulate_batched_persistent(m, sch, bp, true, counters + n_launch,
                                                          chunks, (int)groups, (unsigned)ctas, stream);
        } else {
            e = rsim::launch_accumulate_batched(m, sch, bp, fp64, true,
                                                dim3((unsigned)chunks, (unsigned)groups), stream);
        }
        ++n_launch;
        if (e != cudaSuccess) return cuda_fail(e, "batched summation kernel launch");
        e = rsim::launch_finalize_batched(fb, k, n_vals, fp64, device_sms(), stream);
        if (e != cudaSuccess) return cuda_fail(e, "batched finalize kernel launch");
    }
    return checked_ok(stream);
}

rsim_status rsim_autotune_batched(const rsim_radar* radar, const rsim_platform* platform,
                                  int32_t n_real, const rsim_scatterers* scats, int64_t update0,
                                  int32_t n_updates, int32_t n_fast, int32_t n_doppler,
                                  rsim_precision precision, void* const* spectra, void* workspace,
                                  size_t workspace_bytes, int32_t reps, rsim_tuning* best,
                                  double* best_ms, cudaStream_t stream) {
    if (!best) return fail(RSIM_ERR_INVALID_ARG, "best is NULL");
    if (reps < 1 || reps > 1000) return fail(RSIM_ERR_INVALID_ARG, "reps=%d not in [1, 1000]", reps);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) return cuda_fail(e, "stream query");
    if (cap != cudaStreamCaptureStatusNone)
        return fail(RSIM_ERR_UNSUPPORTED, "autotuning times launches: not allowed during graph capture");
    // candidate plans (duplicates after clamping are skipped)
    const int sets_c[3] = {rsim::kMaxBatch, 32, 8};
    int32_t spg_c[5] = {0, n_updates, (n_updates + 1) / 2, (n_updates + 3) / 4, (n_updates + 7) / 8};
    std::vector<rsim_tuning> cand;
    int nonempty = 0;
    for (int r = 0; r < n_real; ++r) nonempty += (scats && scats[r].n > 0) ? 1 : 0;
    const int n_modes = precision == RSIM_SPLIT ? 2 : 1;   // persistent form: split path only
    for (int mode = 0; mode < n_modes; ++mode) {
        for (int a = 0; a < 3; ++a) {
            if (a > 0 && sets_c[a] >= nonempty) continue;  // same grouping as a larger value
            for (int b = 0; b < 5; ++b) {
                if (b > 0 && spg_c[b] < 1) continue;
                rsim_tuning t;
                memset(&t, 0, sizeof(t));
                t.sets_per_launch = sets_c[a];
                t.samples_per_group = spg_c[b];
                t.persistent = mode == 0 ? 0 : rsim::kMinBlocks;
                bool dup = false;
                for (const rsim_tuning& c : cand)
                    dup = dup || (c.sets_per_launch == t.sets_per_launch &&
                                  c.samples_per_group == t.samples_per_group &&
                                  c.persistent == t.persistent);
                if (!dup) cand.push_back(t);
            }
        }
    }
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return cuda_fail(e, "event");
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(e, "event");
    }
    rsim_status st = RSIM_OK;
    double best_t = -1.0;
    std::vector<float> times;
    for (const rsim_tuning& t : cand) {
        times.clear();
        for (int i = 0; i <= reps && st == RSIM_OK; ++i) {
            if ((e = cudaEventRecord(e0, stream)) != cudaSuccess) { st = cuda_fail(e, "event record"); break; }
            st = rsim_doppler_accumulate_batched(radar, platform, n_real, scats, update0, n_updates,
                                                 n_fast, n_doppler, precision, spectra, &t,
                                                 workspace, workspace_bytes, stream);
            if (st != RSIM_OK) break;
            if ((e = cudaEventRecord(e1, stream)) != cudaSuccess) { st = cuda_fail(e, "event record"); break; }
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { st = cuda_fail(e, "event sync"); break; }
            float ms = 0.f;
            if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) { st = cuda_fail(e, "event time"); break; }
            if (i > 0) times.push_back(ms);  // the first run is untimed (warm-up)
        }
        if (st != RSIM_OK) break;
        std::sort(times.begin(), times.end());
        const double med = times[times.size() / 2];
        if (best_t < 0.0 || med < best_t) {
            best_t = med;
            *best = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != RSIM_OK) return st;
    if (best_ms) *best_ms = best_t < 0.0 ? 0.0 : best_t;
    if (best_t < 0.0) memset(best, 0, sizeof(*best));  // nothing to run: the default plan
    return RSIM_OK;
}

rsim_status rsim_direct_sum_backward(const rsim_radar* radar, const rsim_platform* platform,
                                     const rsim_scatterers* scat, int64_t pulse0,
                                     int32_t n_pulses, rsim_precision precision,
                                     const void* grad_iq, float* grad_z, float* grad_nrcs,
                                     cudaStream_t stream) {
    return run_backward(radar, platform, scat, pulse0, 1, n_pulses, 1, false, precision, grad_iq,
                        grad_z, grad_nrcs, stream);
}

}  // extern "C"
