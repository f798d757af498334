/*
 * rsim.h -- C ABI of the GB300 (sm_103a) radar raw-data summation library.
 *
 * The library computes the coherent summation of many moving sea-surface
 * scatterers into complex IQ range gates, as described in arXiv 2408.11472
 * ("High Performance Simulation of Spaceborne Radar for Remote-Sensing
 * Oceanography"):
 *
 *   - regular mode (Section II.A, Fig. 1 step 4; n_fast = 0 in Section IV):
 *       Y[p, g] = sum_n C_n(t_p) [gate_n(t_p) = g]          -> rsim_direct_sum
 *   - fast mode (Section III): one scatterer pass per surface update i
 *     (pulse p_i = i * n_fast) accumulating a Doppler spectrum per range gate
 *     (Algorithm 1, pulse-pair Doppler + rasterize)          -> rsim_doppler_accumulate
 *     then a batched 1-D inverse FFT per gate, the Eq. (1) weights and the sum
 *     of weighted segments (Section III.B post-processing)  -> rsim_synth_pulses
 *   - adjoints of the three operations (gradients of a real loss w.r.t.
 *     scatterer heights and NRCS)                            -> rsim_*_backward
 *
 * Model (every function uses the same one):
 *   t_p = p / PRF; scatterer n at s(t) = origin + r_n + v_n (t - t0); platform at
 *   P(t) = p0 + v t; d = P - s; R = |d|; range-window reference
 *   r_ref(t) = r_ref0 + r_ref_rate t;
 *   gate = floor((R - r_ref) / gate_width + n_gates / 2), dropped unless
 *   0 <= gate < n_gates;
 *   off-nadir angle theta = atan2(|d_xy|, d_z);
 *   C = sqrt(nrcs * area) * w * (r_ref / R)^2 * exp(-j 4 pi R / lambda),  lambda = c / carrier,
 *   w = exp(-2 ln2 theta^2 / beamwidth^2), or the complex two-way gain of a tabulated
 *   pattern at the facet's direction cosines (rsim_antenna);
 *   pulse-pair Doppler of the pair (p_i, p_i + 1): nu = phase advance of C per
 *   pulse in cycles, wrapped to [-1/2, 1/2); bin = floor(nu * n_doppler + 1/2)
 *   mod n_doppler (so bin k holds the tone exp(+j 2 pi k m / n_doppler));
 *   inverse transform unnormalised: s_i[g, m] = sum_k T[i, g, k] e^{+j 2 pi k m / n_doppler};
 *   Y[x, g] = W(|p_i - x| / n_fast) s_i[g, (x - p_i) mod n_doppler]
 *           + W(|p_{i+1} - x| / n_fast) s_{i+1}[g, (x - p_{i+1}) mod n_doppler],
 *   i = floor(x / n_fast), with the blend window W of rsim_window.
 *
 * Conventions shared by every entry point:
 *   - Memory: every array argument is a DEVICE pointer to caller-owned memory
 *     (structs themselves are host memory, read during the call only).  The
 *     library makes no allocation of its own; scratch space is the explicit
 *     workspace argument, sized by rsim_workspace_size().
 *   - Execution: asynchronous on the given stream (0 = legacy default stream).
 *     A call only enqueues work; outputs are valid after the stream is
 *     synchronised.  Calls are thread-safe; a workspace must not be shared by
 *     calls that may overlap on the device.
 *   - Complex arrays are interleaved (re, im): complex64 (2 x float) when
 *     precision == RSIM_SPLIT, complex128 (2 x double) when RSIM_FP64.
 *   - Errors: a non-zero rsim_status is returned and nothing is enqueued for
 *     RSIM_ERR_INVALID_ARG / RSIM_ERR_UNSUPPORTED / RSIM_ERR_WORKSPACE;
 *     RSIM_ERR_CUDA reports a failed launch.  rsim_last_error() gives a
 *     per-thread message for the last failure.  Nothing throws across the ABI.
 *   - Scatterer order: any order is accepted; RSIM_SPLIT is most accurate when
 *     consecutive scatterers are spatially close (e.g. a row-major grid),
 *     because each block of rsim_block_scatterers() (1024) consecutive
 *     scatterers shares one FP64 reference point.
 *   - Accumulation is deterministic fixed point: each contribution is rounded to
 *     a multiple of 2^-32 (a 64-bit integer) and the integers are summed, so results
 *     are bitwise reproducible run to run regardless of scheduling.  Valid while every
 *     contribution's |re|, |im| < 2^30 and every cell's sum stays within +-2^31; the
 *     default build does not check this, and beyond it the values saturate or wrap
 *     silently (sea-surface facets give contributions of order sqrt(nrcs * area), a few
 *     units).  The debug build (rsim_check_build() == 1) reports an emitted sum at or
 *     beyond 2^30 as RSIM_ERR_CHECK.
 */
#ifndef RSIM_H
#define RSIM_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RSIM_ABI_VERSION 2

typedef enum {
    RSIM_OK = 0,
    RSIM_ERR_INVALID_ARG = 1,  /* null/misaligned pointer, size or value out of range     */
    RSIM_ERR_CUDA = 2,         /* a CUDA launch or stream operation failed                 */
    RSIM_ERR_UNSUPPORTED = 3,  /* valid request the library does not implement           */
    RSIM_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up                       */
    RSIM_ERR_WORKSPACE = 5,    /* workspace missing, misaligned or smaller than required   */
    RSIM_ERR_CHECK = 6         /* -DRSIM_CHECK builds only: a kernel's bounds check failed  */
} rsim_status;

/* Arithmetic of the per-scatterer path.
 * RSIM_FP64  : every per-scatterer quantity in IEEE double (slow on GB300's FP64 pipe).
 * RSIM_SPLIT : FP64 only per (block of scatterers, pulse) -- platform position, reference
 *              range and phase of a block reference point -- and FP32 for the per-scatterer
 *              differential range, phase, sincos and weights; gate and Doppler-bin decisions
 *              that fall within rounding distance of a cell edge are re-taken in FP64. */
typedef enum { RSIM_FP64 = 0, RSIM_SPLIT = 1 } rsim_precision;

/* Blend window W(d), d = |p_i - x| / n_fast in [0, 1], zero at d >= 1.
 * RSIM_WIN_SQRT_LINEAR        : (1 - d)^(1/2)           -- Eq. (1) of the paper.
 * RSIM_WIN_SQRT_RAISED_COSINE : cos(pi d / 2)           -- squared weights form a raised cosine.
 * RSIM_WIN_LINEAR             : 1 - d                   -- linear amplitude crossfade (tests). */
typedef enum {
    RSIM_WIN_SQRT_LINEAR = 0,
    RSIM_WIN_SQRT_RAISED_COSINE = 1,
    RSIM_WIN_LINEAR = 2
} rsim_window;

/* Instrument constants (SI).  1 <= n_gates <= 4096; all doubles finite and > 0. */
/* Two-way antenna pattern tabulated on a u-v grid (Section II.A: every pattern a simulation
 * needs is recorded on a u-v grid, and its complex value at each facet is obtained by
 * interpolation in that grid).  (u, v) are the first two direction cosines of the line of
 * sight from the platform to the facet in the scene frame, u = (s - P)_x / R,
 * v = (s - P)_y / R.  Node (i, j) is at u = u0 + i du, v = v0 + j dv.  Between nodes the
 * real and imaginary parts are interpolated bilinearly; outside
 * [u0, u0 + (nu-1) du) x [v0, v0 + (nv-1) dv) the gain is 0.  The edge decision is taken
 * in the precision of the call, so a table should fall to 0 at its border.
 * gain : DEVICE [nv][nu] complex64 (re, im interleaved), 8-byte aligned, read during the
 *        call's kernels (keep it alive until they finish). */
typedef struct {
    const void *gain;
    int32_t nu, nv;        /* >= 2 each, nu * nv < 2^31 */
    double u0, du;         /* du > 0 */
    double v0, dv;         /* dv > 0 */
} rsim_antenna;

typedef struct {
    double carrier_hz;     /* carrier frequency f_c                               */
    double prf_hz;         /* pulse repetition frequency                          */
    double c_mps;          /* propagation speed                                   */
    double gate_width_m;   /* range-gate width                                    */
    double beamwidth_rad;  /* two-way 3 dB full beamwidth of the Gaussian pattern */
    int32_t n_gates;       /* number of range gates N_g                           */
    int32_t reserved;      /* must be 0                                           */
    const rsim_antenna *antenna;  /* tabulated two-way pattern (host struct, read during the
                                     call), or NULL for the Gaussian pattern of beamwidth_rad */
} rsim_radar;

/* Platform track in the scene frame (metres, seconds): P(t) = p0 + v t;
 * range-window reference r_ref(t) = r_ref0 + r_ref_rate t (gate n_gates/2 starts there). */
typedef struct {
    double p0[3];
    double v[3];
    double r_ref0;
    double r_ref_rate;
} rsim_platform;

/* Scatterer set, structure of arrays of n float32 DEVICE arrays: positions relative
 * to origin (m) at the epoch t0 (s), velocities (m/s), NRCS (linear, >= 0); the scatterer
 * moves as s(t) = origin + r + v (t - t0).  facet_area_m2 > 0.  Give the state at an epoch
 * near the pulses simulated (the surface of Algorithm 1's update_simulation at that time):
 * RSIM_SPLIT carries |r - c + v (t - t0)| in FP32. */
typedef struct {
    int64_t n;
    const float *x, *y, *z, *vx, *vy, *vz, *nrcs;
    double origin[3];
    double facet_area_m2;
    double t0;
} rsim_scatterers;

/* Library version (RSIM_ABI_VERSION). */
int rsim_version(void);

/* 1 if the library was compiled with -DRSIM_CHECK (librsim_check.so), else 0.  In that
 * debug build the summation, cell, echo and adjoint kernels check every Doppler bin when a
 * cell key is formed (0 <= bin < n_doppler), every contribution sum before its fixed-point
 * conversion (|value| < 2^30), every sample slot against the call's samples, and every
 * adjoint gather cell against n_gates x n_doppler.  A failed check skips the addition or
 * read it guards and records itself; the entry point then returns RSIM_ERR_CHECK, with the
 * check and the offending value in rsim_last_error().  Those entry points synchronise their
 * stream to read the record, so the debug build is for testing, not for timing. */
int rsim_check_build(void);

/* Number of consecutive scatterers that share one FP64 reference point in RSIM_SPLIT
 * (the scatterer block of one CTA).  Splitting a scatterer set at multiples of it keeps every
 * scatterer's arithmetic, and so its index decisions, identical to an unsplit call. */
int rsim_block_scatterers(void);

/* Message describing the last failure on the calling thread ("" if none). */
const char *rsim_last_error(void);

/* Bytes of workspace rsim_direct_sum / rsim_doppler_accumulate need for n_samples
 * samples (pulses, or updates) of n_gates x n_doppler cells (n_doppler = 1 for
 * rsim_direct_sum).  Returns 0 for invalid sizes. */
size_t rsim_workspace_size(int32_t n_samples, int32_t n_gates, int32_t n_doppler);

/* Regular mode (Section II.A, Fig. 1 step 4):
 *   iq[p][g] += sum_n C_n(t_{pulse0+p}) [gate_n = g],  p in [0, n_pulses).
 * iq        : [n_pulses][n_gates] complex (see precision), accumulated (+=).
 * workspace : >= rsim_workspace_size(n_pulses, n_gates, 1) bytes, 16-byte aligned.
 * out_of_window : NULL, or DEVICE [n_pulses] uint64, 8-byte aligned, accumulated (+=):
 *             out_of_window[p] += the number of scatterers whose gate at pulse pulse0 + p lies
 *             outside [0, n_gates), so that the call leaves them out.  The decisions are the
 *             summation's own (same precision, same re-decisions near a gate edge); counting
 *             costs one more kernel launch of about a third of the summation's time and
 *             changes nothing in iq.
 * pulse0 >= 0, n_pulses >= 0 (0: no-op). */
rsim_status rsim_direct_sum(const rsim_radar *radar, const rsim_platform *platform,
                            const rsim_scatterers *scat, int64_t pulse0, int32_t n_pulses,
                            rsim_precision precision, void *iq, void *workspace,
                            size_t workspace_bytes, unsigned long long *out_of_window,
                            cudaStream_t stream);

/* Fast-mode Doppler spectra (Algorithm 1 of Section III.B) for the updates
 * i in [update0, update0 + n_updates): pulse pair (p_i, p_i + 1), p_i = i n_fast,
 *   spectra[i - update0][g][k] += sum of C_n(t_{p_i}) over scatterers with gate g, bin k.
 * spectra   : [n_updates][n_gates][n_doppler] complex, accumulated (+=).
 * n_fast >= 1; n_doppler a power of two in [1, 4096]; update0 >= 0.
 * workspace : >= rsim_workspace_size(n_updates, n_gates, n_doppler) bytes, 16-byte aligned.
 * out_of_window : NULL, or DEVICE [n_updates] uint64, 8-byte aligned, accumulated (+=):
 *             out_of_window[i - update0] += the number of scatterers whose gate at pulse p_i
 *             lies outside [0, n_gates) (left out of update i's spectrum), decided as the
 *             summation decides; as rsim_direct_sum's. */
rsim_status rsim_doppler_accumulate(const rsim_radar *radar, const rsim_platform *platform,
                                    const rsim_scatterers *scat, int64_t update0,
                                    int32_t n_updates, int32_t n_fast, int32_t n_doppler,
                                    rsim_precision precision, void *spectra, void *workspace,
                                    size_t workspace_bytes, unsigned long long *out_of_window,
                                    cudaStream_t stream);

/* Workspace bytes of rsim_doppler_accumulate_batched: n_real regions of
 * rsim_workspace_size(n_samples, n_gates, n_doppler) rounded up to 256 bytes, then one
 * 4-byte work counter per launch (rounded up to 256 bytes). */
size_t rsim_batched_workspace_size(int32_t n_real, int32_t n_samples, int32_t n_gates,
                                   int32_t n_doppler);

/* Blockwise summation into one deterministic fixed-point workspace, for a scatterer set that
 * arrives in blocks (streamed from host memory, or larger than device memory):
 *   rsim_workspace_clear, then rsim_doppler_accumulate_partial for every block (each adds
 *   its contributions to the workspace's fixed-point sums; no clear, no conversion), then
 *   rsim_workspace_finalize (adds the sums to the complex spectra, +=).
 * Blocks that start at multiples of rsim_block_scatterers() keep every scatterer's FP64
 * reference point, so the spectra are bit-identical to one rsim_doppler_accumulate call on
 * the whole set.  Arguments as rsim_doppler_accumulate (without the out-of-window
 * counter); workspace 16-byte aligned, of at least
 * rsim_workspace_size(n_updates, n_gates, n_doppler) bytes, and must not be shared by
 * overlapping calls. */
rsim_status rsim_workspace_clear(int32_t n_updates, int32_t n_gates, int32_t n_doppler,
                                 void *workspace, size_t workspace_bytes, cudaStream_t stream);
rsim_status rsim_doppler_accumulate_partial(const rsim_radar *radar,
                                            const rsim_platform *platform,
                                            const rsim_scatterers *scat, int64_t update0,
                                            int32_t n_updates, int32_t n_fast, int32_t n_doppler,
                                            rsim_precision precision, void *workspace,
                                            size_t workspace_bytes, cudaStream_t stream);
rsim_status rsim_workspace_finalize(int32_t n_updates, int32_t n_gates, int32_t n_doppler,
                                    rsim_precision precision, const void *workspace,
                                    size_t workspace_bytes, void *spectra, cudaStream_t stream);

/* One surface update's state (Algorithm 1's update_simulation regenerates the surface at
 * every update): heights and velocities of the scatterer set at epoch t0, DEVICE float32
 * arrays [n], 16-byte aligned (e.g. the fields rsim_surface_at writes for t0). */
typedef struct {
    const float *z, *vx, *vy, *vz;
    double t0;
} rsim_surface_state;

#define RSIM_MAX_STATES 64

/* rsim_doppler_accumulate_partial for updates whose scatterers move between updates
 * (Algorithm 1 with the surface regenerated at every update): update update0 + s takes the
 * positions x, y and NRCS of `scat` (its origin and facet area; its z, vx, vy, vz and t0 are
 * not read and may be NULL / 0) with the heights, velocities and epoch of states[s], and
 * adds its spectrum to slot s of the deterministic fixed-point workspace (cleared before by
 * rsim_workspace_clear, converted after by rsim_workspace_finalize).  One launch covers
 * the n_updates updates: the horizontal positions are read once, each update's heights and
 * velocities (16 bytes per scatterer) once per update.  Every (block, update) pair is
 * evaluated (no range-window culling: pass only updates whose window can see the set).
 * states : HOST array [n_updates], 0 <= n_updates <= RSIM_MAX_STATES;
 * workspace >= rsim_workspace_size(n_updates, n_gates, n_doppler) bytes, 16-byte aligned.
 * Other arguments as rsim_doppler_accumulate. */
rsim_status rsim_doppler_accumulate_states(const rsim_radar *radar, const rsim_platform *platform,
                                           const rsim_scatterers *scat, int64_t update0,
                                           int32_t n_updates, const rsim_surface_state *states,
                                           int32_t n_fast, int32_t n_doppler,
                                           rsim_precision precision, void *workspace,
                                           size_t workspace_bytes, cudaStream_t stream);

/* Launch plan of the batched scatterer pass./* Launch plan of the batched scatterer pass.  Every choice gives bit-identical results;
 * only the speed differs (see rsim_autotune_batched). */
typedef struct {
    int32_t sets_per_launch;   /* scatterer sets per launch, 1..96; 0 = 96 */
    int32_t samples_per_group; /* updates handled by one work item (the rest of the updates go
                                  to further items over the same scatterers); 0 = library's
                                  choice */
    int32_t persistent;        /* 0: one CTA per (block of scatterers, group of updates);
                                  1..8: RSIM_SPLIT only -- one launch of this many CTAs per SM
                                  that stay resident and take (set, block, update group) work
                                  items in order from an atomic counter until none are left */
    int32_t reserved[5];       /* must be 0 */
} rsim_tuning;

/* rsim_doppler_accumulate for n_real independent scatterer sets -- realizations of the same
 * track, as the ~100 realizations behind each SWH/SSH spectrum of Section IV.D -- in one
 * launch per group of up to 96 sets: every CTA of the launch takes a block of scatterers of
 * one set (sets of uneven size share the grid), and samples whose range window no scatterer
 * of a block can reach are skipped by that block.  Each set's spectra are bit-identical to
 * a rsim_doppler_accumulate call of its own.
 * scats   : HOST array [n_real] of scatterer sets (device arrays; each its own origin/area);
 * spectra : HOST array [n_real] of DEVICE pointers, each [n_updates][n_gates][n_doppler]
 *           complex, accumulated (+=);
 * tuning  : launch plan, or NULL for the library's choice (RSIM_ERR_INVALID_ARG when a
 *           field is out of range);
 * workspace >= rsim_batched_workspace_size(n_real, n_updates, n_gates, n_doppler), 256-byte
 * aligned.  Capturable in a CUDA graph (memset + kernels only). */
rsim_status rsim_doppler_accumulate_batched(const rsim_radar *radar,
                                            const rsim_platform *platform, int32_t n_real,
                                            const rsim_scatterers *scats, int64_t update0,
                                            int32_t n_updates, int32_t n_fast, int32_t n_doppler,
                                            rsim_precision precision, void *const *spectra,
                                            const rsim_tuning *tuning, void *workspace,
                                            size_t workspace_bytes, cudaStream_t stream);

/* Autotuner of the batched scatterer pass: runs rsim_doppler_accumulate_batched with the
 * same arguments under candidate launch plans (sets per launch in {96, 32, 8}, samples per
 * group in {library's choice, n_updates, n_updates/2, /4, /8}, each as one CTA per work
 * item and, for RSIM_SPLIT, as a persistent launch of 4 CTAs per SM; limited to what the
 * call can use), times each with CUDA events on `stream` (one untimed run, then the median of
 * `reps` >= 1 runs) and writes the fastest plan to *best and its time in ms to *best_ms
 * (may be NULL).  Tune on a representative part of the job (e.g. a few dozen updates):
 * the plan then applies to any update range of the same sets.
 * SYNCHRONOUS: blocks until the runs finish; RSIM_ERR_UNSUPPORTED while `stream` is being
 * captured into a graph.  The spectra receive unspecified values (accumulated several
 * times): pass scratch buffers or zero them afterwards. */
rsim_status rsim_autotune_batched(const rsim_radar *radar, const rsim_platform *platform,
                                  int32_t n_real, const rsim_scatterers *scats, int64_t update0,
                                  int32_t n_updates, int32_t n_fast, int32_t n_doppler,
                                  rsim_precision precision, void *const *spectra,
                                  void *workspace, size_t workspace_bytes, int32_t reps,
                                  rsim_tuning *best, double *best_ms, cudaStream_t stream);

/* Fast-mode post-processing (Section III.B steps 2-4 with Eq. (1)): batched
 * n_doppler-point inverse FFT per gate of each spectrum, blend window, sum into
 * the pulses x in [pulse0, pulse0 + n_pulses).
 * spectra   : [n_spectra][n_gates][n_doppler] complex; spectra[s] belongs to update update0 + s.
 * iq        : [n_pulses][n_gates] complex, OVERWRITTEN.
 * Every pulse x must find its spectra: floor(x / n_fast) >= update0, and
 * floor(x / n_fast) + 1 < update0 + n_spectra unless x is a multiple of n_fast.
 * n_doppler a power of two in [2, 1024]; n_gates * n_doppler <= 2^20. */
rsim_status rsim_synth_pulses(const rsim_radar *radar, const void *spectra, int32_t n_spectra,
                              int64_t update0, int32_t n_fast, int32_t n_doppler,
                              int64_t pulse0, int32_t n_pulses, rsim_window window,
                              rsim_precision precision, void *iq, cudaStream_t stream);

/* Index decisions (for tests and diagnostics): for every scatterer, the range gate at
 * pulse p and the Doppler bin of the pulse pair (p, p + 1), with the pre-floor
 * coordinates (dR / gate_width + n_gates/2 and nu n_doppler + 1/2).  Gate is reported
 * even when out of the window.  Any output pointer may be NULL.
 * gate, bin : [n] int32;  gate_coord, bin_coord : [n] double. */
rsim_status rsim_scatterer_cells(const rsim_radar *radar, const rsim_platform *platform,
                                 const rsim_scatterers *scat, int64_t pulse, int32_t n_doppler,
                                 rsim_precision precision, int32_t *gate, int32_t *bin,
                                 double *gate_coord, double *bin_coord, cudaStream_t stream);

/* Delay-Doppler focusing of simulated IQ (Section IV.C): the pulses are split into bursts
 * of `burst` consecutive pulses; per burst
 *   1. Doppler centroid correction y_k *= exp(-j 2 pi nu_c k), k = 0 .. burst-1, with
 *      nu_c = -2 v_z / (lambda PRF) the phase advance per pulse of the nadir echo;
 *   2. along-track transform into Doppler beams B_f = sum_k y_k exp(-j 2 pi nu_f k),
 *      nu_f = (f - burst/2) / burst;
 *   3. range-migration correction with delay phase coefficients: beam f sees the
 *      along-track offset x_f = nu_f lambda R_0 PRF / (2 |v_xy|) (flat earth, R_0 = r_ref at
 *      the burst's centre pulse), whose range exceeds the nadir's by s_f = x_f^2 / (2 R_0)
 *      (in gates: / gate_width); Y_f = IDFT(DFT(B_f) exp(+j 2 pi q' s_f / n_gates)), q' the
 *      signed range frequency, IDFT normalised by 1 / n_gates (a shift of s_f gates towards
 *      the nadir gate);
 *   4. multi-look: W[g] = (1 / burst) sum_f |Y_f[g]|^2.
 * iq        : [n_pulses][n_gates] complex64, pulse pulse0 first (pulse0 >= 0 sets the time of
 *             each burst); bursts = floor(n_pulses / burst), trailing pulses unused;
 * focused   : [bursts][burst][n_gates] complex64 (beam-major), OVERWRITTEN, or NULL;
 * multilook : [bursts][n_gates] float, OVERWRITTEN.
 * burst and n_gates must be powers of two >= 2 with burst <= 1024 and
 * burst * n_gates <= 12288 (one burst held on chip), else RSIM_ERR_UNSUPPORTED.
 * Complex64 only (RSIM_SPLIT output). */
rsim_status rsim_delay_doppler(const rsim_radar *radar, const rsim_platform *platform,
                               const void *iq, int64_t pulse0, int32_t n_pulses, int32_t burst,
                               void *focused, float *multilook, cudaStream_t stream);

/* Sea-surface spectrum for the surface update at each update time (Algorithm 1's
 * update_simulation regenerates the surface at every update).  Linear deep-water waves:
 * one-sided complex coefficients A(k) on the L x L wave-number grid k = 2 pi fftfreq(L,
 * spacing) (index [iy][ix]), omega = sqrt(g |k|), and at time t
 *   z   = s Re IFFT2[A e^{-j omega t}],            v_z = s Re IFFT2[-j omega A e^{-j omega t}],
 *   v_x = s Re IFFT2[omega k_x/|k| A e^{-j omega t}], v_y = s Re IFFT2[omega k_y/|k| A ...],
 * IFFT2 normalised by 1 / L^2, on the facet grid x = (ix - (L-1)/2) spacing (y likewise),
 * row-major n = iy L + ix.
 * coef : DEVICE [L][L] complex64, 8-byte aligned; L a power of two in [2, 4096]. */
typedef struct {
    const void *coef;
    int32_t L;
    int32_t reserved;    /* must be 0 */
    double spacing;      /* facet grid step (m), > 0 */
    double scale;        /* amplitude scale s */
    double g;            /* gravity (m/s^2), > 0 */
} rsim_wave_spectrum;

/* Workspace bytes of the surface update: a table of omega / (2 pi) (8 L^2 bytes), two
 * packed L x L complex transforms (16 L^2 bytes), the transform's twiddles and the wave
 * numbers (12 L bytes), rounded up to 256 bytes. */
size_t rsim_surface_workspace_size(int32_t L);

/* Fills the workspace's omega table for `spectrum` (once per spectrum and workspace; the
 * table depends on L, spacing and g only).  Asynchronous on `stream`. */
rsim_status rsim_surface_prepare(const rsim_wave_spectrum *spectrum, void *workspace,
                                 size_t workspace_bytes, cudaStream_t stream);

/* The surface at time t (seconds): heights z and velocities vx, vy, vz ([L*L] float DEVICE
 * arrays, OVERWRITTEN) by two packed L x L inverse transforms per call (eta + j v_z and
 * v_x + j v_y: each real field is the transform of the Hermitian part of its spectrum).
 * The workspace must have been prepared for this spectrum (rsim_surface_prepare).  With
 * the facet grid and NRCS these are a scatterer set whose state epoch t0 is t. */
rsim_status rsim_surface_at(const rsim_wave_spectrum *spectrum, double t, float *z, float *vx,
                            float *vy, float *vz, void *workspace, size_t workspace_bytes,
                            cudaStream_t stream);

/* Per-scatterer complex amplitude C_n(t_pulse) of the radar equation and two-way phase
 * (Section II.A, Fig. 1 step 4; the model above), with the arithmetic of `precision`
 * exactly as the summation entry points evaluate it, for every scatterer whether or not
 * it falls in the range window.  For precision studies (phase and amplitude error of the
 * split path against RSIM_FP64).
 * contrib : [n] complex (complex64 for RSIM_SPLIT, complex128 for RSIM_FP64), OVERWRITTEN. */
rsim_status rsim_scatterer_echo(const rsim_radar *radar, const rsim_platform *platform,
                                const rsim_scatterers *scat, int64_t pulse,
                                rsim_precision precision, void *contrib, cudaStream_t stream);

/* Adjoint of rsim_synth_pulses (gradient convention dL/dRe + j dL/dIm):
 *   grad_spectra[s][g][k] = sum_m exp(-j 2 pi k m / n_doppler)
 *                           sum_x W_s(x) grad_iq[x][g] [ (x - p_s) mod n_doppler = m ].
 * grad_iq      : [n_pulses][n_gates] complex;  grad_spectra : [n_spectra][n_gates][n_doppler]
 * complex, OVERWRITTEN.  Same size rules as rsim_synth_pulses. */
rsim_status rsim_synth_pulses_backward(const rsim_radar *radar, const void *grad_iq,
                                       int32_t n_spectra, int64_t update0, int32_t n_fast,
                                       int32_t n_doppler, int64_t pulse0, int32_t n_pulses,
                                       rsim_window window, rsim_precision precision,
                                       void *grad_spectra, cudaStream_t stream);

/* Adjoint of rsim_doppler_accumulate: for each scatterer n,
 *   grad_z[n]    += sum_i Re(conj(G_i) dC_n/dz_n),
 *   grad_nrcs[n] += sum_i Re(conj(G_i) C_n) / (2 nrcs_n)   (0 where nrcs_n = 0),
 * G_i = grad_spectra[i - update0][gate_n][bin_n] (gate/bin are piecewise constant and
 * carry no gradient).  grad_z, grad_nrcs : [n] float32 (either may be NULL).
 * Per-scatterer phase and amplitude are recomputed, not stored.  Deterministic. */
rsim_status rsim_doppler_accumulate_backward(const rsim_radar *radar,
                                             const rsim_platform *platform,
                                             const rsim_scatterers *scat, int64_t update0,
                                             int32_t n_updates, int32_t n_fast,
                                             int32_t n_doppler, rsim_precision precision,
                                             const void *grad_spectra, float *grad_z,
                                             float *grad_nrcs, cudaStream_t stream);

/* Adjoint of rsim_direct_sum with G = grad_iq[p][gate_n(t_p)] ([n_pulses][n_gates] complex). */
rsim_status rsim_direct_sum_backward(const rsim_radar *radar, const rsim_platform *platform,
                                     const rsim_scatterers *scat, int64_t pulse0,
                                     int32_t n_pulses, rsim_precision precision,
                                     const void *grad_iq, float *grad_z, float *grad_nrcs,
                                     cudaStream_t stream);

/* rsim_doppler_accumulate without a caller workspace, for callers that cannot allocate
 * device memory where they run (allocation-free real-time loops, plug-ins inside a host
 * process whose allocator they do not own, tenants of a pre-partitioned GPU).  The paper
 * has no counterpart: this is a deployment variant of the same computation.
 * Same arguments and results as rsim_doppler_accumulate minus the workspace and the
 * out-of-window counter; the
 * fixed-point scratch is a 16 MiB device array built into the library (held by every GPU
 * that loads the library until the process exits), so
 * rsim_workspace_size(n_updates, n_gates, n_doppler) must be <= 16 MiB, else
 * RSIM_ERR_WORKSPACE.  Nothing is allocated: no cudaMalloc/cudaFree or allocating library
 * call.  The first call in each CUDA context looks the array's device address up
 * (cudaGetSymbolAddress, with that context current) and keeps it under the context's ID,
 * so a non-primary context, or a context made after cudaDeviceReset, gets its own address.
 * All calls in a context share
 * the array and each clears it on entry, so calls that may overlap on the GPU race; order
 * them (one stream, or events). */
rsim_status rsim_doppler_accumulate_noalloc(const rsim_radar *radar,
                                            const rsim_platform *platform,
                                            const rsim_scatterers *scat, int64_t update0,
                                            int32_t n_updates, int32_t n_fast, int32_t n_doppler,
                                            rsim_precision precision, void *spectra,
                                            cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* RSIM_H */
