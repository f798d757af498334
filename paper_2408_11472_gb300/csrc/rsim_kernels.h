// rsim_kernels.h -- host-side launchers of the library's kernels (internal interface
// between the C ABI in abi.cu and the kernel translation units).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rsim {

struct Model;
struct Schedule;
struct Scat;
struct BatchParams;
struct FinalizeBatch;
struct StatesParams;

cudaError_t launch_accumulate(const Model& m, const Schedule& sch, const Scat& sc, bool fp64,
                              bool doppler, unsigned long long* ws, dim3 grid,
                              cudaStream_t stream);
cudaError_t launch_finalize(const void* ws, void* out, int64_t n_vals, bool fp64, int n_sms,
                            cudaStream_t stream);
cudaError_t launch_accumulate_states(const Model& m, const Schedule& sch, const Scat& sc,
                                     const StatesParams& sp, bool fp64, bool doppler,
                                     unsigned long long* ws, unsigned n_chunks,
                                     cudaStream_t stream);
cudaError_t launch_accumulate_batched(const Model& m, const Schedule& sch, const BatchParams& bp,
                                      bool fp64, bool doppler, dim3 grid, cudaStream_t stream);
cudaError_t launch_accumulate_batched_persistent(const Model& m, const Schedule& sch,
                                                 const BatchParams& bp, bool doppler,
                                                 unsigned* counter, int64_t n_chunks, int groups,
                                                 unsigned n_ctas, cudaStream_t stream);
cudaError_t launch_finalize_batched(const FinalizeBatch& fb, int n_real, int64_t n_vals, bool fp64,
                                    int n_sms, cudaStream_t stream);
#ifdef RSIM_CHECK
// -DRSIM_CHECK builds: reads (synchronising `stream`) and clears the check word of the
// summation kernels' translation unit: 0, or the first failed check (code << 56 | value).
cudaError_t check_take(cudaStream_t stream, unsigned long long* word);
#endif
// counts[s] += scatterers the summation over `sch` leaves out (gate outside the window)
cudaError_t launch_window_count(const Model& m, const Schedule& sch, const Scat& sc, bool fp64,
                                bool doppler, unsigned long long* counts, cudaStream_t stream);
cudaError_t launch_cells(const Model& m, int64_t pulse, bool fp64, bool doppler, const Scat& sc,
                         int32_t* gate, int32_t* bin, double* gc, double* bc, void* contrib,
                         cudaStream_t stream);
cudaError_t launch_backward(const Model& m, const Schedule& sch, const Scat& sc, bool fp64,
                            bool doppler, const void* G, float* grad_z, float* grad_nrcs,
                            cudaStream_t stream);

// Sets the calling thread's rsim_last_error() message (abi.cu).
void set_last_error(const char* fmt, ...);

// Post-processing (synth.cu).
struct SynthArgs {
    int n_gates, n_doppler, log2_nd, n_fast, n_spectra, n_pulses;
    int64_t update0, pulse0;
    int window;
};
cudaError_t launch_synth(const SynthArgs& a, bool fp64, const void* spectra, void* iq,
                         cudaStream_t stream);
cudaError_t launch_synth_backward(const SynthArgs& a, bool fp64, const void* grad_iq,
                                  void* grad_spectra, cudaStream_t stream);

// Delay-Doppler focusing (ddfocus.cu).
struct DdArgs {
    int n_gates, burst, log2_g, log2_b;
    int64_t pulse0;
    double nu_c;                 // Doppler centroid, cycles per pulse
    double lambda, prf, inv_prf, vh, gate_width, r_ref0, r_ref_rate;
    double mig_c;                // (lambda PRF / (2 vh))^2 / (2 gate_width n_gates), 0 if vh = 0
};
size_t dd_focus_smem_bytes(int burst, int n_gates);
cudaError_t launch_dd_focus(const DdArgs& a, int64_t n_bursts, const void* iq, void* focused,
                            float* multilook, cudaStream_t stream);

// Spectral surface update (surface.cu).
struct SurfArgs {
    int L, log2L, cols;          // grid side (power of two), columns per column-pass CTA
    double dk, g;                // wave-number step 2 pi / (L spacing), gravity
    float t_hi, t_lo;            // update time as hi + lo
    float scale_over_L2;         // amplitude scale / L^2
};
// The surface workspace: omega / (2 pi) hi + lo [L^2] float2, the two packed transforms
// [2][L^2] float2, the full twiddle table [L] float2, the wave numbers [L] float.
struct SurfTables {
    float2* omega;
    float2* tmp;
    float2* twf;
    float* kf;
};
SurfTables surf_tables(int L, void* workspace);
size_t surf_rows_smem(int L);
size_t surf_cols_smem(int L, int cols);
cudaError_t launch_surf_prepare(const SurfArgs& a, const SurfTables& t, int n_sms,
                                cudaStream_t stream);
cudaError_t launch_surf_at(const SurfArgs& a, const void* coef, const SurfTables& t,
                           float* z, float* vx, float* vy, float* vz, cudaStream_t stream);

}  // namespace rsim
