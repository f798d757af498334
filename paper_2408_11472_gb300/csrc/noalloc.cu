// noalloc.cu -- rsim_doppler_accumulate_noalloc: the fast-mode spectrum pass for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point where they
// run the summation: code inside a real-time or safety-certified loop that forbids
// allocation after start-up, plug-ins living in a host process whose allocator they do
// not own, or hosts that pre-partition device memory among tenants.  This entry point
// needs no workspace from them: its fixed-point scratch lives in a file-scope device
// array that the library image carries, so it is mapped when the library's module is
// loaded and held by every GPU that loads the library until the process exits.
//
// The array holds kNoAllocScratchBytes (16 MiB): rsim_workspace_size(n_updates, n_gates,
// n_doppler) must fit, which covers e.g. 65 updates of 128 gates x 64 bins (8.5 MB).
// Larger requests are rejected with RSIM_ERR_WORKSPACE.  All calls share the one array
// (per device): the pass clears it at the start of each call, but calls that may overlap
// on the GPU (different streams, or host threads without ordering) race on it.
#include <mutex>
#include <string>

#include "rsim.h"
#include "rsim_kernels.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocScratchBytes / 8];

std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device.  In host code the array's
// name is only a host-side stand-in, so the address is looked up once per device (with
// that device current) through cudaGetSymbolAddress and cached.
rsim_status scratch_for_current_device(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        rsim::set_last_error("cudaGetDevice failed: %s", cudaGetErrorString(e));
        return RSIM_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        rsim::set_last_error("device index %d beyond the %d devices the library tracks", dev, kMaxDevices);
        return RSIM_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            rsim::set_last_error("cudaGetSymbolAddress of the built-in scratch failed: %s",
                                 cudaGetErrorString(e));
            return RSIM_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return RSIM_OK;
}

}  // namespace

extern "C" rsim_status rsim_doppler_accumulate_noalloc(
    const rsim_radar* radar, const rsim_platform* platform, const rsim_scatterers* scat,
    int64_t update0, int32_t n_updates, int32_t n_fast, int32_t n_doppler,
    rsim_precision precision, void* spectra, cudaStream_t stream) {
    if (!radar) {
        rsim::set_last_error("radar is NULL");
        return RSIM_ERR_INVALID_ARG;
    }
    const size_t need = rsim_workspace_size(n_updates, radar->n_gates, n_doppler);
    if (n_updates > 0 && need == 0) {
        rsim::set_last_error("invalid sizes: n_updates=%d n_gates=%d n_doppler=%d", n_updates,
                             radar->n_gates, n_doppler);
        return RSIM_ERR_INVALID_ARG;
    }
    if (need > kNoAllocScratchBytes) {
        rsim::set_last_error(
            "rsim_doppler_accumulate_noalloc: %d updates of %d gates x %d bins need %zu bytes of "
            "scratch, more than the %zu-byte built-in array; use rsim_doppler_accumulate with a "
            "caller workspace or fewer updates per call",
            n_updates, radar->n_gates, n_doppler, need, kNoAllocScratchBytes);
        return RSIM_ERR_WORKSPACE;
    }
    void* scratch = nullptr;
    const rsim_status st = scratch_for_current_device(&scratch);
    if (st != RSIM_OK) return st;
    return rsim_doppler_accumulate(radar, platform, scat, update0, n_updates, n_fast, n_doppler,
                                   precision, spectra, scratch, kNoAllocScratchBytes, stream);
}
