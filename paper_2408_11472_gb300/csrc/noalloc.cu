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
// (per context on a device): the pass clears it at the start of each call, but calls that
// may overlap on the GPU (different streams, or host threads without ordering) race on it.
// The first call in each CUDA context looks the array's address up (cudaGetSymbolAddress)
// and keeps it for that context.
#include <mutex>
#include <string>

#include <cuda.h>

#include "rsim.h"
#include "rsim_kernels.h"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
constexpr int kCacheSlots = 64;

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocScratchBytes / 8];

// A __device__ symbol's address belongs to a CUDA context, not to a device: a process may run
// a non-primary context on a device (a host that made its own with the driver API), or make a
// new one after cudaDeviceReset.  The looked-up address is therefore cached per context, keyed
// on the context's unique ID (cuCtxGetId: IDs are never reused within a process).  The two
// driver entry points are resolved through the runtime, so the library needs no link against
// the driver library.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

struct ScratchSlot {
    unsigned long long ctx_id;
    void* ptr;
};

std::mutex g_scratch_mu;
ScratchSlot g_slots[kCacheSlots] = {};
int g_next_slot = 0;
CtxGetCurrentFn g_get_current = nullptr;
CtxGetIdFn g_get_id = nullptr;

rsim_status resolve_driver_calls() {
    if (g_get_current && g_get_id) return RSIM_OK;
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    const cudaError_t e1 = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000,
                                                            cudaEnableDefault, &q1);
    const cudaError_t e2 = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000,
                                                            cudaEnableDefault, &q2);
    if (e1 != cudaSuccess || e2 != cudaSuccess || q1 != cudaDriverEntryPointSuccess ||
        q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
        rsim::set_last_error("could not resolve cuCtxGetCurrent / cuCtxGetId: %s",
                             cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
        return RSIM_ERR_CUDA;
    }
    g_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    g_get_id = reinterpret_cast<CtxGetIdFn>(f2);
    return RSIM_OK;
}

// ID of the calling thread's current context; 0 when none is current yet.
rsim_status current_context_id(unsigned long long* id) {
    *id = 0;
    CUcontext ctx = nullptr;
    if (g_get_current(&ctx) != CUDA_SUCCESS) {
        rsim::set_last_error("cuCtxGetCurrent failed");
        return RSIM_ERR_CUDA;
    }
    if (ctx && g_get_id(ctx, id) != CUDA_SUCCESS) {
        rsim::set_last_error("cuCtxGetId failed");
        return RSIM_ERR_CUDA;
    }
    return RSIM_OK;
}

// Device address of the scratch array in the calling thread's current context.  In host
// code the array's name is only a host-side stand-in, so the address is looked up through
// cudaGetSymbolAddress the first time a context calls (this also makes the runtime's
// primary context current when no context is) and cached under the context's ID.
rsim_status scratch_for_current_context(void** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    rsim_status st = resolve_driver_calls();
    if (st != RSIM_OK) return st;
    unsigned long long id = 0;
    st = current_context_id(&id);
    if (st != RSIM_OK) return st;
    if (id != 0) {
        for (const ScratchSlot& s : g_slots) {
            if (s.ctx_id == id) {
                *out = s.ptr;
                return RSIM_OK;
            }
        }
    }
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        rsim::set_last_error("cudaGetSymbolAddress of the built-in scratch failed: %s",
                             cudaGetErrorString(e));
        return RSIM_ERR_CUDA;
    }
    if (id == 0) {  // no context was current before the look-up: the runtime's now is
        st = current_context_id(&id);
        if (st != RSIM_OK) return st;
    }
    if (id != 0) {
        g_slots[g_next_slot] = ScratchSlot{id, p};
        g_next_slot = (g_next_slot + 1) % kCacheSlots;
    }
    *out = p;
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
    const rsim_status st = scratch_for_current_context(&scratch);
    if (st != RSIM_OK) return st;
    return rsim_doppler_accumulate(radar, platform, scat, update0, n_updates, n_fast, n_doppler,
                                   precision, spectra, scratch, kNoAllocScratchBytes, nullptr,
                                   stream);
}
