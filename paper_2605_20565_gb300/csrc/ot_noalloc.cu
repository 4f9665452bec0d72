// ot_noalloc.cu -- sorted (deterministic) force spreading for callers that cannot allocate
// device memory.
//
// Some callers of this library are not allowed to call cudaMalloc: a solver that has handed
// the whole device memory to its own pool up front, code that runs in a context where an
// allocation (which may synchronise the device or fail under memory pressure) is not
// acceptable, or a host program that only passes buffers it already owns.  For them the
// scratch that the sorted spreading needs (the (leaf, marker, slot) pairs, their sort
// buffer and the radix-sort histograms) lives in one file-scope device array of a fixed size,
// OT_NOALLOC_SCRATCH_BYTES.  Every GPU that loads this library holds that array until the
// process exits.
#include <cuda.h>  // driver types only: the two driver calls below are reached through the runtime

#include <mutex>

#include "ot_internal.h"

namespace {

// The scratch.  In host code this name is only a stand-in for the symbol, never a device
// address: the address comes from cudaGetSymbolAddress, once per device and context.
static __device__ __align__(256) unsigned char g_spread_scratch[OT_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

// Identity of the current CUDA context (0 when the driver does not say).  A context that was
// destroyed and created again -- cudaDeviceReset, for instance -- has a new identity, and the
// library's device array may then sit at a new address, so the address is looked up again.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
    });
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS)
        return id;
    return 0;
}

// Device address of the scratch on the current device: looked up with cudaGetSymbolAddress on
// the first call made with that device current (the set-up; it must not run inside a stream
// capture), and again whenever the device's context is not the one the address came from.
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    // a call without a context yet: the lookup below creates the primary context, after which
    // the identity is read again
    unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev] || g_scratch_ctx[dev] != ctx) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_spread_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
        g_scratch_ctx[dev] = current_context_id();
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

} // namespace

extern "C" ot_status ot_spread_noalloc(const ot_octree* t, int kernel, const double* d_x, const double* d_y,
                                       const double* d_z, const float* d_F, const float* d_dV, int64_t n,
                                       float* d_f, void* stream) {
    if (!t || n < 0 || (kernel != OT_PESKIN4 && kernel != OT_ROMA3)) return OT_ERR_ARG;
    if (n > 0 && (!d_x || !d_y || !d_z || !d_F || !d_f)) return OT_ERR_ARG;
    if (t->lmax < 1) return OT_ERR_ARG;
    if (n == 0) return OT_OK;
    if (n * 64 >= (1LL << 32)) return OT_ERR_LIMIT;
    if (ot::spread_noalloc_bytes(kernel, n) > (size_t)OT_NOALLOC_SCRATCH_BYTES) return OT_ERR_LIMIT;
    void* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return ot::cuda_status(e);
    // Nothing in the scratch needs to start at zero: every pair slot, histogram and scan
    // entry is written before it is read in this call.
    return ot::launch_spread_sorted_noalloc(t, kernel, d_x, d_y, d_z, d_F, d_dV, n, d_f, scratch,
                                            (cudaStream_t)stream);
}
