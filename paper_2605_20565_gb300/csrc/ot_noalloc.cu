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
#include <mutex>

#include "ot_internal.h"

namespace {

// The scratch.  In host code this name is only a stand-in for the symbol, never a device
// address: the address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_spread_scratch[OT_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up on the first call made with
// that device current.
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_spread_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
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
