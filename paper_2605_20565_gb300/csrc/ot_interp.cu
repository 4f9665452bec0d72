// ot_interp.cu -- single-op kernels: locate, trilinear and delta-kernel interpolation.
// Persistent grid-stride launches (a few blocks per SM).
#include <algorithm>
#include <type_traits>

#include "ot_internal.h"
#include "ot_points.cuh"
#include "ot_queue.cuh"

namespace ot {

namespace {

template <bool LEARNED>
__global__ void __launch_bounds__(256) k_locate(TreeView t, const double* __restrict__ x,
                                                const double* __restrict__ y, const double* __restrict__ z, int64_t n,
                                                int32_t* __restrict__ host, unsigned long long* n_miss) {
    unsigned miss = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t X[3];
        int h = -1;
        if (fixpoint3(x[i], y[i], z[i], X))
            h = search<LEARNED>(t,
                                morton3((uint32_t)(X[0] >> 32), (uint32_t)(X[1] >> 32), (uint32_t)(X[2] >> 32)));
        else
            ++miss;
        host[i] = h;
    }
    if (miss) {
        atomicOr(t.err, (unsigned)OT_DEV_OUTSIDE);
        if (n_miss) atomicAdd(n_miss, (unsigned long long)miss);
    }
}

template <typename T, bool LEARNED, bool MATES>
__global__ void __launch_bounds__(256) k_trilinear(TreeView t, const double* __restrict__ x,
                                                   const double* __restrict__ y, const double* __restrict__ z,
                                                   int64_t n, const int32_t* __restrict__ host_in,
                                                   const T* __restrict__ field, const T* __restrict__ pyr,
                                                   T* __restrict__ u, int32_t* __restrict__ host_out) {
    // warp-aligned iteration: every lane of a warp runs the same trip count (the trilinear
    // routine is warp-cooperative)
    using Q = typename std::conditional<MATES, HostQueue, WarpQueue>::type;
    __shared__ Q s_queue[256 / 32];
    __shared__ RootModel s_root;
    Q& wq = s_queue[threadIdx.x >> 5];
    stage_root<LEARNED>(t, s_root);
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp0 * 32; base < n; base += nwarps * 32) {
        const int64_t i = base + lane;
        const bool inr = i < n;
        T o[3];
        int hin = -1;
        bool active = inr;
        if (inr && host_in) {
            hin = host_in[i];
            if (hin < 0 || hin >= t.n) {
                // no host (outside the cube) or an index that is not a leaf: no value
                if (hin >= t.n) atomicOr(t.err, (unsigned)OT_DEV_OUTSIDE);
                active = false;
            }
        }
        const double xi = inr ? x[i] : 0.0, yi = inr ? y[i] : 0.0, zi = inr ? z[i] : 0.0;
        int h;
        if constexpr (MATES)
            h = trilinear_mates<T, LEARNED>(t, s_root, field, pyr, wq, active, xi, yi, zi, hin, o);
        else
            h = trilinear_queued<T, LEARNED>(t, s_root, field, pyr, wq, active, xi, yi, zi, hin, o);
        if (inr) {
            u[i] = o[0];
            u[n + i] = o[1];
            u[2 * n + i] = o[2];
            if (host_out) host_out[i] = h;
        }
    }
}

template <typename T, int K, bool LEARNED>
__global__ void __launch_bounds__(256) k_delta(TreeView t, const double* __restrict__ x,
                                               const double* __restrict__ y, const double* __restrict__ z, int64_t n,
                                               const T* __restrict__ field, T* __restrict__ u,
                                               int32_t* __restrict__ host_out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        T o[3];
        const int h = delta_point<T, K, LEARNED>(t, field, x[i], y[i], z[i], host_out != nullptr, o);
        u[i] = o[0];
        u[n + i] = o[1];
        u[2 * n + i] = o[2];
        if (host_out) host_out[i] = h;
    }
}

template <typename Kern>
unsigned persistent_grid(Kern k, int block, size_t smem, int64_t n) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem);
    per_sm = std::max(per_sm, 1);
    int64_t need = (n + block - 1) / block;
    int64_t g = std::min<int64_t>((int64_t)num_sms() * per_sm, need);
    return (unsigned)std::max<int64_t>(g, 1);
}

template <typename Kern>
ot_status prep_smem(Kern k, size_t smem) {
    if (smem > 48 * 1024) OT_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return OT_OK;
}

} // namespace

ot_status launch_locate(const ot_octree* t, const double* x, const double* y, const double* z, int64_t n, int search,
                        int32_t* host, unsigned long long* n_miss, cudaStream_t s) {
    if (n == 0) return OT_OK;
    const bool learned = search == OT_LEARNED;
    TreeView v = tree_view(t);
    const size_t smem = 0;
    const int block = 256;
    if (learned) {
        auto k = k_locate<true>;
        ot_status st = prep_smem(k, smem);
        if (st != OT_OK) return st;
        k<<<persistent_grid(k, block, smem, n), block, smem, s>>>(v, x, y, z, n, host, n_miss);
    } else {
        auto k = k_locate<false>;
        ot_status st = prep_smem(k, smem);
        if (st != OT_OK) return st;
        k<<<persistent_grid(k, block, smem, n), block, smem, s>>>(v, x, y, z, n, host, n_miss);
    }
    count_launch();
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

template <typename T>
ot_status launch_interp(const ot_octree* t, int kernel, const double* x, const double* y, const double* z, int64_t n,
                        const int32_t* host_in, int search, const T* field, T* u, int32_t* host_out, void* ws,
                        size_t ws_bytes, cudaStream_t s) {
    if (n == 0) return OT_OK;
    if (kernel == OT_TRILINEAR && (ws_bytes < interp_ws_bytes(t, kernel, sizeof(T)) || !ws || ((uintptr_t)ws & 15)))
        return OT_ERR_ARG;
    const bool learned = search == OT_LEARNED;
    TreeView v = tree_view(t);
    const size_t smem = 0;
    const int block = 256;
    ot_status st = OT_OK;
#define OT_LAUNCH(KERN, ...)                                                               \
    do {                                                                                   \
        auto k_ = KERN;                                                                    \
        if ((st = prep_smem(k_, smem)) != OT_OK) return st;                                \
        k_<<<persistent_grid(k_, block, smem, n), block, smem, s>>>(__VA_ARGS__);          \
    } while (0)
    if (kernel == OT_TRILINEAR) {
        // cell means of the field (refined level-mates), in the caller's workspace
        T* pyr = static_cast<T*>(ws);
        if ((st = launch_pyramid<T>(t, field, pyr, s)) != OT_OK) return st;
        if (t->d_mates && learned)
            OT_LAUNCH((k_trilinear<T, true, true>), v, x, y, z, n, host_in, field, pyr, u, host_out);
        else if (t->d_mates)
            OT_LAUNCH((k_trilinear<T, false, true>), v, x, y, z, n, host_in, field, pyr, u, host_out);
        else if (learned)
            OT_LAUNCH((k_trilinear<T, true, false>), v, x, y, z, n, host_in, field, pyr, u, host_out);
        else
            OT_LAUNCH((k_trilinear<T, false, false>), v, x, y, z, n, host_in, field, pyr, u, host_out);
    } else if (kernel == OT_PESKIN4) {
        if (learned)
            OT_LAUNCH((k_delta<T, OT_PESKIN4, true>), v, x, y, z, n, field, u, host_out);
        else
            OT_LAUNCH((k_delta<T, OT_PESKIN4, false>), v, x, y, z, n, field, u, host_out);
    } else {
        if (learned)
            OT_LAUNCH((k_delta<T, OT_ROMA3, true>), v, x, y, z, n, field, u, host_out);
        else
            OT_LAUNCH((k_delta<T, OT_ROMA3, false>), v, x, y, z, n, field, u, host_out);
    }
#undef OT_LAUNCH
    count_launch();
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

template ot_status launch_interp<float>(const ot_octree*, int, const double*, const double*, const double*, int64_t,
                                        const int32_t*, int, const float*, float*, int32_t*, void*, size_t,
                                        cudaStream_t);
template ot_status launch_interp<double>(const ot_octree*, int, const double*, const double*, const double*, int64_t,
                                         const int32_t*, int, const double*, double*, int32_t*, void*, size_t,
                                         cudaStream_t);

size_t interp_ws_bytes(const ot_octree* t, int kernel, size_t elem) {
    return kernel == OT_TRILINEAR ? pyramid_bytes(t, elem) : 0;
}

} // namespace ot
