// ot_spread.cu -- force spreading, the adjoint of the delta-kernel interpolation (Sec. 2.2):
//   f(cell) += sum_k F_k phi(rx) phi(ry) phi(rz) dV_k / h^3.
// OT_ATOMIC: each marker adds its stencil contributions with float atomics.
// OT_SORTED: each marker emits one 64-bit pair per stencil slot, (leaf << 32) | (k W^3 + slot);
//   a stable radix sort by leaf groups the pairs of a leaf in marker order; one thread per
//   leaf then recomputes the weights and sums in that order and adds once to f (no atomics,
//   bit-identical from run to run and for any launch shape).
#include <algorithm>

#include "ot_internal.h"
#include "ot_points.cuh"

namespace ot {

namespace {

constexpr uint64_t INVALID_HI = 0xFFFFFFFFull;

template <typename T> __device__ __forceinline__ void add3(T* f, int leaf, T a, T b, T c);
template <> __device__ __forceinline__ void add3<float>(float* f, int leaf, float a, float b, float c) {
    atomicAdd(reinterpret_cast<float4*>(f) + leaf, make_float4(a, b, c, 0.0f));
}
template <> __device__ __forceinline__ void add3<double>(double* f, int leaf, double a, double b, double c) {
    double* p = f + 4 * (size_t)leaf;
    atomicAdd(p, a);
    atomicAdd(p + 1, b);
    atomicAdd(p + 2, c);
}

template <typename T>
__device__ __forceinline__ T marker_volume(const T* __restrict__ dV, int64_t k, int lmax) {
    return dV ? dV[k] * (T)ldexp(1.0, 3 * lmax) : T(1);
}

template <typename T, int K>
__global__ void __launch_bounds__(256) k_spread_atomic(TreeView t, RootModel rm, const double* __restrict__ x,
                                                       const double* __restrict__ y, const double* __restrict__ z,
                                                       const T* __restrict__ F, const T* __restrict__ dV, int64_t n,
                                                       T* __restrict__ f) {
    extern __shared__ uint64_t s_sample[];
    const bool staged = t.nsample > 1;
    if (staged) load_sample(t, s_sample);
    const uint64_t* ss = staged ? s_sample : nullptr;
    constexpr int W = Stencil<K>::W;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        uint64_t X[3];
        if (!fixpoint3(x[k], y[k], z[k], X)) {
            atomicOr(t.err, (unsigned)OT_DEV_OUTSIDE);
            continue;
        }
        int i0[3];
        T w[3][W];
        stencil_weights<K, T>(t.lmax, X, i0, w);
        const T vol = marker_volume(dV, k, t.lmax);
        const T F0 = F[k] * vol, F1 = F[n + k] * vol, F2 = F[2 * n + k] * vol;
        const bool ok = visit_stencil<K, false>(t, rm, ss, i0, [&](int leaf, int ax, int ay, int az) {
            const T wt = w[0][ax] * w[1][ay] * w[2][az];
            add3<T>(f, leaf, F0 * wt, F1 * wt, F2 * wt);
        });
        if (!ok) atomicOr(t.err, (unsigned)OT_DEV_STENCIL);
    }
}

template <int K>
__global__ void __launch_bounds__(256) k_spread_emit(TreeView t, RootModel rm, const double* __restrict__ x,
                                                     const double* __restrict__ y, const double* __restrict__ z,
                                                     int64_t n, uint64_t* __restrict__ pairs) {
    extern __shared__ uint64_t s_sample[];
    const bool staged = t.nsample > 1;
    if (staged) load_sample(t, s_sample);
    const uint64_t* ss = staged ? s_sample : nullptr;
    constexpr int W = Stencil<K>::W, W3 = W * W * W;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        uint64_t* out = pairs + k * W3;
        const uint64_t id0 = (uint64_t)k * W3;
        for (int sl = 0; sl < W3; ++sl) out[sl] = (INVALID_HI << 32) | (id0 + sl);
        uint64_t X[3];
        if (!fixpoint3(x[k], y[k], z[k], X)) {
            atomicOr(t.err, (unsigned)OT_DEV_OUTSIDE);
            continue;
        }
        int i0[3];
        for (int d = 0; d < 3; ++d)
            i0[d] = Stencil<K>::first((int)fix_cell(X[d], t.lmax), fix_upper_half(X[d], t.lmax) ? 1 : 0);
        const bool ok = visit_stencil<K, false>(t, rm, ss, i0, [&](int leaf, int ax, int ay, int az) {
            const int sl = ax + W * (ay + W * az);
            out[sl] = ((uint64_t)(uint32_t)leaf << 32) | (id0 + sl);
        });
        if (!ok) atomicOr(t.err, (unsigned)OT_DEV_STENCIL);
    }
}

// One thread per sorted pair; the first pair of each leaf walks its run in order.
template <typename T, int K>
__global__ void __launch_bounds__(256) k_spread_reduce(const uint64_t* __restrict__ pairs, int64_t npairs, int lmax,
                                                       const double* __restrict__ x, const double* __restrict__ y,
                                                       const double* __restrict__ z, const T* __restrict__ F,
                                                       const T* __restrict__ dV, int64_t n, T* __restrict__ f) {
    constexpr int W = Stencil<K>::W, W3 = W * W * W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npairs;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t pv = pairs[i];
        const uint32_t leaf = (uint32_t)(pv >> 32);
        if (leaf == (uint32_t)INVALID_HI) continue;
        if (i > 0 && (uint32_t)(pairs[i - 1] >> 32) == leaf) continue;
        T a0 = T(0), a1 = T(0), a2 = T(0);
        for (int64_t j = i; j < npairs; ++j) {
            const uint64_t pj = pairs[j];
            if ((uint32_t)(pj >> 32) != leaf) break;
            const uint32_t id = (uint32_t)pj;
            const int64_t k = id / W3;
            const int sl = (int)(id - (uint32_t)(k * W3));
            const int slot[3] = {sl % W, (sl / W) % W, sl / (W * W)};
            uint64_t X[3];
            fixpoint3(x[k], y[k], z[k], X);  // inside: the pair was emitted
            T wt = T(1);
#pragma unroll
            for (int d = 0; d < 3; ++d) wt *= stencil_weight_1d<K, T>(lmax, X[d], slot[d]);
            const T vol = marker_volume(dV, k, lmax);
            a0 += F[k] * vol * wt;
            a1 += F[n + k] * vol * wt;
            a2 += F[2 * n + k] * vol * wt;
        }
        T* fp = f + 4 * (size_t)leaf;
        fp[0] += a0;
        fp[1] += a1;
        fp[2] += a2;
    }
}

template <typename Kern>
unsigned grid_for(Kern k, int block, size_t smem, int64_t n) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem);
    per_sm = std::max(per_sm, 1);
    int64_t need = (n + block - 1) / block;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms() * per_sm, need));
}

template <typename Kern>
ot_status prep(Kern k, size_t smem) {
    if (smem > 48 * 1024) OT_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return OT_OK;
}

int leaf_bits(int64_t n) {
    int b = 1;
    while (b < 32 && ((int64_t)1 << b) <= n) ++b; // n <= 2^b - 1: the all-ones key stays above every leaf
    return b;
}

inline int stencil_cells(int kernel) { return kernel == OT_PESKIN4 ? 64 : 27; }

template <typename T, int K>
ot_status spread_sorted(const ot_octree* t, const double* x, const double* y, const double* z, const T* F,
                        const T* dV, int64_t n, T* f, void* ws, cudaStream_t s) {
    constexpr int W3 = Stencil<K>::W * Stencil<K>::W * Stencil<K>::W;
    const int64_t np = n * W3;
    uint64_t* pairs = static_cast<uint64_t*>(ws);
    uint64_t* tmp = pairs + np;
    void* rws = tmp + np;
    TreeView v = tree_view(t, true);
    const size_t smem = (size_t)v.nsample * sizeof(uint64_t);
    ot_status st;
    auto ke = k_spread_emit<K>;
    if ((st = prep(ke, smem)) != OT_OK) return st;
    ke<<<grid_for(ke, 256, smem, n), 256, smem, s>>>(v, t->root, x, y, z, n, pairs);
    count_launch();
    OT_CUDA(cudaGetLastError());
    const int bits = leaf_bits(t->n);
    if ((st = radix_sort_u64_ws(pairs, tmp, np, 32, 32 + bits, rws, s)) != OT_OK) return st;
    auto kr = k_spread_reduce<T, K>;
    kr<<<grid_for(kr, 256, 0, np), 256, 0, s>>>(pairs, np, t->lmax, x, y, z, F, dV, n, f);
    count_launch();
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

} // namespace

size_t spread_ws_bytes(const ot_octree* t, int kernel, int64_t n) {
    (void)t;
    const int64_t np = n * stencil_cells(kernel);
    return (size_t)np * 16 + radix_ws_bytes(np) + 256;
}

template <typename T>
ot_status launch_spread(const ot_octree* t, int kernel, int mode, const double* x, const double* y, const double* z,
                        const T* F, const T* dV, int64_t n, T* f, void* ws, size_t ws_bytes, cudaStream_t s) {
    if (n == 0) return OT_OK;
    if (mode == OT_SORTED) {
        if (ws_bytes < spread_ws_bytes(t, kernel, n)) return OT_ERR_ARG;
        if (kernel == OT_PESKIN4) return spread_sorted<T, OT_PESKIN4>(t, x, y, z, F, dV, n, f, ws, s);
        return spread_sorted<T, OT_ROMA3>(t, x, y, z, F, dV, n, f, ws, s);
    }
    TreeView v = tree_view(t, true);
    const size_t smem = (size_t)v.nsample * sizeof(uint64_t);
    ot_status st;
    if (kernel == OT_PESKIN4) {
        auto k = k_spread_atomic<T, OT_PESKIN4>;
        if ((st = prep(k, smem)) != OT_OK) return st;
        k<<<grid_for(k, 256, smem, n), 256, smem, s>>>(v, t->root, x, y, z, F, dV, n, f);
    } else {
        auto k = k_spread_atomic<T, OT_ROMA3>;
        if ((st = prep(k, smem)) != OT_OK) return st;
        k<<<grid_for(k, 256, smem, n), 256, smem, s>>>(v, t->root, x, y, z, F, dV, n, f);
    }
    count_launch();
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

template ot_status launch_spread<float>(const ot_octree*, int, int, const double*, const double*, const double*,
                                        const float*, const float*, int64_t, float*, void*, size_t, cudaStream_t);
template ot_status launch_spread<double>(const ot_octree*, int, int, const double*, const double*, const double*,
                                         const double*, const double*, int64_t, double*, void*, size_t, cudaStream_t);

} // namespace ot

// ------------------------------------------------------------------------------------------
// Sorted spreading with caller scratch only (no allocation of any kind).
// ------------------------------------------------------------------------------------------
namespace ot {

size_t spread_noalloc_bytes(int kernel, int64_t n) {
    const int64_t np = n * stencil_cells(kernel);
    return (size_t)np * 16 + radix_noalloc_bytes(np) + 256;
}

namespace {
template <int K>
ot_status sorted_noalloc(const ot_octree* t, const double* x, const double* y, const double* z, const float* F,
                         const float* dV, int64_t n, float* f, void* scratch, cudaStream_t s) {
    constexpr int W3 = Stencil<K>::W * Stencil<K>::W * Stencil<K>::W;
    const int64_t np = n * W3;
    uint64_t* pairs = static_cast<uint64_t*>(scratch);
    uint64_t* tmp = pairs + np;
    void* rws = tmp + np;
    TreeView v = tree_view(t, true);
    const size_t smem = (size_t)v.nsample * sizeof(uint64_t);
    ot_status st;
    auto ke = k_spread_emit<K>;
    if ((st = prep(ke, smem)) != OT_OK) return st;
    ke<<<grid_for(ke, 256, smem, n), 256, smem, s>>>(v, t->root, x, y, z, n, pairs);
    count_launch();
    OT_CUDA(cudaGetLastError());
    if ((st = radix_sort_u64_noalloc(pairs, tmp, np, 32, 32 + leaf_bits(t->n), rws, s)) != OT_OK) return st;
    auto kr = k_spread_reduce<float, K>;
    kr<<<grid_for(kr, 256, 0, np), 256, 0, s>>>(pairs, np, t->lmax, x, y, z, F, dV, n, f);
    count_launch();
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}
} // namespace

ot_status launch_spread_sorted_noalloc(const ot_octree* t, int kernel, const double* x, const double* y,
                                       const double* z, const float* F, const float* dV, int64_t n, float* f,
                                       void* scratch, cudaStream_t s) {
    if (n == 0) return OT_OK;
    if (kernel == OT_PESKIN4) return sorted_noalloc<OT_PESKIN4>(t, x, y, z, F, dV, n, f, scratch, s);
    return sorted_noalloc<OT_ROMA3>(t, x, y, z, F, dV, n, f, scratch, s);
}

} // namespace ot
