// ot_pyramid.cu -- means of the field over refined cells: the value a refined trilinear
// level-mate takes, the volume-weighted mean of the leaves inside it (the coalescence average
// of Sec. 2.1.1), in one load whatever its level.
//   Node means, levels Lc+1 .. lmax-1 (Lc = min(lmax, 7)): one array of N entries per level,
//   indexed by the refined cell's first leaf (the leaf holding its anchor, which the level-mate
//   search finds).  The refined cells of each level are listed once per octree; every
//   recomputation takes each listed cell as the mean of its 8 children, deepest level first, a
//   child being a leaf or a refined cell of the next level whose leaf count (kept in the 4th
//   component, as integer bits) gives the start of the next child.
//   Dense pyramid, levels 0 .. Lc: level Lc holds each cell's mean (the covering leaf's value,
//   or the mean of its 8 children as above); every coarser level the mean of its 8 children.
// Recomputed whenever the field changes (every replay of a batch graph).
#include <algorithm>
#include <vector>

#include "ot_internal.h"

namespace ot {

namespace {

// bit-exact integer count in the 4th component
__device__ __forceinline__ float count_bits(int c, float) { return __int_as_float(c); }
__device__ __forceinline__ double count_bits(int c, double) { return __longlong_as_double((long long)c); }
__device__ __forceinline__ int bits_count(float v) { return __float_as_int(v); }
__device__ __forceinline__ int bits_count(double v) { return (int)__double_as_longlong(v); }

// Mean of the 8 children of the refined cell of level l whose first leaf is a, written to p
// with the cell's leaf count.  child: node means of level l + 1 (null when l + 1 == lmax: every
// child is a leaf).
template <typename T>
__device__ __forceinline__ void children_mean(const uint8_t* __restrict__ level, int l, const T* __restrict__ field,
                                              const T* __restrict__ child, int a, T* __restrict__ p) {
    using V = Vec4<T>;
    int pos = a;
    T s0 = T(0), s1 = T(0), s2 = T(0);
    for (int ch = 0; ch < 8; ++ch) {
        typename V::type f;
        int step = 1;
        if ((int)level[pos] == l + 1) {
            f = V::load(field, pos);
        } else {
            f = V::load(child, pos);
            step = bits_count(f.w);
        }
        s0 += f.x;
        s1 += f.y;
        s2 += f.z;
        pos += step;
    }
    p[0] = s0 * T(0.125), p[1] = s1 * T(0.125), p[2] = s2 * T(0.125), p[3] = count_bits(pos - a, T(0));
}

// Level Lc of the pyramid: cell c holds leaves [pmap[c], pmap[c+1]); one leaf covers it when
// that range has at most one leaf.
template <typename T>
__device__ __forceinline__ void base_mean(const uint32_t* __restrict__ pmap, const uint8_t* __restrict__ level, int n,
                                          int Lc, const T* __restrict__ field, const T* __restrict__ child, int64_t c,
                                          T* __restrict__ out) {
    using V = Vec4<T>;
    const int64_t ncell = (int64_t)1 << (3 * Lc);
    const int a = (int)pmap[c];
    const int e = c + 1 < ncell ? (int)pmap[c + 1] : n;
    T* p = out + 4 * c;
    if (e - a <= 1) {
        const auto f = V::load(field, a);
        p[0] = f.x, p[1] = f.y, p[2] = f.z, p[3] = T(0);
    } else {
        children_mean<T>(level, Lc, field, child, a, p);
    }
}

// need (nullable): only the cells flagged there
template <typename T>
__global__ void __launch_bounds__(256) k_pyr_base(const uint32_t* __restrict__ pmap, const uint8_t* __restrict__ level,
                                                  int n, int Lc, const T* __restrict__ field,
                                                  const T* __restrict__ child, T* __restrict__ out,
                                                  const uint8_t* __restrict__ need) {
    const int64_t ncell = (int64_t)1 << (3 * Lc);
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x)
        if (!need || need[c]) base_mean<T>(pmap, level, n, Lc, field, child, c, out);
}

// Refined cells of level l listed in nodes[0, cnt): their means, at index first leaf (need,
// nullable: only the cells flagged there, by first leaf).
template <typename T>
__global__ void __launch_bounds__(256) k_node_means(const int* __restrict__ nodes, int64_t cnt,
                                                    const uint8_t* __restrict__ level, int l,
                                                    const T* __restrict__ field, const T* __restrict__ child,
                                                    T* __restrict__ out, const uint8_t* __restrict__ need) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        const int a = nodes[i];
        if (!need || need[a]) children_mean<T>(level, l, field, child, a, out + 4 * (int64_t)a);
    }
}

template <typename T>
__device__ __forceinline__ void up_mean(const T* __restrict__ fine, T* __restrict__ coarse, int64_t c) {
    using V = Vec4<T>;
    T s0 = T(0), s1 = T(0), s2 = T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const auto f = V::load(fine, 8 * c + k);
        s0 += f.x;
        s1 += f.y;
        s2 += f.z;
    }
    T* p = coarse + 4 * c;
    p[0] = s0 * T(0.125), p[1] = s1 * T(0.125), p[2] = s2 * T(0.125), p[3] = T(0);
}

template <typename T>
__global__ void __launch_bounds__(256) k_pyr_up(const T* __restrict__ fine, T* __restrict__ coarse, int64_t ncell,
                                                const uint8_t* __restrict__ need) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x)
        if (!need || need[c]) up_mean<T>(fine, coarse, c);
}

// ---- the cell means the level-mate table reads, closed under "a mean needs its children's" ----

// needed dense cell c of level l -> its 8 children of level l + 1
__global__ void k_close_dense(const uint8_t* __restrict__ need, int64_t ncell, uint8_t* __restrict__ child_need) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x)
        if (need[c])
#pragma unroll
            for (int k = 0; k < 8; ++k) child_need[8 * c + k] = 1;
}

// The refined children of a refined cell of level l whose first leaf is a (anchor key[a]): each
// child's first leaf is the leaf holding its anchor, searched within the cell's leaves from a.
__device__ __forceinline__ void mark_refined_children(const uint64_t* __restrict__ key,
                                                      const uint8_t* __restrict__ level, int n, int l, int a,
                                                      int e, uint8_t* __restrict__ child_need) {
    const uint64_t anchor = key[a] & ~(key_span(l) - 1);
    for (int k = 0; k < 8; ++k) {
        const uint64_t ca = anchor + (uint64_t)k * key_span(l + 1);
        const int f = search_range(key, a, e - a, ca);
        if ((int)level[f] > l + 1) child_need[f] = 1;
    }
}

// needed base cells (level Lc) that are refined -> their refined children (node level 0)
__global__ void k_close_base(const uint8_t* __restrict__ need, const uint32_t* __restrict__ pmap,
                             const uint64_t* __restrict__ key, const uint8_t* __restrict__ level, int n, int Lc,
                             uint8_t* __restrict__ child_need) {
    const int64_t ncell = (int64_t)1 << (3 * Lc);
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        if (!need[c]) continue;
        const int a = (int)pmap[c];
        const int e = c + 1 < ncell ? (int)pmap[c + 1] : n;
        if (e - a > 1) mark_refined_children(key, level, n, Lc, a, e, child_need);
    }
}

// needed refined cells of level l (by first leaf) -> their refined children (level l + 1)
__global__ void k_close_node(const uint8_t* __restrict__ need, const uint64_t* __restrict__ key,
                             const uint8_t* __restrict__ level, int n, int l, uint8_t* __restrict__ child_need) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n; a += (int64_t)gridDim.x * blockDim.x) {
        if (!need[a]) continue;
        // the cell's leaves end where the next cell of level l begins (at most 8^(lmax - l) leaves;
        // the search range is capped at the leaf count)
        const uint64_t next = (key[a] & ~(key_span(l) - 1)) + key_span(l);
        const int e = next == 0 ? n : search_range(key, (int)a, n - (int)a, next - 1) + 1;
        mark_refined_children(key, level, n, l, (int)a, e, child_need);
    }
}

// The leaves that start a refined cell of level l: level > l and key aligned to level l.
__global__ void k_flag_nodes(const uint64_t* __restrict__ key, const uint8_t* __restrict__ level, int n, int l,
                             uint32_t* __restrict__ flag) {
    const uint64_t mask = key_span(l) - 1;
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n; a += (int64_t)gridDim.x * blockDim.x)
        flag[a] = ((int)level[a] > l && (key[a] & mask) == 0) ? 1u : 0u;
}

__global__ void k_scatter_nodes(const uint32_t* __restrict__ flag, const uint32_t* __restrict__ pos, int n,
                                int* __restrict__ out) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n; a += (int64_t)gridDim.x * blockDim.x)
        if (flag[a]) out[pos[a]] = (int)a;
}

unsigned grid_n(int64_t n, int b) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + b - 1) / b, (int64_t)num_sms() * 16));
}

} // namespace

int64_t pyramid_offset(int l) { return ((int64_t)1 << (3 * l)) / 7; }  // sum_{k<l} 8^k = (8^l - 1)/7

int node_levels(const ot_octree* t) { return std::max(0, t->lmax - 1 - t->pyr_level); }

size_t pyramid_bytes(const ot_octree* t, size_t elem) {
    return elem * 4 * ((size_t)pyramid_offset(t->pyr_level + 1) + (size_t)node_levels(t) * (size_t)t->n) + 256;
}

// Lists, once per octree, the refined cells of every node level (by first leaf, in key order).
ot_status build_node_lists(ot_octree* t, cudaStream_t s) {
    const int nl = node_levels(t);
    if (t->d_nodes) cudaFree(t->d_nodes);
    t->d_nodes = nullptr;
    if (nl == 0 || t->n == 0) return OT_OK;
    uint32_t *flag = nullptr, *pos = nullptr, *tot = nullptr;
    OT_CUDA(cudaMallocAsync(&flag, sizeof(uint32_t) * t->n, s));
    OT_CUDA(cudaMallocAsync(&pos, sizeof(uint32_t) * t->n, s));
    OT_CUDA(cudaMallocAsync(&tot, sizeof(uint32_t), s));
    std::vector<int64_t> cnt(nl);
    for (int k = 0; k < nl; ++k) {  // counts first, then one allocation
        k_flag_nodes<<<grid_n(t->n, 256), 256, 0, s>>>(t->d_key, t->d_level, (int)t->n, t->pyr_level + 1 + k, flag);
        count_launch();
        ot_status st = scan_u32(flag, pos, t->n, tot, s);
        if (st != OT_OK) return st;
        uint32_t h = 0;
        OT_CUDA(cudaMemcpyAsync(&h, tot, sizeof(h), cudaMemcpyDeviceToHost, s));
        OT_CUDA(cudaStreamSynchronize(s));
        cnt[k] = h;
    }
    int64_t total = 0;
    for (int k = 0; k < nl; ++k) {
        t->node_off[k] = total;
        t->node_cnt[k] = cnt[k];
        total += cnt[k];
    }
    OT_CUDA(cudaMalloc(&t->d_nodes, sizeof(int) * std::max<int64_t>(total, 1)));
    for (int k = 0; k < nl; ++k) {
        k_flag_nodes<<<grid_n(t->n, 256), 256, 0, s>>>(t->d_key, t->d_level, (int)t->n, t->pyr_level + 1 + k, flag);
        ot_status st = scan_u32(flag, pos, t->n, nullptr, s);
        if (st != OT_OK) return st;
        k_scatter_nodes<<<grid_n(t->n, 256), 256, 0, s>>>(flag, pos, (int)t->n, t->d_nodes + t->node_off[k]);
        count_launch(2);
    }
    cudaFreeAsync(flag, s);
    cudaFreeAsync(pos, s);
    cudaFreeAsync(tot, s);
    OT_CUDA(cudaGetLastError());
    OT_CUDA(cudaStreamSynchronize(s));
    return OT_OK;
}

size_t need_flag_bytes(const ot_octree* t) {
    return (size_t)pyramid_offset(t->pyr_level + 1) + (size_t)node_levels(t) * (size_t)t->n;
}

// Closes the flags of the means the level-mate table reads (need: one byte per entry of the
// means array, dense pyramid then node levels, set by the table builder) under "a mean needs
// its children's"; the octree keeps them, and every later pyramid computes the flagged means
// only.
ot_status close_need_flags(ot_octree* t, uint8_t* need, cudaStream_t s) {
    const int Lc = t->pyr_level;
    const int nl = node_levels(t);
    const int n = (int)t->n;
    for (int l = 0; l < Lc; ++l) {
        const int64_t nc = (int64_t)1 << (3 * l);
        k_close_dense<<<grid_n(nc, 256), 256, 0, s>>>(need + pyramid_offset(l), nc, need + pyramid_offset(l + 1));
        count_launch();
    }
    uint8_t* node_need = need + pyramid_offset(Lc + 1);
    if (nl > 0) {
        const int64_t nc = (int64_t)1 << (3 * Lc);
        k_close_base<<<grid_n(nc, 256), 256, 0, s>>>(need + pyramid_offset(Lc), t->d_pmap, t->d_key, t->d_level, n, Lc,
                                                     node_need);
        count_launch();
    }
    for (int k = 0; k + 1 < nl; ++k) {
        k_close_node<<<grid_n(n, 256), 256, 0, s>>>(node_need + (int64_t)k * n, t->d_key, t->d_level, n, Lc + 1 + k,
                                                     node_need + (int64_t)(k + 1) * n);
        count_launch();
    }
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

template <typename T>
ot_status launch_pyramid(const ot_octree* t, const T* field, T* pyr, cudaStream_t s) {
    const int Lc = t->pyr_level;
    const int nl = node_levels(t);
    T* nodes = pyr + 4 * pyramid_offset(Lc + 1);
    // with the level-mate table, only the means it reads and the ones they are made of
    const uint8_t* need = t->d_need_flags;
    // node means, deepest level first (each reads the next level's)
    for (int k = nl - 1; k >= 0; --k) {
        T* out = nodes + 4 * (int64_t)k * t->n;
        const T* child = k + 1 < nl ? out + 4 * (int64_t)t->n : nullptr;
        if (t->node_cnt[k] > 0) {
            const uint8_t* nk = need ? need + pyramid_offset(Lc + 1) + (int64_t)k * t->n : nullptr;
            k_node_means<T><<<grid_n(t->node_cnt[k], 256), 256, 0, s>>>(t->d_nodes + t->node_off[k], t->node_cnt[k],
                                                                       t->d_level, Lc + 1 + k, field, child, out, nk);
            count_launch();
        }
    }
    const int64_t ncell = (int64_t)1 << (3 * Lc);
    k_pyr_base<T><<<grid_n(ncell, 256), 256, 0, s>>>(t->d_pmap, t->d_level, (int)t->n, Lc, field,
                                                    nl > 0 ? nodes : nullptr, pyr + 4 * pyramid_offset(Lc),
                                                    need ? need + pyramid_offset(Lc) : nullptr);
    count_launch();
    for (int l = Lc - 1; l >= 0; --l) {
        const int64_t nc = (int64_t)1 << (3 * l);
        k_pyr_up<T><<<grid_n(nc, 256), 256, 0, s>>>(pyr + 4 * pyramid_offset(l + 1), pyr + 4 * pyramid_offset(l), nc,
                                                    need ? need + pyramid_offset(l) : nullptr);
        count_launch();
    }
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

template ot_status launch_pyramid<float>(const ot_octree*, const float*, float*, cudaStream_t);
template ot_status launch_pyramid<double>(const ot_octree*, const double*, double*, cudaStream_t);

} // namespace ot
