// ot_pyramid.cu -- pyramid of cell means of the field over the top levels of the tree (0 .. the
// pyramid level Lc = min(lmax, 7)): the value a refined trilinear level-mate of level l <= Lc takes, the
// volume-weighted mean of the leaves inside it (the coalescence average of Sec. 2.1.1), in one
// load.  Level Lc: each map cell's mean (the covering leaf's value, or the volume-weighted mean
// of its leaves, one warp per cell, fixed-order reduction); every coarser level: the mean of the
// 8 children.  Recomputed whenever the field changes (every replay of a batch graph).
#include <algorithm>

#include "ot_internal.h"

namespace ot {

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_pyr_base(const uint64_t* __restrict__ key, const uint8_t* __restrict__ level,
                                                  int n, const uint32_t* __restrict__ lmap, int Lc,
                                                  const T* __restrict__ field, T* __restrict__ out) {
    using V = Vec4<T>;
    const int lane = threadIdx.x & 31;
    const int64_t ncell = (int64_t)1 << (3 * Lc);
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = w0; c < ncell; c += nw) {
        const int a = (int)lmap[c];
        const int la = level[a];
        T s0 = T(0), s1 = T(0), s2 = T(0);
        if (la <= Lc) {  // one leaf covers the cell
            if (lane == 0) {
                const auto f = V::load(field, a);
                s0 = f.x, s1 = f.y, s2 = f.z;
            }
        } else {  // the cell's leaves [a, e), weight 8^-(level - Lc)
            const int e = c + 1 < ncell ? (int)lmap[c + 1] : n;
            for (int b = a + lane; b < e; b += 32) {
                const T vol = (T)exp2_neg(3 * ((int)level[b] - Lc));
                const auto f = V::load(field, b);
                s0 += vol * f.x;
                s1 += vol * f.y;
                s2 += vol * f.z;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (lane == 0) {
            T* p = out + 4 * c;
            p[0] = s0, p[1] = s1, p[2] = s2, p[3] = T(0);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_pyr_up(const T* __restrict__ fine, T* __restrict__ coarse, int64_t ncell) {
    using V = Vec4<T>;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
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
}

// bit-exact integer count in the 4th component
__device__ __forceinline__ float count_bits(int c, float) { return __int_as_float(c); }
__device__ __forceinline__ double count_bits(int c, double) { return __longlong_as_double((long long)c); }
__device__ __forceinline__ int bits_count(float v) { return __float_as_int(v); }
__device__ __forceinline__ int bits_count(double v) { return (int)__double_as_longlong(v); }

// Refined cells of level l (l >= Lc + 1): the ones whose first leaf a has level > l and a key
// aligned to level l.  child: node means of level l + 1 (unused when l + 1 == lmax: all
// children are leaves).
template <typename T>
__global__ void __launch_bounds__(256) k_nodes(const uint64_t* __restrict__ key, const uint8_t* __restrict__ level,
                                               int n, int l, const T* __restrict__ field, const T* __restrict__ child,
                                               T* __restrict__ out) {
    using V = Vec4<T>;
    const uint64_t mask = key_span(l) - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)i;
        if ((int)level[a] <= l || (key[a] & mask) != 0) continue;
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
        T* p = out + 4 * (int64_t)a;
        p[0] = s0 * T(0.125), p[1] = s1 * T(0.125), p[2] = s2 * T(0.125), p[3] = count_bits(pos - a, T(0));
    }
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

template <typename T>
ot_status launch_pyramid(const ot_octree* t, const T* field, T* pyr, cudaStream_t s) {
    const int Lc = t->pyr_level;
    const int64_t ncell = (int64_t)1 << (3 * Lc);
    k_pyr_base<T><<<grid_n(ncell * 32, 256), 256, 0, s>>>(t->d_key, t->d_level, (int)t->n, t->d_pmap, Lc, field,
                                                         pyr + 4 * pyramid_offset(Lc));
    count_launch();
    // node means below the pyramid, deepest level first
    T* nodes = pyr + 4 * pyramid_offset(Lc + 1);
    const int nl = node_levels(t);
    for (int k = nl - 1; k >= 0; --k) {
        const int l = Lc + 1 + k;
        T* out = nodes + 4 * (int64_t)k * t->n;
        const T* child = k + 1 < nl ? out + 4 * (int64_t)t->n : nullptr;
        k_nodes<T><<<grid_n(t->n, 256), 256, 0, s>>>(t->d_key, t->d_level, (int)t->n, l, field, child, out);
        count_launch();
    }
    for (int l = Lc - 1; l >= 0; --l) {
        const int64_t nc = (int64_t)1 << (3 * l);
        k_pyr_up<T><<<grid_n(nc, 256), 256, 0, s>>>(pyr + 4 * pyramid_offset(l + 1), pyr + 4 * pyramid_offset(l), nc);
        count_launch();
    }
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

template ot_status launch_pyramid<float>(const ot_octree*, const float*, float*, cudaStream_t);
template ot_status launch_pyramid<double>(const ot_octree*, const double*, double*, cudaStream_t);

} // namespace ot
