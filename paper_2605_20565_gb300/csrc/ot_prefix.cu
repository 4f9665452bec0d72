// ot_prefix.cu -- exclusive prefix sums of the volume-weighted field, P[i] = sum_{j<i} f_j 8^-level_j
// (FP64, per component), so that the volume-weighted mean of the leaves of any refined cell of
// level l -- a contiguous index range [a, e) -- is (P[e] - P[a]) 8^l: the coalescence average of
// Sec. 2.1.1 that a refined trilinear level-mate takes, in O(1) per lookup.
#include <algorithm>

#include "ot_internal.h"

namespace ot {

namespace {

constexpr int PT = 256, PI = 8, PTILE = PT * PI;

template <typename T>
__device__ __forceinline__ void weighted(const T* __restrict__ field, const uint8_t* __restrict__ level, int64_t i,
                                        double& a, double& b, double& c) {
    const double v = ldexp(1.0, -3 * (int)level[i]);
    a = v * (double)field[4 * i];
    b = v * (double)field[4 * i + 1];
    c = v * (double)field[4 * i + 2];
}

// Block-wide exclusive scan of 3 doubles (fixed order: thread serial, then warp shuffles,
// then warp totals).  tot receives the block sums.
__device__ __forceinline__ void block_scan3(double v[3], double* s_w, double tot[3]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double x[3] = {v[0], v[1], v[2]};
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double y = __shfl_up_sync(0xffffffffu, x[d], o);
            if (lane >= o) x[d] += y;
        }
    }
    if (lane == 31)
        for (int d = 0; d < 3; ++d) s_w[3 * warp + d] = x[d];
    __syncthreads();
    if (threadIdx.x == 0) {
        double run[3] = {0.0, 0.0, 0.0};
        for (int w = 0; w < nw; ++w)
            for (int d = 0; d < 3; ++d) {
                const double t = s_w[3 * w + d];
                s_w[3 * w + d] = run[d];
                run[d] += t;
            }
        for (int d = 0; d < 3; ++d) s_w[3 * 32 + d] = run[d];
    }
    __syncthreads();
    for (int d = 0; d < 3; ++d) {
        tot[d] = s_w[3 * 32 + d];
        v[d] = s_w[3 * warp + d] + x[d] - v[d];  // exclusive
    }
    __syncthreads();
}

// Pass 1: per-tile sums.
template <typename T>
__global__ void __launch_bounds__(PT) k_tile_sums(const T* __restrict__ field, const uint8_t* __restrict__ level,
                                                  int64_t n, double* __restrict__ tsum) {
    __shared__ double s_w[3 * 33];
    const int64_t base = (int64_t)blockIdx.x * PTILE + (int64_t)threadIdx.x * PI;
    double v[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < PI; ++k)
        if (base + k < n) {
            double a, b, c;
            weighted(field, level, base + k, a, b, c);
            v[0] += a, v[1] += b, v[2] += c;
        }
    double tot[3];
    block_scan3(v, s_w, tot);
    if (threadIdx.x == 0)
        for (int d = 0; d < 3; ++d) tsum[3 * blockIdx.x + d] = tot[d];
}

// Pass 2: exclusive scan of the tile sums (one block, serial over chunks of blockDim).
__global__ void __launch_bounds__(PT) k_scan_tile_sums(double* __restrict__ tsum, int64_t ntiles) {
    __shared__ double s_w[3 * 33];
    double carry[3] = {0.0, 0.0, 0.0};
    for (int64_t base = 0; base < ntiles; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        double v[3] = {0.0, 0.0, 0.0};
        if (i < ntiles)
            for (int d = 0; d < 3; ++d) v[d] = tsum[3 * i + d];
        double tot[3];
        block_scan3(v, s_w, tot);
        if (i < ntiles)
            for (int d = 0; d < 3; ++d) tsum[3 * i + d] = v[d] + carry[d];
        for (int d = 0; d < 3; ++d) carry[d] += tot[d];
    }
}

// Pass 3: the prefix itself, P[i] = tile offset + exclusive scan inside the tile; P[n] = total.
template <typename T>
__global__ void __launch_bounds__(PT) k_prefix(const T* __restrict__ field, const uint8_t* __restrict__ level,
                                               int64_t n, const double* __restrict__ toff, double4* __restrict__ P) {
    __shared__ double s_w[3 * 33];
    const int64_t base = (int64_t)blockIdx.x * PTILE + (int64_t)threadIdx.x * PI;
    double w[PI][3];
    double v[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < PI; ++k) {
        w[k][0] = w[k][1] = w[k][2] = 0.0;
        if (base + k < n) weighted(field, level, base + k, w[k][0], w[k][1], w[k][2]);
        for (int d = 0; d < 3; ++d) v[d] += w[k][d];
    }
    double tot[3];
    block_scan3(v, s_w, tot);
    double run[3] = {toff[3 * blockIdx.x] + v[0], toff[3 * blockIdx.x + 1] + v[1], toff[3 * blockIdx.x + 2] + v[2]};
#pragma unroll
    for (int k = 0; k < PI; ++k) {
        if (base + k <= n) P[base + k] = make_double4(run[0], run[1], run[2], 0.0);
        for (int d = 0; d < 3; ++d) run[d] += w[k][d];
    }
}

} // namespace

size_t prefix_bytes(int64_t n) {
    const int64_t nt = (n + 1 + PTILE - 1) / PTILE;
    return sizeof(double4) * (size_t)(n + 1) + sizeof(double) * 3 * (size_t)nt + 256;
}

template <typename T>
ot_status launch_prefix(const ot_octree* t, const T* field, void* ws, cudaStream_t s) {
    const int64_t n = t->n;
    const int64_t nt = (n + 1 + PTILE - 1) / PTILE;  // covers index n as well
    double4* P = static_cast<double4*>(ws);
    double* tsum = reinterpret_cast<double*>(P + (n + 1));
    k_tile_sums<T><<<(unsigned)nt, PT, 0, s>>>(field, t->d_level, n, tsum);
    k_scan_tile_sums<<<1, PT, 0, s>>>(tsum, nt);
    k_prefix<T><<<(unsigned)nt, PT, 0, s>>>(field, t->d_level, n, tsum, P);
    count_launch(3);
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

template ot_status launch_prefix<float>(const ot_octree*, const float*, void*, cudaStream_t);
template ot_status launch_prefix<double>(const ot_octree*, const double*, void*, cudaStream_t);

} // namespace ot
