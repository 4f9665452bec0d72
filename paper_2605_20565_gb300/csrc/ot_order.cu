// ot_order.cu -- the Morton (Z-curve) order of a point set: the permutation that sorts the
// points (stably) by the key of the level-L cell holding them.  Points stored in this order give
// a warp neighbouring points (the same host leaf and level-mates), which is how the paper's
// ranks keep their Lagrangian points grouped by cell (Sec. 3.2); the tracking driver reorders
// its particles this way at every re-adaptation.
#include <algorithm>

#include "ot_internal.h"

namespace ot {

namespace {

// (level-L cell key << ib) | index; a point outside the cube gets the all-ones key (last).
__global__ void __launch_bounds__(256) k_point_keys(const double* __restrict__ x, const double* __restrict__ y,
                                                   const double* __restrict__ z, int64_t n, int L, int ib,
                                                   uint64_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t X[3];
        uint64_t cell = (1ULL << (3 * L)) - 1;
        if (fixpoint3(x[i], y[i], z[i], X))
            cell = morton3((uint32_t)(X[0] >> 32), (uint32_t)(X[1] >> 32), (uint32_t)(X[2] >> 32)) >>
                   (3 * (MAXLEVEL - L));
        out[i] = (cell << ib) | (uint64_t)i;
    }
}

__global__ void __launch_bounds__(256) k_pair_index(const uint64_t* __restrict__ pairs, int64_t n, uint64_t mask,
                                                    int32_t* __restrict__ perm) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        perm[i] = (int32_t)(pairs[i] & mask);
}

int index_bits(int64_t n) {
    int b = 1;
    while (b < 31 && ((int64_t)1 << b) < n) ++b;
    return b;
}

unsigned grid_o(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8));
}

} // namespace

size_t order_ws_bytes(int64_t n) { return 2 * sizeof(uint64_t) * (size_t)n + radix_ws_bytes(n) + 512; }

bool order_fits(int64_t n, int level) { return level >= 1 && level <= MAXLEVEL && 3 * level + index_bits(n) <= 64; }

// Sorts (cell key << ib | index) pairs of the n points into `pairs` (workspace: pairs, tmp and
// the radix histograms, order_ws_bytes(n) bytes from `pairs`); the low ib bits of each sorted
// pair are a point index.  Capturable in a CUDA graph.
ot_status launch_point_sort(const double* x, const double* y, const double* z, int64_t n, int level,
                            uint64_t* pairs, int* ib_out, cudaStream_t s) {
    const int ib = index_bits(n);
    *ib_out = ib;
    uint64_t* tmp = pairs + n;
    void* rws = tmp + n;
    k_point_keys<<<grid_o(n), 256, 0, s>>>(x, y, z, n, level, ib, pairs);
    count_launch();
    return radix_sort_u64_ws(pairs, tmp, n, ib, ib + 3 * level, rws, s);
}

} // namespace ot

using namespace ot;

extern "C" ot_status ot_points_order_workspace_size(int64_t n, size_t* bytes) {
    if (!bytes || n < 0) return OT_ERR_ARG;
    *bytes = order_ws_bytes(n);
    return OT_OK;
}

extern "C" ot_status ot_points_morton_order(const double* d_x, const double* d_y, const double* d_z, int64_t n,
                                            int level, int32_t* d_perm, void* d_workspace, size_t ws_bytes,
                                            void* stream) {
    if (n < 0 || n > ((int64_t)1 << 31) - 1 || level < 1 || level > MAXLEVEL) return OT_ERR_ARG;
    if (3 * level + index_bits(std::max<int64_t>(n, 1)) > 64) return OT_ERR_ARG;
    if (n == 0) return OT_OK;
    if (!d_x || !d_y || !d_z || !d_perm || !d_workspace || ((uintptr_t)d_workspace & 15) ||
        ws_bytes < order_ws_bytes(n))
        return OT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t* pairs = static_cast<uint64_t*>(d_workspace);
    uint64_t* tmp = pairs + n;
    void* rws = tmp + n;
    const int ib = index_bits(n);
    k_point_keys<<<grid_o(n), 256, 0, s>>>(d_x, d_y, d_z, n, level, ib, pairs);
    count_launch();
    ot_status st = radix_sort_u64_ws(pairs, tmp, n, ib, ib + 3 * level, rws, s);
    if (st != OT_OK) return st;
    k_pair_index<<<grid_o(n), 256, 0, s>>>(pairs, n, ((uint64_t)1 << ib) - 1, d_perm);
    count_launch();
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}
