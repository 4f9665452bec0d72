// ot_mates.cu -- the level-mate table: the trilinear level-mate rule (Sec. 2.3.2 reading:
// host cell c of level l, level-mates c + {0, s_d}) resolved once per octree instead of at
// every query.  For leaf h and octant o of its cell (bit d of o: the upper half on axis d, so
// s_d = +1), row 8h + o holds the 8 value slots of the level-mates in corner order (bit d of
// the corner: the neighbour on axis d), 32 bytes:
//   slot < 2^31: a leaf index -- a leaf of level l, or the coarser leaf covering the level-mate;
//   slot >= 2^31: (slot - 2^31) indexes the array of cell means of a refined level-mate (the
//   dense pyramid for l <= pyr_level, else the node means of level l by first leaf).
// Out-of-cube neighbours take the host's index on that axis, or wrap when the cube is periodic.
// A query then needs its host leaf, one 32-byte row and the 8 values: the values are those the
// per-query search finds, so results are bit-identical either way.
// 256 bytes per leaf; the table depends on the leaves and the periodic setting only.
#include <algorithm>

#include "ot_internal.h"
#include "ot_points.cuh"

namespace ot {

namespace {

// One warp per leaf: lanes 0..26 resolve the 27 cells c + {-1, 0, 1}^3 (lane = sum (dir_d + 1)
// 3^d; lane 13 is the host itself), then lane j writes corners 2(j & 3), 2(j & 3) + 1 of row
// j >> 2 -- the warp stores the leaf's 256 bytes contiguously.
__global__ void __launch_bounds__(256) k_mates(TreeView t, uint2* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int Lp = t.pyr_level;
    for (int64_t h = warp0; h < t.n; h += nwarps) {
        const uint64_t kh = ldg_key(t.key + h);
        const int l = t.level[h];
        const int sh = MAXLEVEL - l;
        const int ncell = 1 << l;
        uint32_t cu[3];
        demorton3(kh >> (3 * sh), cu[0], cu[1], cu[2]);
        uint32_t slot = (uint32_t)h;
        if (lane < 27 && lane != 13) {
            const int dir[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
            uint32_t m[3];
            bool self = true;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                int v = (int)cu[d] + dir[d];
                if (v < 0 || v >= ncell) v = t.periodic ? (v + ncell) & (ncell - 1) : (int)cu[d];
                m[d] = (uint32_t)v;
                self = self && m[d] == cu[d];
            }
            if (!self) {
                const uint64_t cell = morton3(m[0], m[1], m[2]);
                const int a = search_plain(t, cell << (3 * sh));
                if ((int)t.level[a] <= l) {
                    slot = (uint32_t)a;
                } else {
                    const long long ri = l <= Lp ? pyr_offset(l) + (long long)cell
                                                 : pyr_offset(Lp + 1) + (long long)(l - Lp - 1) * t.n + a;
                    slot = 0x80000000u | (uint32_t)ri;
                }
            }
        }
        const int o = lane >> 2;
        uint32_t pr[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int corner = 2 * (lane & 3) + k;
            int src = 0, p3 = 1;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int dd = ((corner >> d) & 1) ? (((o >> d) & 1) ? 1 : -1) : 0;
                src += (dd + 1) * p3;
                p3 *= 3;
            }
            pr[k] = __shfl_sync(0xffffffffu, slot, src);
        }
        out[32 * h + lane] = make_uint2(pr[0], pr[1]);
    }
}

} // namespace

ot_status build_mates(ot_octree* t, cudaStream_t s) {
    if (t->d_mates) cudaFree(t->d_mates);
    t->d_mates = nullptr;
    // every slot must fit in 31 bits
    const int64_t means = pyramid_offset(t->pyr_level + 1) + (int64_t)node_levels(t) * t->n;
    if (means >= ((int64_t)1 << 31) || t->n >= ((int64_t)1 << 31)) return OT_ERR_LIMIT;
    OT_CUDA(cudaMalloc(&t->d_mates, (size_t)256 * (size_t)t->n));
    TreeView v = tree_view(t);
    int per_sm = 0;
    OT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mates, 256, 0));
    const int64_t grid = std::min<int64_t>((t->n + 7) / 8, (int64_t)num_sms() * std::max(per_sm, 1));
    k_mates<<<(unsigned)std::max<int64_t>(grid, 1), 256, 0, s>>>(v, reinterpret_cast<uint2*>(t->d_mates));
    count_launch();
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

} // namespace ot

using namespace ot;

extern "C" ot_status ot_octree_build_mates(ot_octree* t, int enable, void* stream) {
    if (!t || (enable != 0 && enable != 1)) return OT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!enable) {
        if (t->d_mates) {
            OT_CUDA(cudaStreamSynchronize(s));
            cudaFree(t->d_mates);
        }
        t->d_mates = nullptr;
        return OT_OK;
    }
    const ot_status st = build_mates(t, s);
    if (st != OT_OK) {
        if (t->d_mates) cudaFree(t->d_mates);
        t->d_mates = nullptr;
        return st;
    }
    OT_CUDA(cudaStreamSynchronize(s));
    return OT_OK;
}

extern "C" ot_status ot_octree_has_mates(const ot_octree* t, int* has) {
    if (!t || !has) return OT_ERR_ARG;
    *has = t->d_mates != nullptr;
    return OT_OK;
}
