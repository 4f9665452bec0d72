// ot_batch.cu -- persistent launches over every group of points (IBM markers with a delta
// kernel, point particles with trilinear interpolation), replayed from a CUDA graph.
//
// A graph replay first recomputes the pyramid of cell means of the field (refined trilinear
// level-mates read it; a few small launches), then runs the batch kernel: one launch over all
// groups, or, with the octree's level-mate table, a launch for the delta-kernel groups and
// one for the trilinear groups, each at its own occupancy.  Work is cut into tiles of
// 32 * tile points; warps take tiles from a global counter, the expensive marker groups first
// (their tiles come first in the tile space), so uneven groups balance across the SMs without
// a host round trip.  The counters are reset by a memset node captured in the same graph.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "ot_internal.h"
#include "ot_points.cuh"
#include "ot_queue.cuh"

struct ot_batch {
    const ot_octree* tree = nullptr;
    int n_groups = 0;
    std::vector<void*> bufs;   // per ordered group: point-order workspace and the ordered copies
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned* d_counter = nullptr;
    float* d_pyr = nullptr;    // pyramid of cell means, recomputed at every replay
    int kernels = 1;           // kernels in one replay of the graph
    // value records of the hot leaves (trilinear launch with the level-mate table): per
    // level-map cell its entry, per hot leaf its index, per (hot leaf, octant) the 8 level-mate
    // values, rewritten from the field at every replay
    uint2* d_ent = nullptr;
    int* d_hot_leaf = nullptr;
    float* d_rec = nullptr;
    int64_t n_rec = 0;
};

namespace ot {

constexpr int MAX_GROUPS = 16;
constexpr int TRI_MINB = 4;  // register budget of the trilinear-only launch (level-mate table)

struct GroupDev {
    int kernel;
    const double *x, *y, *z;
    int64_t n;
    float* u;
    int32_t* host;
    int64_t tile0; // first tile of the group
};

struct BatchArgs {
    GroupDev g[MAX_GROUPS];
    int ng;
    int64_t ntiles;
    int tile; // points per lane per tile
};

// MINB: the register budget (blocks of 256 resident per SM it is compiled for); 3 is the
// default, 2 trades occupancy for no register spills and is picked with blocks_per_sm = 2.
// MATES: trilinear level-mates read from the octree's level-mate table instead of searched.
// KINDS: the group kinds the instance serves -- K_ALL, K_DELTA (delta-kernel groups only) or
// K_TRI (trilinear groups only: with the table it needs far fewer registers than the delta
// path, so it runs as its own launch at a higher occupancy).
enum { K_ALL = 0, K_DELTA = 1, K_TRI = 2 };
template <bool LEARNED, int MINB, bool MATES, int KINDS = K_ALL>
__global__ void __launch_bounds__(256, MINB) k_batch(TreeView t, BatchArgs a, const float* __restrict__ field,
                                               const float* __restrict__ pyr, unsigned* __restrict__ counter) {
    // with the table a trilinear-only launch searches hosts only: a 32-task list per warp; the
    // delta-kernel launch needs none (one task slot): the less shared memory, the more of the
    // SM's memory is left to the L1 cache
    using Q = typename std::conditional<
        KINDS == K_DELTA, WarpQueueN<1>,
        typename std::conditional<MATES && KINDS == K_TRI, HostQueue, WarpQueue>::type>::type;
    __shared__ Q s_queue[256 / 32];
    __shared__ RootModel s_root;
    Q& wq = s_queue[threadIdx.x >> 5];
    stage_root<LEARNED>(t, s_root);
    const int lane = threadIdx.x & 31;
    const int64_t tile_pts = 32 * (int64_t)a.tile;
    for (;;) {
        unsigned tl = 0;
        if (lane == 0) tl = atomicAdd(counter, 1u);
        tl = __shfl_sync(0xffffffffu, tl, 0);
        if ((int64_t)tl >= a.ntiles) break;
        int g = 0;
        while (g + 1 < a.ng && (int64_t)tl >= a.g[g + 1].tile0) ++g;
        const GroupDev& gr = a.g[g];
        const int64_t base = ((int64_t)tl - gr.tile0) * tile_pts;
        for (int j = 0; j < a.tile; ++j) {
            const int64_t i = base + (int64_t)j * 32 + lane;
            const bool active = i < gr.n;
            if (!__any_sync(0xffffffffu, active)) break;  // warp-uniform
            float o[3];
            int h;
            const double x = active ? gr.x[i] : 0.0, y = active ? gr.y[i] : 0.0, z = active ? gr.z[i] : 0.0;
            bool tri = false;
            if constexpr (KINDS != K_DELTA) {
                tri = KINDS == K_TRI || gr.kernel == OT_TRILINEAR;
                if (tri) {
                    if constexpr (MATES)
                        h = trilinear_mates<float, LEARNED>(t, s_root, field, pyr, wq, active, x, y, z, -1, o);
                    else
                        h = trilinear_queued<float, LEARNED>(t, s_root, field, pyr, wq, active, x, y, z, -1, o);
                }
            }
            if (tri) {
            } else if (!active) {
                h = -1;
            } else if (gr.kernel == OT_PESKIN4) {
                h = delta_point<float, OT_PESKIN4, LEARNED>(t, field, x, y, z, gr.host != nullptr, o);
            } else {
                h = delta_point<float, OT_ROMA3, LEARNED>(t, field, x, y, z, gr.host != nullptr, o);
            }
            if (active) {
                gr.u[i] = o[0];
                gr.u[gr.n + i] = o[1];
                gr.u[2 * gr.n + i] = o[2];
                if (gr.host) gr.host[i] = h;
            }
        }
    }
}


// ------------------------------------------------------------------------------------------
// Value records of the hot leaves.  A level-map cell that lies inside one leaf of level at most
// the hot level (a level whose leaves receive several points per launch) gets the entry
// (leaf, level << 27 | hot ordinal); every other cell (leaf, ~0).  For every hot leaf and octant
// of its cell, the record holds the 8 level-mate values of its level-mate row (24 floats, corner
// order), copied from the field and the cell means at every replay.  A point in such a cell then
// reads one cell entry and one 96-byte record (three 32-byte loads) instead of the row and 8
// scattered values; the values and the sum are the same, so the results are bit-identical.
// ------------------------------------------------------------------------------------------
constexpr uint32_t REC_NONE = 0xFFFFFFFFu;
constexpr int REC_FLOATS = 24;

__global__ void k_hot_flags(const uint8_t* __restrict__ level, int64_t n, int hot_l, uint32_t* __restrict__ flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = level[i] <= hot_l ? 1u : 0u;
}

__global__ void k_hot_list(const uint32_t* __restrict__ flag, const uint32_t* __restrict__ ord, int64_t n,
                           int* __restrict__ hot_leaf) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) hot_leaf[ord[i]] = (int)i;
}

__global__ void k_cell_entries(TreeView t, const uint32_t* __restrict__ ord, int hot_l, uint2* __restrict__ ent) {
    const int64_t ncell = (int64_t)1 << (3 * t.lmap_level);
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)t.lmap[c];
        const int e = c + 1 < ncell ? (int)t.lmap[c + 1] : t.n;
        const int lv = t.level[a];
        const bool hot = e - a <= 1 && lv <= hot_l;
        ent[c] = make_uint2((uint32_t)a, hot ? ((uint32_t)lv << 27) | ord[a] : REC_NONE);
    }
}

// One record per (hot leaf, octant), rewritten from the field and the cell means.
__global__ void __launch_bounds__(256) k_hot_records(TreeView t, const int* __restrict__ hot_leaf, int64_t n_rec,
                                                     const float* __restrict__ field, const float* __restrict__ pyr,
                                                     float* __restrict__ rec) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rec; r += (int64_t)gridDim.x * blockDim.x) {
        const int h = hot_leaf[r >> 3];
        const uint4* row = t.mates + 2 * (8 * (long long)h + (r & 7));
        const uint4 r0 = __ldg(row), r1 = __ldg(row + 1);
        const uint32_t sl[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
        float v[REC_FLOATS];
#pragma unroll
        for (int corner = 0; corner < 8; ++corner) {
            const uint32_t sv = sl[corner];
            const float4 f = Vec4<float>::load((sv >> 31) ? pyr : field, (long long)(sv & 0x7FFFFFFFu));
            v[3 * corner] = f.x, v[3 * corner + 1] = f.y, v[3 * corner + 2] = f.z;
        }
        float4* dst = reinterpret_cast<float4*>(rec + REC_FLOATS * r);
#pragma unroll
        for (int k = 0; k < REC_FLOATS / 4; ++k) dst[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    }
}

// L2 policies: keep lines resident ahead of others (evict-last), or the default priority.
__device__ __forceinline__ uint64_t policy_keep() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t policy_normal() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// 32 bytes from global memory in one load (sm_100 and later), read-only path, L2 policy pol.
__device__ __forceinline__ void ld_nc_v8(const float* p, float* r, uint64_t pol) {
    asm("ld.global.nc.L2::cache_hint.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], %9;"
        : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7])
        : "l"(p), "l"(pol));
}

__device__ __forceinline__ uint2 ld_nc_u2(const uint2* p, uint64_t pol) {
    uint2 e;
    asm("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(e.x), "=r"(e.y) : "l"(p), "l"(pol));
    return e;
}

// The trilinear launch with value records.  Per 32-point row: quantise, read the level-map
// cell's entry; a point in a hot cell takes its octant's record and is done; the others (cold:
// deeper leaves, uncovered cells) are queued per warp and, whenever 32 are queued (and at the
// end), interpolated together by the level-mate-table routine with every lane busy.
template <bool LEARNED>
__global__ void __launch_bounds__(256, TRI_MINB) k_tri_rec(TreeView t, BatchArgs a, const float* __restrict__ field,
                                                          const float* __restrict__ pyr,
                                                          unsigned* __restrict__ counter,
                                                          const uint2* __restrict__ ent,
                                                          const float* __restrict__ rec) {
    // per warp of the block: its host task list and its queue of cold points (dynamic shared
    // memory sized by the block's warps: what the block does not use is left to the L1 cache)
    extern __shared__ __align__(16) unsigned char tri_smem[];
    HostQueue* s_queue = reinterpret_cast<HostQueue*>(tri_smem);
    long long (*s_cold)[64] = reinterpret_cast<long long (*)[64]>(tri_smem + sizeof(HostQueue) * (blockDim.x >> 5));
    __shared__ RootModel s_root;
    // Morton spreading of 8-bit cell coordinates (bit b -> bit 3b): the level-map cell of a point
    // is spread[cx] | spread[cy] << 1 | spread[cz] << 2 (map levels are at most 8)
    __shared__ uint32_t s_spread[256];
    for (int v = threadIdx.x; v < 256; v += blockDim.x) s_spread[v] = (uint32_t)part1by2((uint32_t)v);
    const int wid = threadIdx.x >> 5;
    HostQueue& wq = s_queue[wid];
    long long* cq = s_cold[wid];
    stage_root<LEARNED>(t, s_root);
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int cell_shift = MAXLEVEL - t.lmap_level;  // of the 21-bit coordinates
    const int64_t tile_pts = 32 * (int64_t)a.tile;
    // the cell entries (16 MB at map level 7) are read by every point: evict-last in L2; the
    // records (about 100 MB) at the default priority (evict-last on them as well measured 3%
    // slower on the many-bubble step, evict-first 15% slower); the positions and results
    // stream through once: evict-first (.cs), so they push out neither
    const uint64_t keep = policy_keep(), normal = policy_normal();
    int qn = 0;  // queued cold points (warp-uniform)
    // the first cnt queued points, one per lane (warp-wide)
    auto drain = [&](int cnt) {
        const bool act = lane < cnt;
        const long long it = act ? cq[lane] : 0;
        const GroupDev& gq = a.g[(int)(it >> 40)];
        const int64_t i = it & ((1LL << 40) - 1);
        const double x = act ? gq.x[i] : 0.0, y = act ? gq.y[i] : 0.0, z = act ? gq.z[i] : 0.0;
        float o[3];
        const int h = trilinear_mates<float, LEARNED>(t, s_root, field, pyr, wq, act, x, y, z, -1, o);
        if (act) {
            gq.u[i] = o[0];
            gq.u[gq.n + i] = o[1];
            gq.u[2 * gq.n + i] = o[2];
            if (gq.host) gq.host[i] = h;
        }
    };
    for (;;) {
        unsigned tl = 0;
        if (lane == 0) tl = atomicAdd(counter, 1u);
        tl = __shfl_sync(0xffffffffu, tl, 0);
        if ((int64_t)tl >= a.ntiles) break;
        int g = 0;
        while (g + 1 < a.ng && (int64_t)tl >= a.g[g + 1].tile0) ++g;
        const GroupDev& gr = a.g[g];
        const int64_t base = ((int64_t)tl - gr.tile0) * tile_pts;
        for (int j = 0; j < a.tile; ++j) {
            const int64_t i = base + (int64_t)j * 32 + lane;
            const bool active = i < gr.n;
            if (!__any_sync(0xffffffffu, active)) break;  // warp-uniform
            const double x = active ? __ldcs(gr.x + i) : 0.0, y = active ? __ldcs(gr.y + i) : 0.0,
                         z = active ? __ldcs(gr.z + i) : 0.0;
            uint64_t X[3];
            const bool ok = active && fixpoint3(x, y, z, X);
            uint2 e = make_uint2(0u, REC_NONE);
            if (ok) {
                const uint32_t c = s_spread[(uint32_t)(X[0] >> 32) >> cell_shift] |
                                   (s_spread[(uint32_t)(X[1] >> 32) >> cell_shift] << 1) |
                                   (s_spread[(uint32_t)(X[2] >> 32) >> cell_shift] << 2);
                e = ld_nc_u2(ent + c, keep);
            }
            const bool hot = e.y != REC_NONE;
            if (hot) {
                float at[3];
                const int oc = tri_octant<float>(X, (int)(e.y >> 27), at);
                const float* rp = rec + (8 * (size_t)(e.y & 0x7FFFFFFu) + oc) * REC_FLOATS;
                float vv[REC_FLOATS];
                ld_nc_v8(rp, vv, normal);
                ld_nc_v8(rp + 8, vv + 8, normal);
                ld_nc_v8(rp + 16, vv + 16, normal);
                float v[8][3];
#pragma unroll
                for (int c = 0; c < 8; ++c) v[c][0] = vv[3 * c], v[c][1] = vv[3 * c + 1], v[c][2] = vv[3 * c + 2];
                float o[3];
                tri_sum<float>(at, v, o);
                __stcs(gr.u + i, o[0]);
                __stcs(gr.u + gr.n + i, o[1]);
                __stcs(gr.u + 2 * gr.n + i, o[2]);
                if (gr.host) __stcs(gr.host + i, (int)e.x);
            } else if (active && !ok) {  // outside the cube: no host, no value
                atomicOr(t.err, (unsigned)OT_DEV_OUTSIDE);
                const float nan = qnan<float>();
                gr.u[i] = nan;
                gr.u[gr.n + i] = nan;
                gr.u[2 * gr.n + i] = nan;
                if (gr.host) gr.host[i] = -1;
            }
            const bool cold = ok && !hot;
            const unsigned m = __ballot_sync(0xffffffffu, cold);
            if (cold) cq[qn + __popc(m & lt)] = ((long long)g << 40) | i;
            qn += __popc(m);
            __syncwarp();
            if (qn >= 32) {
                drain(32);
                __syncwarp();
                qn -= 32;
                if (lane < qn) cq[lane] = cq[32 + lane];
                __syncwarp();
            }
        }
    }
    if (qn > 0) drain(qn);
}

// Ordered copies of a group's positions: the i-th ordered point is point (pairs[i] & mask).
__global__ void __launch_bounds__(256) k_gather_points(const uint64_t* __restrict__ pairs, int64_t n, uint64_t mask,
                                                       const double* __restrict__ x, const double* __restrict__ y,
                                                       const double* __restrict__ z, double* __restrict__ xs,
                                                       double* __restrict__ ys, double* __restrict__ zs) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = (int64_t)(pairs[i] & mask);
        xs[i] = x[j];
        ys[i] = y[j];
        zs[i] = z[j];
    }
}

// Results back to the caller's order.
__global__ void __launch_bounds__(256) k_scatter_results(const uint64_t* __restrict__ pairs, int64_t n, uint64_t mask,
                                                         const float* __restrict__ us, const int32_t* __restrict__ hs,
                                                         float* __restrict__ u, int32_t* __restrict__ host) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = (int64_t)(pairs[i] & mask);
        u[j] = us[i];
        u[n + j] = us[n + i];
        u[2 * n + j] = us[2 * n + i];
        if (host) host[j] = hs[i];
    }
}

unsigned grid_b(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8));
}

// Cell entries, hot-leaf list and record buffer of a batch (synchronises the legacy stream;
// batch creation is not stream-ordered work).  Leaves b->n_rec = 0 when no leaf is hot or the
// ordinals would not fit the entry's 27 bits.
ot_status build_hot_records(const ot_octree* t, int hot_l, ot_batch* b) {
    const int64_t n = t->n;
    uint32_t *flag = nullptr, *ord = nullptr, *tot = nullptr;
    auto cleanup = [&]() {
        if (flag) cudaFree(flag);
        if (ord) cudaFree(ord);
        if (tot) cudaFree(tot);
    };
    cudaStream_t s = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&flag, sizeof(uint32_t) * n)) != cudaSuccess || (e = cudaMalloc(&ord, sizeof(uint32_t) * n)) != cudaSuccess ||
        (e = cudaMalloc(&tot, sizeof(uint32_t))) != cudaSuccess) {
        cleanup();
        return cuda_status(e);
    }
    k_hot_flags<<<grid_b(n), 256, 0, s>>>(t->d_level, n, hot_l, flag);
    count_launch();
    ot_status st = scan_u32(flag, ord, n, tot, s);
    uint32_t n_hot = 0;
    if (st == OT_OK && (e = cudaMemcpy(&n_hot, tot, sizeof(uint32_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
        st = cuda_status(e);
    if (st != OT_OK || n_hot == 0 || n_hot >= (1u << 27)) {
        cleanup();
        return st;
    }
    const int64_t ncell = (int64_t)1 << (3 * t->lmap_level);
    if ((e = cudaMalloc(&b->d_hot_leaf, sizeof(int) * (size_t)n_hot)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_ent, sizeof(uint2) * (size_t)ncell)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_rec, sizeof(float) * REC_FLOATS * 8 * (size_t)n_hot)) != cudaSuccess) {
        cleanup();
        return cuda_status(e);
    }
    TreeView v = tree_view(t);
    k_hot_list<<<grid_b(n), 256, 0, s>>>(flag, ord, n, b->d_hot_leaf);
    k_cell_entries<<<grid_b(ncell), 256, 0, s>>>(v, ord, hot_l, b->d_ent);
    count_launch(2);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) return cuda_status(e);
    b->n_rec = 8 * (int64_t)n_hot;
    return OT_OK;
}

} // namespace ot

using namespace ot;

extern "C" ot_status ot_batch_create(const ot_octree* t, const ot_group* groups, int n_groups, const float* d_field,
                                     int search, const ot_launch* launch, void* stream, ot_batch** out) {
    if (!t || !groups || !out || !d_field || n_groups < 1 || n_groups > MAX_GROUPS) return OT_ERR_ARG;
    if (search != OT_BINARY && search != OT_LEARNED) return OT_ERR_ARG;
    if (search == OT_LEARNED && !t->has_index) return OT_ERR_NO_INDEX;
    *out = nullptr;
    const int block = (launch && launch->block) ? launch->block : 256;
    const int tile = (launch && launch->tile) ? launch->tile : 4;
    const int order_level = launch ? launch->order_level : 0;
    const int tri_tile = (launch && launch->tri_tile) ? launch->tri_tile : tile;
    const int tri_per_sm = (launch && launch->tri_blocks_per_sm) ? launch->tri_blocks_per_sm : 2;
    const int tri_records = launch ? launch->tri_records : 0;
    if (tri_records < -1 || tri_records > MAXLEVEL) return OT_ERR_ARG;
    if (block < 64 || block > 256 || block % 32 || tile < 1 || tile > 64) return OT_ERR_ARG;
    if (tri_tile < 1 || tri_tile > 64 || tri_per_sm < 1 || (launch && launch->blocks_per_sm < 0)) return OT_ERR_ARG;
    if (order_level < 0 || order_level > MAXLEVEL) return OT_ERR_ARG;
    BatchArgs a{};
    a.ng = n_groups;
    a.tile = tile;
    // delta-kernel groups first: the longest work is taken first
    std::vector<int> order;
    for (int pass = 0; pass < 2; ++pass)
        for (int g = 0; g < n_groups; ++g)
            if ((groups[g].kernel != OT_TRILINEAR) == (pass == 0)) order.push_back(g);
    int64_t tile0 = 0;
    for (int k = 0; k < n_groups; ++k) {
        const ot_group& gi = groups[order[k]];
        if (gi.kernel != OT_TRILINEAR && gi.kernel != OT_PESKIN4 && gi.kernel != OT_ROMA3) return OT_ERR_ARG;
        if (gi.n < 0 || (gi.n > 0 && (!gi.d_x || !gi.d_y || !gi.d_z || !gi.d_u))) return OT_ERR_ARG;
        if (gi.kernel != OT_TRILINEAR && t->lmax < 1) return OT_ERR_ARG;
        GroupDev& d = a.g[k];
        d = GroupDev{gi.kernel, gi.d_x, gi.d_y, gi.d_z, gi.n, gi.d_u, gi.d_host, tile0};
        tile0 += (gi.n + 32 * (int64_t)tile - 1) / (32 * (int64_t)tile);
    }
    a.ntiles = tile0;
    if (a.ntiles >= (1LL << 32)) return OT_ERR_LIMIT;

    ot_batch* b = new ot_batch();
    b->tree = t;
    b->n_groups = n_groups;
    // trilinear groups processed in Morton order of their points' level-order_level cells:
    // per group, the sort workspace and ordered copies of positions and results
    struct Ordered {
        int k;                 // slot in a.g
        GroupDev user;         // the caller's arrays
        uint64_t* pairs;
        double *xs, *ys, *zs;
        float* us;
        int32_t* hs;
    };
    std::vector<Ordered> ordered;
    cudaStream_t cs = nullptr;
    auto fail = [&](cudaError_t e) {
        if (cs) cudaStreamDestroy(cs);
        ot_batch_destroy(b);
        return cuda_status(e);
    };
    cudaError_t e;
    if ((e = cudaMalloc(&b->d_counter, sizeof(unsigned))) != cudaSuccess) return fail(e);
    for (int k = 0; order_level > 0 && k < n_groups; ++k) {
        GroupDev& d = a.g[k];
        if (d.kernel != OT_TRILINEAR || d.n < 64 || !order_fits(d.n, order_level)) continue;
        Ordered o{k, d, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
        void* p = nullptr;
        const size_t bytes = order_ws_bytes(d.n) + 3 * sizeof(double) * (size_t)d.n + 3 * sizeof(float) * (size_t)d.n +
                             sizeof(int32_t) * (size_t)d.n + 4 * 256;
        if ((e = cudaMalloc(&p, bytes)) != cudaSuccess) return fail(e);
        b->bufs.push_back(p);
        char* c = static_cast<char*>(p);
        auto take = [&](size_t sz) {
            char* r = c;
            c += (sz + 255) & ~(size_t)255;
            return r;
        };
        o.pairs = reinterpret_cast<uint64_t*>(take(order_ws_bytes(d.n)));
        o.xs = reinterpret_cast<double*>(take(sizeof(double) * d.n));
        o.ys = reinterpret_cast<double*>(take(sizeof(double) * d.n));
        o.zs = reinterpret_cast<double*>(take(sizeof(double) * d.n));
        o.us = reinterpret_cast<float*>(take(3 * sizeof(float) * d.n));
        o.hs = d.host ? reinterpret_cast<int32_t*>(take(sizeof(int32_t) * d.n)) : nullptr;
        d.x = o.xs, d.y = o.ys, d.z = o.zs, d.u = o.us, d.host = o.hs;
        ordered.push_back(o);
    }
    bool has_tri = false;
    for (int k = 0; k < n_groups; ++k) has_tri = has_tri || groups[k].kernel == OT_TRILINEAR;
    if (has_tri && (e = cudaMalloc(&b->d_pyr, pyramid_bytes(t, sizeof(float)))) != cudaSuccess) return fail(e);
    TreeView v = tree_view(t);
    const size_t smem = 0;
    const bool two = launch && launch->blocks_per_sm == 2;
    const bool learned = search == OT_LEARNED;
    // The launches of one replay: without the level-mate table, one kernel over every group;
    // with it, the delta-kernel groups and the trilinear groups as two launches (the trilinear
    // one at its own, higher, occupancy), each over its own tile range and counter.
    struct Launch {
        void* fn;
        BatchArgs args;
        unsigned grid;
        bool records;  // k_tri_rec: two more arguments
        size_t dsmem;  // dynamic shared memory per block
    };
    std::vector<Launch> launches;
    auto add_launch = [&](void* fn, const BatchArgs& args, int cap, size_t dsmem = 0) -> cudaError_t {
        int per_sm = 0;
        cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, dsmem);
        if (err != cudaSuccess) return err;
        if (cap > 0) per_sm = std::min(per_sm, cap);
        per_sm = std::max(per_sm, 1);
        launches.push_back(Launch{fn, args, (unsigned)(num_sms() * per_sm), false, dsmem});
        return cudaSuccess;
    };
    // every warp takes one tile number past the last tile before it stops: the 32-bit tile
    // counter must hold ntiles plus one per warp of the launch without wrapping
    auto counter_fits = [&]() {
        for (const Launch& l : launches)
            if ((uint64_t)l.args.ntiles + (uint64_t)l.grid * (uint64_t)(block / 32) >= (1ULL << 32)) return false;
        return true;
    };
    if (!t->d_mates) {
        void* fn = learned ? (two ? (void*)k_batch<true, 2, false> : (void*)k_batch<true, 3, false>)
                           : (two ? (void*)k_batch<false, 2, false> : (void*)k_batch<false, 3, false>);
        if ((e = add_launch(fn, a, launch ? launch->blocks_per_sm : 0)) != cudaSuccess) return fail(e);
    } else {
        BatchArgs part[2] = {};
        for (int k = 0; k < a.ng; ++k) {
            BatchArgs& p = part[a.g[k].kernel == OT_TRILINEAR ? 1 : 0];
            GroupDev d = a.g[k];
            d.tile0 = p.ntiles;
            p.tile = a.g[k].kernel == OT_TRILINEAR ? tri_tile : tile;
            p.g[p.ng++] = d;
            p.ntiles += (d.n + 32 * (int64_t)p.tile - 1) / (32 * (int64_t)p.tile);
        }
        if (part[1].ntiles >= (1LL << 32)) {
            ot_batch_destroy(b);
            return OT_ERR_LIMIT;
        }
        if (part[0].ng > 0) {
            void* fn = learned ? (two ? (void*)k_batch<true, 2, true, K_DELTA> : (void*)k_batch<true, 3, true, K_DELTA>)
                               : (two ? (void*)k_batch<false, 2, true, K_DELTA> : (void*)k_batch<false, 3, true, K_DELTA>);
            if ((e = add_launch(fn, part[0], launch ? launch->blocks_per_sm : 0)) != cudaSuccess) return fail(e);
        }
        if (part[1].ng > 0) {
            // value records of the hot leaves: leaves of level <= min(map level, hot level), where
            // the hot level is the deepest whose leaves would receive at least 4 of the trilinear
            // points if these were spread evenly over the cube (n 8^-l >= 4)
            int64_t n_tri = 0;
            for (int k = 0; k < part[1].ng; ++k) n_tri += part[1].g[k].n;
            int hot_l = 0;
            while (hot_l < MAXLEVEL && (n_tri >> (3 * (hot_l + 1))) >= 4) ++hot_l;
            hot_l = std::min(hot_l, t->lmap_level);
            if (tri_records > 0) hot_l = std::min(hot_l, tri_records);
            if (tri_records >= 0 && t->d_lmap) {
                ot_status st = build_hot_records(t, hot_l, b);
                if (st != OT_OK) {
                    ot_batch_destroy(b);
                    return st;
                }
            }
            const bool rec = b->n_rec > 0;
            void* fn = rec ? (learned ? (void*)k_tri_rec<true> : (void*)k_tri_rec<false>)
                           : (learned ? (void*)k_batch<true, TRI_MINB, true, K_TRI>
                                      : (void*)k_batch<false, TRI_MINB, true, K_TRI>);
            const size_t dsmem = rec ? (sizeof(HostQueue) + 64 * sizeof(long long)) * (size_t)(block / 32) : 0;
            if ((e = add_launch(fn, part[1], tri_per_sm, dsmem)) != cudaSuccess) return fail(e);
            launches.back().records = rec;
        }
    }
    if (!counter_fits()) {
        ot_batch_destroy(b);
        return OT_ERR_LIMIT;
    }
    if (launches.size() > 1) {
        cudaFree(b->d_counter);
        b->d_counter = nullptr;
        if ((e = cudaMalloc(&b->d_counter, sizeof(unsigned) * launches.size())) != cudaSuccess) return fail(e);
    }

    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
    // the kernels captured below run at every replay: count them once here, as the replay's
    const uint64_t launches0 = g_launches.load();
    if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return fail(e);
    cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned) * launches.size(), cs);
    bool cap_ok = true;
    std::vector<int> ibs;
    for (const Ordered& o : ordered) {
        int ib = 0;
        cap_ok = cap_ok && launch_point_sort(o.user.x, o.user.y, o.user.z, o.user.n, order_level, o.pairs, &ib, cs) == OT_OK;
        ibs.push_back(ib);
        k_gather_points<<<grid_b(o.user.n), 256, 0, cs>>>(o.pairs, o.user.n, (1ULL << ib) - 1, o.user.x, o.user.y,
                                                          o.user.z, o.xs, o.ys, o.zs);
        count_launch();
    }
    if (cap_ok && has_tri) cap_ok = launch_pyramid<float>(t, d_field, b->d_pyr, cs) == OT_OK;
    if (cap_ok && b->n_rec > 0) {
        k_hot_records<<<grid_b(b->n_rec), 256, 0, cs>>>(v, b->d_hot_leaf, b->n_rec, d_field, b->d_pyr, b->d_rec);
        count_launch();
    }
    for (size_t i = 0; cap_ok && i < launches.size(); ++i) {
        unsigned* ctr = b->d_counter + i;
        void* args[] = {&v, &launches[i].args, (void*)&d_field, (void*)&b->d_pyr, &ctr, (void*)&b->d_ent,
                        (void*)&b->d_rec};
        cap_ok = cudaLaunchKernel(launches[i].fn, dim3(launches[i].grid), dim3(block), args, launches[i].dsmem, cs) ==
                 cudaSuccess;
        count_launch();
    }
    for (size_t i = 0; cap_ok && i < ordered.size(); ++i) {
        const Ordered& o = ordered[i];
        k_scatter_results<<<grid_b(o.user.n), 256, 0, cs>>>(o.pairs, o.user.n, (1ULL << ibs[i]) - 1, o.us, o.hs,
                                                            o.user.u, o.user.host);
        count_launch();
    }
    b->kernels = (int)(g_launches.load() - launches0);
    g_launches.fetch_sub((uint64_t)b->kernels);
    if (!cap_ok) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(cs, &g);
        if (g) cudaGraphDestroy(g);
        return fail(cudaErrorUnknown);
    }
    e = cudaStreamEndCapture(cs, &b->graph);
    if (e != cudaSuccess) return fail(e);
    if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) return fail(e);
    cudaStreamDestroy(cs);
    *out = b;
    return OT_OK;
}

extern "C" ot_status ot_batch_run(ot_batch* b, void* stream) {
    if (!b || !b->exec) return OT_ERR_ARG;
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_status(e);
    count_launch((uint64_t)b->kernels);
    return OT_OK;
}

extern "C" ot_status ot_batch_destroy(ot_batch* b) {
    if (!b) return OT_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->d_counter) cudaFree(b->d_counter);
    if (b->d_pyr) cudaFree(b->d_pyr);
    if (b->d_ent) cudaFree(b->d_ent);
    if (b->d_hot_leaf) cudaFree(b->d_hot_leaf);
    if (b->d_rec) cudaFree(b->d_rec);
    for (void* p : b->bufs) cudaFree(p);
    delete b;
    return OT_OK;
}
