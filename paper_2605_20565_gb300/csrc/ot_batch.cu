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
    // with the table a trilinear-only launch searches hosts only: a 32-task list per warp
    // (more of the SM's memory left to the L1 cache)
    using Q = typename std::conditional<MATES && KINDS == K_TRI, HostQueue, WarpQueue>::type;
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
            if (KINDS != K_DELTA && (KINDS == K_TRI || gr.kernel == OT_TRILINEAR)) {
                if constexpr (MATES)
                    h = trilinear_mates<float, LEARNED>(t, s_root, field, pyr, wq, active, x, y, z, -1, o);
                else
                    h = trilinear_queued<float, LEARNED>(t, s_root, field, pyr, wq, active, x, y, z, -1, o);
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
    };
    std::vector<Launch> launches;
    auto add_launch = [&](void* fn, const BatchArgs& args, int cap) -> cudaError_t {
        int per_sm = 0;
        cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, smem);
        if (err != cudaSuccess) return err;
        if (cap > 0) per_sm = std::min(per_sm, cap);
        per_sm = std::max(per_sm, 1);
        launches.push_back(Launch{fn, args, (unsigned)(num_sms() * per_sm)});
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
            void* fn = learned ? (void*)k_batch<true, TRI_MINB, true, K_TRI> : (void*)k_batch<false, TRI_MINB, true, K_TRI>;
            if ((e = add_launch(fn, part[1], tri_per_sm)) != cudaSuccess) return fail(e);
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
    for (size_t i = 0; cap_ok && i < launches.size(); ++i) {
        unsigned* ctr = b->d_counter + i;
        void* args[] = {&v, &launches[i].args, (void*)&d_field, (void*)&b->d_pyr, &ctr};
        cap_ok = cudaLaunchKernel(launches[i].fn, dim3(launches[i].grid), dim3(block), args, smem, cs) == cudaSuccess;
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
    for (void* p : b->bufs) cudaFree(p);
    delete b;
    return OT_OK;
}
