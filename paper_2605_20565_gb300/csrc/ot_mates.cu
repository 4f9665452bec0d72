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
//
// Built with it, the parent-block table of the delta kernels (Sec. 2.2 stencils on the finest
// level): for every parent block -- a cell of level lmax-1 whose 8 children are leaves of
// level lmax, identified by its first child's index a0 (a0 >> 3 is unique per block) -- row
// a0 >> 3 holds the first child of each of the 27 blocks (b + {-1, 0, 1}^3, entry
// sum (delta_d + 1) 3^d), or -1 for a block outside the cube (wrapped when periodic) or not
// refined to the finest level; 32 entries per row (128 bytes).  A delta stencil's 2-3 blocks
// per axis all lie within one block's neighbourhood, so a marker needs one lookup and one row
// instead of one lookup per block (visit_parents).
#include <algorithm>

#include "ot_internal.h"
#include "ot_points.cuh"

namespace ot {

namespace {

// One warp per MATES_U consecutive leaves at a time (their lookups in flight together).  Per
// leaf, lanes 0..8 form the dilated (Morton-interleaved) coordinate c_d + delta of axis d = j / 3,
// delta = j % 3 - 1 (clamped to the host's index or wrapped at the cube's faces; bit 63 marks
// "equals c_d"); lane k < 27 ORs the three of its direction (k = sum (delta_d + 1) 3^d, lane 13
// the host itself) into the level-mate cell's key and resolves it; then lane j writes corners
// 2(j & 3), 2(j & 3) + 1 of row j >> 2 -- the warp stores each leaf's 256 bytes contiguously.
constexpr int MATES_U = 3;
constexpr uint64_t SAME = 1ULL << 63;

__global__ void __launch_bounds__(256, 4) k_mates(TreeView t, uint2* __restrict__ out, uint8_t* __restrict__ need) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // the shuffle source of each of this lane's two corners
    const int o = lane >> 2;
    int src[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int corner = 2 * (lane & 3) + k;
        int sidx = 0, p3 = 1;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int dd = ((corner >> d) & 1) ? (((o >> d) & 1) ? 1 : -1) : 0;
            sidx += (dd + 1) * p3;
            p3 *= 3;
        }
        src[k] = sidx;
    }
    // this lane's producer role (lanes 0..8: axis pd, offset pdel) and its direction's producers
    const int pd = lane / 3, pdel = lane % 3 - 1;
    const int sx = lane % 3, sy = 3 + (lane / 3) % 3, sz = 6 + (lane / 9) % 3;
    const bool is_mate = lane < 27 && lane != 13;
    const int Lsh = 3 * (MAXLEVEL - t.lmap_level);
    const uint32_t nmap = 1u << (3 * t.lmap_level);
    // keys and levels of the warp's leaves, one lane each (then broadcast), loaded one
    // iteration ahead
    uint64_t kl = 0;
    int ll = 0;
    if (lane < MATES_U && warp0 * MATES_U + lane < t.n) {
        kl = ldg_key(t.key + warp0 * MATES_U + lane);
        ll = t.level[warp0 * MATES_U + lane];
    }
    for (int64_t base = warp0 * MATES_U; base < t.n; base += nwarps * MATES_U) {
        const int64_t nxt = base + nwarps * MATES_U + lane;
        uint64_t kl_next = 0;
        int ll_next = 0;
        if (lane < MATES_U && nxt < t.n) {
            kl_next = ldg_key(t.key + nxt);
            ll_next = t.level[nxt];
        }
        // every leaf's level-map lookups issued before any is resolved (one round of loads)
        int lv[MATES_U], a[MATES_U], e[MATES_U], la[MATES_U];
        uint64_t q[MATES_U];
        uint4 dsc[MATES_U];
        bool nb[MATES_U];
#pragma unroll
        for (int u = 0; u < MATES_U; ++u) {
            const uint64_t kh = __shfl_sync(0xffffffffu, kl, u);
            const int l = __shfl_sync(0xffffffffu, ll, u);
            lv[u] = l;
            const int sh3 = 3 * (MAXLEVEL - l);
            uint64_t dil = 0;
            if (lane < 9) {
                const int ncell = 1 << l;
                const int cd = (int)compact1by2(kh >> (sh3 + pd));
                int v = cd + pdel;
                if (v < 0 || v >= ncell) v = t.periodic ? (v + ncell) & (ncell - 1) : cd;
                dil = (part1by2((uint32_t)v) << pd) | (v == cd ? SAME : 0ULL);
            }
            const uint64_t dx = __shfl_sync(0xffffffffu, dil, sx);
            const uint64_t dy = __shfl_sync(0xffffffffu, dil, sy);
            const uint64_t dz = __shfl_sync(0xffffffffu, dil, sz);
            nb[u] = is_mate && base + u < t.n && !(dx & dy & dz & SAME);
            q[u] = ((dx | dy | dz) & ~SAME) << sh3;  // the level-mate cell's anchor key
            const uint32_t c = nb[u] ? (uint32_t)(q[u] >> Lsh) : 0u;
            a[u] = (int)t.lmap[c];
            e[u] = c + 1 < nmap ? (int)t.lmap[c + 1] : t.n;
            la[u] = t.lmap_lv[c];
            dsc[u] = t.desc ? __ldg(t.desc + c) : make_uint4(0u, 0u, 0u, 0u);
        }
        const int Lp = t.pyr_level;
#pragma unroll
        for (int u = 0; u < MATES_U; ++u) {
            uint32_t slot = (uint32_t)(base + u);
            if (nb[u]) {
                const int l = lv[u];
                int leaf = a[u], lvl = la[u];
                if (e[u] - a[u] > 1) {
                    if (dsc[u].z & DESC_VALID) {
                        leaf = desc_leaf(dsc[u], t.lmap_level, q[u], a[u], lvl);
                    } else {
                        leaf = search_range(t.key, a[u], e[u] - a[u], q[u]);
                        lvl = t.level[leaf];
                    }
                }
                if (lvl <= l) {
                    slot = (uint32_t)leaf;
                } else {
                    const long long ri = l <= Lp ? pyr_offset(l) + (long long)(q[u] >> (3 * (MAXLEVEL - l)))
                                                 : pyr_offset(Lp + 1) + (long long)(l - Lp - 1) * t.n + leaf;
                    slot = 0x80000000u | (uint32_t)ri;
                need[ri] = 1;  // a mean the table reads
                }
            }
            const uint32_t p0 = __shfl_sync(0xffffffffu, slot, src[0]);
            const uint32_t p1 = __shfl_sync(0xffffffffu, slot, src[1]);
            if (base + u < t.n) out[32 * (base + u) + lane] = make_uint2(p0, p1);
        }
        kl = kl_next;
        ll = ll_next;
    }
}

// One warp per row slot s (leaves 8s .. 8s+7 hold at most one first child of a block): lanes
// 0..7 find it, then lane k < 27 resolves block b + delta(k); lanes 27..31 write -1 padding.
__global__ void __launch_bounds__(256) k_pnbr(TreeView t, int64_t nslots, int* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int lp = t.lmax - 1;
    const int sh = MAXLEVEL - lp;
    const uint64_t pmask = key_span(lp) - 1;
    const int ncell = 1 << lp;
    for (int64_t sl = warp0; sl < nslots; sl += nwarps) {
        const int64_t a = 8 * sl + lane;
        bool first = false;
        if (lane < 8 && a < t.n) first = (int)t.level[a] == t.lmax && (ldg_key(t.key + a) & pmask) == 0;
        const unsigned m = __ballot_sync(0xffffffffu, first);
        if (!m) continue;  // warp-uniform
        const int64_t a0 = 8 * sl + (__ffs(m) - 1);
        uint32_t b[3];
        demorton3(ldg_key(t.key + a0) >> (3 * sh), b[0], b[1], b[2]);
        int v = -1;
        if (lane < 27) {
            const int dir[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
            int q[3];
            bool inside = true;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                q[d] = (int)b[d] + dir[d];
                if (t.periodic) q[d] = (q[d] + ncell) & (ncell - 1);
                inside = inside && q[d] >= 0 && q[d] < ncell;
            }
            if (inside) {
                const uint64_t anchor = morton3((uint32_t)q[0], (uint32_t)q[1], (uint32_t)q[2]) << (3 * sh);
                const int f = search_plain(t, anchor);
                if ((int)t.level[f] == t.lmax && ldg_key(t.key + f) == anchor) v = f;
            }
        }
        out[32 * sl + lane] = v;
    }
}

} // namespace

size_t pnbr_slots(const ot_octree* t) { return t->lmax >= 1 ? (size_t)(t->n / 8 + 1) : 0; }

// level-mate table, then the parent-block table
size_t mates_bytes(const ot_octree* t) { return (size_t)256 * (size_t)t->n + 128 * pnbr_slots(t); }

// Every slot must fit in 31 bits.
bool mates_fit(const ot_octree* t) {
    const int64_t means = pyramid_offset(t->pyr_level + 1) + (int64_t)node_levels(t) * t->n;
    return means < ((int64_t)1 << 31) && t->n < ((int64_t)1 << 31);
}

// Fills the octree's table (t->d_mates, mates_bytes(t) bytes) on stream s.
ot_status build_mates(ot_octree* t, cudaStream_t s) {
    if (!t->d_mates) return OT_ERR_ARG;
    if (!mates_fit(t)) return OT_ERR_LIMIT;
    TreeView v = tree_view(t);
    int per_sm = 0;
    OT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mates, 256, 0));
    const int64_t warps = (t->n + MATES_U - 1) / MATES_U;
    const int64_t grid = std::min<int64_t>((warps + 7) / 8, (int64_t)num_sms() * std::max(per_sm, 1));
    // flags of the cell means the table reads (kept by the octree: later pyramids compute
    // those only)
    const size_t nbytes = std::max<size_t>(need_flag_bytes(t), 1);
    if (t->d_need_flags) cudaFree(t->d_need_flags);
    t->d_need_flags = nullptr;
    uint8_t* need = nullptr;
    OT_CUDA(cudaMalloc(&need, nbytes));
    OT_CUDA(cudaMemsetAsync(need, 0, nbytes, s));
    k_mates<<<(unsigned)std::max<int64_t>(grid, 1), 256, 0, s>>>(v, reinterpret_cast<uint2*>(t->d_mates), need);
    count_launch();
    const int64_t nslots = (int64_t)pnbr_slots(t);
    if (nslots > 0) {
        int* pn = reinterpret_cast<int*>(reinterpret_cast<char*>(t->d_mates) + (size_t)256 * t->n);
        OT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pnbr, 256, 0));
        const int64_t g2 = std::min<int64_t>((nslots + 7) / 8, (int64_t)num_sms() * std::max(per_sm, 1));
        k_pnbr<<<(unsigned)std::max<int64_t>(g2, 1), 256, 0, s>>>(v, nslots, pn);
        count_launch();
    }
    OT_CUDA(cudaGetLastError());
    const ot_status st = close_need_flags(t, need, s);
    if (st != OT_OK) {
        cudaFree(need);
        return st;
    }
    t->d_need_flags = need;
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

} // namespace ot

using namespace ot;

namespace {

// Drops the octree's table (freed when the library owns it).
void drop_mates(ot_octree* t) {
    if (t->d_need_flags) cudaFree(t->d_need_flags);  // without the table every mean is computed again
    t->d_need_flags = nullptr;
    if (t->d_mates && t->mates_owned) cudaFree(t->d_mates);
    t->d_mates = nullptr;
    t->mates_owned = false;
}

} // namespace

extern "C" ot_status ot_octree_build_mates(ot_octree* t, int enable, void* stream) {
    if (!t || (enable != 0 && enable != 1)) return OT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!enable) {
        if (t->d_mates) OT_CUDA(cudaStreamSynchronize(s));
        drop_mates(t);
        return OT_OK;
    }
    if (!mates_fit(t)) return OT_ERR_LIMIT;
    if (!t->d_mates) {
        const cudaError_t e = cudaMalloc(&t->d_mates, mates_bytes(t));
        if (e != cudaSuccess) {
            t->d_mates = nullptr;
            return cuda_status(e);
        }
        t->mates_owned = true;
    }
    ot_status st = build_mates(t, s);
    if (st == OT_OK && cudaStreamSynchronize(s) != cudaSuccess) st = OT_ERR_CUDA;
    if (st != OT_OK) drop_mates(t);
    return st;
}

extern "C" ot_status ot_octree_mates_bytes(const ot_octree* t, size_t* bytes) {
    if (!t || !bytes) return OT_ERR_ARG;
    *bytes = mates_bytes(t);
    return OT_OK;
}

extern "C" ot_status ot_octree_build_mates_in(ot_octree* t, void* d_buffer, size_t bytes, void* stream) {
    if (!t || !d_buffer || ((uintptr_t)d_buffer & 15) || bytes < mates_bytes(t)) return OT_ERR_ARG;
    if (!mates_fit(t)) return OT_ERR_LIMIT;
    cudaStream_t s = (cudaStream_t)stream;
    if (t->d_mates) OT_CUDA(cudaStreamSynchronize(s));
    drop_mates(t);
    t->d_mates = static_cast<uint32_t*>(d_buffer);
    ot_status st = build_mates(t, s);
    if (st == OT_OK && cudaStreamSynchronize(s) != cudaSuccess) st = OT_ERR_CUDA;
    if (st != OT_OK) drop_mates(t);
    return st;
}

extern "C" ot_status ot_octree_has_mates(const ot_octree* t, int* has) {
    if (!t || !has) return OT_ERR_ARG;
    *has = t->d_mates != nullptr;
    return OT_OK;
}
