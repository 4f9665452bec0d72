// ot_queue.cuh -- warp-cooperative host-cell search over a per-warp task list, and the
// trilinear interpolation (Sec. 2.3.2, level-mate rule) built on it.
//
// A point needs up to 8 searches (its host, then the level-mates that are not siblings of the
// host) and each search takes 0 to ~12 dependent key probes, so a warp that gives each lane its
// own searches idles most lanes: every corner costs the longest lane's search.  Here the lanes
// first append every search they need to a task list in shared memory (ballot + popc, no
// atomics); then each lane takes the next task whenever its current one ends and performs one
// probe per step.  The warp's step count follows the total number of probes / 32 instead of the
// sum over corners of the longest lane's.  Results are exactly those of the per-lane searches
// (the same halving over the same range).
#pragma once

#include "ot_points.cuh"

namespace ot {

constexpr int QCAP = 7 * 32;  // level-mate searches of a warp's 32 points (the host's need 32)
constexpr unsigned FULL = 0xffffffffu;

// A warp's task list: key searched, and the range to search (the uncovered level-map cell);
// lo holds the answer once the task has run.  CAP tasks: QCAP for the level-mate searches, 32
// where only the hosts are searched (the level-mate table gives the rest).
template <int CAP>
struct WarpQueueN {
    static constexpr int cap = CAP;
    uint64_t q[CAP];
    int lo[CAP];
    int len[CAP];
    signed char lv[CAP];  // the answer leaf's level when the search learned it, else -1
};
using WarpQueue = WarpQueueN<QCAP>;
using HostQueue = WarpQueueN<32>;

// The root model of the learned index, staged in shared memory by every block that searches
// with it (block-wide call; a no-op for the plain form).
template <bool LEARNED>
__device__ __forceinline__ void stage_root(const TreeView& t, RootModel& s_root) {
    if (LEARNED) {
        const int* src = reinterpret_cast<const int*>(t.root);
        int* dst = reinterpret_cast<int*>(&s_root);
        for (int i = threadIdx.x; i < (int)(sizeof(RootModel) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
}

// Level-map lookup of key q: the leaf holding its cell's anchor (a) and the next cell's (e).
// The cell is covered by one leaf -- leaf a, the answer -- exactly when e - a <= 1 (a refined
// cell holds at least 8 leaves, its first one starting at its anchor).  Returns true with the
// answer in a when covered, else false with the cell's leaf range [a, e) to search.
// lv: the level of leaf a (from the per-cell level table, in the same round trip).
__device__ __forceinline__ bool map_lookup(const TreeView& t, uint64_t q, int& a, int& e, int& lv) {
    const uint32_t cell = (uint32_t)(q >> (3 * (MAXLEVEL - t.lmap_level)));
    a = (int)t.lmap[cell];
    e = cell < (1u << (3 * t.lmap_level)) - 1u ? (int)t.lmap[cell + 1] : t.n;
    lv = t.lmap_lv[cell];
    return e - a <= 1;
}

// Appends a task for every lane with need set (warp-wide call); returns the lane's task index
// or -1.  n is the warp-uniform task count.
template <typename Q>
__device__ __forceinline__ int push_task(Q& w, int& n, bool need, uint64_t q, int lo, int len, unsigned lt) {
    const unsigned m = __ballot_sync(FULL, need);
    const int idx = n + __popc(m & lt);
    n += __popc(m);
    if (need) {
        w.q[idx] = q;
        w.lo[idx] = lo;
        w.len[idx] = len;
    }
    return need ? idx : -1;
}

// Runs the warp's ntask tasks (warp-wide call).  Each step, a lane without a task takes the
// next one, and every lane with a task advances it by one step of at most one memory round
// trip:
//   plain:   the cell's subtree descriptor, which answers directly when the subtree is at most
//            3 levels deep; else halving probes over the cell's leaves;
//   learned: route (root model from shared memory, then the middle model's load), leaf model
//            load and window (its prediction widened by the stored error bounds, clamped to
//            the cell), halving probes over the window, and the check key[a] <= q < key[a+1];
//            a window that missed is replaced by the whole cell (a counted fallback).
// A finished task's answer (the last index in its range whose key is <= q) replaces its lo;
// its level goes to lv when the descriptor gave it (-1 otherwise).
// (Routing all tasks side by side before the loop was measured slower: it adds a round trip
// and registers.)
enum { ST_ROUTE = 0, ST_MODEL = 1, ST_PROBE = 2, ST_CHECK = 3, ST_DONE = 4, ST_DESC = 5 };

template <bool LEARNED, typename Q>
__device__ __forceinline__ void run_tasks(const TreeView& t, const RootModel& root, Q& w, int ntask,
                                          unsigned lt) {
    __syncwarp();
    int cur = -1, lo = 0, len = 0, next = 0, st = ST_DONE, clo = 0, clen = 0, j = 0, lvr = -1;
    bool checked = false;
    uint64_t q = 0;
    for (;;) {
        const bool fin = cur >= 0 && st == ST_DONE;
        if (fin) {
            w.lo[cur] = lo;
            w.lv[cur] = (signed char)lvr;
        }
        const bool need = cur < 0 || fin;
        const unsigned m = __ballot_sync(FULL, need);
        if (need) {
            const int idx = next + __popc(m & lt);
            cur = -1;
            if (idx < ntask) {
                cur = idx;
                q = w.q[idx];
                lo = clo = w.lo[idx];
                len = clen = w.len[idx];
                st = LEARNED ? ST_ROUTE : (t.desc ? ST_DESC : ST_PROBE);
                checked = false;
                lvr = -1;
            }
        }
        next += __popc(m);
        if (!__any_sync(FULL, cur >= 0)) break;
        if (cur < 0) continue;
        if (!LEARNED && st == ST_DESC) {
            const uint4 d = __ldg(t.desc + (q >> (3 * (MAXLEVEL - t.lmap_level))));
            if (d.z & DESC_VALID) {
                lo = desc_leaf(d, t.lmap_level, q, lo, lvr);
                st = ST_DONE;
            } else {
                st = ST_PROBE;
            }
        } else if (LEARNED && st == ST_ROUTE) {
            j = root_route(root, q);
            if (t.mids) j = (int)(((int64_t)leaf_predict(t.mids[j], q, t.n) * t.n_leaf) / t.n);
            st = ST_MODEL;
        } else if (LEARNED && st == ST_MODEL) {
            const LeafModel md = t.models[j];
            int wl = clo, wh = clo + clen - 1;
            if (md.count > 0) {
                const int pc = leaf_predict(md, q, t.n);
                wl = max(pc - md.err_lo - 1, clo);
                wh = min(pc + md.err_hi + 1, clo + clen - 1);
            }
            if (md.count > 0 && wl <= wh) {
                lo = wl;
                len = wh - wl + 1;
            } else {
                atomicAdd(t.fallbacks, 1ULL);
                atomicOr(t.err, (unsigned)OT_DEV_WINDOW);
                checked = true;  // the whole cell: its answer needs no check
            }
            st = ST_PROBE;
        } else if (st == ST_PROBE) {
            if (len > 1) {
                const int half = len >> 1;
                const uint64_t k = ldg_key(t.key + lo + half);
                lo = (k <= q) ? lo + half : lo;
                len -= half;
            }
            if (len <= 1) st = (LEARNED && !checked) ? ST_CHECK : ST_DONE;
        } else if (LEARNED && st == ST_CHECK) {
            const uint64_t k0 = ldg_key(t.key + lo);
            const uint64_t k1 = lo + 1 < t.n ? ldg_key(t.key + lo + 1) : ~0ULL;
            checked = true;
            st = ST_DONE;
            if (!(k0 <= q && q < k1)) {
                atomicAdd(t.fallbacks, 1ULL);
                atomicOr(t.err, (unsigned)OT_DEV_WINDOW);
                lo = clo;
                len = clen;
                st = len > 1 ? ST_PROBE : ST_DONE;
            }
        }
    }
    __syncwarp();
}

// Host leaf of the point with fixed-point coordinates X, for the lanes with ok set and no host
// given (h < 0) (warp-wide call): the level-map lookup, then the warp's task list for the lanes
// whose cell is not covered.  hl receives the leaf's level when the lookup or the descriptor
// gave it, else stays -1.
template <bool LEARNED, typename Q>
__device__ __forceinline__ void host_queued(const TreeView& t, const RootModel& root, Q& w, bool ok,
                                            const uint64_t X[3], int& h, int& hl) {
    const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
    const uint64_t q = morton3((uint32_t)(X[0] >> 32), (uint32_t)(X[1] >> 32), (uint32_t)(X[2] >> 32));
    int ca = 0, ce = 0, clv = -1;
    const bool need = ok && h < 0 && !map_lookup(t, q, ca, ce, clv);
    if (ok && h < 0 && !need) h = ca, hl = clv;
    if (__any_sync(FULL, need)) {
        int n = 0;
        const int ix = push_task(w, n, need, q, ca, ce - ca, lt);
        run_tasks<LEARNED>(t, root, w, n, lt);
        if (ix >= 0) h = w.lo[ix], hl = w.lv[ix];
        __syncwarp();
    }
}

// Trilinear interpolation at one point per lane (warp-wide call; Sec. 2.3.2 with the
// level-mate rule):
//   host leaf of level l, cell c; t_d = offset from the cell centre; s_d = +1 if t_d >= 0;
//   level-mates c + {0, s_d}; weights prod (1 - |t_d|) or |t_d|;
//   level-mate value: leaf of level l -> its value; inside a coarser leaf -> that leaf's
//   value; refined -> volume-weighted mean of its leaves, one load: from the dense pyramid of
//   cell means for l <= the pyramid level, else from the node means of level l (both in pyr);
//   outside the cube -> the host's index on that axis, or the wrapped index when periodic.
// Lanes with active == false take part in the warp's steps only.  host_in >= 0 gives the host.
// Returns the host leaf (-1 when inactive or outside the cube, out = NaN).
template <typename T, bool LEARNED>
__device__ __forceinline__ int trilinear_queued(const TreeView& t, const RootModel& root, const T* __restrict__ field,
                                                const T* __restrict__ pyr, WarpQueue& w, bool active, double x,
                                                double y, double z, int host_in, T out[3]) {
    using V = Vec4<T>;
    const unsigned lt = (1u << (threadIdx.x & 31)) - 1u;
    uint64_t X[3] = {0, 0, 0};
    const bool ok = active && fixpoint3(x, y, z, X);
    if (active && !ok) atomicOr(t.err, (unsigned)OT_DEV_OUTSIDE);

    // host (and its level, when the lookup gives it)
    int h = host_in, hl = -1;
    host_queued<LEARNED>(t, root, w, ok, X, h, hl);
    if (!ok) h = 0, hl = -1;  // keeps the lane's reads in bounds; its result is discarded

    const int l = hl >= 0 ? hl : (int)t.level[h];
    const int ncell = 1 << l;
    int c[3], sg[3];
    T at[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        c[d] = (int)fix_cell(X[d], l);
        sg[d] = fix_upper_half(X[d], l) ? 1 : -1;
        const T td = fix_offset<T>(X[d], l);
        at[d] = td < T(0) ? -td : td;
    }
    const int sh = MAXLEVEL - l;
    // The level-mates are resolved in stages, each issuing its loads for all 8 corners at once
    // (independent loads in flight together instead of one dependent chain per corner).
    // Stage 1: anchors, weights, and the sibling guess h + (difference of child numbers) for
    // level-mates in the host's parent cell.
    uint64_t anc[8];
    T wt[8];
    int a[8], gi[8];
    unsigned self_m = 1u, sib_m = 0u;
    // per axis the level-mate index (the host's, or the neighbour's clamped into the cube) and
    // its Morton bits: each corner's anchor is the OR of three of these six
    int nb[3];
    uint64_t dil[3][2];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        nb[d] = c[d] + sg[d];
        if (nb[d] < 0 || nb[d] >= ncell) nb[d] = t.periodic ? (nb[d] + ncell) & (ncell - 1) : c[d];
        dil[d][0] = (part1by2((uint32_t)c[d]) << d) << (3 * sh);
        dil[d][1] = (part1by2((uint32_t)nb[d]) << d) << (3 * sh);
    }
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
        int m[3];
        T wc = T(1);
        bool self = true, sib = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int off = (corner >> d) & 1;
            const int v = off ? nb[d] : c[d];
            m[d] = v;
            self = self && (v == c[d]);
            sib = sib && ((v >> 1) == (c[d] >> 1));
            wc *= off ? at[d] : T(1) - at[d];
        }
        wt[corner] = wc;
        anc[corner] = dil[0][corner & 1] | dil[1][(corner >> 1) & 1] | dil[2][(corner >> 2) & 1];
        a[corner] = h;
        gi[corner] = min(max(h + ((m[0] & 1) | ((m[1] & 1) << 1) | ((m[2] & 1) << 2)) -
                                 ((c[0] & 1) | ((c[1] & 1) << 1) | ((c[2] & 1) << 2)),
                             0),
                         t.n - 1);
        if (self) self_m |= 1u << corner;
        if (sib && !self) sib_m |= 1u << corner;
    }
    if (!ok) self_m = 0xffu, sib_m = 0u;
    // Stage 2: the guessed siblings' keys (a match proves the guess: keys are unique) and, in
    // the same round of loads, the level-map lookups of the other level-mates (a covered cell
    // settles its level-mate).  Stage 3: a failed guess's lookup.  Stage 4: the rest become
    // tasks of the warp's list.
    unsigned pend_m = ~self_m & 0xffu;
    int ca[8], ce[8];
    {
        uint64_t gk[8];
        int unused_lv;
#pragma unroll
        for (int corner = 1; corner < 8; ++corner) {
            ca[corner] = 0;
            ce[corner] = 0;
            gk[corner] = 0;
            if ((sib_m >> corner) & 1u) {
                gk[corner] = ldg_key(t.key + gi[corner]);
            } else if ((pend_m >> corner) & 1u) {
                if (map_lookup(t, anc[corner], ca[corner], ce[corner], unused_lv)) {
                    a[corner] = ca[corner];
                    pend_m &= ~(1u << corner);
                }
            }
        }
#pragma unroll
        for (int corner = 1; corner < 8; ++corner) {
            if (!((sib_m >> corner) & 1u)) continue;
            if (gk[corner] == anc[corner] || map_lookup(t, anc[corner], ca[corner], ce[corner], unused_lv)) {
                a[corner] = gk[corner] == anc[corner] ? gi[corner] : ca[corner];
                pend_m &= ~(1u << corner);
            }
        }
    }
    if (__any_sync(FULL, pend_m != 0u)) {
        int n = 0;
        int tix[8];
#pragma unroll
        for (int corner = 1; corner < 8; ++corner)
            tix[corner] = push_task(w, n, (pend_m >> corner) & 1u, anc[corner], ca[corner], ce[corner] - ca[corner], lt);
        run_tasks<LEARNED>(t, root, w, n, lt);
#pragma unroll
        for (int corner = 1; corner < 8; ++corner)
            if (tix[corner] >= 0) a[corner] = w.lo[tix[corner]];
        __syncwarp();
    }
    if (!ok) {
        out[0] = out[1] = out[2] = qnan<T>();
        return -1;
    }
    // Stage 6: the levels of the level-mates' leaves (carrying them along from the lookups was
    // measured slower: registers); stage 7: the values.
    int lvl[8];
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) lvl[corner] = ((self_m >> corner) & 1u) ? l : (int)t.level[a[corner]];
    // a refined level-mate: the pyramid cell (l <= pyramid level) or the node mean of level l
    // indexed by its first leaf
    const bool in_pyr = l <= t.pyr_level;
    const T* rbase = in_pyr ? pyr + 4 * pyr_offset(l) : pyr + 4 * (pyr_offset(t.pyr_level + 1) +
                                                               (long long)(l - t.pyr_level - 1) * t.n);
    T v[8][3];
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
        const bool refined = lvl[corner] > l;
        const long long ri = in_pyr ? (long long)(anc[corner] >> (3 * sh)) : (long long)a[corner];
        const auto f = V::load(refined ? rbase : field, refined ? ri : (long long)a[corner]);
        v[corner][0] = f.x, v[corner][1] = f.y, v[corner][2] = f.z;
    }
    T acc0 = T(0), acc1 = T(0), acc2 = T(0);
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
        acc0 += wt[corner] * v[corner][0];
        acc1 += wt[corner] * v[corner][1];
        acc2 += wt[corner] * v[corner][2];
    }
    out[0] = acc0;
    out[1] = acc1;
    out[2] = acc2;
    return h;
}

// Octant of the point with fixed-point coordinates X in its host leaf of level l (bit d: the
// upper half on axis d) and the distances |t_d| of the point from the leaf's centre in cell
// units (Sec. 2.3.2 trilinear weights).
template <typename T>
__device__ __forceinline__ int tri_octant(const uint64_t X[3], int l, T at[3]) {
    int o = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        o |= (fix_upper_half(X[d], l) ? 1 : 0) << d;
        const T td = fix_offset<T>(X[d], l);
        at[d] = td < T(0) ? -td : td;
    }
    return o;
}

// The trilinear sum over the 8 level-mate values v (corner order: bit d of the corner set for
// the neighbour on axis d), weights prod (1 - |t_d|) or |t_d|, accumulated in corner order.
// Every form of the trilinear interpolation ends here, so their results are bit-identical.
template <typename T>
__device__ __forceinline__ void tri_sum(const T at[3], const T v[8][3], T out[3]) {
    // corner weight (f_0 f_1) f_2 with f_d = |t_d| or 1 - |t_d|: the four x-y products once
    const T b0 = T(1) - at[0], b1 = T(1) - at[1], b2 = T(1) - at[2];
    const T wxy[4] = {b0 * b1, at[0] * b1, b0 * at[1], at[0] * at[1]};
    T acc0 = T(0), acc1 = T(0), acc2 = T(0);
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
        const T wc = wxy[corner & 3] * ((corner & 4) ? at[2] : b2);
        acc0 += wc * v[corner][0];
        acc1 += wc * v[corner][1];
        acc2 += wc * v[corner][2];
    }
    out[0] = acc0;
    out[1] = acc1;
    out[2] = acc2;
}

// The same interpolation with the level-mates read from the octree's level-mate table (built
// by ot_octree_build_mates): host leaf h of level l, octant o of its cell (bit d: the upper
// half on axis d), then row 8h + o gives the 8 value slots -- a leaf index, or (top bit set)
// an index into the cell means in pyr.  The weights, values and summation order are those of
// trilinear_queued: the results are bit-identical.  Warp-wide call (the host search).
template <typename T, bool LEARNED, typename Q>
__device__ __forceinline__ int trilinear_mates(const TreeView& t, const RootModel& root, const T* __restrict__ field,
                                               const T* __restrict__ pyr, Q& w, bool active, double x,
                                               double y, double z, int host_in, T out[3]) {
    using V = Vec4<T>;
    uint64_t X[3] = {0, 0, 0};
    const bool ok = active && fixpoint3(x, y, z, X);
    if (active && !ok) atomicOr(t.err, (unsigned)OT_DEV_OUTSIDE);
    int h = host_in, hl = -1;
    host_queued<LEARNED>(t, root, w, ok, X, h, hl);
    if (!ok) {
        out[0] = out[1] = out[2] = qnan<T>();
        return -1;
    }
    const int l = hl >= 0 ? hl : (int)t.level[h];
    T at[3];
    const int o = tri_octant<T>(X, l, at);
    const uint4* row = t.mates + 2 * (8 * (long long)h + o);
    const uint4 r0 = __ldg(row), r1 = __ldg(row + 1);
    const uint32_t sl[8] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w};
    T v[8][3];
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
        const uint32_t sv = sl[corner];
        const auto f = V::load((sv >> 31) ? pyr : field, (long long)(sv & 0x7FFFFFFFu));
        v[corner][0] = f.x, v[corner][1] = f.y, v[corner][2] = f.z;
    }
    tri_sum<T>(at, v, out);
    return h;
}

} // namespace ot
