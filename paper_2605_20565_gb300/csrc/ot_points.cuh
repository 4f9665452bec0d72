// ot_points.cuh -- per-point device routines: trilinear interpolation with level-mates,
// delta-kernel interpolation and stencil enumeration, all on exact fixed-point coordinates.
// Used by the single-op kernels, the persistent batched kernel and the spreading kernels.
#pragma once

#include "ot_common.cuh"

namespace ot {

constexpr unsigned FULL_MASK = 0xffffffffu;

__device__ __forceinline__ int floordiv2(int v) { return v >> 1; } // arithmetic shift: floor

template <typename T> __device__ __forceinline__ T qnan();
template <> __device__ __forceinline__ float qnan<float>() { return __int_as_float(0x7fc00000); }
template <> __device__ __forceinline__ double qnan<double>() { return __longlong_as_double(0x7ff8000000000000LL); }

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

// Volume-weighted sum over the leaves [a, ...) whose keys are below `end`, weight 8^-(level-l):
// the value of a refined level-mate of level l (the coalescence average of Sec. 2.1.1).  The
// whole warp works on one range at a time, 32 consecutive leaves per step; every lane gets the
// sum.  Must be reached by all 32 lanes together.  Bounded by OT_REFINED_CAP leaves.
template <typename T>
__device__ __forceinline__ void warp_range_mean(const TreeView& t, const T* __restrict__ field, int a, uint64_t end,
                                                int l, T& s0, T& s1, T& s2, bool& capped) {
    using V = Vec4<T>;
    const int lane = threadIdx.x & 31;
    T p0 = T(0), p1 = T(0), p2 = T(0);
    int b = a + lane;
    bool done = false;
    for (int it = 0; it < OT_REFINED_CAP / 32; ++it) {
        bool in = false;
        if (b < t.n) in = ldg_key(t.key + b) < end;
        if (in) {
            const T vol = (T)exp2_neg(3 * ((int)t.level[b] - l));
            const auto f = V::load(field, b);
            p0 += vol * f.x;
            p1 += vol * f.y;
            p2 += vol * f.z;
        }
        if (__ballot_sync(FULL_MASK, in) != FULL_MASK) {  // sorted keys: the range ended here
            done = true;
            break;
        }
        b += 32;
    }
    if (!done) capped = true;
    s0 = warp_sum(p0);
    s1 = warp_sum(p1);
    s2 = warp_sum(p2);
}

// Trilinear interpolation at one point per lane (Sec. 2.3.2) with the level-mate rule:
//   host leaf of level l, cell c; t_d = offset from the cell centre; s_d = +1 if t_d >= 0;
//   level-mates c + {0, s_d}; weights prod (1 - |t_d|) or |t_d|;
//   level-mate value: leaf of level l -> its value; inside a coarser leaf -> that leaf's
//   value; refined -> volume-weighted mean of its leaves; outside the cube -> the host's
//   index on that axis.
// All 32 lanes of the warp must call this together; lanes with active == false idle.
// Returns the host leaf (-1 when inactive or outside the cube, out = NaN).
template <typename T, bool LEARNED>
__device__ __forceinline__ int trilinear_warp(const TreeView& t, const RootModel& rm, const uint64_t* s_sample,
                                              const T* __restrict__ field, bool active, double x, double y, double z,
                                              int host_in, T out[3]) {
    using V = Vec4<T>;
    const int lane = threadIdx.x & 31;
    uint64_t X[3] = {0, 0, 0};
    bool ok = active && fixpoint3(x, y, z, X);
    if (active && !ok) atomicOr(t.err, (unsigned)OT_DEV_OUTSIDE);
    int h = -1, l = 0, c[3] = {0, 0, 0}, sg[3] = {1, 1, 1}, ncell = 1;
    T at[3] = {T(0), T(0), T(0)};
    if (ok) {
        h = host_in >= 0 ? host_in
                         : search<LEARNED>(t, rm, s_sample,
                                           morton3((uint32_t)(X[0] >> 32), (uint32_t)(X[1] >> 32), (uint32_t)(X[2] >> 32)));
        l = t.level[h];
        ncell = 1 << l;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            c[d] = (int)fix_cell(X[d], l);
            sg[d] = fix_upper_half(X[d], l) ? 1 : -1;
            const T td = fix_offset<T>(X[d], l);
            at[d] = td < T(0) ? -td : td;
        }
    }
    const int sh = MAXLEVEL - l;
    const uint64_t span = key_span(l);
    // level-mates: anchors, weights; a sibling of the host cell is usually h + (difference of
    // child numbers), which one key comparison proves (keys are unique); the rest are searched
    // together in lockstep
    uint64_t anc[8];
    T w[8];
    int a[8];
    unsigned need = 0, self_mask = 0;
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
        int m[3];
        T wc = T(1);
        bool self = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int off = (corner >> d) & 1;
            int v = c[d] + off * sg[d];
            if (v < 0 || v >= ncell) v = c[d];
            m[d] = v;
            self = self && (v == c[d]);
            wc *= off ? at[d] : T(1) - at[d];
        }
        w[corner] = wc;
        anc[corner] = morton3((uint32_t)m[0] << sh, (uint32_t)m[1] << sh, (uint32_t)m[2] << sh);
        a[corner] = h;
        if (self) self_mask |= 1u << corner;
        if (ok && !self) {
            bool hit = false;
            if ((m[0] >> 1) == (c[0] >> 1) && (m[1] >> 1) == (c[1] >> 1) && (m[2] >> 1) == (c[2] >> 1)) {
                const int gi = h + ((m[0] & 1) | ((m[1] & 1) << 1) | ((m[2] & 1) << 2)) -
                               ((c[0] & 1) | ((c[1] & 1) << 1) | ((c[2] & 1) << 2));
                if (gi >= 0 && gi < t.n && ldg_key(t.key + gi) == anc[corner]) {
                    a[corner] = gi;
                    hit = true;
                }
            }
            if (!hit) need |= 1u << corner;
        }
    }
#pragma unroll
    for (int corner = 0; corner < 8; ++corner)
        if ((need >> corner) & 1u) a[corner] = search<LEARNED>(t, rm, s_sample, anc[corner]);
    // values: leaves of level <= l directly; refined level-mates afterwards, warp-cooperatively
    T acc0 = T(0), acc1 = T(0), acc2 = T(0);
    unsigned rmask = 0;
    int lv[8];
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) lv[corner] = ok ? (int)t.level[a[corner]] : 0;
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
        if (!ok) continue;
        if (!((self_mask >> corner) & 1u) && lv[corner] > l) {
            rmask |= 1u << corner;
        } else {
            const auto f = V::load(field, a[corner]);
            acc0 += w[corner] * f.x;
            acc1 += w[corner] * f.y;
            acc2 += w[corner] * f.z;
        }
    }
    bool capped = false;
    while (__any_sync(FULL_MASK, rmask != 0)) {
        // each lane's next refined level-mate
        const int k = rmask ? __ffs(rmask) - 1 : 0;
        int ak = 0;
        uint64_t ek = 0;
        T wk = T(0);
#pragma unroll
        for (int kk = 0; kk < 8; ++kk)
            if (kk == k) {
                ak = a[kk];
                ek = anc[kk] + span;
                wk = w[kk];
            }
        unsigned pend = __ballot_sync(FULL_MASK, rmask != 0);
        while (pend) {
            const int owner = __ffs(pend) - 1;
            pend &= pend - 1;
            const int ao = __shfl_sync(FULL_MASK, ak, owner);
            const uint64_t eo = __shfl_sync(FULL_MASK, ek, owner);
            const int lo_ = __shfl_sync(FULL_MASK, l, owner);
            T r0, r1, r2;
            warp_range_mean<T>(t, field, ao, eo, lo_, r0, r1, r2, capped);
            if (lane == owner) {
                acc0 += wk * r0;
                acc1 += wk * r1;
                acc2 += wk * r2;
            }
        }
        if (rmask) rmask &= rmask - 1;
    }
    if (capped) atomicOr(t.err, (unsigned)OT_DEV_REFINED_CAP);
    if (!ok) {
        out[0] = out[1] = out[2] = qnan<T>();
        return -1;
    }
    out[0] = acc0;
    out[1] = acc1;
    out[2] = acc2;
    return h;
}

// Stencil origin and per-axis weights of a point with fixed-point coordinates X on the
// finest level lmax (Sec. 2.2: W(x) = prod phi(x_d/dx)/dx).
template <int K, typename T>
__device__ __forceinline__ void stencil_weights(int lmax, const uint64_t X[3], int i0[3], T w[3][Stencil<K>::W]) {
    constexpr int W = Stencil<K>::W;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int c = (int)fix_cell(X[d], lmax);
        const int hi = fix_upper_half(X[d], lmax) ? 1 : 0;
        const T t = fix_offset<T>(X[d], lmax);
        i0[d] = Stencil<K>::first(c, hi);
#pragma unroll
        for (int a = 0; a < W; ++a) w[d][a] = Stencil<K>::template phi<T>(Stencil<K>::template r<T>(a, hi, t));
    }
}

// One axis weight of stencil slot a (used when a pair is reduced on its own).
template <int K, typename T>
__device__ __forceinline__ T stencil_weight_1d(int lmax, uint64_t X, int a) {
    const int hi = fix_upper_half(X, lmax) ? 1 : 0;
    return Stencil<K>::template phi<T>(Stencil<K>::template r<T>(a, hi, fix_offset<T>(X, lmax)));
}

// Delta-kernel stencil on the finest level.  For every parent block (2x2x2 cells of level
// lmax) overlapping the stencil, one search finds its first child; a parent whose first child
// is a leaf of level lmax has all 8 children as consecutive leaves.  The visitor gets
// (leaf, ax, ay, az) for each valid stencil cell.  Returns false when some stencil cell was
// outside the cube or not a finest-level leaf (its weight is dropped).
template <int K, bool LEARNED, typename Visit>
__device__ __forceinline__ bool visit_stencil(const TreeView& t, const RootModel& rm, const uint64_t* s_sample,
                                              const int i0[3], Visit&& visit) {
    constexpr int W = Stencil<K>::W;
    const int lp = t.lmax - 1;     // parent level
    const int np_cells = 1 << lp;  // parents per axis
    const int shp = MAXLEVEL - lp;
    int p0[3], pn[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        p0[d] = floordiv2(i0[d]);
        pn[d] = floordiv2(i0[d] + W - 1) - p0[d] + 1;
    }
    bool ok_all = true;
    int prevP[3] = {-1, -1, -1}, prev_a0 = -1;  // last parent found with its 8 finest leaves
    for (int bz = 0; bz < pn[2]; ++bz)
        for (int by = 0; by < pn[1]; ++by)
            for (int bx = 0; bx < pn[0]; ++bx) {
                const int P[3] = {p0[0] + bx, p0[1] + by, p0[2] + bz};
                const bool inside = P[0] >= 0 && P[1] >= 0 && P[2] >= 0 && P[0] < np_cells && P[1] < np_cells &&
                                    P[2] < np_cells;
                int a0 = -1;
                if (inside) {
                    const uint64_t anchor =
                        morton3((uint32_t)P[0] << shp, (uint32_t)P[1] << shp, (uint32_t)P[2] << shp);
                    int a = -1;
                    if (prev_a0 >= 0 && (P[0] >> 1) == (prevP[0] >> 1) && (P[1] >> 1) == (prevP[1] >> 1) &&
                        (P[2] >> 1) == (prevP[2] >> 1)) {
                        const int g = prev_a0 + 8 * (((P[0] & 1) | ((P[1] & 1) << 1) | ((P[2] & 1) << 2)) -
                                                     ((prevP[0] & 1) | ((prevP[1] & 1) << 1) | ((prevP[2] & 1) << 2)));
                        if (g >= 0 && g < t.n && ldg_key(t.key + g) == anchor) a = g;
                    }
                    if (a < 0) a = search<LEARNED>(t, rm, s_sample, anchor);
                    if (ldg_key(t.key + a) == anchor && t.level[a] == t.lmax) {
                        a0 = a;
                        prevP[0] = P[0], prevP[1] = P[1], prevP[2] = P[2];
                        prev_a0 = a;
                    }
                }
#pragma unroll
                for (int ch = 0; ch < 8; ++ch) {
                    const int ax = 2 * P[0] + (ch & 1) - i0[0];
                    const int ay = 2 * P[1] + ((ch >> 1) & 1) - i0[1];
                    const int az = 2 * P[2] + ((ch >> 2) & 1) - i0[2];
                    if (ax < 0 || ay < 0 || az < 0 || ax >= W || ay >= W || az >= W) continue;
                    if (a0 < 0) {
                        ok_all = false;
                        continue;
                    }
                    visit(a0 + ch, ax, ay, az);
                }
            }
    return ok_all;
}

// Delta-kernel interpolation at one marker (Sec. 2.2, Eq. ibm_interpolate).  Returns the host
// leaf (-1 outside the cube).
template <typename T, int K, bool LEARNED>
__device__ __forceinline__ int delta_point(const TreeView& t, const RootModel& rm, const uint64_t* s_sample,
                                           const T* __restrict__ field, double x, double y, double z, bool want_host,
                                           T out[3]) {
    using V = Vec4<T>;
    constexpr int W = Stencil<K>::W;
    uint64_t X[3];
    if (!fixpoint3(x, y, z, X)) {
        out[0] = out[1] = out[2] = qnan<T>();
        atomicOr(t.err, (unsigned)OT_DEV_OUTSIDE);
        return -1;
    }
    int i0[3];
    T w[3][W];
    stencil_weights<K, T>(t.lmax, X, i0, w);
    // host: the finest cell holding X, one of the stencil cells
    const int hc[3] = {(int)fix_cell(X[0], t.lmax) - i0[0], (int)fix_cell(X[1], t.lmax) - i0[1],
                       (int)fix_cell(X[2], t.lmax) - i0[2]};
    int host = -1;
    T a0 = T(0), a1 = T(0), a2 = T(0);
    const bool ok = visit_stencil<K, LEARNED>(t, rm, s_sample, i0, [&](int leaf, int ax, int ay, int az) {
        const T wt = w[0][ax] * w[1][ay] * w[2][az];
        const auto f = V::load(field, leaf);
        a0 += wt * f.x;
        a1 += wt * f.y;
        a2 += wt * f.z;
        if (ax == hc[0] && ay == hc[1] && az == hc[2]) host = leaf;
    });
    if (!ok) atomicOr(t.err, (unsigned)OT_DEV_STENCIL);
    if (want_host && host < 0)
        host = search_plain(t, s_sample,
                            morton3((uint32_t)(X[0] >> 32), (uint32_t)(X[1] >> 32), (uint32_t)(X[2] >> 32)));
    out[0] = a0;
    out[1] = a1;
    out[2] = a2;
    return host;
}

} // namespace ot
