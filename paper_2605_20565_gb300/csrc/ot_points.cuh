// ot_points.cuh -- per-point device routines: trilinear interpolation with level-mates,
// delta-kernel interpolation and stencil enumeration, all on exact fixed-point coordinates.
// Used by the single-op kernels, the persistent batched kernel and the spreading kernels.
#pragma once

#include "ot_common.cuh"

namespace ot {

__device__ __forceinline__ int floordiv2(int v) { return v >> 1; } // arithmetic shift: floor

template <typename T> __device__ __forceinline__ T qnan();
template <> __device__ __forceinline__ float qnan<float>() { return __int_as_float(0x7fc00000); }
template <> __device__ __forceinline__ double qnan<double>() { return __longlong_as_double(0x7ff8000000000000LL); }


// 2^k as a double, built from the bits (0 <= k < 1000).
__device__ __forceinline__ double exp2_pos(int k) { return __longlong_as_double((long long)(1023 + k) << 52); }

// Trilinear interpolation at one point (Sec. 2.3.2) with the level-mate rule:
//   host leaf of level l, cell c; t_d = offset from the cell centre; s_d = +1 if t_d >= 0;
//   level-mates c + {0, s_d}; weights prod (1 - |t_d|) or |t_d|;
//   level-mate value: leaf of level l -> its value; inside a coarser leaf -> that leaf's
//   value; refined -> volume-weighted mean of its leaves, (P[e] - P[a]) 8^l from the prefix P
//   of the volume-weighted field over its leaf range [a, e); outside the cube -> the host's
//   index on that axis.
// Lanes with active == false do nothing.  Returns the host leaf (-1 when inactive or outside
// the cube, out = NaN).
template <typename T, bool LEARNED>
__device__ __forceinline__ int trilinear_point(const TreeView& t, const T* __restrict__ field,
                                               const double4* __restrict__ P, bool active, double x, double y,
                                               double z, int host_in, T out[3]) {
    using V = Vec4<T>;
    uint64_t X[3] = {0, 0, 0};
    const bool ok = active && fixpoint3(x, y, z, X);
    if (active && !ok) atomicOr(t.err, (unsigned)OT_DEV_OUTSIDE);
    if (!ok) {
        out[0] = out[1] = out[2] = qnan<T>();
        return -1;
    }
    const int h = host_in >= 0 ? host_in
                               : search<LEARNED>(t,
                                                 morton3((uint32_t)(X[0] >> 32), (uint32_t)(X[1] >> 32),
                                                         (uint32_t)(X[2] >> 32)));
    const int l = t.level[h];
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
    const uint64_t span = key_span(l);
    // level-mates: anchors, weights; a sibling of the host cell is usually h + (difference of
    // child numbers), which one key comparison proves (keys are unique); the rest are searched
    uint64_t anc[8];
    T w[8];
    int a[8];
    unsigned self_mask = 0;
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
        if (self) {
            self_mask |= 1u << corner;
            continue;
        }
        int g = -1;
        if ((m[0] >> 1) == (c[0] >> 1) && (m[1] >> 1) == (c[1] >> 1) && (m[2] >> 1) == (c[2] >> 1)) {
            const int gi = h + ((m[0] & 1) | ((m[1] & 1) << 1) | ((m[2] & 1) << 2)) -
                           ((c[0] & 1) | ((c[1] & 1) << 1) | ((c[2] & 1) << 2));
            if (gi >= 0 && gi < t.n && ldg_key(t.key + gi) == anc[corner]) g = gi;
        }
        a[corner] = g >= 0 ? g : search<LEARNED>(t, anc[corner]);
    }
    T acc0 = T(0), acc1 = T(0), acc2 = T(0);
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
        const int ak = a[corner];
        T v0, v1, v2;
        if (((self_mask >> corner) & 1u) || (int)t.level[ak] <= l) {
            const auto f = V::load(field, ak);
            v0 = f.x, v1 = f.y, v2 = f.z;
        } else {
            // refined: its leaves are [ak, e); e is the leaf that starts right after the cell
            const uint64_t endkey = anc[corner] + span;
            int e;
            if (endkey >> 63) {
                e = t.n;
            } else if (l <= t.lmap_level) {
                const uint32_t ca = (uint32_t)(endkey >> (3 * (MAXLEVEL - t.lmap_level)));
                e = (int)t.lmap[ca];
            } else {
                e = search<LEARNED>(t, endkey);
            }
            const double4 pa = P[ak], pe = P[e];
            const double sc = exp2_pos(3 * l);
            v0 = (T)((pe.x - pa.x) * sc);
            v1 = (T)((pe.y - pa.y) * sc);
            v2 = (T)((pe.z - pa.z) * sc);
        }
        acc0 += w[corner] * v0;
        acc1 += w[corner] * v1;
        acc2 += w[corner] * v2;
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

// Parent blocks (2x2x2 cells of level lmax, i.e. cells of level lmax-1) overlapping the
// delta-kernel stencil whose first cell is i0.  For each one, one search finds its first
// child; a parent whose first child is a leaf of level lmax has all 8 children as
// consecutive leaves.  A parent in the same grandparent as the last one found is usually 8
// leaves per child-number step away, which one key comparison proves.  The visitor gets
// (a0, bx, by, bz, P) with a0 the first child's index, or -1 when the parent is outside the
// cube or not refined to the finest level.
template <int K, bool LEARNED, typename PVisit>
__device__ __forceinline__ void visit_parents(const TreeView& t, const int i0[3], PVisit&& pvisit) {
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
    int prevP[3] = {-1, -1, -1}, prev_a0 = -1;
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
                    if (a < 0) a = search<LEARNED>(t, anchor);
                    if (ldg_key(t.key + a) == anchor && t.level[a] == t.lmax) {
                        a0 = a;
                        prevP[0] = P[0], prevP[1] = P[1], prevP[2] = P[2];
                        prev_a0 = a;
                    }
                }
                pvisit(a0, bx, by, bz, P);
            }
}

// The stencil cells themselves: the visitor gets (leaf, ax, ay, az) for each valid stencil
// cell.  Returns false when some stencil cell was outside the cube or not a finest-level leaf
// (its weight is dropped).
template <int K, bool LEARNED, typename Visit>
__device__ __forceinline__ bool visit_stencil(const TreeView& t, const int i0[3], Visit&& visit) {
    constexpr int W = Stencil<K>::W;
    bool ok_all = true;
    visit_parents<K, LEARNED>(t, i0, [&](int a0, int, int, int, const int P[3]) {
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
    });
    return ok_all;
}

// Delta-kernel interpolation at one marker (Sec. 2.2, Eq. ibm_interpolate).  Returns the host
// leaf (-1 outside the cube).
template <typename T, int K, bool LEARNED>
__device__ __forceinline__ int delta_point(const TreeView& t, const T* __restrict__ field, double x, double y, double z, bool want_host,
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
    const bool ok = visit_stencil<K, LEARNED>(t, i0, [&](int leaf, int ax, int ay, int az) {
        const T wt = w[0][ax] * w[1][ay] * w[2][az];
        const auto f = V::load(field, leaf);
        a0 += wt * f.x;
        a1 += wt * f.y;
        a2 += wt * f.z;
        if (ax == hc[0] && ay == hc[1] && az == hc[2]) host = leaf;
    });
    if (!ok) atomicOr(t.err, (unsigned)OT_DEV_STENCIL);
    if (want_host && host < 0)
        host = search_plain(t, morton3((uint32_t)(X[0] >> 32), (uint32_t)(X[1] >> 32), (uint32_t)(X[2] >> 32)));
    out[0] = a0;
    out[1] = a1;
    out[2] = a2;
    return host;
}

} // namespace ot
