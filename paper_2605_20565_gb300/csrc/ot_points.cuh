// ot_points.cuh -- per-point device routines: delta-kernel interpolation and stencil
// enumeration on exact fixed-point coordinates (the trilinear routine, which searches
// cooperatively across the warp, is in ot_queue.cuh).
// Used by the single-op kernels, the persistent batched kernel and the spreading kernels.
#pragma once

#include "ot_common.cuh"

namespace ot {

__device__ __forceinline__ int floordiv2(int v) { return v >> 1; } // arithmetic shift: floor

template <typename T> __device__ __forceinline__ T qnan();
template <> __device__ __forceinline__ float qnan<float>() { return __int_as_float(0x7fc00000); }
template <> __device__ __forceinline__ double qnan<double>() { return __longlong_as_double(0x7ff8000000000000LL); }


// First cell of level l in the pyramid of cell means: sum_{k<l} 8^k = (8^l - 1) / 7, the octal
// number 11...1 of l digits, i.e. the top l of the 21 octal ones of 0x1249249249249249 (no
// 64-bit division).
__device__ __forceinline__ long long pyr_offset(int l) { return (long long)(0x1249249249249249ULL >> (3 * (21 - l))); }

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
// delta-kernel stencil whose first cell is i0.  With the parent-block table, the middle block's
// row gives every block's first child; otherwise one search per block finds it.  A parent
// whose first child is a leaf of level lmax has all 8 children as consecutive leaves.  A parent in the same grandparent as the last one found is usually 8
// leaves per child-number step away, which one key comparison proves.  The visitor gets
// (a0, bx, by, bz, P) with a0 the first child's index, or -1 when the parent is outside the
// cube (a periodic cube wraps it instead) or not refined to the finest level.
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
    if (t.pnbr) {
        // the parent-block table: every stencil block lies within one block of the middle one,
        // whose row gives all their first children -- one lookup and one row of loads
        int pm[3], qm[3];
        bool inside = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            pm[d] = p0[d] + (pn[d] == 3 ? 1 : 0);
            qm[d] = t.periodic ? (pm[d] + np_cells) & (np_cells - 1) : pm[d];
            inside = inside && qm[d] >= 0 && qm[d] < np_cells;
        }
        int am = -1;
        if (inside) {
            const uint64_t anchor = morton3((uint32_t)qm[0] << shp, (uint32_t)qm[1] << shp, (uint32_t)qm[2] << shp);
            const int a = search<LEARNED>(t, anchor);
            if (ldg_key(t.key + a) == anchor && t.level[a] == t.lmax) am = a;
        }
        if (am >= 0) {  // else (the middle block is not refined to the finest level) the walk below
            const int* __restrict__ row = t.pnbr + 32 * (size_t)(am >> 3);
            for (int bz = 0; bz < pn[2]; ++bz)
                for (int by = 0; by < pn[1]; ++by)
                    for (int bx = 0; bx < pn[0]; ++bx) {
                        const int P[3] = {p0[0] + bx, p0[1] + by, p0[2] + bz};
                        const int k = (P[0] - pm[0] + 1) + 3 * (P[1] - pm[1] + 1) + 9 * (P[2] - pm[2] + 1);
                        pvisit(__ldg(row + k), bx, by, bz, P);
                    }
            return;
        }
    }
    int prevP[3] = {-1, -1, -1}, prev_a0 = -1;
    for (int bz = 0; bz < pn[2]; ++bz)
        for (int by = 0; by < pn[1]; ++by)
            for (int bx = 0; bx < pn[0]; ++bx) {
                const int P[3] = {p0[0] + bx, p0[1] + by, p0[2] + bz};
                // the parent's own index (wrapped around a periodic cube); P stays unwrapped for
                // the stencil offsets the visitor computes
                int Q[3] = {P[0], P[1], P[2]};
                if (t.periodic)
#pragma unroll
                    for (int d = 0; d < 3; ++d) Q[d] = (Q[d] + np_cells) & (np_cells - 1);
                const bool inside = Q[0] >= 0 && Q[1] >= 0 && Q[2] >= 0 && Q[0] < np_cells && Q[1] < np_cells &&
                                    Q[2] < np_cells;
                int a0 = -1;
                if (inside) {
                    const uint64_t anchor =
                        morton3((uint32_t)Q[0] << shp, (uint32_t)Q[1] << shp, (uint32_t)Q[2] << shp);
                    int a = -1;
                    if (prev_a0 >= 0 && (Q[0] >> 1) == (prevP[0] >> 1) && (Q[1] >> 1) == (prevP[1] >> 1) &&
                        (Q[2] >> 1) == (prevP[2] >> 1)) {
                        const int g = prev_a0 + 8 * (((Q[0] & 1) | ((Q[1] & 1) << 1) | ((Q[2] & 1) << 2)) -
                                                     ((prevP[0] & 1) | ((prevP[1] & 1) << 1) | ((prevP[2] & 1) << 2)));
                        if (g >= 0 && g < t.n && ldg_key(t.key + g) == anchor) a = g;
                    }
                    if (a < 0) a = search<LEARNED>(t, anchor);
                    if (ldg_key(t.key + a) == anchor && t.level[a] == t.lmax) {
                        a0 = a;
                        prevP[0] = Q[0], prevP[1] = Q[1], prevP[2] = Q[2];
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

// w[i] for a run-time stencil index i (0 <= i < W) by register selects, not an indexed (local
// memory) load.
template <int W, typename T>
__device__ __forceinline__ T sel_w(const T (&w)[W], int i) {
    T r = w[0];
#pragma unroll
    for (int k = 1; k < W; ++k) r = i == k ? w[k] : r;
    return r;
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
        const T wt = sel_w<W>(w[0], ax) * sel_w<W>(w[1], ay) * sel_w<W>(w[2], az);
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
