// ot_points.cuh -- per-point device routines: host search, trilinear interpolation with
// level-mates, delta-kernel interpolation and stencil enumeration.  Used by the single-op
// kernels, the persistent batched kernel and the spreading kernels.
#pragma once

#include "ot_common.cuh"

namespace ot {

__device__ __forceinline__ int floordiv2(int v) { return v >> 1; } // arithmetic shift: floor

template <typename T> __device__ __forceinline__ T qnan();
template <> __device__ __forceinline__ float qnan<float>() { return __int_as_float(0x7fc00000); }
template <> __device__ __forceinline__ double qnan<double>() { return __longlong_as_double(0x7ff8000000000000LL); }

// Trilinear interpolation at one point (Sec. 2.3.2) with the level-mate rule:
//   host leaf of level l, cell c; t_d = x_d 2^l - (c_d + 1/2); s_d = sign(t_d) (+1 at 0);
//   level-mates c + {0, s_d}; weights prod (1 - |t_d|) or |t_d|;
//   level-mate value: leaf of level l -> its value; inside a coarser leaf -> that leaf's value;
//   refined -> volume-weighted mean of its leaves; outside the cube -> host index on that axis.
// Returns the host leaf (-1 outside the cube; out = NaN).
template <typename T, bool LEARNED>
__device__ __forceinline__ int trilinear_point(const TreeView& t, const RootModel& rm, const uint64_t* s_sample,
                                               const T* __restrict__ field, double x, double y, double z, int host_in,
                                               T out[3]) {
    using V = Vec4<T>;
    uint32_t q[3];
    if (!quantise(x, y, z, q[0], q[1], q[2])) {
        out[0] = out[1] = out[2] = qnan<T>();
        atomicOr(t.err, (unsigned)OT_DEV_OUTSIDE);
        return -1;
    }
    const int h = host_in >= 0 ? host_in : search<LEARNED>(t, rm, s_sample, morton3(q[0], q[1], q[2]));
    const int l = t.level[h];
    const int sh = MAXLEVEL - l;
    const int ncell = 1 << l;
    const double p[3] = {x, y, z};
    const double sc = (double)ncell;
    int c[3], sg[3];
    T at[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        c[d] = (int)(q[d] >> sh);
        const double td = p[d] * sc - ((double)c[d] + 0.5);
        sg[d] = td >= 0.0 ? 1 : -1;
        at[d] = (T)fabs(td);
    }
    T acc0 = T(0), acc1 = T(0), acc2 = T(0);
    const uint64_t span = key_span(l);
#pragma unroll 1
    for (int corner = 0; corner < 8; ++corner) {
        int m[3];
        T w = T(1);
        bool self = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int off = (corner >> d) & 1;
            int v = c[d] + off * sg[d];
            if (v < 0 || v >= ncell) v = c[d];
            m[d] = v;
            self = self && (v == c[d]);
            w *= off ? at[d] : T(1) - at[d];
        }
        T v0, v1, v2;
        if (self) {
            auto f = V::load(field, h);
            v0 = f.x, v1 = f.y, v2 = f.z;
        } else {
            const uint64_t anchor =
                morton3((uint32_t)m[0] << sh, (uint32_t)m[1] << sh, (uint32_t)m[2] << sh);
            const int a = search<LEARNED>(t, rm, s_sample, anchor);
            const int la = t.level[a];
            if (la <= l) {
                auto f = V::load(field, a);
                v0 = f.x, v1 = f.y, v2 = f.z;
            } else {
                // refined: leaves with keys in [anchor, anchor + span), weight 8^-(level - l)
                v0 = v1 = v2 = T(0);
                const uint64_t end = anchor + span;
                int b = a, it = 0;
                for (; b < t.n && it < OT_REFINED_CAP; ++b, ++it) {
                    if (ldg_key(t.key + b) >= end) break;
                    const T vol = (T)ldexp(1.0, -3 * ((int)t.level[b] - l));
                    auto f = V::load(field, b);
                    v0 += vol * f.x;
                    v1 += vol * f.y;
                    v2 += vol * f.z;
                }
                if (it >= OT_REFINED_CAP) atomicOr(t.err, (unsigned)OT_DEV_REFINED_CAP);
            }
        }
        acc0 += w * v0;
        acc1 += w * v1;
        acc2 += w * v2;
    }
    out[0] = acc0;
    out[1] = acc1;
    out[2] = acc2;
    return h;
}

// Delta-kernel stencil around one point on the finest level.  For every parent block (2x2x2
// cells of level lmax) that overlaps the stencil, one search finds its first child; a parent
// whose first child is a leaf of level lmax has all 8 children as consecutive leaves.  The
// visitor gets (leaf, weight index ax, ay, az) for each valid stencil cell.  Returns false
// when some stencil cell was outside the cube or not a finest-level leaf.
template <int K, bool LEARNED, typename Visit>
__device__ __forceinline__ bool visit_stencil(const TreeView& t, const RootModel& rm, const uint64_t* s_sample,
                                              const int i0[3], Visit&& visit) {
    constexpr int W = Stencil<K>::W;
    const int lp = t.lmax - 1;          // parent level
    const int np_cells = 1 << lp;       // parents per axis
    const int shp = MAXLEVEL - lp;
    int p0[3], pn[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        p0[d] = floordiv2(i0[d]);
        pn[d] = floordiv2(i0[d] + W - 1) - p0[d] + 1;
    }
    bool ok_all = true;
    for (int bz = 0; bz < pn[2]; ++bz)
        for (int by = 0; by < pn[1]; ++by)
            for (int bx = 0; bx < pn[0]; ++bx) {
                const int P[3] = {p0[0] + bx, p0[1] + by, p0[2] + bz};
                const bool inside = P[0] >= 0 && P[1] >= 0 && P[2] >= 0 && P[0] < np_cells && P[1] < np_cells &&
                                    P[2] < np_cells;
                int a0 = -1;
                if (inside && t.lmax > 0) {
                    const uint64_t anchor =
                        morton3((uint32_t)P[0] << shp, (uint32_t)P[1] << shp, (uint32_t)P[2] << shp);
                    const int a = search<LEARNED>(t, rm, s_sample, anchor);
                    if (ldg_key(t.key + a) == anchor && t.level[a] == t.lmax) a0 = a;
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

// Stencil origin and per-axis weights of a point at X (finest spacing 2^-lmax).
template <int K, typename T>
__device__ __forceinline__ void stencil_weights(int lmax, double x, double y, double z, int i0[3],
                                                T w[3][Stencil<K>::W]) {
    constexpr int W = Stencil<K>::W;
    const double sc = ldexp(1.0, lmax);
    const double s[3] = {x * sc - 0.5, y * sc - 0.5, z * sc - 0.5};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        i0[d] = Stencil<K>::first(s[d]);
#pragma unroll
        for (int a = 0; a < W; ++a) w[d][a] = Stencil<K>::template phi<T>((T)(s[d] - (double)(i0[d] + a)));
    }
}

// Delta-kernel interpolation at one marker (Sec. 2.2, Eq. ibm_interpolate).  Returns the host
// leaf (-1 outside the cube).
template <typename T, int K, bool LEARNED>
__device__ __forceinline__ int delta_point(const TreeView& t, const RootModel& rm, const uint64_t* s_sample,
                                           const T* __restrict__ field, double x, double y, double z, bool want_host,
                                           T out[3]) {
    using V = Vec4<T>;
    constexpr int W = Stencil<K>::W;
    uint32_t q[3];
    if (!quantise(x, y, z, q[0], q[1], q[2])) {
        out[0] = out[1] = out[2] = qnan<T>();
        atomicOr(t.err, (unsigned)OT_DEV_OUTSIDE);
        return -1;
    }
    int i0[3];
    T w[3][W];
    stencil_weights<K, T>(t.lmax, x, y, z, i0, w);
    // host cell of level lmax: floor(X 2^lmax), one of the stencil cells
    const int sh = MAXLEVEL - t.lmax;
    const int hc[3] = {(int)(q[0] >> sh) - i0[0], (int)(q[1] >> sh) - i0[1], (int)(q[2] >> sh) - i0[2]};
    int host = -1;
    T a0 = T(0), a1 = T(0), a2 = T(0);
    const bool ok = visit_stencil<K, LEARNED>(t, rm, s_sample, i0, [&](int leaf, int ax, int ay, int az) {
        const T wt = w[0][ax] * w[1][ay] * w[2][az];
        auto f = V::load(field, leaf);
        a0 += wt * f.x;
        a1 += wt * f.y;
        a2 += wt * f.z;
        if (ax == hc[0] && ay == hc[1] && az == hc[2]) host = leaf;
    });
    if (!ok) atomicOr(t.err, (unsigned)OT_DEV_STENCIL);
    if (want_host && host < 0) host = search_plain(t, s_sample, morton3(q[0], q[1], q[2]));
    out[0] = a0;
    out[1] = a1;
    out[2] = a2;
    return host;
}

} // namespace ot
