// ot_common.cuh -- device building blocks shared by the library's kernels: Morton keys,
// FP64 quantisation, host-cell search (plain and learned), delta functions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "octtrack.h"

namespace ot {

constexpr int MAXLEVEL = 21;
constexpr int MLP_H = 32;
constexpr int MLP_NPARAM = 3 * MLP_H + 1;

// ------------------------------------------------------------------------------------------
// Morton keys: x bit b -> key bit 3b, y -> 3b+1, z -> 3b+2 (the Z-order of p4est, Sec. 3.1).
// ------------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t part1by2(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffULL;
    x = (x | (x << 16)) & 0x1f0000ff0000ffULL;
    x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
    x = (x | (x << 2)) & 0x1249249249249249ULL;
    return x;
}
__host__ __device__ __forceinline__ uint32_t compact1by2(uint64_t x) {
    x &= 0x1249249249249249ULL;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ULL;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00fULL;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffULL;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffULL;
    x = (x ^ (x >> 32)) & 0x1fffffULL;
    return (uint32_t)x;
}
__host__ __device__ __forceinline__ uint64_t morton3(uint32_t x, uint32_t y, uint32_t z) {
    return part1by2(x) | (part1by2(y) << 1) | (part1by2(z) << 2);
}
__host__ __device__ __forceinline__ void demorton3(uint64_t k, uint32_t& x, uint32_t& y, uint32_t& z) {
    x = compact1by2(k);
    y = compact1by2(k >> 1);
    z = compact1by2(k >> 2);
}
// Number of MAXLEVEL keys covered by a leaf of level l: 8^(21-l).
__host__ __device__ __forceinline__ uint64_t key_span(int l) { return 1ULL << (3 * (MAXLEVEL - l)); }

// ------------------------------------------------------------------------------------------
// Exact fixed-point coordinates, integer operations only.
// X = floor(x 2^53) is read off the IEEE-754 bits of x: every cell index and in-cell fraction
// the path needs is a shift of X, so the integer cell of a point (Algorithm 1, get_cell_at:
// floor(x 2^level)) is exactly the FP64 floor, faces go to the upper cell, and no FP64
// arithmetic (a slow pipe on this GPU) is spent on it.
// ------------------------------------------------------------------------------------------
// False for x outside [0,1) or NaN; -0.0 counts as 0 (it compares equal to 0).
__device__ __forceinline__ bool fixpoint(double x, uint64_t& X) {
    const uint64_t u = (uint64_t)__double_as_longlong(x);
    X = 0;
    if (u == 0x8000000000000000ULL) return true;  // -0.0
    if (u >> 63) return false;                      // negative
    const int e = (int)(u >> 52);                   // biased exponent
    if (e >= 1023) return false;                    // >= 1, inf, NaN
    if (e == 0) return true;                        // +0, subnormal: floor(x 2^53) = 0
    const uint64_t m = (u & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
    const int sh = 1022 - e;                        // x 2^53 = m 2^(e - 1022)
    X = sh >= 64 ? 0 : (m >> sh);
    return true;
}
__device__ __forceinline__ bool fixpoint3(double x, double y, double z, uint64_t X[3]) {
    const bool a = fixpoint(x, X[0]), b = fixpoint(y, X[1]), c = fixpoint(z, X[2]);
    return a && b && c;
}
// floor(x 2^l), l <= 21.
__device__ __forceinline__ uint32_t fix_cell(uint64_t X, int l) { return (uint32_t)(X >> (53 - l)); }
// The top 24 bits of the fraction of x 2^l.
__device__ __forceinline__ uint32_t fix_frac24(uint64_t X, int l) { return (uint32_t)(X >> (29 - l)) & 0xFFFFFFu; }
// Offset from the centre of the level-l cell, frac(x 2^l) - 1/2: exact in FP64 from all bits,
// from the top 24 fraction bits in FP32 (itself exact: 24 significant bits).
template <typename T> __device__ __forceinline__ T fix_offset(uint64_t X, int l);
template <> __device__ __forceinline__ float fix_offset<float>(uint64_t X, int l) {
    return __fmaf_rn((float)fix_frac24(X, l), 0x1p-24f, -0.5f);
}
template <> __device__ __forceinline__ double fix_offset<double>(uint64_t X, int l) {
    const uint64_t f = X & ((1ULL << (53 - l)) - 1ULL);
    return ldexp((double)f, l - 53) - 0.5;
}
// Whether the point lies in the upper half of its level-l cell (offset >= 0): one bit of X.
__device__ __forceinline__ bool fix_upper_half(uint64_t X, int l) { return (X >> (52 - l)) & 1ULL; }

// Unsigned 64-bit integer -> float, rounding toward zero, built from the bits (no 64-bit
// conversion instruction).  Used identically at index training and query time.
__device__ __forceinline__ float u64_to_float_rz(uint64_t v) {
    if (v == 0) return 0.0f;
    const int lz = __clzll((long long)v);
    const int e = 63 - lz;                                   // position of the leading one
    const uint32_t mant = (uint32_t)((v << lz) >> 40) & 0x7FFFFFu;  // 23 bits after it
    return __int_as_float(((e + 127) << 23) | (int)mant);
}
__device__ __forceinline__ float i64_to_float_rz(int64_t v) {
    return v < 0 ? -u64_to_float_rz(0ULL - (uint64_t)v) : u64_to_float_rz((uint64_t)v);
}
// 2^-k as float for 0 <= k < 126.
__device__ __forceinline__ float exp2_neg(int k) { return __int_as_float((127 - k) << 23); }

// ------------------------------------------------------------------------------------------
// Views passed by value to kernels.
// ------------------------------------------------------------------------------------------
struct __align__(32) LeafModel {
    uint64_t base; // smallest key routed to the model (prediction input is key - base)
    float slope;
    float icpt; // relative to `first`
    int err_lo; // window below the prediction
    int err_hi; // window above the prediction
    int first;  // index of the model's first key (prediction origin)
    int count;  // keys routed here; a model no key routed to is filled (err_lo = -1, below)
};

struct RootModel {
    int kind;   // OT_ROOT_LINEAR / OT_ROOT_MLP
    int n_models;
    float a, b; // linear root: y = a + b x
    float w1[MLP_H], b1[MLP_H], w2[MLP_H];
    float b2;
    // the trained network in its piecewise-linear form (a 1 -> H ReLU -> 1 network is linear
    // between the breakpoints -b1/w1 of its units): nknot sorted breakpoints inside (0, 1) and
    // one line y = sa x + sb per segment.  Index building and queries both evaluate this form.
    int nknot;
    float knot[MLP_H];
    float sa[MLP_H + 1], sb[MLP_H + 1];
};

struct TreeView {
    const uint64_t* __restrict__ key;
    const uint8_t* __restrict__ level;
    int n;
    int lmin, lmax;
    // level map: lmap[c] = the leaf holding the anchor of cell c of level lmap_level (the
    // top levels of the tree, staged as a dense table)
    const uint32_t* __restrict__ lmap;
    int lmap_level;
    // per level-map cell, the shape of its subtree when it is at most 3 levels deep (see
    // desc_leaf); null when not built
    const uint4* __restrict__ desc;
    const uint8_t* __restrict__ lmap_lv;  // level of leaf lmap[c]
    int pyr_level;  // deepest level of the pyramid of cell means (refined trilinear level-mates)
    int periodic;   // the unit cube is periodic: stencils and level-mates wrap around
    // level-mate table: for leaf h and octant o, the 8 value slots of its trilinear
    // level-mates at mates[2 (8h + o)], two uint4 (null when not built)
    const uint4* __restrict__ mates;
    // parent-block table: row b = first children of the 27 blocks around the block whose first
    // child is leaf 8b.. (32 entries per row), -1 where none (null when not built)
    const int* __restrict__ pnbr;
    // learned search: root -> (optional mid models) -> leaf models
    const RootModel* __restrict__ root;  // device copy
    const LeafModel* __restrict__ models;
    const LeafModel* __restrict__ mids;  // null for a two-stage index
    int n_leaf;                          // leaf models
    unsigned* err;                      // device error word
    unsigned long long* fallbacks;      // learned-query fallbacks
};

__device__ __forceinline__ uint64_t ldg_key(const uint64_t* p) { return __ldg(reinterpret_cast<const unsigned long long*>(p)); }

// Last index in [lo, lo+len) whose key <= q, given key[lo] <= q (branch-free halving).
__device__ __forceinline__ int search_range(const uint64_t* __restrict__ key, int lo, int len, uint64_t q) {
    while (len > 1) {
        int half = len >> 1;
        uint64_t k = ldg_key(key + lo + half);
        lo = (k <= q) ? lo + half : lo;
        len -= half;
    }
    return lo;
}

// Cell of the level map holding key q, and the leaf range [a, e) of that cell: a is the leaf
// holding the cell's anchor, e the one holding the next cell's.  One leaf covers the whole cell
// (and is the answer for every key in it) exactly when e - a <= 1: a refined cell holds at
// least 8 leaves, the first starting at its anchor.
__device__ __forceinline__ void map_range(const TreeView& t, uint64_t q, int& a, int& e, bool& covered) {
    const uint32_t c = (uint32_t)(q >> (3 * (MAXLEVEL - t.lmap_level)));
    a = (int)t.lmap[c];
    e = (c + 1 < (1u << (3 * t.lmap_level))) ? (int)t.lmap[c + 1] : t.n;
    covered = e - a <= 1;
}

// Plain host search (Algorithm 1's answer, upper bound - 1): the level map gives the leaf
// directly for a cell covered by one leaf, else the cell's range of leaves, which a
// branch-free binary search finishes (key[a] <= q: a holds the cell's anchor).
// Leaf holding key q inside an uncovered level-map cell (level L, first leaf a) whose subtree is
// at most 3 levels deep, from the cell's descriptor d: m1 (d.z bits 0-7) marks the refined
// children (level L+1, Morton child order), byte i of m2 (d.x | d.y << 32) the refined
// grandchildren of child i; every deeper cell is a leaf.  A refined child holds 8 + 7 popc(its
// m2 byte) leaves, so the leaves before child c1 number c1 + 7 popc(m1 below c1) + 7 popc(m2
// bytes below c1); inside a refined child the same count one level down, and inside a refined
// grandchild the great-grandchild's index.
// The leaf's level comes with it: L+1, L+2 or L+3 by the depth reached.
__device__ __forceinline__ int desc_leaf(uint4 d, int L, uint64_t q, int a, int& lv) {
    const uint32_t m1 = d.z & 0xFFu;
    const uint64_t m2 = ((uint64_t)d.y << 32) | d.x;
    const int c1 = (int)(q >> (3 * (MAXLEVEL - L - 1))) & 7;
    const uint64_t low = c1 ? (~0ULL >> (64 - 8 * c1)) : 0ULL;
    int idx = a + c1 + 7 * __popc(m1 & ((1u << c1) - 1u)) + 7 * __popcll(m2 & low);
    lv = L + 1;
    if ((m1 >> c1) & 1u) {
        const int c2 = (int)(q >> (3 * (MAXLEVEL - L - 2))) & 7;
        const uint32_t g = (uint32_t)(m2 >> (8 * c1)) & 0xFFu;
        idx += c2 + 7 * __popc(g & ((1u << c2) - 1u));
        lv = L + 2;
        if ((g >> c2) & 1u) {
            idx += (int)(q >> (3 * (MAXLEVEL - L - 3))) & 7;
            lv = L + 3;
        }
    }
    return idx;
}
constexpr uint32_t DESC_VALID = 0x100u;

// The cell's map entries and its descriptor are loaded together (one round trip).
__device__ __forceinline__ int search_plain(const TreeView& t, uint64_t q) {
    const uint32_t c = (uint32_t)(q >> (3 * (MAXLEVEL - t.lmap_level)));
    const int a = (int)t.lmap[c];
    const int e = (c + 1 < (1u << (3 * t.lmap_level))) ? (int)t.lmap[c + 1] : t.n;
    const uint4 d = t.desc ? __ldg(t.desc + c) : make_uint4(0u, 0u, 0u, 0u);
    if (e - a <= 1) return a;
    int lv;
    if (d.z & DESC_VALID) return desc_leaf(d, t.lmap_level, q, a, lv);
    return search_range(t.key, a, e - a, q);
}

// Input of the root model: key 2^-63 in FP32 (rounded toward zero).
__device__ __forceinline__ float key_to_x(uint64_t q) { return u64_to_float_rz(q) * 0x1p-63f; }

// Root model: predicted fractional position y ~ i/N of key q.
__device__ __forceinline__ float root_predict(const RootModel& r, uint64_t q) {
    const float x = key_to_x(q);
    if (r.kind == OT_ROOT_LINEAR) return __fadd_rn(r.a, __fmul_rn(r.b, x));
    // segment: the number of breakpoints <= x (branch-free halving over the sorted breakpoints)
    int s = 0;
#pragma unroll
    for (int step = 32; step > 0; step >>= 1)
        if (s + step <= r.nknot && r.knot[s + step - 1] <= x) s += step;
    return __fadd_rn(__fmul_rn(r.sa[s], x), r.sb[s]);
}
__device__ __forceinline__ int root_route(const RootModel& r, uint64_t q) {
    float y = root_predict(r, q) * (float)r.n_models;
    y = fminf(fmaxf(y, 0.0f), (float)(r.n_models - 1));
    return (int)y; // y >= 0: truncation is floor
}
// Leaf model prediction (integer), the same arithmetic at training and query time:
// first + floor(slope (q - base) + icpt), clamped to the model's own index range widened by
// one on each side (the answer for a key routed here lies there unless routing is not
// monotone, which the search verifies), then to [0, n).
__device__ __forceinline__ int leaf_predict(const LeafModel& m, uint64_t q, int n) {
    const float off = i64_to_float_rz((int64_t)(q - m.base));
    float p = __fadd_rn(__fmul_rn(m.slope, off), m.icpt);
    p = fminf(fmaxf(p, -1.0f), (float)m.count);
    const int pc = m.first + (int)floorf(p);
    return min(max(pc, 0), n - 1);
}

// Leaf model serving key q: the root's choice, or, with a middle stage, the mid model's
// position estimate scaled to the leaf count (integer, monotone within a mid model).
__device__ __forceinline__ int route_leaf(const RootModel& r, const LeafModel* mids, int n_leaf, int n, uint64_t q) {
    const int j = root_route(r, q);
    if (!mids) return j;
    const int pc = leaf_predict(mids[j], q, n);
    return (int)(((int64_t)pc * n_leaf) / n);
}

// Learned search inside a level-map cell [ca, ce) that one leaf does not cover: the models give
// a window [pc - err_lo - 1, pc + err_hi + 1], clamped to the cell, searched by halving; the
// answer a is verified by key[a] <= q < key[a+1], and a window that missed is answered by a
// binary search of the cell (counted as a fallback).  Out of line: one copy serves every call
// site, and the root network stays in device memory.
static __device__ __noinline__ int learned_in_cell(const uint64_t* __restrict__ key, const RootModel* __restrict__ root,
                                            const LeafModel* __restrict__ mids, const LeafModel* __restrict__ models,
                                            int n, int n_leaf, int ca, int ce, uint64_t q,
                                            unsigned long long* fallbacks, unsigned* err) {
    const int j = route_leaf(*root, mids, n_leaf, n, q);
    const LeafModel m = models[j];
    if (m.count > 0) {
        const int pc = leaf_predict(m, q, n);
        const int lo = max(pc - m.err_lo - 1, ca);
        const int hi = min(pc + m.err_hi + 1, ce - 1);
        if (lo <= hi) {
            const int a = search_range(key, lo, hi - lo + 1, q);
            const uint64_t a0 = ldg_key(key + a);
            const uint64_t a1 = a + 1 < n ? ldg_key(key + a + 1) : ~0ULL;
            if (a0 <= q && q < a1) return a;
        }
    }
    atomicAdd(fallbacks, 1ULL);
    atomicOr(err, (unsigned)OT_DEV_WINDOW);
    return search_range(key, ca, ce - ca, q);
}

// Learned host search: the level map first (a covered cell answers directly), the models
// inside an uncovered cell.
__device__ __forceinline__ int search_learned(const TreeView& t, uint64_t q) {
    int ca, ce;
    bool covered;
    map_range(t, q, ca, ce, covered);
    if (covered) return ca;
    return learned_in_cell(t.key, t.root, t.mids, t.models, t.n, t.n_leaf, ca, ce, q, t.fallbacks, t.err);
}

template <bool LEARNED>
__device__ __forceinline__ int search(const TreeView& t, uint64_t q) {
    if (LEARNED) return search_learned(t, q);
    return search_plain(t, q);
}


// ------------------------------------------------------------------------------------------
// Discrete delta functions (Sec. 2.2), argument in grid units.  Square-root arguments are
// written in the factored forms 2 - (2a-1)^2, 2 - (2a-3)^2 (Peskin) and 1 - 3(1-a)^2 (Roma),
// which equal the printed polynomials and lose less to cancellation in FP32.
// ------------------------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T dsqrt(T v);
template <> __device__ __forceinline__ float dsqrt<float>(float v) { return sqrtf(fmaxf(v, 0.0f)); }
template <> __device__ __forceinline__ double dsqrt<double>(double v) { return sqrt(fmax(v, 0.0)); }

template <typename T> __device__ __forceinline__ T phi_peskin4(T r) {
    T a = r < T(0) ? -r : r;
    if (a <= T(1)) {
        T e = T(2) * a - T(1);
        return (T(3) - T(2) * a + dsqrt<T>(T(2) - e * e)) * T(0.125);
    }
    if (a <= T(2)) {
        T e = T(2) * a - T(3);
        return (T(5) - T(2) * a - dsqrt<T>(T(2) - e * e)) * T(0.125);
    }
    return T(0);
}
template <typename T> __device__ __forceinline__ T phi_roma3(T r) {
    T a = r < T(0) ? -r : r;
    if (a <= T(0.5)) return (T(1) + dsqrt<T>(T(1) - T(3) * a * a)) * (T(1) / T(3));
    if (a <= T(1.5)) {
        T e = T(1) - a;
        return (T(5) - T(3) * a - dsqrt<T>(T(1) - T(3) * e * e)) * (T(1) / T(6));
    }
    return T(0);
}

// Stencil of one axis on the finest level.  With the point's finest cell c, the upper-half bit
// hi and the offset t = frac - 1/2 from the cell centre (cell j is centred at s = j when
// s = X 2^lmax - 1/2):
//   Peskin-4: cells floor(s) - 1 .. floor(s) + 2, floor(s) = c - 1 + hi; r_a = (2 - hi - a) + t;
//   Roma-3:   cells c - 1 .. c + 1 (nearest centre and its neighbours); r_a = (1 - a) + t.
template <int KERNEL> struct Stencil;
template <> struct Stencil<OT_PESKIN4> {
    static constexpr int W = 4;
    __device__ static int first(int c, int hi) { return c - 2 + hi; }
    template <typename T> __device__ static T r(int a, int hi, T t) { return (T)(2 - hi - a) + t; }
    template <typename T> __device__ static T phi(T r) { return phi_peskin4<T>(r); }
};
template <> struct Stencil<OT_ROMA3> {
    static constexpr int W = 3;
    __device__ static int first(int c, int hi) { (void)hi; return c - 1; }
    template <typename T> __device__ static T r(int a, int hi, T t) { (void)hi; return (T)(1 - a) + t; }
    template <typename T> __device__ static T phi(T r) { return phi_roma3<T>(r); }
};

// Per-leaf field vectors.
template <typename T> struct Vec4;
template <> struct Vec4<float> {
    using type = float4;
    __device__ static float4 load(const float* f, long long i) { return __ldg(reinterpret_cast<const float4*>(f) + i); }
};
struct __align__(32) dbl4 {
    double x, y, z, w;
};
template <> struct Vec4<double> {
    using type = dbl4;
    __device__ static dbl4 load(const double* f, long long i) {
        const double2* p = reinterpret_cast<const double2*>(f) + 2 * (size_t)i;
        double2 a = __ldg(p), b = __ldg(p + 1);
        return dbl4{a.x, a.y, b.x, b.y};
    }
};

} // namespace ot
