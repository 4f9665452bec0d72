// ot_spread.cu -- force spreading, the adjoint of the delta-kernel interpolation (Sec. 2.2):
//   f(cell) += sum_k F_k phi(rx) phi(ry) phi(rz) dV_k / h^3.
// OT_ATOMIC: each marker adds its stencil contributions with float atomics.
// OT_SORTED: each marker emits one 64-bit pair per overlapping parent block (2x2x2 finest
//   cells), (first child leaf << 32) | (k PS + slot); a stable radix sort by parent groups the
//   pairs of a block in marker order; one thread per block then recomputes the weights, sums
//   its 8 children in that order and adds each once to f (no atomics, bit-identical from run
//   to run and for any launch shape; per leaf the same sum in the same order as a per-cell
//   reduction).
#include <algorithm>

#include "ot_internal.h"
#include "ot_points.cuh"

namespace ot {

namespace {

constexpr uint64_t INVALID_HI = 0xFFFFFFFFull;

template <typename T> __device__ __forceinline__ void add3(T* f, int leaf, T a, T b, T c);
template <> __device__ __forceinline__ void add3<float>(float* f, int leaf, float a, float b, float c) {
    atomicAdd(reinterpret_cast<float4*>(f) + leaf, make_float4(a, b, c, 0.0f));
}
template <> __device__ __forceinline__ void add3<double>(double* f, int leaf, double a, double b, double c) {
    double* p = f + 4 * (size_t)leaf;
    atomicAdd(p, a);
    atomicAdd(p + 1, b);
    atomicAdd(p + 2, c);
}

template <typename T>
__device__ __forceinline__ T marker_volume(const T* __restrict__ dV, int64_t k, int lmax) {
    return dV ? dV[k] * (T)ldexp(1.0, 3 * lmax) : T(1);
}

template <typename T, int K>
__global__ void __launch_bounds__(256) k_spread_atomic(TreeView t, const double* __restrict__ x,
                                                       const double* __restrict__ y, const double* __restrict__ z,
                                                       const T* __restrict__ F, const T* __restrict__ dV, int64_t n,
                                                       T* __restrict__ f) {
    constexpr int W = Stencil<K>::W;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        uint64_t X[3];
        if (!fixpoint3(x[k], y[k], z[k], X)) {
            atomicOr(t.err, (unsigned)OT_DEV_OUTSIDE);
            continue;
        }
        int i0[3];
        T w[3][W];
        stencil_weights<K, T>(t.lmax, X, i0, w);
        const T vol = marker_volume(dV, k, t.lmax);
        const T F0 = F[k] * vol, F1 = F[n + k] * vol, F2 = F[2 * n + k] * vol;
        const bool ok = visit_stencil<K, false>(t, i0, [&](int leaf, int ax, int ay, int az) {
            const T wt = w[0][ax] * w[1][ay] * w[2][az];
            add3<T>(f, leaf, F0 * wt, F1 * wt, F2 * wt);
        });
        if (!ok) atomicOr(t.err, (unsigned)OT_DEV_STENCIL);
    }
}

// Parent slots per marker: the stencil spans up to PW parent blocks per axis.
template <int K> struct ParentSlots {
    static constexpr int PW = Stencil<K>::W == 4 ? 3 : 2;
    static constexpr int PS = PW * PW * PW;
};

// One pair per (marker, overlapping parent block): (first child leaf << 32) | (k PS + slot).
template <int K>
__global__ void __launch_bounds__(256) k_spread_emit(TreeView t, const double* __restrict__ x,
                                                     const double* __restrict__ y, const double* __restrict__ z,
                                                     int64_t n, uint64_t* __restrict__ pairs) {
    constexpr int PW = ParentSlots<K>::PW, PS = ParentSlots<K>::PS;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        uint64_t* out = pairs + k * PS;
        const uint64_t id0 = (uint64_t)k * PS;
        for (int sl = 0; sl < PS; ++sl) out[sl] = (INVALID_HI << 32) | (id0 + sl);
        uint64_t X[3];
        if (!fixpoint3(x[k], y[k], z[k], X)) {
            atomicOr(t.err, (unsigned)OT_DEV_OUTSIDE);
            continue;
        }
        int i0[3];
        for (int d = 0; d < 3; ++d)
            i0[d] = Stencil<K>::first((int)fix_cell(X[d], t.lmax), fix_upper_half(X[d], t.lmax) ? 1 : 0);
        bool ok = true;
        visit_parents<K, false>(t, i0, [&](int a0, int bx, int by, int bz, const int*) {
            if (a0 < 0) {
                ok = false;
                return;
            }
            const int sl = bx + PW * (by + PW * bz);
            out[sl] = ((uint64_t)(uint32_t)a0 << 32) | (id0 + sl);
        });
        if (!ok) atomicOr(t.err, (unsigned)OT_DEV_STENCIL);
    }
}

// Each thread owns a chunk of RC consecutive sorted pairs and reduces every run (all pairs of
// one parent block, markers in index order) that starts inside its chunk, reading past the
// chunk's end to finish its last run: balanced work, no compaction of run heads.  Each run
// accumulates its 8 children and adds each touched child to f once.
constexpr int RC = 64;

template <typename T, int K>
__global__ void __launch_bounds__(256) k_spread_reduce(const uint64_t* __restrict__ pairs, int64_t npairs, int lmax,
                                                       const double* __restrict__ x, const double* __restrict__ y,
                                                       const double* __restrict__ z, const T* __restrict__ F,
                                                       const T* __restrict__ dV, int64_t n, T* __restrict__ f) {
    constexpr int W = Stencil<K>::W;
    constexpr int PW = ParentSlots<K>::PW, PS = ParentSlots<K>::PS;
    const int64_t nchunks = (npairs + RC - 1) / RC;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nchunks;
         c += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = c * RC;
        const int64_t jend = min(j + RC, npairs);
        if (j > 0) {  // the run in progress at the chunk start belongs to an earlier chunk
            const uint32_t prev = (uint32_t)(pairs[j - 1] >> 32);
            while (j < jend && (uint32_t)(pairs[j] >> 32) == prev) ++j;
        }
        while (j < jend) {
            const uint32_t a0 = (uint32_t)(pairs[j] >> 32);
            if (a0 == (uint32_t)INVALID_HI) break;  // invalid pairs sort last
            T acc[8][3];
#pragma unroll
            for (int ch = 0; ch < 8; ++ch) acc[ch][0] = acc[ch][1] = acc[ch][2] = T(0);
            unsigned touched = 0;
            for (; j < npairs; ++j) {
                const uint64_t pj = pairs[j];
                if ((uint32_t)(pj >> 32) != a0) break;
                const uint32_t id = (uint32_t)pj;
                const int64_t k = id / PS;
                const int sl = (int)(id - (uint32_t)(k * PS));
                uint64_t X[3];
                fixpoint3(x[k], y[k], z[k], X);  // inside: the pair was emitted
                int i0[3];
                T w[3][W];
                stencil_weights<K, T>(lmax, X, i0, w);
                const int P[3] = {floordiv2(i0[0]) + sl % PW, floordiv2(i0[1]) + (sl / PW) % PW,
                                  floordiv2(i0[2]) + sl / (PW * PW)};
                const T vol = marker_volume(dV, k, lmax);
                const T F0 = F[k] * vol, F1 = F[n + k] * vol, F2 = F[2 * n + k] * vol;
#pragma unroll
                for (int ch = 0; ch < 8; ++ch) {
                    const int ax = 2 * P[0] + (ch & 1) - i0[0];
                    const int ay = 2 * P[1] + ((ch >> 1) & 1) - i0[1];
                    const int az = 2 * P[2] + ((ch >> 2) & 1) - i0[2];
                    if (ax < 0 || ay < 0 || az < 0 || ax >= W || ay >= W || az >= W) continue;
                    const T wt = w[0][ax] * w[1][ay] * w[2][az];
                    acc[ch][0] += F0 * wt;
                    acc[ch][1] += F1 * wt;
                    acc[ch][2] += F2 * wt;
                    touched |= 1u << ch;
                }
            }
#pragma unroll
            for (int ch = 0; ch < 8; ++ch) {
                if (!((touched >> ch) & 1u)) continue;
                T* fp = f + 4 * ((size_t)a0 + ch);
                fp[0] += acc[ch][0];
                fp[1] += acc[ch][1];
                fp[2] += acc[ch][2];
            }
        }
    }
}

// Per-marker record of the sorted spreading, written once by the emit pass: the stencil's
// per-axis weights, the marker's force times its volume factor, and the parity of the stencil's
// first cell per axis (which fixes where a parent block's children sit in the stencil).
template <typename T>
struct __align__(16) MarkerRec {
    T w[3][4];
    T F[3];
    int par;  // bit d: i0[d] & 1
};

// A marker's record in two 32-byte loads (sm_100 and later; FP32 records are 64 bytes and
// 64-byte aligned in the workspace), read-only path, default L2 priority; FP64 records whole.
template <typename T>
__device__ __forceinline__ MarkerRec<T> load_rec(const MarkerRec<T>* p) {
    return *p;
}
template <>
__device__ __forceinline__ MarkerRec<float> load_rec<float>(const MarkerRec<float>* p) {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
    float v[16];
    const float* q = reinterpret_cast<const float*>(p);
    asm("ld.global.nc.L2::cache_hint.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], %9;"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
        : "l"(q), "l"(pol));
    asm("ld.global.nc.L2::cache_hint.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], %9;"
        : "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11]), "=f"(v[12]), "=f"(v[13]), "=f"(v[14]), "=f"(v[15])
        : "l"(q + 8), "l"(pol));
    MarkerRec<float> r;
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
        for (int a = 0; a < 4; ++a) r.w[d][a] = v[4 * d + a];
    r.F[0] = v[12], r.F[1] = v[13], r.F[2] = v[14];
    r.par = __float_as_int(v[15]);
    return r;
}

// Parent blocks overlapping a marker's stencil (2 or 3 per axis for Peskin-4, by the parity
// of the stencil's first cell); 0 outside the cube.
template <int K>
__global__ void __launch_bounds__(256) k_spread_count(const double* __restrict__ x, const double* __restrict__ y,
                                                      const double* __restrict__ z, int64_t n, int lmax,
                                                      uint32_t* __restrict__ cnt) {
    constexpr int W = Stencil<K>::W;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        uint64_t X[3];
        uint32_t c = 0;
        if (fixpoint3(x[k], y[k], z[k], X)) {
            c = 1;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int i0 = Stencil<K>::first((int)fix_cell(X[d], lmax), fix_upper_half(X[d], lmax) ? 1 : 0);
                c *= (uint32_t)(floordiv2(i0 + W - 1) - floordiv2(i0) + 1);
            }
        }
        cnt[k] = c;
    }
}

// Emit pass: the marker's record and, from offset off[k], one pair per overlapping parent block
// in slot order (a block outside the cube or not refined to the finest level gets an invalid
// pair, which sorts last).
template <typename T, int K>
__global__ void __launch_bounds__(256) k_spread_emit_rec(TreeView t, const double* __restrict__ x,
                                                         const double* __restrict__ y, const double* __restrict__ z,
                                                         const T* __restrict__ F, const T* __restrict__ dV,
                                                         int64_t n, const uint32_t* __restrict__ off,
                                                         uint64_t* __restrict__ pairs,
                                                         MarkerRec<T>* __restrict__ recs) {
    constexpr int W = Stencil<K>::W;
    constexpr int PW = ParentSlots<K>::PW, PS = ParentSlots<K>::PS;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        uint64_t* out = pairs + off[k];
        const uint64_t id0 = (uint64_t)k * PS;
        uint64_t X[3];
        if (!fixpoint3(x[k], y[k], z[k], X)) {
            atomicOr(t.err, (unsigned)OT_DEV_OUTSIDE);
            continue;
        }
        int i0[3];
        T w[3][W];
        stencil_weights<K, T>(t.lmax, X, i0, w);
        MarkerRec<T> r;
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int a = 0; a < 4; ++a) r.w[d][a] = a < W ? w[d][a] : T(0);
        const T vol = marker_volume(dV, k, t.lmax);
        r.F[0] = F[k] * vol, r.F[1] = F[n + k] * vol, r.F[2] = F[2 * n + k] * vol;
        r.par = (i0[0] & 1) | ((i0[1] & 1) << 1) | ((i0[2] & 1) << 2);
        recs[k] = r;
        bool ok = true;
        int m = 0;
        visit_parents<K, false>(t, i0, [&](int a0, int bx, int by, int bz, const int*) {
            const int sl = bx + PW * (by + PW * bz);
            if (a0 < 0) ok = false;
            out[m++] = ((a0 < 0 ? INVALID_HI : (uint64_t)(uint32_t)a0) << 32) | (id0 + sl);
        });
        if (!ok) atomicOr(t.err, (unsigned)OT_DEV_STENCIL);
    }
}

// Reduce pass over the sorted pairs, reading each pair's marker record instead of recomputing
// its weights: a child (cx, cy, cz) of parent slot (bx, by, bz) is stencil cell 2 b + c - parity
// on each axis.  Same products, same order as k_spread_reduce: the result is bit-identical.
// Work split: runs (all pairs of one parent block) average ~50 pairs (1 to ~100), so instead
// of a thread per fixed chunk (idle when no run starts in it) every warp owns an equal range
// of the sorted pairs, lists the runs that start in it (32 pairs per ballot) and hands them
// to its lanes round-robin in batches of up to 256, each lane reducing whole runs in order
// (reading past the range's end to finish its last one).
constexpr int RB = 256;  // run heads per warp batch

template <typename T, int K>
__device__ __forceinline__ void reduce_run(const uint64_t* __restrict__ pairs, int64_t npairs, int64_t j,
                                           const MarkerRec<T>* __restrict__ recs, T* __restrict__ f) {
    constexpr int W = Stencil<K>::W;
    constexpr int PW = ParentSlots<K>::PW, PS = ParentSlots<K>::PS;
    const uint32_t a0 = (uint32_t)(pairs[j] >> 32);
    // the 8 children's lines of f, fetched into L2 now: the read-modify-write at the run's end
    // then hits L2 instead of waiting on DRAM (runs are short on trees with many markers)
    {
        const char* fa = reinterpret_cast<const char*>(f + 4 * (size_t)a0);
        constexpr int span = 8 * 4 * (int)sizeof(T);
#pragma unroll
        for (int o = 0; o < span; o += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(fa + o));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(fa + span - 1));
    }
    T acc[8][3];
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) acc[ch][0] = acc[ch][1] = acc[ch][2] = T(0);
    unsigned touched = 0;
    for (; j < npairs; ++j) {
        const uint64_t pj = pairs[j];
        if ((uint32_t)(pj >> 32) != a0) break;
        const uint32_t id = (uint32_t)pj;
        const int64_t k = id / PS;
        const int sl = (int)(id - (uint32_t)(k * PS));
        const MarkerRec<T> r = load_rec<T>(recs + k);
        const int b[3] = {sl % PW, (sl / PW) % PW, sl / (PW * PW)};
        // per axis, the two children's stencil cells 2 b + e - parity (register selects)
        T wa[3][2];
        bool va[3][2];
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int cc = 2 * b[d] + e - ((r.par >> d) & 1);
                va[d][e] = cc >= 0 && cc < W;
                wa[d][e] = cc == 1 ? r.w[d][1] : cc == 2 ? r.w[d][2] : cc == 3 ? r.w[d][3] : r.w[d][0];
            }
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
            const int ex = ch & 1, ey = (ch >> 1) & 1, ez = (ch >> 2) & 1;
            if (!(va[0][ex] && va[1][ey] && va[2][ez])) continue;
            const T wt = wa[0][ex] * wa[1][ey] * wa[2][ez];
            acc[ch][0] += r.F[0] * wt;
            acc[ch][1] += r.F[1] * wt;
            acc[ch][2] += r.F[2] * wt;
            touched |= 1u << ch;
        }
    }
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) {
        if (!((touched >> ch) & 1u)) continue;
        T* fp = f + 4 * ((size_t)a0 + ch);
        fp[0] += acc[ch][0];
        fp[1] += acc[ch][1];
        fp[2] += acc[ch][2];
    }
}

template <typename T, int K>
__global__ void __launch_bounds__(256) k_spread_reduce_rec(const uint64_t* __restrict__ pairs,
                                                           const uint32_t* __restrict__ d_np,
                                                           const MarkerRec<T>* __restrict__ recs,
                                                           T* __restrict__ f) {
    __shared__ uint32_t s_heads[256 / 32][RB];
    __shared__ uint32_t s_len[256 / 32][RB];
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    uint32_t* heads = s_heads[threadIdx.x >> 5];
    uint32_t* len = s_len[threadIdx.x >> 5];
    const int64_t npairs = *d_np;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t wg = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t j0 = npairs * wg / nwarps, j1 = npairs * (wg + 1) / nwarps;
    int nh = 0;  // listed run heads (warp-uniform)
    // the listed runs, longest first (lengths up to the scan position end; the last one's is a
    // lower bound), dealt to the lanes in snake order so that every lane gets about the same
    // number of pairs
    auto run_batch = [&](int64_t end) {
        __syncwarp();
        int P = 32;
        while (P < nh) P <<= 1;
        for (int r = lane; r < P; r += 32) {
            if (r < nh) {
                const int64_t e = r + 1 < nh ? (int64_t)heads[r + 1] : end;
                const int64_t l_ = e - (int64_t)heads[r];
                len[r] = (uint32_t)(l_ > 1 ? l_ : 1);
            } else {
                len[r] = 0;
            }
        }
        __syncwarp();
        // (with at most one run per lane there is nothing to balance)
        for (int k = 2; nh > 32 && k <= P; k <<= 1)
            for (int jj = k >> 1; jj > 0; jj >>= 1) {
                for (int i = lane; i < P; i += 32) {
                    const int ix = i ^ jj;
                    if (ix > i) {
                        const uint32_t li = len[i], lx = len[ix];
                        if (((i & k) == 0) ? (li < lx) : (li > lx)) {
                            len[i] = lx, len[ix] = li;
                            const uint32_t h = heads[i];
                            heads[i] = heads[ix], heads[ix] = h;
                        }
                    }
                }
                __syncwarp();
            }
        for (int q = 0; q * 32 < nh; ++q) {
            const int r = q * 32 + ((q & 1) ? 31 - lane : lane);
            if (r < nh) reduce_run<T, K>(pairs, npairs, (int64_t)heads[r], recs, f);
        }
        __syncwarp();
        nh = 0;
    };
    bool tail = false;  // invalid pairs (blocks outside the cube or not refined) sort last
    for (int64_t base = j0; base < j1 && !tail; base += 32) {
        const int64_t j = base + lane;
        uint32_t a = (uint32_t)INVALID_HI;
        if (j < j1) a = (uint32_t)(pairs[j] >> 32);
        uint32_t prev = __shfl_up_sync(0xffffffffu, a, 1);
        if (lane == 0) prev = j > 0 ? (uint32_t)(pairs[j - 1] >> 32) : (uint32_t)INVALID_HI;
        const bool head = j < j1 && a != (uint32_t)INVALID_HI && (j == 0 || a != prev);
        tail = __any_sync(0xffffffffu, j < j1 && a == (uint32_t)INVALID_HI);
        const unsigned m = __ballot_sync(0xffffffffu, head);
        if (head) heads[nh + __popc(m & lt)] = (uint32_t)j;
        nh += __popc(m);
        if (nh > RB - 32) run_batch(base + 32);
    }
    if (nh > 0) run_batch(j1);
}

template <typename Kern>
unsigned grid_for(Kern k, int block, size_t smem, int64_t n) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem);
    per_sm = std::max(per_sm, 1);
    int64_t need = (n + block - 1) / block;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms() * per_sm, need));
}

template <typename Kern>
ot_status prep(Kern k, size_t smem) {
    if (smem > 48 * 1024) OT_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return OT_OK;
}

size_t align_up(size_t b) { return (b + 255) & ~(size_t)255; }

int leaf_bits(int64_t n) {
    int b = 1;
    while (b < 32 && ((int64_t)1 << b) <= n) ++b; // n <= 2^b - 1: the all-ones key stays above every leaf
    return b;
}

// Pairs per marker in the sorted spreading: one per overlapping parent block slot.
inline int stencil_cells(int kernel) { return kernel == OT_PESKIN4 ? ParentSlots<OT_PESKIN4>::PS : ParentSlots<OT_ROMA3>::PS; }

template <typename T, int K>
ot_status spread_sorted(const ot_octree* t, const double* x, const double* y, const double* z, const T* F,
                        const T* dV, int64_t n, T* f, void* ws, cudaStream_t s) {
    const int64_t np = n * ParentSlots<K>::PS;
    uint64_t* pairs = static_cast<uint64_t*>(ws);
    uint64_t* tmp = pairs + np;
    void* rws = tmp + np;
    TreeView v = tree_view(t);
    const size_t smem = 0;
    ot_status st;
    char* p = static_cast<char*>(rws) + align_up(radix_ws_bytes(np));
    // records 64-byte aligned (the reduce reads an FP32 record as two 32-byte loads)
    p = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(p) + 63) & ~(uintptr_t)63);
    MarkerRec<T>* recs = reinterpret_cast<MarkerRec<T>*>(p);
    p += align_up((size_t)n * sizeof(MarkerRec<double>));
    uint32_t* cnt = reinterpret_cast<uint32_t*>(p);
    p += align_up((size_t)n * sizeof(uint32_t));
    uint32_t* off = reinterpret_cast<uint32_t*>(p);
    p += align_up((size_t)n * sizeof(uint32_t));
    uint32_t* d_np = reinterpret_cast<uint32_t*>(p);
    p += 256;
    void* scan_ws = p;
    auto kc = k_spread_count<K>;
    kc<<<grid_for(kc, 256, 0, n), 256, 0, s>>>(x, y, z, n, t->lmax, cnt);
    count_launch();
    if ((st = scan_u32_ws(cnt, off, n, d_np, scan_ws, s)) != OT_OK) return st;
    auto ke = k_spread_emit_rec<T, K>;
    if ((st = prep(ke, smem)) != OT_OK) return st;
    ke<<<grid_for(ke, 256, smem, n), 256, smem, s>>>(v, x, y, z, F, dV, n, off, pairs, recs);
    count_launch();
    OT_CUDA(cudaGetLastError());
    // a parent block is identified by its first child leaf a0; blocks are 8 consecutive leaves,
    // so a0 >> 3 is distinct for distinct blocks and keeps their order: sorting on it skips 3 bits
    const int bits = leaf_bits(t->n + 8);
    uint64_t* sorted = pairs;
    if ((st = radix_sort_u64_dn(pairs, tmp, np, d_np, 35, 32 + bits, rws, &sorted, s)) != OT_OK) return st;
    auto kr = k_spread_reduce_rec<T, K>;
    kr<<<grid_for(kr, 256, 0, (np + RC - 1) / RC), 256, 0, s>>>(sorted, d_np, recs, f);  // warps split the pairs
    count_launch();
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

} // namespace

size_t spread_ws_bytes(const ot_octree* t, int kernel, int64_t n) {
    (void)t;
    const int64_t np = n * stencil_cells(kernel);
    return (size_t)np * 16 + align_up(radix_ws_bytes(np)) + align_up((size_t)n * sizeof(MarkerRec<double>)) +
           2 * align_up((size_t)n * sizeof(uint32_t)) + 256 + align_up(scan_ws_bytes(n)) + 512 + 64;
}

template <typename T>
ot_status launch_spread(const ot_octree* t, int kernel, int mode, const double* x, const double* y, const double* z,
                        const T* F, const T* dV, int64_t n, T* f, void* ws, size_t ws_bytes, cudaStream_t s) {
    if (n == 0) return OT_OK;
    if (mode == OT_SORTED) {
        if (ws_bytes < spread_ws_bytes(t, kernel, n)) return OT_ERR_ARG;
        if (kernel == OT_PESKIN4) return spread_sorted<T, OT_PESKIN4>(t, x, y, z, F, dV, n, f, ws, s);
        return spread_sorted<T, OT_ROMA3>(t, x, y, z, F, dV, n, f, ws, s);
    }
    TreeView v = tree_view(t);
    const size_t smem = 0;
    ot_status st;
    if (kernel == OT_PESKIN4) {
        auto k = k_spread_atomic<T, OT_PESKIN4>;
        if ((st = prep(k, smem)) != OT_OK) return st;
        k<<<grid_for(k, 256, smem, n), 256, smem, s>>>(v, x, y, z, F, dV, n, f);
    } else {
        auto k = k_spread_atomic<T, OT_ROMA3>;
        if ((st = prep(k, smem)) != OT_OK) return st;
        k<<<grid_for(k, 256, smem, n), 256, smem, s>>>(v, x, y, z, F, dV, n, f);
    }
    count_launch();
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

template ot_status launch_spread<float>(const ot_octree*, int, int, const double*, const double*, const double*,
                                        const float*, const float*, int64_t, float*, void*, size_t, cudaStream_t);
template ot_status launch_spread<double>(const ot_octree*, int, int, const double*, const double*, const double*,
                                         const double*, const double*, int64_t, double*, void*, size_t, cudaStream_t);

} // namespace ot

// ------------------------------------------------------------------------------------------
// Sorted spreading with caller scratch only (no allocation of any kind).
// ------------------------------------------------------------------------------------------
namespace ot {

size_t spread_noalloc_bytes(int kernel, int64_t n) {
    const int64_t np = n * stencil_cells(kernel);
    return (size_t)np * 16 + radix_noalloc_bytes(np) + 256;
}

namespace {
template <int K>
ot_status sorted_noalloc(const ot_octree* t, const double* x, const double* y, const double* z, const float* F,
                         const float* dV, int64_t n, float* f, void* scratch, cudaStream_t s) {
    const int64_t np = n * ParentSlots<K>::PS;
    uint64_t* pairs = static_cast<uint64_t*>(scratch);
    uint64_t* tmp = pairs + np;
    void* rws = tmp + np;
    TreeView v = tree_view(t);
    const size_t smem = 0;
    ot_status st;
    auto ke = k_spread_emit<K>;
    if ((st = prep(ke, smem)) != OT_OK) return st;
    ke<<<grid_for(ke, 256, smem, n), 256, smem, s>>>(v, x, y, z, n, pairs);
    count_launch();
    OT_CUDA(cudaGetLastError());
    if ((st = radix_sort_u64_noalloc(pairs, tmp, np, 32, 32 + leaf_bits(t->n), rws, s)) != OT_OK) return st;
    auto kr = k_spread_reduce<float, K>;
    kr<<<grid_for(kr, 256, 0, (np + RC - 1) / RC), 256, 0, s>>>(pairs, np, t->lmax, x, y, z, F, dV, n, f);
    count_launch();
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}
} // namespace

ot_status launch_spread_sorted_noalloc(const ot_octree* t, int kernel, const double* x, const double* y,
                                       const double* z, const float* F, const float* dV, int64_t n, float* f,
                                       void* scratch, cudaStream_t s) {
    if (n == 0) return OT_OK;
    if (kernel == OT_PESKIN4) return sorted_noalloc<OT_PESKIN4>(t, x, y, z, F, dV, n, f, scratch, s);
    return sorted_noalloc<OT_ROMA3>(t, x, y, z, F, dV, n, f, scratch, s);
}

} // namespace ot
