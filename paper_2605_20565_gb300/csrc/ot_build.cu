// ot_build.cu -- octree construction on the device, leaf validation, centres, level map.
//
// Construction (Sec. 3.1 refinement + 2:1 balance, Sec. 3.3 surface-driven auxiliary forest)
// works on per-level sorted key arrays R[l] of the REFINED cells of level l (3l-bit keys):
//   1. top-down: R[lmin] = cells of level lmin meeting the criterion; R[l+1] = children of
//      R[l] meeting it;
//   2. balance, finest level first: a refined cell p of level l needs every neighbour cell
//      of level l to exist, i.e. the parents of p's neighbours (and p's own parent) must be
//      refined; missing ones are added to R[l-1].  Requirements only flow to coarser levels,
//      so one descending pass reaches the fixed point (the coarsest balanced refinement);
//   3. leaves: nodes of level l+1 are the children of R[l] (already Morton-sorted); subtree
//      leaf counts bottom-up and offsets top-down place every leaf at its rank without a
//      global sort.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ot_internal.h"

namespace ot {

namespace {

unsigned grid1d(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    int64_t cap = (int64_t)num_sms() * 16;
    return (unsigned)std::max<int64_t>(1, std::min(g, cap));
}

#define GRID_STRIDE(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// The refinement test in FP64 with every operation rounded as written (no fused multiply-add),
// in x, y, z order: max(0, |c - box|_near - r, r - |c - box|_far) <= shell.
__device__ bool box_near_surface(const double lo[3], double h, const ot_sphere& s) {
    double near2 = 0.0, far2 = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double c = s.c[d];
        const double hi = __dadd_rn(lo[d], h);
        const double below = __dsub_rn(lo[d], c);
        const double above = __dsub_rn(c, hi);
        double e = 0.0;
        if (below > e) e = below;
        if (above > e) e = above;
        near2 = __dadd_rn(near2, __dmul_rn(e, e));
        const double f0 = fabs(__dsub_rn(c, lo[d]));
        const double f1 = fabs(__dsub_rn(c, hi));
        const double f = f0 > f1 ? f0 : f1;
        far2 = __dadd_rn(far2, __dmul_rn(f, f));
    }
    double dist = 0.0;
    const double t0 = __dsub_rn(__dsqrt_rn(near2), s.r);
    const double t1 = __dsub_rn(s.r, __dsqrt_rn(far2));
    if (t0 > dist) dist = t0;
    if (t1 > dist) dist = t1;
    return dist <= s.shell;
}

// Conservative FP32 pre-test: false only when the box is certainly farther than r + shell from
// the centre (then the exact test fails too).  Skips most spheres cheaply.
__device__ __forceinline__ bool maybe_near(const float lo[3], float h, const ot_sphere& s) {
    float d2 = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float c = (float)s.c[k];
        float e = fmaxf(fmaxf(lo[k] - c, 0.0f), c - (lo[k] + h));
        d2 += e * e;
    }
    float lim = (float)(s.r + s.shell) * 1.0001f + 1e-5f;
    return d2 <= lim * lim;
}

// Candidate cells of level l: the 8^l cells (parent == null, l == lmin) or the children of the
// refined parents; flag[j] = criterion, cand[j] = key.  With the sphere bins (l >= Lb), only the
// spheres listed for the cell's bin of level Lb are tested: a bin lists every sphere whose
// centre is within (r + shell) + margin of it, a superset of those the pre-test can accept for
// any cell inside it, so the result is the same as testing every sphere.
__global__ void k_refine(const uint64_t* __restrict__ parent, int64_t ncand, int l, const ot_sphere* __restrict__ sph,
                         int nsph, const int* __restrict__ bin_off, const int* __restrict__ bin_sph, int Lb,
                         uint64_t* __restrict__ cand, uint32_t* __restrict__ flag) {
    const double h = ldexp(1.0, -l);
    const float hf = (float)h;
    const bool binned = bin_off && l >= Lb;
    GRID_STRIDE(j, ncand) {
        uint64_t key = parent ? ((parent[j >> 3] << 3) | (uint64_t)(j & 7)) : (uint64_t)j;
        uint32_t i0, i1, i2;
        demorton3(key, i0, i1, i2);
        const double lo[3] = {__dmul_rn((double)i0, h), __dmul_rn((double)i1, h), __dmul_rn((double)i2, h)};
        const float lof[3] = {(float)lo[0], (float)lo[1], (float)lo[2]};
        uint32_t hit = 0;
        if (binned) {
            const int sh = l - Lb, nb = 1 << Lb;
            const int b = (int)(i0 >> sh) + nb * ((int)(i1 >> sh) + nb * (int)(i2 >> sh));
            for (int k = bin_off[b]; k < bin_off[b + 1] && !hit; ++k) {
                const ot_sphere sp = sph[bin_sph[k]];
                if (maybe_near(lof, hf, sp) && box_near_surface(lo, h, sp)) hit = 1;
            }
        } else {
            for (int s = 0; s < nsph && !hit; ++s) {
                const ot_sphere sp = sph[s];
                if (maybe_near(lof, hf, sp) && box_near_surface(lo, h, sp)) hit = 1;
            }
        }
        cand[j] = key;
        flag[j] = hit;
    }
}

__device__ __forceinline__ bool contains_sorted(const uint64_t* __restrict__ a, int64_t n, uint64_t q, int64_t* at) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < q)
            lo = mid + 1;
        else
            hi = mid;
    }
    if (at) *at = lo;
    return lo < n && a[lo] == q;
}

// Balance requirement of refined cells p of level l: the parents (level l-1) of p's neighbour
// cells and of p itself must be refined.  Missing ones are appended to `miss`.
__global__ void k_balance_req(const uint64_t* __restrict__ R, int64_t nR, int l, const uint64_t* __restrict__ Rp,
                              int64_t nRp, int full, uint64_t* __restrict__ miss, uint32_t* __restrict__ nmiss,
                              int64_t cap) {
    const int64_t ncell = (int64_t)1 << l;
    GRID_STRIDE(j, nR) {
        uint32_t c[3];
        demorton3(R[j], c[0], c[1], c[2]);
        // candidate parent coordinates per axis
        int64_t plo[3], phi[3];
        for (int d = 0; d < 3; ++d) {
            const int64_t a = (int64_t)c[d] - 1, b = (int64_t)c[d] + 1;
            plo[d] = (a < 0 ? 0 : a) >> 1;
            phi[d] = (b > ncell - 1 ? ncell - 1 : b) >> 1;
        }
        for (int64_t pz = plo[2]; pz <= phi[2]; ++pz)
            for (int64_t py = plo[1]; py <= phi[1]; ++py)
                for (int64_t px = plo[0]; px <= phi[0]; ++px) {
                    if (!full) {
                        // face balance: p's own parent, or the parent of a face neighbour
                        int differ = (px != (c[0] >> 1)) + (py != (c[1] >> 1)) + (pz != (c[2] >> 1));
                        if (differ > 1) continue;
                    }
                    uint64_t key = morton3((uint32_t)px, (uint32_t)py, (uint32_t)pz);
                    if (!contains_sorted(Rp, nRp, key, nullptr)) {
                        uint32_t at = atomicAdd(nmiss, 1u);
                        if (at < cap) miss[at] = key;
                    }
                }
    }
}

__device__ __forceinline__ uint64_t node_key(const uint64_t* __restrict__ Rparent, int64_t j) {
    return Rparent ? ((Rparent[j >> 3] << 3) | (uint64_t)(j & 7)) : (uint64_t)j;
}

__global__ void k_rank(const uint64_t* __restrict__ Rparent, int64_t M, const uint64_t* __restrict__ R, int64_t nR,
                       int32_t* __restrict__ rank) {
    GRID_STRIDE(j, M) {
        int64_t at;
        rank[j] = contains_sorted(R, nR, node_key(Rparent, j), &at) ? (int32_t)at : -1;
    }
}

__global__ void k_count(const int32_t* __restrict__ rank, int64_t M, const uint32_t* __restrict__ cnt_child,
                        uint32_t* __restrict__ cnt) {
    GRID_STRIDE(j, M) {
        int32_t r = rank[j];
        if (r < 0) {
            cnt[j] = 1;
        } else if (!cnt_child) {
            cnt[j] = 8;
        } else {
            uint32_t s = 0;
            for (int c = 0; c < 8; ++c) s += cnt_child[8 * (int64_t)r + c];
            cnt[j] = s;
        }
    }
}

__global__ void k_child_off(const int32_t* __restrict__ rank, const uint32_t* __restrict__ off, int64_t M,
                            const uint32_t* __restrict__ cnt_child, uint32_t* __restrict__ off_child) {
    GRID_STRIDE(j, M) {
        int32_t r = rank[j];
        if (r < 0) continue;
        uint32_t run = off[j];
        for (int c = 0; c < 8; ++c) {
            off_child[8 * (int64_t)r + c] = run;
            run += cnt_child ? cnt_child[8 * (int64_t)r + c] : 1u;
        }
    }
}

__global__ void k_emit(const uint64_t* __restrict__ Rparent, const int32_t* __restrict__ rank,
                       const uint32_t* __restrict__ off, int64_t M, int l, uint64_t* __restrict__ key_out,
                       uint8_t* __restrict__ lev_out) {
    GRID_STRIDE(j, M) {
        if (rank && rank[j] >= 0) continue;
        uint32_t o = off[j];
        key_out[o] = node_key(Rparent, j) << (3 * (MAXLEVEL - l));
        lev_out[o] = (uint8_t)l;
    }
}

template <typename T>
ot_status dalloc(T** p, int64_t n, cudaStream_t s) {
    *p = nullptr;
    if (n <= 0) return OT_OK;
    OT_CUDA(cudaMallocAsync((void**)p, sizeof(T) * (size_t)n, s));
    return OT_OK;
}

struct Guard {
    cudaStream_t s;
    std::vector<void*> ptrs;
    ~Guard() {
        for (void* p : ptrs)
            if (p) cudaFreeAsync(p, s);
    }
    template <typename T> T* keep(T* p) {
        ptrs.push_back((void*)p);
        return p;
    }
};

} // namespace

ot_status build_tree(const ot_sphere* h_spheres, int nsph, const ot_build_params* p, cudaStream_t s, ot_octree* t) {
    const int lmin = p->lmin, lmax = p->lmax;
    Guard g{s, {}};
    ot_sphere* d_sph = nullptr;
    if (nsph > 0) {
        OT_CUDA(cudaMallocAsync(&d_sph, sizeof(ot_sphere) * nsph, s));
        g.keep(d_sph);
        OT_CUDA(cudaMemcpyAsync(d_sph, h_spheres, sizeof(ot_sphere) * nsph, cudaMemcpyHostToDevice, s));
    }
    // sphere bins: the cells of level Lb, each listing the spheres whose centre lies within
    // (r + shell) (1 + 1e-4) + 1e-4 of the bin's box (bounding-box overlap; a superset)
    const int Lb = std::min(lmin, 5);
    int* d_bin_off = nullptr;
    int* d_bin_sph = nullptr;
    if (nsph > 0 && Lb >= 1) {
        const int nb = 1 << Lb;
        std::vector<std::vector<int>> bins((size_t)nb * nb * nb);
        for (int k = 0; k < nsph; ++k) {
            const ot_sphere& sp = h_spheres[k];
            const double R = (sp.r + sp.shell) * 1.0001 + 1e-4;
            int lo[3], hi[3];
            const auto bin_of = [nb](double v) {  // clamped in FP64 before the conversion
                return (int)std::floor(std::max(0.0, std::min((double)(nb - 1), v * nb)));
            };
            for (int d = 0; d < 3; ++d) {
                lo[d] = bin_of(sp.c[d] - R);
                hi[d] = bin_of(sp.c[d] + R);
            }
            for (int z = lo[2]; z <= hi[2]; ++z)
                for (int y = lo[1]; y <= hi[1]; ++y)
                    for (int x = lo[0]; x <= hi[0]; ++x) bins[(size_t)x + nb * ((size_t)y + nb * (size_t)z)].push_back(k);
        }
        std::vector<int> off(bins.size() + 1, 0), idx;
        for (size_t b = 0; b < bins.size(); ++b) {
            off[b + 1] = off[b] + (int)bins[b].size();
            idx.insert(idx.end(), bins[b].begin(), bins[b].end());
        }
        OT_CUDA(cudaMallocAsync(&d_bin_off, sizeof(int) * off.size(), s));
        g.keep(d_bin_off);
        OT_CUDA(cudaMallocAsync(&d_bin_sph, sizeof(int) * std::max<size_t>(idx.size(), 1), s));
        g.keep(d_bin_sph);
        OT_CUDA(cudaMemcpyAsync(d_bin_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, s));
        if (!idx.empty())
            OT_CUDA(cudaMemcpyAsync(d_bin_sph, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, s));
        OT_CUDA(cudaStreamSynchronize(s));  // the host vectors go out of scope
    }
    const int L = lmax + 1;
    std::vector<uint64_t*> R(L, nullptr);
    std::vector<int64_t> nR(L, 0);

    // 1. top-down refinement by the criterion
    for (int l = lmin; l < lmax; ++l) {
        const int64_t ncand = (l == lmin) ? ((int64_t)1 << (3 * lmin)) : 8 * nR[l - 1];
        if (ncand == 0) break;
        uint64_t* cand = nullptr;
        uint32_t *flag = nullptr, *pos = nullptr;
        ot_status st;
        if ((st = dalloc(&cand, ncand, s)) != OT_OK) return st;
        g.keep(cand);
        if ((st = dalloc(&flag, ncand, s)) != OT_OK) return st;
        g.keep(flag);
        if ((st = dalloc(&pos, ncand, s)) != OT_OK) return st;
        g.keep(pos);
        k_refine<<<grid1d(ncand, 256), 256, 0, s>>>(l == lmin ? nullptr : R[l - 1], ncand, l, d_sph, nsph, d_bin_off,
                                                    d_bin_sph, Lb, cand, flag);
        count_launch();
        OT_CUDA(cudaGetLastError());
        uint64_t* out = nullptr;
        if ((st = dalloc(&out, ncand, s)) != OT_OK) return st;
        g.keep(out);
        if ((st = compact_u64(cand, flag, pos, ncand, out, &nR[l], s)) != OT_OK) return st;
        R[l] = out;
    }

    // 2. balance, finest refined level first
    for (int l = lmax - 1; l >= lmin + 1; --l) {
        if (nR[l] == 0) continue;
        const int64_t cap = 8 * nR[l];
        uint64_t* miss = nullptr;
        uint32_t* nmiss = nullptr;
        ot_status st;
        if ((st = dalloc(&miss, cap, s)) != OT_OK) return st;
        g.keep(miss);
        if ((st = dalloc(&nmiss, 1, s)) != OT_OK) return st;
        g.keep(nmiss);
        OT_CUDA(cudaMemsetAsync(nmiss, 0, sizeof(uint32_t), s));
        k_balance_req<<<grid1d(nR[l], 256), 256, 0, s>>>(R[l], nR[l], l, R[l - 1], nR[l - 1], p->balance_full, miss,
                                                        nmiss, cap);
        count_launch();
        OT_CUDA(cudaGetLastError());
        uint32_t hm = 0;
        OT_CUDA(cudaMemcpyAsync(&hm, nmiss, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        OT_CUDA(cudaStreamSynchronize(s));
        if (hm > 0) {
            const int64_t tot = nR[l - 1] + hm;
            uint64_t *u = nullptr, *tmp = nullptr;
            if ((st = dalloc(&u, tot, s)) != OT_OK) return st;
            g.keep(u);
            if ((st = dalloc(&tmp, tot, s)) != OT_OK) return st;
            g.keep(tmp);
            if (nR[l - 1] > 0)
                OT_CUDA(cudaMemcpyAsync(u, R[l - 1], sizeof(uint64_t) * nR[l - 1], cudaMemcpyDeviceToDevice, s));
            OT_CUDA(cudaMemcpyAsync(u + nR[l - 1], miss, sizeof(uint64_t) * hm, cudaMemcpyDeviceToDevice, s));
            if ((st = radix_sort_u64(u, tmp, tot, 0, 3 * (l - 1), s)) != OT_OK) return st;
            int64_t m = 0;
            if ((st = unique_u64(u, tot, &m, s)) != OT_OK) return st;
            R[l - 1] = u;
            nR[l - 1] = m;
        }
    }

    // 3. leaves: ranks, subtree counts (bottom-up), offsets (top-down), emission
    std::vector<int64_t> M(L + 1, 0);
    std::vector<int32_t*> rank(L + 1, nullptr);
    std::vector<uint32_t*> cnt(L + 1, nullptr), off(L + 1, nullptr);
    M[lmin] = (int64_t)1 << (3 * lmin);
    for (int l = lmin; l < lmax; ++l) M[l + 1] = 8 * nR[l];
    ot_status st;
    for (int l = lmin; l <= lmax; ++l) {
        if (M[l] == 0) continue;
        if (l < lmax) {
            if ((st = dalloc(&rank[l], M[l], s)) != OT_OK) return st;
            g.keep(rank[l]);
            k_rank<<<grid1d(M[l], 256), 256, 0, s>>>(l == lmin ? nullptr : R[l - 1], M[l], R[l], nR[l], rank[l]);
            count_launch();
        }
        if ((st = dalloc(&cnt[l], M[l], s)) != OT_OK) return st;
        g.keep(cnt[l]);
        if ((st = dalloc(&off[l], M[l], s)) != OT_OK) return st;
        g.keep(off[l]);
    }
    for (int l = lmax - 1; l >= lmin; --l) {
        if (M[l] == 0) continue;
        const uint32_t* child = (l + 1 < lmax && M[l + 1] > 0) ? cnt[l + 1] : nullptr;
        k_count<<<grid1d(M[l], 256), 256, 0, s>>>(rank[l], M[l], child, cnt[l]);
        count_launch();
    }
    uint32_t* d_tot = nullptr;
    if ((st = dalloc(&d_tot, 1, s)) != OT_OK) return st;
    g.keep(d_tot);
    if (lmin == lmax) {
        // uniform tree: every node of level lmin is a leaf
        OT_CUDA(cudaMemsetAsync(cnt[lmin], 0, sizeof(uint32_t) * M[lmin], s));
    }
    if (lmin < lmax) {
        if ((st = scan_u32(cnt[lmin], off[lmin], M[lmin], d_tot, s)) != OT_OK) return st;
    }
    for (int l = lmin; l < lmax; ++l) {
        if (M[l] == 0 || M[l + 1] == 0) continue;
        const uint32_t* child = (l + 1 < lmax) ? cnt[l + 1] : nullptr;
        k_child_off<<<grid1d(M[l], 256), 256, 0, s>>>(rank[l], off[l], M[l], child, off[l + 1]);
        count_launch();
    }
    int64_t nleaf = 0;
    if (lmin < lmax) {
        uint32_t h = 0;
        OT_CUDA(cudaMemcpyAsync(&h, d_tot, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        OT_CUDA(cudaStreamSynchronize(s));
        nleaf = h;
    } else {
        nleaf = M[lmin];
    }
    if (nleaf <= 0 || nleaf > OT_MAX_LEAVES) return OT_ERR_LIMIT;
    OT_CUDA(cudaMalloc(&t->d_key, sizeof(uint64_t) * nleaf));
    OT_CUDA(cudaMalloc(&t->d_level, nleaf));
    for (int l = lmin; l <= lmax; ++l) {
        if (M[l] == 0) continue;
        const uint32_t* o = off[l];
        if (lmin == lmax) {
            // off = identity for a uniform tree
            std::vector<uint32_t> id(M[l]);
            for (int64_t j = 0; j < M[l]; ++j) id[j] = (uint32_t)j;
            OT_CUDA(cudaMemcpyAsync(off[l], id.data(), sizeof(uint32_t) * M[l], cudaMemcpyHostToDevice, s));
            OT_CUDA(cudaStreamSynchronize(s));
        }
        k_emit<<<grid1d(M[l], 256), 256, 0, s>>>(l == lmin ? nullptr : R[l - 1], l < lmax ? rank[l] : nullptr, o, M[l],
                                                l, t->d_key, t->d_level);
        count_launch();
    }
    OT_CUDA(cudaGetLastError());
    OT_CUDA(cudaStreamSynchronize(s));
    t->n = nleaf;
    t->lmin = lmin;
    t->lmax = lmax;
    return OT_OK;
}

// ------------------------------------------------------------------------------------------
// Validation of caller leaves.
// ------------------------------------------------------------------------------------------
namespace {

__global__ void k_check_tiling(const uint64_t* __restrict__ key, const uint8_t* __restrict__ lev, int64_t n,
                               unsigned* __restrict__ bad, int* __restrict__ lrange) {
    GRID_STRIDE(i, n) {
        int l = lev[i];
        bool ok = l <= OT_MAX_LEVEL;
        uint64_t sp = ok ? key_span(l) : 0;
        if (ok) {
            ok = (key[i] & (sp - 1)) == 0;
            if (i == 0) ok = ok && key[0] == 0;
            if (i + 1 < n)
                ok = ok && key[i] + sp == key[i + 1];
            else
                ok = ok && key[i] + sp == (1ULL << 63);
        }
        if (!ok) atomicAdd(bad, 1u);
        atomicMin(&lrange[0], l);
        atomicMax(&lrange[1], l);
    }
}

__global__ void k_check_balance(const uint64_t* __restrict__ key, const uint8_t* __restrict__ lev, int n, int full,
                                unsigned* __restrict__ bad) {
    GRID_STRIDE(b, (int64_t)n) {
        const int lb = lev[b];
        uint32_t x, y, z;
        demorton3(key[b], x, y, z);
        const int sh = MAXLEVEL - lb;
        const int64_t ci = x >> sh, cj = y >> sh, ck = z >> sh, nc = (int64_t)1 << lb;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int nz = (dx != 0) + (dy != 0) + (dz != 0);
                    if (nz == 0 || (!full && nz != 1)) continue;
                    int64_t a = ci + dx, bq = cj + dy, c = ck + dz;
                    if (a < 0 || bq < 0 || c < 0 || a >= nc || bq >= nc || c >= nc) continue;
                    uint64_t q = morton3((uint32_t)(a << sh), (uint32_t)(bq << sh), (uint32_t)(c << sh));
                    int at = search_range(key, 0, n, q);
                    if ((int)lev[at] + 2 <= lb) atomicAdd(bad, 1u);
                }
    }
}

} // namespace

ot_status validate_leaves(const uint64_t* d_key, const uint8_t* d_level, int64_t n, int full, cudaStream_t s, int* lmin,
                          int* lmax) {
    unsigned* bad = nullptr;
    int* lr = nullptr;
    OT_CUDA(cudaMallocAsync(&bad, 2 * sizeof(unsigned), s));
    OT_CUDA(cudaMallocAsync(&lr, 2 * sizeof(int), s));
    int init[2] = {1 << 20, -1};
    OT_CUDA(cudaMemsetAsync(bad, 0, 2 * sizeof(unsigned), s));
    OT_CUDA(cudaMemcpyAsync(lr, init, sizeof(init), cudaMemcpyHostToDevice, s));
    k_check_tiling<<<grid1d(n, 256), 256, 0, s>>>(d_key, d_level, n, bad, lr);
    count_launch();
    unsigned hb[2] = {0, 0};
    int hr[2];
    OT_CUDA(cudaMemcpyAsync(hb, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    OT_CUDA(cudaMemcpyAsync(hr, lr, sizeof(hr), cudaMemcpyDeviceToHost, s));
    OT_CUDA(cudaStreamSynchronize(s));
    ot_status st = OT_OK;
    if (hb[0] != 0) {
        st = OT_ERR_UNSORTED;
    } else {
        k_check_balance<<<grid1d(n, 256), 256, 0, s>>>(d_key, d_level, (int)n, full, bad + 1);
        count_launch();
        OT_CUDA(cudaMemcpyAsync(hb + 1, bad + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        OT_CUDA(cudaStreamSynchronize(s));
        if (hb[1] != 0) st = OT_ERR_UNBALANCED;
    }
    cudaFreeAsync(bad, s);
    cudaFreeAsync(lr, s);
    *lmin = hr[0];
    *lmax = hr[1];
    OT_CUDA(cudaGetLastError());
    return st;
}

// ------------------------------------------------------------------------------------------
// Centres, search sample, diagnostics words.
// ------------------------------------------------------------------------------------------
namespace {

__global__ void k_centres(const uint64_t* __restrict__ key, const uint8_t* __restrict__ lev, int64_t n,
                          double* __restrict__ out) {
    GRID_STRIDE(i, n) {
        uint32_t x, y, z;
        demorton3(key[i], x, y, z);
        const double half = 0.5 * (double)(1u << (MAXLEVEL - lev[i]));
        const double sc = 0x1p-21;
        out[i] = ((double)x + half) * sc;
        out[n + i] = ((double)y + half) * sc;
        out[2 * n + i] = ((double)z + half) * sc;
    }
}

// lmap[c] = the leaf holding the anchor of level-L cell c: the last key <= its anchor.
__global__ void k_lmap(const uint64_t* __restrict__ key, int n, int L, int64_t ncell, uint32_t* __restrict__ out) {
    GRID_STRIDE(c, ncell) out[c] = (uint32_t)search_range(key, 0, n, (uint64_t)c << (3 * (MAXLEVEL - L)));
}

} // namespace

ot_status leaf_centres(const ot_octree* t, double* d_xyz, cudaStream_t s) {
    k_centres<<<grid1d(t->n, 256), 256, 0, s>>>(t->d_key, t->d_level, t->n, d_xyz);
    count_launch();
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

// Descriptor of every level-map cell of level L (see desc_leaf): the refined children and
// grandchildren of an uncovered cell, valid when no leaf of the cell is deeper than L + 3.
__global__ void k_desc(const uint64_t* __restrict__ key, const uint8_t* __restrict__ level, int n,
                       const uint32_t* __restrict__ lmap, int L, int64_t ncell, uint4* __restrict__ desc) {
    GRID_STRIDE(c, ncell) {
        const int a = (int)lmap[c];
        const int e = c + 1 < ncell ? (int)lmap[c + 1] : n;
        uint32_t m1 = 0, valid = 1;
        uint64_t m2 = 0;
        if (e - a <= 1) {
            valid = 0;  // covered: the map answers
        } else {
            for (int b = a; b < e; ++b) {
                const int lb = level[b];
                if (lb > L + 3) {
                    valid = 0;
                    break;
                }
                const uint64_t kb = key[b];
                const int c1 = (int)(kb >> (3 * (MAXLEVEL - L - 1))) & 7;
                if (lb >= L + 2) m1 |= 1u << c1;
                if (lb >= L + 3) m2 |= 1ULL << (8 * c1 + ((int)(kb >> (3 * (MAXLEVEL - L - 2))) & 7));
            }
        }
        desc[c] = valid ? make_uint4((uint32_t)m2, (uint32_t)(m2 >> 32), m1 | DESC_VALID, 0u) : make_uint4(0u, 0u, 0u, 0u);
    }
}

__global__ void k_lmap_lv(const uint32_t* __restrict__ lmap, const uint8_t* __restrict__ level, int64_t ncell,
                          uint8_t* __restrict__ out) {
    GRID_STRIDE(c, ncell) out[c] = level[lmap[c]];
}

ot_status finish_tree(ot_octree* t, cudaStream_t s, int map_level) {
    // default: level 7, or 8 for trees deeper than 10 levels (the descriptors then reach lmax)
    const int L = map_level >= 0 ? std::min(map_level, t->lmax)
                                 : std::min(t->lmax, std::max(7, std::min(8, t->lmax - 3)));
    const int Lp = std::min(t->lmax, 7);
    if (!t->d_pmap) {
        const int64_t np = (int64_t)1 << (3 * Lp);
        OT_CUDA(cudaMalloc(&t->d_pmap, sizeof(uint32_t) * np));
        k_lmap<<<grid1d(np, 256), 256, 0, s>>>(t->d_key, (int)t->n, Lp, np, t->d_pmap);
        count_launch();
        t->pyr_level = Lp;
        ot_status st = build_node_lists(t, s);
        if (st != OT_OK) return st;
    }
    if (t->d_lmap && t->d_lmap != t->d_pmap) cudaFree(t->d_lmap);
    t->d_lmap = nullptr;
    if (L == Lp) {
        t->d_lmap = t->d_pmap;
    } else {
        const int64_t ncell = (int64_t)1 << (3 * L);
        OT_CUDA(cudaMalloc(&t->d_lmap, sizeof(uint32_t) * ncell));
        k_lmap<<<grid1d(ncell, 256), 256, 0, s>>>(t->d_key, (int)t->n, L, ncell, t->d_lmap);
        count_launch();
    }
    t->lmap_level = L;
    if (t->d_lmap_lv) cudaFree(t->d_lmap_lv);
    {
        const int64_t ncell = (int64_t)1 << (3 * L);
        OT_CUDA(cudaMalloc(&t->d_lmap_lv, ncell));
        k_lmap_lv<<<grid1d(ncell, 256), 256, 0, s>>>(t->d_lmap, t->d_level, ncell, t->d_lmap_lv);
        count_launch();
    }
    if (t->d_desc) cudaFree(t->d_desc);
    t->d_desc = nullptr;
    if (L + 1 <= t->lmax && L + 1 < MAXLEVEL) {
        const int64_t ncell = (int64_t)1 << (3 * L);
        OT_CUDA(cudaMalloc(&t->d_desc, sizeof(uint4) * ncell));
        k_desc<<<grid1d(ncell, 256), 256, 0, s>>>(t->d_key, t->d_level, (int)t->n, t->d_lmap, L, ncell, t->d_desc);
        count_launch();
    }
    if (!t->d_err) {
        OT_CUDA(cudaMalloc(&t->d_err, 64));
        OT_CUDA(cudaMemsetAsync(t->d_err, 0, 64, s));
        t->d_fallbacks = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(t->d_err) + 8);
    }
    OT_CUDA(cudaGetLastError());
    OT_CUDA(cudaStreamSynchronize(s));
    return OT_OK;
}

TreeView tree_view(const ot_octree* t) {
    TreeView v{};
    v.key = t->d_key;
    v.level = t->d_level;
    v.n = (int)t->n;
    v.lmin = t->lmin;
    v.lmax = t->lmax;
    v.lmap = t->d_lmap;
    v.lmap_level = t->lmap_level;
    v.desc = t->d_desc;
    v.lmap_lv = t->d_lmap_lv;
    v.pyr_level = t->pyr_level;
    v.periodic = t->periodic;
    v.mates = reinterpret_cast<const uint4*>(t->d_mates);
    v.pnbr = (t->d_mates && t->lmax >= 1)
                 ? reinterpret_cast<const int*>(reinterpret_cast<const char*>(t->d_mates) + (size_t)256 * t->n)
                 : nullptr;
    v.root = t->d_root;
    v.models = t->d_models;
    v.mids = t->d_mids;
    v.n_leaf = t->n_models;
    v.err = t->d_err;
    v.fallbacks = t->d_fallbacks;
    return v;
}

} // namespace ot
