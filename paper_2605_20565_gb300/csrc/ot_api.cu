// ot_api.cu -- the C ABI: argument validation, octree ownership, dispatch to the kernels.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "ot_internal.h"

using namespace ot;

namespace {

bool kernel_ok(int k) { return k == OT_TRILINEAR || k == OT_PESKIN4 || k == OT_ROMA3; }
bool search_ok(int s) { return s == OT_BINARY || s == OT_LEARNED; }

ot_status check_points(const ot_octree* t, const void* x, const void* y, const void* z, int64_t n) {
    if (!t || n < 0) return OT_ERR_ARG;
    if (n > 0 && (!x || !y || !z)) return OT_ERR_ARG;
    return OT_OK;
}

// AB2 step of point-particle velocity and position, FP32 state, FP64 positions.
__global__ void k_advect(double* __restrict__ x, float* __restrict__ v, float* __restrict__ ap,
                         float* __restrict__ vp, const float* __restrict__ u, int64_t n, float tau, float re_coef,
                         float dt, int first, int periodic) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float rel[3], mag2 = 0.0f;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            rel[d] = u[d * n + i] - v[d * n + i];
            mag2 += rel[d] * rel[d];
        }
        float fp = 1.0f;
        if (re_coef > 0.0f) fp = 1.0f + 0.15f * powf(re_coef * sqrtf(mag2), 0.687f);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float vn = v[d * n + i];
            const float an = fp * rel[d] / tau;
            const float am = first ? an : ap[d * n + i];
            const float vm = first ? vn : vp[d * n + i];
            v[d * n + i] = vn + dt * (1.5f * an - 0.5f * am);
            // the displacement (well below one cell) in FP32, one FP64 add for the position:
            // GB300's FP64 rate made the all-FP64 update the bound of this kernel
            double xn = x[d * n + i] + (double)(dt * (1.5f * vn - 0.5f * vm));
            // outside [0, 1) <=> the bit pattern, read as a signed integer, is negative (sign
            // set, or -0.0 excluded below) or at least that of 1.0: integer compares, not FP64
            const long long xb = __double_as_longlong(xn);
            if (periodic && (xb < 0 || xb >= 0x3FF0000000000000LL) && xb != (long long)0x8000000000000000ULL) {
                xn -= floor(xn);
                if (xn >= 1.0) xn = 0.0;  // -tiny - floor(-tiny) rounds to 1
            }
            x[d * n + i] = xn;
            ap[d * n + i] = an;
            vp[d * n + i] = vn;
        }
    }
}

// The same step for 4 consecutive particles per thread with 16-byte loads and stores (every
// component plane 16-byte aligned: n % 4 == 0 and aligned bases); identical arithmetic.
__device__ __forceinline__ void advect_one(double& x, float& v, float& ap, float& vp, float rel, float fp,
                                           float tau, float dt, int first, int periodic) {
    const float vn = v;
    const float an = fp * rel / tau;
    const float am = first ? an : ap;
    const float vm = first ? vn : vp;
    v = vn + dt * (1.5f * an - 0.5f * am);
    double xn = x + (double)(dt * (1.5f * vn - 0.5f * vm));
    const long long xb = __double_as_longlong(xn);
    if (periodic && (xb < 0 || xb >= 0x3FF0000000000000LL) && xb != (long long)0x8000000000000000ULL) {
        xn -= floor(xn);
        if (xn >= 1.0) xn = 0.0;
    }
    x = xn;
    ap = an;
    vp = vn;
}

__global__ void __launch_bounds__(256) k_advect4(double* __restrict__ x, float* __restrict__ v,
                                                 float* __restrict__ ap, float* __restrict__ vp,
                                                 const float* __restrict__ u, int64_t n, float tau, float re_coef,
                                                 float dt, int first, int periodic) {
    const int64_t nq = n / 4;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
        float4 uu[3], vv[3], aa[3], pp[3];
        double2 xx[3][2];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            uu[d] = reinterpret_cast<const float4*>(u + d * n)[q];
            vv[d] = reinterpret_cast<const float4*>(v + d * n)[q];
            if (!first) {
                aa[d] = reinterpret_cast<const float4*>(ap + d * n)[q];
                pp[d] = reinterpret_cast<const float4*>(vp + d * n)[q];
            }
            xx[d][0] = reinterpret_cast<const double2*>(x + d * n)[2 * q];
            xx[d][1] = reinterpret_cast<const double2*>(x + d * n)[2 * q + 1];
        }
        float* uf[3] = {&uu[0].x, &uu[1].x, &uu[2].x};
        float* vf[3] = {&vv[0].x, &vv[1].x, &vv[2].x};
        float* af[3] = {&aa[0].x, &aa[1].x, &aa[2].x};
        float* pf[3] = {&pp[0].x, &pp[1].x, &pp[2].x};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float rel[3], mag2 = 0.0f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                rel[d] = uf[d][j] - vf[d][j];
                mag2 += rel[d] * rel[d];
            }
            float fp = 1.0f;
            if (re_coef > 0.0f) fp = 1.0f + 0.15f * powf(re_coef * sqrtf(mag2), 0.687f);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                double& xr = j < 2 ? (j == 0 ? xx[d][0].x : xx[d][0].y) : (j == 2 ? xx[d][1].x : xx[d][1].y);
                advect_one(xr, vf[d][j], af[d][j], pf[d][j], rel[d], fp, tau, dt, first, periodic);
            }
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            reinterpret_cast<float4*>(v + d * n)[q] = vv[d];
            reinterpret_cast<float4*>(ap + d * n)[q] = aa[d];
            reinterpret_cast<float4*>(vp + d * n)[q] = pp[d];
            reinterpret_cast<double2*>(x + d * n)[2 * q] = xx[d][0];
            reinterpret_cast<double2*>(x + d * n)[2 * q + 1] = xx[d][1];
        }
    }
}

template <typename T>
ot_status interp_any(const ot_octree* t, int kernel, const double* x, const double* y, const double* z,
                            int64_t n, const int32_t* host_in, int search, const T* field, T* u, int32_t* host_out,
                            void* ws, size_t ws_bytes, void* stream) {
    ot_status st = check_points(t, x, y, z, n);
    if (st != OT_OK) return st;
    if (!kernel_ok(kernel) || !search_ok(search) || (n > 0 && (!field || !u))) return OT_ERR_ARG;
    if (kernel != OT_TRILINEAR && t->lmax < 1) return OT_ERR_ARG;
    if (search == OT_LEARNED && !t->has_index && !(kernel == OT_TRILINEAR && host_in)) return OT_ERR_NO_INDEX;
    return launch_interp<T>(t, kernel, x, y, z, n, host_in, search, field, u, host_out, ws, ws_bytes,
                            (cudaStream_t)stream);
}

template <typename T>
ot_status spread_any(const ot_octree* t, int kernel, int mode, const double* x, const double* y, const double* z,
                            const T* F, const T* dV, int64_t n, T* f, void* ws, size_t ws_bytes, void* stream) {
    ot_status st = check_points(t, x, y, z, n);
    if (st != OT_OK) return st;
    if ((kernel != OT_PESKIN4 && kernel != OT_ROMA3) || (mode != OT_SORTED && mode != OT_ATOMIC)) return OT_ERR_ARG;
    if (n > 0 && (!F || !f)) return OT_ERR_ARG;
    if (t->lmax < 1) return OT_ERR_ARG;
    if (n * 64 >= (1LL << 32)) return OT_ERR_LIMIT; // pair ids are 32-bit
    if (mode == OT_SORTED && n > 0 && (!ws || ((uintptr_t)ws & 15))) return OT_ERR_ARG;
    return launch_spread<T>(t, kernel, mode, x, y, z, F, dV, n, f, ws, ws_bytes, (cudaStream_t)stream);
}

} // namespace

extern "C" {

const char* ot_status_string(ot_status s) {
    switch (s) {
    case OT_OK: return "ok";
    case OT_ERR_ARG: return "invalid argument";
    case OT_ERR_CUDA: return "CUDA error";
    case OT_ERR_OOM: return "out of device memory";
    case OT_ERR_UNSORTED: return "leaves do not tile the unit cube in Morton order";
    case OT_ERR_UNBALANCED: return "leaves violate the 2:1 balance";
    case OT_ERR_NOT_FOUND: return "not found";
    case OT_ERR_STENCIL: return "stencil cell not on the finest level";
    case OT_ERR_LIMIT: return "size limit exceeded";
    case OT_ERR_NO_INDEX: return "no learned index trained";
    }
    return "unknown status";
}

uint64_t ot_launch_count(void) { return g_launches.load(); }

ot_status ot_octree_build(const ot_sphere* h_spheres, int n, const ot_build_params* p, void* stream, ot_octree** out) {
    if (!p || !out || n < 0 || n > OT_MAX_SPHERES || (n > 0 && !h_spheres)) return OT_ERR_ARG;
    if (p->lmin < 0 || p->lmax < p->lmin || p->lmax > OT_MAX_LEVEL) return OT_ERR_ARG;
    if (p->lmin > 7) return OT_ERR_LIMIT; // 8^lmin root cells
    for (int i = 0; i < n; ++i)
        if (!(h_spheres[i].r >= 0.0) || !(h_spheres[i].shell >= 0.0) || !std::isfinite(h_spheres[i].c[0]) ||
            !std::isfinite(h_spheres[i].c[1]) || !std::isfinite(h_spheres[i].c[2]))
            return OT_ERR_ARG;
    *out = nullptr;
    ot_octree* t = new (std::nothrow) ot_octree();
    if (!t) return OT_ERR_OOM;
    cudaGetDevice(&t->device);
    cudaStream_t s = (cudaStream_t)stream;
    ot_status st = build_tree(h_spheres, n, p, s, t);
    if (st == OT_OK) st = finish_tree(t, s);
    if (st != OT_OK) {
        ot_octree_destroy(t);
        return st;
    }
    *out = t;
    return OT_OK;
}

ot_status ot_octree_from_leaves(const uint64_t* d_keys, const uint8_t* d_levels, int64_t n, int balance_full,
                                void* stream, ot_octree** out) {
    if (!d_keys || !d_levels || !out || n < 1) return OT_ERR_ARG;
    if (n > OT_MAX_LEAVES) return OT_ERR_LIMIT;
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    int lmin = 0, lmax = 0;
    ot_status st = validate_leaves(d_keys, d_levels, n, balance_full ? 1 : 0, s, &lmin, &lmax);
    if (st != OT_OK) return st;
    ot_octree* t = new (std::nothrow) ot_octree();
    if (!t) return OT_ERR_OOM;
    cudaGetDevice(&t->device);
    cudaError_t e = cudaMalloc(&t->d_key, sizeof(uint64_t) * n);
    if (e == cudaSuccess) e = cudaMalloc(&t->d_level, n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->d_key, d_keys, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->d_level, d_levels, n, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        ot_octree_destroy(t);
        return cuda_status(e);
    }
    t->n = n;
    t->lmin = lmin;
    t->lmax = lmax;
    st = finish_tree(t, s);
    if (st != OT_OK) {
        ot_octree_destroy(t);
        return st;
    }
    *out = t;
    return OT_OK;
}

ot_status ot_octree_info(const ot_octree* t, int64_t* n, int* lmin, int* lmax) {
    if (!t) return OT_ERR_ARG;
    if (n) *n = t->n;
    if (lmin) *lmin = t->lmin;
    if (lmax) *lmax = t->lmax;
    return OT_OK;
}

ot_status ot_octree_leaves(const ot_octree* t, int64_t* n, const uint64_t** d_keys, const uint8_t** d_levels) {
    if (!t) return OT_ERR_ARG;
    if (n) *n = t->n;
    if (d_keys) *d_keys = t->d_key;
    if (d_levels) *d_levels = t->d_level;
    return OT_OK;
}

ot_status ot_octree_copy_leaves(const ot_octree* t, uint64_t* d_keys, uint8_t* d_levels, void* stream) {
    if (!t) return OT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (d_keys) OT_CUDA(cudaMemcpyAsync(d_keys, t->d_key, sizeof(uint64_t) * t->n, cudaMemcpyDeviceToDevice, s));
    if (d_levels) OT_CUDA(cudaMemcpyAsync(d_levels, t->d_level, t->n, cudaMemcpyDeviceToDevice, s));
    return OT_OK;
}

ot_status ot_octree_set_periodic(ot_octree* t, int periodic) {
    if (!t || (periodic != 0 && periodic != 1)) return OT_ERR_ARG;
    if (t->periodic == periodic) return OT_OK;
    t->periodic = periodic;
    // the level-mate table wraps or clamps at the faces: refilled for the new setting
    if (t->d_mates) {
        OT_CUDA(cudaDeviceSynchronize());
        const ot_status st = build_mates(t, nullptr);
        if (st != OT_OK) return st;
        OT_CUDA(cudaStreamSynchronize(nullptr));
    }
    return OT_OK;
}

ot_status ot_octree_get_map_level(const ot_octree* t, int* level) {
    if (!t || !level) return OT_ERR_ARG;
    *level = t->lmap_level;
    return OT_OK;
}

ot_status ot_octree_set_map_level(ot_octree* t, int level, void* stream) {
    if (!t || level < 0 || level > 8) return OT_ERR_ARG;
    return finish_tree(t, (cudaStream_t)stream, level);
}

ot_status ot_octree_centres(const ot_octree* t, double* d_xyz, void* stream) {
    if (!t || !d_xyz) return OT_ERR_ARG;
    return leaf_centres(t, d_xyz, (cudaStream_t)stream);
}

ot_status ot_octree_destroy(ot_octree* t) {
    if (!t) return OT_OK;
    if (t->d_key) cudaFree(t->d_key);
    if (t->d_level) cudaFree(t->d_level);
    if (t->d_lmap && t->d_lmap != t->d_pmap) cudaFree(t->d_lmap);
    if (t->d_pmap) cudaFree(t->d_pmap);
    if (t->d_nodes) cudaFree(t->d_nodes);
    if (t->d_desc) cudaFree(t->d_desc);
    if (t->d_lmap_lv) cudaFree(t->d_lmap_lv);
    if (t->d_mates && t->mates_owned) cudaFree(t->d_mates);
    if (t->d_need_flags) cudaFree(t->d_need_flags);
    if (t->d_models) cudaFree(t->d_models);
    if (t->d_mids) cudaFree(t->d_mids);
    if (t->d_root) cudaFree(t->d_root);
    if (t->d_err) cudaFree(t->d_err);
    delete t;
    return OT_OK;
}

ot_status ot_index_train(ot_octree* t, const ot_index_params* p, void* stream) {
    if (!t || !p) return OT_ERR_ARG;
    if (p->root != OT_ROOT_LINEAR && p->root != OT_ROOT_MLP) return OT_ERR_ARG;
    if (p->n_leaf_models < 1 || p->n_leaf_models > (1 << 22)) return OT_ERR_ARG;
    if (p->n_mid_models < 0 || p->n_mid_models > (1 << 20)) return OT_ERR_ARG;
    if (p->root == OT_ROOT_MLP && (p->epochs < 0 || p->steps < 0 || p->batch < 1 || !(p->lr >= 0.0f)))
        return OT_ERR_ARG;
    return train_index(t, p, (cudaStream_t)stream);
}

ot_status ot_index_get_root_params(const ot_octree* t, float* h) {
    if (!t || !h) return OT_ERR_ARG;
    if (!t->has_index || t->root.kind != OT_ROOT_MLP) return OT_ERR_NO_INDEX;
    for (int k = 0; k < MLP_H; ++k) {
        h[k] = t->root.w1[k];
        h[MLP_H + k] = t->root.b1[k];
        h[2 * MLP_H + k] = t->root.w2[k];
    }
    h[3 * MLP_H] = t->root.b2;
    return OT_OK;
}

ot_status ot_index_get_stats(const ot_octree* t, ot_index_stats* s, int reset) {
    if (!t || !s) return OT_ERR_ARG;
    if (!t->has_index) return OT_ERR_NO_INDEX;
    std::vector<LeafModel> m(t->n_models);
    OT_CUDA(cudaMemcpy(m.data(), t->d_models, sizeof(LeafModel) * m.size(), cudaMemcpyDeviceToHost));
    double sum = 0.0, probes = 0.0;
    int64_t mx = 0, empty = 0, used = 0;
    for (const LeafModel& x : m) {
        if (x.count == 0 || x.err_lo < 0) {  // no stored key routed here (filled model)
            ++empty;
            continue;
        }
        const int64_t w = (int64_t)x.err_lo + x.err_hi + 3;
        sum += (double)w * x.count; // weighted by the keys the model serves
        probes += std::ceil(std::log2((double)w)) * x.count;
        used += x.count;
        mx = std::max(mx, w);
    }
    s->mean_window = used ? sum / (double)used : 0.0;
    s->mean_probes = used ? probes / (double)used : 0.0;
    s->max_window = mx;
    s->empty_models = empty;
    unsigned long long fb = 0;
    OT_CUDA(cudaMemcpy(&fb, t->d_fallbacks, sizeof(fb), cudaMemcpyDeviceToHost));
    s->fallbacks = fb;
    s->final_loss = t->final_loss;
    if (reset) OT_CUDA(cudaMemset(t->d_fallbacks, 0, sizeof(unsigned long long)));
    return OT_OK;
}

ot_status ot_index_mlp_grad(const float* d_params, const float* d_x, const float* d_t, int64_t n, float* d_grad,
                            float* d_loss, void* stream) {
    if (!d_params || !d_x || !d_t || !d_grad || n < 1) return OT_ERR_ARG;
    return mlp_grad(d_params, d_x, d_t, n, d_grad, d_loss, (cudaStream_t)stream);
}

ot_status ot_locate(const ot_octree* t, const double* x, const double* y, const double* z, int64_t n, int search,
                    int32_t* host, unsigned long long* n_miss, void* stream) {
    ot_status st = check_points(t, x, y, z, n);
    if (st != OT_OK) return st;
    if (!search_ok(search) || (n > 0 && !host)) return OT_ERR_ARG;
    if (search == OT_LEARNED && !t->has_index) return OT_ERR_NO_INDEX;
    return launch_locate(t, x, y, z, n, search, host, n_miss, (cudaStream_t)stream);
}

ot_status ot_interpolate_workspace_size(const ot_octree* t, int kernel, int fp64, size_t* bytes) {
    if (!t || !bytes || !kernel_ok(kernel)) return OT_ERR_ARG;
    *bytes = interp_ws_bytes(t, kernel, fp64 ? sizeof(double) : sizeof(float));
    return OT_OK;
}

ot_status ot_interpolate(const ot_octree* t, int kernel, const double* x, const double* y, const double* z, int64_t n,
                         const int32_t* host_in, int search, const float* field, float* u, int32_t* host_out,
                         void* ws, size_t ws_bytes, void* stream) {
    return interp_any<float>(t, kernel, x, y, z, n, host_in, search, field, u, host_out, ws, ws_bytes, stream);
}

ot_status ot_interpolate_f64(const ot_octree* t, int kernel, const double* x, const double* y, const double* z,
                             int64_t n, const int32_t* host_in, int search, const double* field, double* u,
                             int32_t* host_out, void* ws, size_t ws_bytes, void* stream) {
    return interp_any<double>(t, kernel, x, y, z, n, host_in, search, field, u, host_out, ws, ws_bytes, stream);
}

ot_status ot_spread_workspace_size(const ot_octree* t, int kernel, int64_t n, size_t* bytes) {
    if (!t || !bytes || n < 0 || (kernel != OT_PESKIN4 && kernel != OT_ROMA3)) return OT_ERR_ARG;
    *bytes = spread_ws_bytes(t, kernel, n);
    return OT_OK;
}

ot_status ot_spread(const ot_octree* t, int kernel, int mode, const double* x, const double* y, const double* z,
                    const float* F, const float* dV, int64_t n, float* f, void* ws, size_t ws_bytes, void* stream) {
    return spread_any<float>(t, kernel, mode, x, y, z, F, dV, n, f, ws, ws_bytes, stream);
}

ot_status ot_spread_f64(const ot_octree* t, int kernel, int mode, const double* x, const double* y, const double* z,
                        const double* F, const double* dV, int64_t n, double* f, void* ws, size_t ws_bytes,
                        void* stream) {
    return spread_any<double>(t, kernel, mode, x, y, z, F, dV, n, f, ws, ws_bytes, stream);
}

ot_status ot_advect_ab2(double* x, float* v, float* ap, float* vp, const float* u, int64_t n, float tau, float re_coef,
                        float dt, int first, int periodic, void* stream) {
    if (n < 0 || (n > 0 && (!x || !v || !ap || !vp || !u)) || !(tau > 0.0f) || !(re_coef >= 0.0f)) return OT_ERR_ARG;
    if (n == 0) return OT_OK;
    const bool aligned = n % 4 == 0 && ((uintptr_t)x & 15) == 0 && ((uintptr_t)v & 15) == 0 &&
                         ((uintptr_t)ap & 15) == 0 && ((uintptr_t)vp & 15) == 0 && ((uintptr_t)u & 15) == 0;
    if (aligned) {
        const int64_t g = std::min<int64_t>((n / 4 + 255) / 256, (int64_t)num_sms() * 8);
        k_advect4<<<(unsigned)g, 256, 0, (cudaStream_t)stream>>>(x, v, ap, vp, u, n, tau, re_coef, dt, first,
                                                                 periodic);
    } else {
        const int64_t g = std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8);
        k_advect<<<(unsigned)g, 256, 0, (cudaStream_t)stream>>>(x, v, ap, vp, u, n, tau, re_coef, dt, first,
                                                                periodic);
    }
    count_launch();
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

ot_status ot_last_error(const ot_octree* t, unsigned* bits, int clear, void* stream) {
    if (!t || !bits) return OT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    OT_CUDA(cudaMemcpyAsync(bits, t->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    OT_CUDA(cudaStreamSynchronize(s));
    if (clear) {
        OT_CUDA(cudaMemsetAsync(t->d_err, 0, sizeof(unsigned), s));
        OT_CUDA(cudaStreamSynchronize(s));
    }
    return OT_OK;
}

} // extern "C"
