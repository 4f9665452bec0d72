// ot_mdf.cu -- multi-direct forcing (Sec. 2.2): n_iter rounds of
//   u_k = I u (delta-kernel interpolation), F_k = (U_k - u_k) / dt, F = S F_k (sorted,
//   deterministic spreading), u += dt F / rho, f += F,
// on the device, with one more interpolation at the end for the final slip.  Every step is a
// library kernel on the caller's stream; the workspace is the caller's.
#include <algorithm>

#include "ot_internal.h"

namespace ot {

namespace {

// F_k = (U_k - u_k) / dt; the squared slip summed into *slip2 (FP64, one atomic per block).
__global__ void __launch_bounds__(256) k_mdf_force(const float* __restrict__ U, const float* __restrict__ uk,
                                                   int64_t n, float inv_dt, float* __restrict__ Fk,
                                                   double* __restrict__ slip2) {
    __shared__ double s_part[8];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * n; i += (int64_t)gridDim.x * blockDim.x) {
        const float e = U[i] - uk[i];
        Fk[i] = e * inv_dt;
        acc += (double)e * (double)e;
    }
    if (!slip2) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += s_part[w];
        atomicAdd(slip2, b);
    }
}

// F_k = (0 - u_k) / dt: markers of a body at rest.
__global__ void __launch_bounds__(256) k_rest_force(const float* __restrict__ uk, int64_t n, float inv_dt,
                                                    float* __restrict__ Fk) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * n; i += (int64_t)gridDim.x * blockDim.x)
        Fk[i] = (0.0f - uk[i]) * inv_dt;
}

// u += scale F, f += F over the leaves (component 3 untouched).
__global__ void __launch_bounds__(256) k_mdf_correct(float4* __restrict__ u, float4* __restrict__ f,
                                                     const float4* __restrict__ F, int64_t n, float scale) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 d = F[i];
        if (d.x == 0.0f && d.y == 0.0f && d.z == 0.0f) continue;  // leaves the force does not reach
        float4 a = u[i], b = f[i];
        a.x += scale * d.x, a.y += scale * d.y, a.z += scale * d.z;
        b.x += d.x, b.y += d.y, b.z += d.z;
        u[i] = a;
        f[i] = b;
    }
}

__global__ void k_sqrt_slip(const double* __restrict__ s2, float* __restrict__ slip, int m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) slip[i] = (float)sqrt(s2[i]);
}

unsigned grid_of(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 8));
}

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

} // namespace

size_t mdf_ws_bytes(const ot_octree* t, int kernel, int64_t n, int n_iter) {
    return 2 * up256(sizeof(float) * 3 * (size_t)n) + up256(sizeof(float4) * (size_t)t->n) +
           up256(sizeof(double) * (size_t)(n_iter + 1)) + up256(spread_ws_bytes(t, kernel, n)) + 256;
}

ot_status launch_mdf(const ot_octree* t, int kernel, const double* x, const double* y, const double* z,
                     const float* U, const float* dV, int64_t n, float rho, float dt, int n_iter, float* u, float* f,
                     float* slip, void* ws, cudaStream_t s) {
    char* p = static_cast<char*>(ws);
    float* uk = reinterpret_cast<float*>(p);
    p += up256(sizeof(float) * 3 * (size_t)n);
    float* Fk = reinterpret_cast<float*>(p);
    p += up256(sizeof(float) * 3 * (size_t)n);
    float4* F = reinterpret_cast<float4*>(p);
    p += up256(sizeof(float4) * (size_t)t->n);
    double* s2 = reinterpret_cast<double*>(p);
    p += up256(sizeof(double) * (size_t)(n_iter + 1));
    void* sws = p;
    const size_t sws_bytes = spread_ws_bytes(t, kernel, n);
    OT_CUDA(cudaMemsetAsync(f, 0, sizeof(float4) * (size_t)t->n, s));
    if (slip) OT_CUDA(cudaMemsetAsync(s2, 0, sizeof(double) * (size_t)(n_iter + 1), s));
    ot_status st;
    for (int it = 0; it <= n_iter; ++it) {
        if ((st = launch_interp<float>(t, kernel, x, y, z, n, nullptr, OT_BINARY, u, uk, nullptr, nullptr, 0, s)) != OT_OK)
            return st;
        k_mdf_force<<<grid_of(3 * n), 256, 0, s>>>(U, uk, n, 1.0f / dt, Fk, slip ? s2 + it : nullptr);
        count_launch();
        if (it == n_iter) break;
        OT_CUDA(cudaMemsetAsync(F, 0, sizeof(float4) * (size_t)t->n, s));
        if ((st = launch_spread<float>(t, kernel, OT_SORTED, x, y, z, Fk, dV, n, reinterpret_cast<float*>(F), sws,
                                       sws_bytes, s)) != OT_OK)
            return st;
        k_mdf_correct<<<grid_of(t->n), 256, 0, s>>>(reinterpret_cast<float4*>(u), reinterpret_cast<float4*>(f), F,
                                                    t->n, dt / rho);
        count_launch();
    }
    if (slip) {
        k_sqrt_slip<<<(n_iter + 1 + 63) / 64, 64, 0, s>>>(s2, slip, n_iter + 1);
        count_launch();
    }
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

} // namespace ot

using namespace ot;

extern "C" ot_status ot_marker_force(const float* d_U, const float* d_u, int64_t n, float dt, float* d_F,
                                     void* stream) {
    if (n < 0 || !(dt > 0.0f) || (n > 0 && (!d_u || !d_F))) return OT_ERR_ARG;
    if (n == 0) return OT_OK;
    if (d_U) {
        k_mdf_force<<<grid_of(3 * n), 256, 0, (cudaStream_t)stream>>>(d_U, d_u, n, 1.0f / dt, d_F, nullptr);
    } else {
        k_rest_force<<<grid_of(3 * n), 256, 0, (cudaStream_t)stream>>>(d_u, n, 1.0f / dt, d_F);
    }
    count_launch();
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

extern "C" ot_status ot_ibm_mdf_workspace_size(const ot_octree* t, int kernel, int64_t n, int n_iter, size_t* bytes) {
    if (!t || !bytes || n < 0 || n_iter < 0 || (kernel != OT_PESKIN4 && kernel != OT_ROMA3)) return OT_ERR_ARG;
    *bytes = mdf_ws_bytes(t, kernel, n, n_iter);
    return OT_OK;
}

extern "C" ot_status ot_ibm_mdf(const ot_octree* t, int kernel, const double* d_x, const double* d_y,
                                const double* d_z, const float* d_U, const float* d_dV, int64_t n, float rho, float dt,
                                int n_iter, float* d_u, float* d_f, float* d_slip, void* d_workspace,
                                size_t ws_bytes, void* stream) {
    if (!t || (kernel != OT_PESKIN4 && kernel != OT_ROMA3) || n < 0 || n_iter < 0 || !d_u || !d_f) return OT_ERR_ARG;
    if (!(rho > 0.0f) || !(dt > 0.0f) || t->lmax < 1) return OT_ERR_ARG;
    if (n > 0 && (!d_x || !d_y || !d_z || !d_U)) return OT_ERR_ARG;
    if (n * 64 >= (1LL << 32)) return OT_ERR_LIMIT;
    if (!d_workspace || ((uintptr_t)d_workspace & 255) || ws_bytes < mdf_ws_bytes(t, kernel, n, n_iter))
        return OT_ERR_ARG;
    return launch_mdf(t, kernel, d_x, d_y, d_z, d_U, d_dV, n, rho, dt, n_iter, d_u, d_f, d_slip, d_workspace,
                      (cudaStream_t)stream);
}
