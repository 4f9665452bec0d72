// ot_body.cu -- per-body linear and angular sums of a marker quantity (Sec. 2.3, rigid bodies):
//   lin_b = scale sum_{k in b} v_k w_k,   ang_b = scale sum_{k in b} (X_k - x_b) x v_k w_k.
// With v the velocity interpolated at the internal markers and scale = rho_f these are the
// internal fluid's linear and angular momenta P and L; with v = F_k at the surface markers and
// scale = -1, the IBM force and torque.  One block per body, FP64 accumulation in a fixed
// order (thread-strided, then a fixed tree): bit-identical from run to run.
#include "ot_internal.h"

namespace ot {

namespace {

constexpr int BT = 256;

__global__ void __launch_bounds__(BT) k_body_sums(const double* __restrict__ x, const double* __restrict__ y,
                                                  const double* __restrict__ z, const float* __restrict__ v,
                                                  const float* __restrict__ dV, float w, int64_t n,
                                                  const int64_t* __restrict__ start, const double* __restrict__ xb,
                                                  double scale, double* __restrict__ lin, double* __restrict__ ang) {
    __shared__ double s[6][BT];
    const int b = blockIdx.x;
    const int64_t k0 = start[b], k1 = start[b + 1];
    const double cx = xb[3 * b], cy = xb[3 * b + 1], cz = xb[3 * b + 2];
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t k = k0 + threadIdx.x; k < k1; k += BT) {
        const double wk = dV ? (double)dV[k] : (double)w;
        const double v0 = (double)v[k] * wk, v1 = (double)v[n + k] * wk, v2 = (double)v[2 * n + k] * wk;
        const double r0 = x[k] - cx, r1 = y[k] - cy, r2 = z[k] - cz;
        acc[0] += v0;
        acc[1] += v1;
        acc[2] += v2;
        acc[3] += r1 * v2 - r2 * v1;
        acc[4] += r2 * v0 - r0 * v2;
        acc[5] += r0 * v1 - r1 * v0;
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) s[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int o = BT / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
#pragma unroll
            for (int c = 0; c < 6; ++c) s[c][threadIdx.x] += s[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 3) {
        lin[3 * b + threadIdx.x] = scale * s[threadIdx.x][0];
        ang[3 * b + threadIdx.x] = scale * s[3 + threadIdx.x][0];
    }
}

} // namespace

} // namespace ot

using namespace ot;

extern "C" ot_status ot_body_sums(const double* d_x, const double* d_y, const double* d_z, const float* d_v,
                                  const float* d_dV, float w, int64_t n, const int64_t* d_start, int n_bodies,
                                  const double* d_xb, double scale, double* d_lin, double* d_ang, void* stream) {
    if (n < 0 || n_bodies < 0 || n_bodies > (1 << 24)) return OT_ERR_ARG;
    if (n_bodies == 0) return OT_OK;
    if (!d_start || !d_xb || !d_lin || !d_ang || (n > 0 && (!d_x || !d_y || !d_z || !d_v))) return OT_ERR_ARG;
    k_body_sums<<<n_bodies, BT, 0, (cudaStream_t)stream>>>(d_x, d_y, d_z, d_v, d_dV, w, n, d_start, d_xb, scale,
                                                            d_lin, d_ang);
    count_launch();
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}
