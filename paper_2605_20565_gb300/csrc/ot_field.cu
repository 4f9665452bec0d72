// ot_field.cu -- an analytic cell-centred field on the leaves: u(x) = sum_m A_m cos(2 pi n_m . x
// + phi_m) at every leaf centre, for integer wave vectors n_m (the random solenoidal fields the
// tracking driver re-samples on each new octree, standing in for the fluid solver's field).
// The phase is exact fixed point: a leaf centre at level l is (2 x + 2^(21-l)) 2^-22 per axis
// (x its level-21 anchor coordinate), so n . x in turns is an integer times 2^-22; with the
// phase rounded to 2^-32 turns the whole argument reduces modulo one turn in integer
// arithmetic, and only the final cosine is FP32 (cospif).
#include <algorithm>
#include <cmath>

#include "ot_internal.h"

namespace ot {

namespace {

constexpr int MAX_MODES = 64;

struct Modes {
    int m;
    int n[MAX_MODES][3];
    float amp[MAX_MODES][3];
    uint32_t phase[MAX_MODES];  // turns, 2^-32 units
};

__global__ void __launch_bounds__(256) k_field_fourier(const uint64_t* __restrict__ key,
                                                       const uint8_t* __restrict__ level, int64_t n, Modes md,
                                                       float4* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x, y, z;
        demorton3(key[i], x, y, z);
        const int64_t off = (int64_t)1 << (MAXLEVEL - level[i]);
        const int64_t cx = 2 * (int64_t)x + off, cy = 2 * (int64_t)y + off, cz = 2 * (int64_t)z + off;
        float u0 = 0.0f, u1 = 0.0f, u2 = 0.0f;
        for (int k = 0; k < md.m; ++k) {
            const int64_t t = md.n[k][0] * cx + md.n[k][1] * cy + md.n[k][2] * cz;  // turns, 2^-22 units
            const uint32_t T = ((uint32_t)(uint64_t)t << 10) + md.phase[k];          // mod 1 turn, 2^-32 units
            const float fr = (float)(int32_t)T * 0x1p-32f;                             // in [-1/2, 1/2)
            const float c = cospif(2.0f * fr);
            u0 += md.amp[k][0] * c;
            u1 += md.amp[k][1] * c;
            u2 += md.amp[k][2] * c;
        }
        out[i] = make_float4(u0, u1, u2, 0.0f);
    }
}

// Volume-weighted field sums, FP64: block b adds the leaves of its stride in a fixed order,
// then a fixed tree; a single block then adds the block partials in order.
constexpr int MT = 256;

__global__ void __launch_bounds__(MT) k_field_sum(const uint8_t* __restrict__ level, int64_t n,
                                                  const float4* __restrict__ f, double* __restrict__ part) {
    __shared__ double s[3][MT];
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)MT + threadIdx.x; i < n; i += (int64_t)gridDim.x * MT) {
        const double vol = __longlong_as_double((long long)(1023 - 3 * (int)level[i]) << 52);  // 8^-level
        const float4 v = f[i];
        a0 += vol * v.x, a1 += vol * v.y, a2 += vol * v.z;
    }
    s[0][threadIdx.x] = a0, s[1][threadIdx.x] = a1, s[2][threadIdx.x] = a2;
    __syncthreads();
    for (int o = MT / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int c = 0; c < 3; ++c) s[c][threadIdx.x] += s[c][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 3) part[3 * blockIdx.x + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void k_field_mean_finish(const double* __restrict__ part, int nb, double* __restrict__ mean) {
    if (threadIdx.x < 3) {
        double a = 0.0;
        for (int b = 0; b < nb; ++b) a += part[3 * b + threadIdx.x];
        mean[threadIdx.x] = a;  // the unit cube's volume is 1
    }
}

__global__ void __launch_bounds__(MT) k_field_sub(float4* __restrict__ f, int64_t n, const double* __restrict__ mean) {
    const float m0 = (float)mean[0], m1 = (float)mean[1], m2 = (float)mean[2];
    for (int64_t i = blockIdx.x * (int64_t)MT + threadIdx.x; i < n; i += (int64_t)gridDim.x * MT) {
        float4 v = f[i];
        v.x -= m0, v.y -= m1, v.z -= m2;
        f[i] = v;
    }
}

} // namespace

} // namespace ot

using namespace ot;

// Block partials of the mean: at most MEAN_BLOCKS blocks, so the workspace has a fixed size.
constexpr int MEAN_BLOCKS = 1024;

extern "C" ot_status ot_field_mean_workspace_size(const ot_octree* t, size_t* bytes) {
    if (!t || !bytes) return OT_ERR_ARG;
    *bytes = sizeof(double) * (3 * (size_t)MEAN_BLOCKS + 3);
    return OT_OK;
}

extern "C" ot_status ot_field_subtract_mean(const ot_octree* t, float* d_field, double* d_mean, void* d_workspace,
                                            size_t ws_bytes, void* stream) {
    if (!t || !d_field || !d_workspace || ((uintptr_t)d_workspace & 7) ||
        ws_bytes < sizeof(double) * (3 * (size_t)MEAN_BLOCKS + 3))
        return OT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (int)std::max<int64_t>(
        1, std::min<int64_t>({(t->n + MT - 1) / MT, (int64_t)num_sms() * 4, (int64_t)MEAN_BLOCKS}));
    double* part = static_cast<double*>(d_workspace);
    double* mean = part + 3 * nb;
    k_field_sum<<<nb, MT, 0, s>>>(t->d_level, t->n, reinterpret_cast<const float4*>(d_field), part);
    k_field_mean_finish<<<1, 32, 0, s>>>(part, nb, mean);
    k_field_sub<<<nb, MT, 0, s>>>(reinterpret_cast<float4*>(d_field), t->n, mean);
    count_launch(3);
    if (d_mean) OT_CUDA(cudaMemcpyAsync(d_mean, mean, sizeof(double) * 3, cudaMemcpyDeviceToDevice, s));
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

extern "C" ot_status ot_field_fourier(const ot_octree* t, int n_modes, const int32_t* h_wave, const double* h_amp,
                                      const double* h_phase, float* d_field, void* stream) {
    if (!t || n_modes < 0 || n_modes > MAX_MODES || (n_modes > 0 && (!h_wave || !h_amp || !h_phase)) || !d_field)
        return OT_ERR_ARG;
    Modes md{};
    md.m = n_modes;
    for (int k = 0; k < n_modes; ++k) {
        for (int d = 0; d < 3; ++d) {
            const int32_t w = h_wave[3 * k + d];
            if (w < -(1 << 12) || w > (1 << 12)) return OT_ERR_ARG;
            md.n[k][d] = w;
            md.amp[k][d] = (float)h_amp[3 * k + d];
        }
        double turns = h_phase[k] / (2.0 * M_PI);
        turns -= std::floor(turns);
        md.phase[k] = (uint32_t)(uint64_t)std::llround(turns * 4294967296.0);
    }
    if (t->n == 0) return OT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((t->n + 255) / 256, (int64_t)num_sms() * 8));
    k_field_fourier<<<grid, 256, 0, s>>>(t->d_key, t->d_level, t->n, md, reinterpret_cast<float4*>(d_field));
    count_launch();
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}
