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

} // namespace

} // namespace ot

using namespace ot;

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
