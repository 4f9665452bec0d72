// ot_learned.cu -- two-stage learned index over the octree's Morton keys, trained on the device.
//
// Root: a linear model fitted in closed form, or a 1 -> 32 (ReLU) -> 1 network trained with
// Adam on minibatches of (key 2^-63, i / N).  The network starts as the 32-knot linear spline of
// the empirical key CDF (knots at x = k/32) and is refined by its own forward and backward
// kernels.  Leaves: every key is routed by the root; each leaf model is a least-squares line
// through (key - base, i) of the keys routed to it, with the largest under- and
// over-prediction over those keys stored as its search window (computed with the query's
// own arithmetic).
#include <algorithm>
#include <cmath>
#include <vector>

#include "ot_internal.h"

namespace ot {

namespace {

#define GSTRIDE(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// Block sum of `v` (doubles), result valid in thread 0.  Fixed reduction order.
template <int NT>
__device__ double block_sum_d(double v, double* s) {
    s[threadIdx.x] = v;
    __syncthreads();
#pragma unroll
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    double r = s[0];
    __syncthreads();
    return r;
}

// ----- linear root: closed-form least squares over (x_i, i/N), two passes, FP64 ------------
constexpr int LT = 256;

__global__ void k_lin_sums(const uint64_t* __restrict__ key, int64_t n, double* __restrict__ part, int pass,
                           const double* __restrict__ means) {
    __shared__ double s[LT];
    double a = 0, b = 0;
    const double mx = pass ? means[0] : 0.0, my = pass ? means[1] : 0.0;
    GSTRIDE(i, n) {
        const double x = (double)key_to_x(key[i]);
        const double y = (double)i / (double)n;
        if (pass == 0) {
            a += x;
            b += y;
        } else {
            a += (x - mx) * (y - my);
            b += (x - mx) * (x - mx);
        }
    }
    a = block_sum_d<LT>(a, s);
    b = block_sum_d<LT>(b, s);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

// A model that no stored key was routed to: under monotone routing every query that reaches it
// lies between the last key of the previous non-empty model and the first key of the next
// one, so its answer is the index just before the next model's first key.  The model
// predicts that index with the window [pc, pc + 1] (err_lo = -1 marks it as filled); a query
// that breaks the premise fails verification and falls back.
__global__ void k_fill_empty(const LeafModel* __restrict__ fitted, LeafModel* __restrict__ models, int nm,
                             int nkeys) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nm; j += gridDim.x * blockDim.x) {
        if (fitted[j].count > 0) continue;
        int k = j + 1;
        while (k < nm && fitted[k].count <= 0) ++k;
        const int first_next = k < nm ? fitted[k].first : nkeys;
        LeafModel m{};
        m.base = 0;
        m.slope = 0.0f;
        m.icpt = 0.0f;
        m.first = max(first_next - 1, 0);
        m.count = 1;
        m.err_lo = -1;
        m.err_hi = 0;
        models[j] = m;
    }
}

__global__ void k_lin_finish(const double* __restrict__ part, int nb, int64_t n, double* __restrict__ means, int pass) {
    if (threadIdx.x != 0) return;
    double a = 0, b = 0;
    for (int i = 0; i < nb; ++i) {
        a += part[2 * i];
        b += part[2 * i + 1];
    }
    if (pass == 0) {
        means[0] = a / (double)n;
        means[1] = b / (double)n;
    } else {
        const double slope = b > 0 ? a / b : 0.0;
        means[2] = slope;
        means[3] = means[1] - slope * means[0];
    }
}

// ----- MLP root ---------------------------------------------------------------------------
constexpr int MT = 256;

struct Adam {
    float m[MLP_NPARAM], v[MLP_NPARAM];
};

__device__ __forceinline__ void mlp_fwd_bwd(const float* __restrict__ p, float x, float t, float inv_n, float* g,
                                            float& loss) {
    float z[MLP_H];
    float y = p[3 * MLP_H];
#pragma unroll
    for (int k = 0; k < MLP_H; ++k) {
        z[k] = __fadd_rn(__fmul_rn(p[k], x), p[MLP_H + k]);
        y = __fadd_rn(y, __fmul_rn(p[2 * MLP_H + k], fmaxf(z[k], 0.0f)));
    }
    const float e = y - t;
    loss += e * e * inv_n;
    const float gy = 2.0f * e * inv_n;
    g[3 * MLP_H] += gy;
#pragma unroll
    for (int k = 0; k < MLP_H; ++k) {
        const float h = fmaxf(z[k], 0.0f);
        g[2 * MLP_H + k] += gy * h;
        const float dz = z[k] > 0.0f ? gy * p[2 * MLP_H + k] : 0.0f;
        g[k] += dz * x;
        g[MLP_H + k] += dz;
    }
}

// Partial gradients of one block, reduced in shared memory in a fixed order.
__device__ void block_reduce_grad(float* g, float loss, float* s_red, float* out) {
    // s_red: MT floats
    for (int j = 0; j <= MLP_NPARAM; ++j) {
        const float v = j < MLP_NPARAM ? g[j] : loss;
        s_red[threadIdx.x] = v;
        __syncthreads();
        for (int o = MT / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) s_red[threadIdx.x] += s_red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[j] = s_red[0];
        __syncthreads();
    }
}

// Gradient of the MSE loss over given samples: one partial row per block.
__global__ void __launch_bounds__(MT) k_mlp_grad_samples(const float* __restrict__ p, const float* __restrict__ xs,
                                                         const float* __restrict__ ts, int64_t n,
                                                         float* __restrict__ part) {
    __shared__ float s_p[MLP_NPARAM];
    __shared__ float s_red[MT];
    for (int j = threadIdx.x; j < MLP_NPARAM; j += blockDim.x) s_p[j] = p[j];
    __syncthreads();
    float g[MLP_NPARAM];
#pragma unroll
    for (int j = 0; j < MLP_NPARAM; ++j) g[j] = 0.0f;
    float loss = 0.0f;
    const float inv_n = 1.0f / (float)n;
    GSTRIDE(i, n) mlp_fwd_bwd(s_p, xs[i], ts[i], inv_n, g, loss);
    block_reduce_grad(g, loss, s_red, part + (size_t)blockIdx.x * (MLP_NPARAM + 1));
}

__global__ void k_sum_rows(const float* __restrict__ part, int nb, float* __restrict__ grad, float* __restrict__ loss) {
    for (int j = threadIdx.x; j <= MLP_NPARAM; j += blockDim.x) {
        float a = 0.0f;
        for (int b = 0; b < nb; ++b) a += part[(size_t)b * (MLP_NPARAM + 1) + j];
        if (j < MLP_NPARAM)
            grad[j] = a;
        else if (loss)
            *loss = a;
    }
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// One training step on a minibatch drawn by a counter-based hash of (seed, step, sample).
__global__ void __launch_bounds__(MT) k_mlp_step_grad(const float* __restrict__ p, const uint64_t* __restrict__ key,
                                                      int64_t n, int batch, uint64_t seed, int step,
                                                      float* __restrict__ part) {
    __shared__ float s_p[MLP_NPARAM];
    __shared__ float s_red[MT];
    for (int j = threadIdx.x; j < MLP_NPARAM; j += blockDim.x) s_p[j] = p[j];
    __syncthreads();
    float g[MLP_NPARAM];
#pragma unroll
    for (int j = 0; j < MLP_NPARAM; ++j) g[j] = 0.0f;
    float loss = 0.0f;
    const float inv_n = 1.0f / (float)batch;
    GSTRIDE(b, (int64_t)batch) {
        const uint64_t r = mix64(seed * 0x9E3779B97F4A7C15ULL + ((uint64_t)step << 32) + (uint64_t)b + 1);
        const int64_t i = (int64_t)(r % (uint64_t)n);
        mlp_fwd_bwd(s_p, key_to_x(key[i]), (float)((double)i / (double)n), inv_n, g, loss);
    }
    block_reduce_grad(g, loss, s_red, part + (size_t)blockIdx.x * (MLP_NPARAM + 1));
}

__global__ void k_adam(float* __restrict__ p, Adam* __restrict__ st, const float* __restrict__ part, int nb, int step,
                       float lr, float* __restrict__ loss_out) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - powf(b1, (float)(step + 1)), c2 = 1.0f - powf(b2, (float)(step + 1));
    for (int j = threadIdx.x; j <= MLP_NPARAM; j += blockDim.x) {
        float gj = 0.0f;
        for (int b = 0; b < nb; ++b) gj += part[(size_t)b * (MLP_NPARAM + 1) + j];
        if (j == MLP_NPARAM) {
            *loss_out = gj;
            continue;
        }
        st->m[j] = b1 * st->m[j] + (1.0f - b1) * gj;
        st->v[j] = b2 * st->v[j] + (1.0f - b2) * gj * gj;
        const float mh = st->m[j] / c1, vh = st->v[j] / c2;
        p[j] -= lr * mh / (sqrtf(vh) + eps);
    }
}

// Empirical CDF at the knots x = k/32: first index with key >= k 2^58.
__global__ void k_knot_cdf(const uint64_t* __restrict__ key, int64_t n, float* __restrict__ cdf) {
    const int k = threadIdx.x;
    if (k > MLP_H) return;
    const uint64_t q = (k == MLP_H) ? ~0ULL : ((uint64_t)k << 58);
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (key[mid] < q)
            lo = mid + 1;
        else
            hi = mid;
    }
    cdf[k] = (float)((double)lo / (double)n);
}

// ----- leaf models -------------------------------------------------------------------------
// (model, index) pairs of every stored key, routed exactly as a query would be.
__global__ void k_route(const uint64_t* __restrict__ key, int64_t n, RootModel rm, const LeafModel* __restrict__ mids,
                        int n_leaf, uint64_t* __restrict__ pairs) {
    GSTRIDE(i, n) {
        const int j = route_leaf(rm, mids, n_leaf, (int)n, key[i]);
        pairs[i] = ((uint64_t)(uint32_t)j << 32) | (uint64_t)i;
    }
}

// Run [start, end) of every model in the sorted pairs (untouched for empty models).
__global__ void k_model_bounds(const uint64_t* __restrict__ pairs, int64_t n, int* __restrict__ start,
                               int* __restrict__ end) {
    GSTRIDE(i, n) {
        const int m = (int)(pairs[i] >> 32);
        if (i == 0 || (int)(pairs[i - 1] >> 32) != m) start[m] = (int)i;
        if (i == n - 1 || (int)(pairs[i + 1] >> 32) != m) end[m] = (int)i + 1;
    }
}

// One block per model: FP64 least squares (two passes), then the error window with the query's
// float arithmetic.  start/cnt: run of the model in the sorted pairs.
__global__ void __launch_bounds__(LT) k_fit_models(const uint64_t* __restrict__ key, const uint64_t* __restrict__ pairs,
                                                   const int* __restrict__ start, const int* __restrict__ end, int nkeys,
                                                   LeafModel* __restrict__ models) {
    __shared__ double s[LT];
    __shared__ int s_i[2 * LT];
    const int m = blockIdx.x;
    const int c = start[m] >= 0 ? end[m] - start[m] : 0;
    LeafModel md{};
    if (c == 0) {
        if (threadIdx.x == 0) {
            md.count = 0;
            md.first = -1;
            models[m] = md;
        }
        return;
    }
    const int s0 = start[m];
    const int first = (int)(uint32_t)pairs[s0];
    const uint64_t base = key[first];
    // means
    double sx = 0, sy = 0;
    for (int j = threadIdx.x; j < c; j += LT) {
        const int i = (int)(uint32_t)pairs[s0 + j];
        sx += (double)(int64_t)(key[i] - base);
        sy += (double)(i - first);
    }
    sx = block_sum_d<LT>(sx, s);
    sy = block_sum_d<LT>(sy, s);
    const double mx = sx / c, my = sy / c;
    double sxy = 0, sxx = 0;
    for (int j = threadIdx.x; j < c; j += LT) {
        const int i = (int)(uint32_t)pairs[s0 + j];
        const double dx = (double)(int64_t)(key[i] - base) - mx;
        sxy += dx * ((double)(i - first) - my);
        sxx += dx * dx;
    }
    sxy = block_sum_d<LT>(sxy, s);
    sxx = block_sum_d<LT>(sxx, s);
    const double slope = sxx > 0 ? sxy / sxx : 0.0;
    md.base = base;
    md.slope = (float)slope;
    md.icpt = (float)(my - slope * mx);
    md.first = first;
    md.count = c;
    md.err_lo = 0;
    md.err_hi = 0;
    // error window over the stored keys
    int elo = 0, ehi = 0;
    for (int j = threadIdx.x; j < c; j += LT) {
        const int i = (int)(uint32_t)pairs[s0 + j];
        const int pc = leaf_predict(md, key[i], nkeys);
        elo = max(elo, pc - i);
        ehi = max(ehi, i - pc);
    }
    s_i[threadIdx.x] = elo;
    s_i[LT + threadIdx.x] = ehi;
    __syncthreads();
    for (int o = LT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s_i[threadIdx.x] = max(s_i[threadIdx.x], s_i[threadIdx.x + o]);
            s_i[LT + threadIdx.x] = max(s_i[LT + threadIdx.x], s_i[LT + threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        md.err_lo = s_i[0];
        md.err_hi = s_i[LT];
        models[m] = md;
    }
}

unsigned g1(int64_t n, int b) {
    int64_t g = (n + b - 1) / b;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)num_sms() * 8));
}

} // namespace

ot_status mlp_grad(const float* d_params, const float* d_x, const float* d_t, int64_t n, float* d_grad, float* d_loss,
                   cudaStream_t s) {
    const int nb = (int)std::min<int64_t>(std::max<int64_t>(1, (n + MT - 1) / MT), 64);
    float* part = nullptr;
    OT_CUDA(cudaMallocAsync(&part, sizeof(float) * nb * (MLP_NPARAM + 1), s));
    k_mlp_grad_samples<<<nb, MT, 0, s>>>(d_params, d_x, d_t, n, part);
    k_sum_rows<<<1, 128, 0, s>>>(part, nb, d_grad, d_loss);
    count_launch(2);
    OT_CUDA(cudaFreeAsync(part, s));
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

// The trained 1 -> H ReLU -> 1 network as a piecewise-linear function on [0, 1): the units'
// breakpoints -b1/w1 inside (0, 1), sorted, and on each segment the line through the units
// active there (slope sum w2 w1, intercept b2 + sum w2 b1; a unit with w1 = 0 is a constant,
// active when b1 > 0).  Computed in FP64 and rounded once.
static void piecewise_form(RootModel& rm) {
    std::vector<double> kn;
    for (int k = 0; k < MLP_H; ++k)
        if (rm.w1[k] != 0.0f) {
            const double x = -(double)rm.b1[k] / (double)rm.w1[k];
            if (x > 0.0 && x < 1.0) kn.push_back(x);
        }
    std::sort(kn.begin(), kn.end());
    kn.erase(std::unique(kn.begin(), kn.end()), kn.end());
    rm.nknot = (int)kn.size();
    for (int k = 0; k < MLP_H; ++k) rm.knot[k] = k < rm.nknot ? (float)kn[k] : 2.0f;
    for (int sgm = 0; sgm <= rm.nknot; ++sgm) {
        const double lo = sgm == 0 ? 0.0 : kn[sgm - 1], hi = sgm == rm.nknot ? 1.0 : kn[sgm];
        const double xm = 0.5 * (lo + hi);
        double a = 0.0, b = (double)rm.b2;
        for (int k = 0; k < MLP_H; ++k)
            if ((double)rm.w1[k] * xm + (double)rm.b1[k] > 0.0) {
                a += (double)rm.w2[k] * rm.w1[k];
                b += (double)rm.w2[k] * rm.b1[k];
            }
        rm.sa[sgm] = (float)a;
        rm.sb[sgm] = (float)b;
    }
    for (int sgm = rm.nknot + 1; sgm <= MLP_H; ++sgm) rm.sa[sgm] = rm.sb[sgm] = 0.0f;
}

ot_status train_index(ot_octree* t, const ot_index_params* prm, cudaStream_t s) {
    const int64_t n = t->n;
    const int M = prm->n_leaf_models;
    RootModel rm{};
    rm.kind = prm->root;
    rm.n_models = M;
    float final_loss = 0.0f;
    if (prm->root == OT_ROOT_LINEAR) {
        const int nb = 256;
        double *part = nullptr, *means = nullptr;
        OT_CUDA(cudaMallocAsync(&part, sizeof(double) * 2 * nb, s));
        OT_CUDA(cudaMallocAsync(&means, sizeof(double) * 4, s));
        for (int pass = 0; pass < 2; ++pass) {
            k_lin_sums<<<nb, LT, 0, s>>>(t->d_key, n, part, pass, means);
            k_lin_finish<<<1, 32, 0, s>>>(part, nb, n, means, pass);
            count_launch(2);
        }
        double h[4];
        OT_CUDA(cudaMemcpyAsync(h, means, sizeof(h), cudaMemcpyDeviceToHost, s));
        OT_CUDA(cudaStreamSynchronize(s));
        cudaFreeAsync(part, s);
        cudaFreeAsync(means, s);
        rm.b = (float)h[2];
        rm.a = (float)h[3];
    } else {
        // knot initialisation: the linear spline through (k/32, CDF(k/32))
        float* d_cdf = nullptr;
        OT_CUDA(cudaMallocAsync(&d_cdf, sizeof(float) * (MLP_H + 1), s));
        k_knot_cdf<<<1, 64, 0, s>>>(t->d_key, n, d_cdf);
        count_launch();
        float cdf[MLP_H + 1];
        OT_CUDA(cudaMemcpyAsync(cdf, d_cdf, sizeof(cdf), cudaMemcpyDeviceToHost, s));
        OT_CUDA(cudaStreamSynchronize(s));
        cudaFreeAsync(d_cdf, s);
        float p[MLP_NPARAM];
        float prev = 0.0f;
        for (int k = 0; k < MLP_H; ++k) {
            const float slope = (cdf[k + 1] - cdf[k]) * (float)MLP_H;
            p[k] = 1.0f;                       // w1
            p[MLP_H + k] = -(float)k / MLP_H;  // b1: knot at k/32
            p[2 * MLP_H + k] = slope - prev;   // w2: change of slope at the knot
            prev = slope;
        }
        p[3 * MLP_H] = cdf[0];
        if (prm->h_init)
            for (int k = 0; k < MLP_NPARAM; ++k) p[k] = prm->h_init[k];
        float* d_p = nullptr;
        Adam* d_adam = nullptr;
        float* d_loss = nullptr;
        const int nb = 32;
        float* part = nullptr;
        OT_CUDA(cudaMallocAsync(&d_p, sizeof(p), s));
        OT_CUDA(cudaMallocAsync(&d_adam, sizeof(Adam), s));
        OT_CUDA(cudaMallocAsync(&d_loss, sizeof(float), s));
        OT_CUDA(cudaMallocAsync(&part, sizeof(float) * nb * (MLP_NPARAM + 1), s));
        OT_CUDA(cudaMemcpyAsync(d_p, p, sizeof(p), cudaMemcpyHostToDevice, s));
        OT_CUDA(cudaMemsetAsync(d_adam, 0, sizeof(Adam), s));
        OT_CUDA(cudaMemsetAsync(d_loss, 0, sizeof(float), s));
        const int batch = std::max(1, prm->batch);
        const int64_t per_epoch = std::max<int64_t>(1, std::min<int64_t>(n / batch, 512));
        const int64_t steps = prm->steps > 0 ? prm->steps : (int64_t)std::max(0, prm->epochs) * per_epoch;
        for (int64_t st = 0; st < steps; ++st) {
            k_mlp_step_grad<<<nb, MT, 0, s>>>(d_p, t->d_key, n, batch, prm->seed, (int)st, part);
            k_adam<<<1, 128, 0, s>>>(d_p, d_adam, part, nb, (int)st, prm->lr, d_loss);
        }
        count_launch(2 * (uint64_t)steps);
        OT_CUDA(cudaGetLastError());
        OT_CUDA(cudaMemcpyAsync(p, d_p, sizeof(p), cudaMemcpyDeviceToHost, s));
        OT_CUDA(cudaMemcpyAsync(&final_loss, d_loss, sizeof(float), cudaMemcpyDeviceToHost, s));
        OT_CUDA(cudaStreamSynchronize(s));
        cudaFreeAsync(d_p, s);
        cudaFreeAsync(d_adam, s);
        cudaFreeAsync(d_loss, s);
        cudaFreeAsync(part, s);
        for (int k = 0; k < MLP_H; ++k) {
            rm.w1[k] = p[k];
            rm.b1[k] = p[MLP_H + k];
            rm.w2[k] = p[2 * MLP_H + k];
        }
        rm.b2 = p[3 * MLP_H];
        piecewise_form(rm);
    }
    const bool three = prm->n_mid_models > 0;
    rm.n_models = three ? prm->n_mid_models : M;
    // models of one stage: route every key as a query would be, stable-sort the (model, index)
    // pairs by model, fit each model's line and error window
    auto fit_stage = [&](const LeafModel* mids, int n_route, LeafModel* out) -> ot_status {
        uint64_t *pairs = nullptr, *tmp = nullptr;
        int *start = nullptr, *end = nullptr;
        OT_CUDA(cudaMallocAsync(&pairs, sizeof(uint64_t) * n, s));
        OT_CUDA(cudaMallocAsync(&tmp, sizeof(uint64_t) * n, s));
        OT_CUDA(cudaMallocAsync(&start, sizeof(int) * n_route, s));
        OT_CUDA(cudaMallocAsync(&end, sizeof(int) * n_route, s));
        k_route<<<g1(n, 256), 256, 0, s>>>(t->d_key, n, rm, mids, M, pairs);
        count_launch();
        int bits = 1;
        while ((1 << bits) < n_route) ++bits;
        ot_status st = radix_sort_u64(pairs, tmp, n, 32, 32 + bits, s);
        if (st != OT_OK) return st;
        OT_CUDA(cudaMemsetAsync(start, 0xff, sizeof(int) * n_route, s));
        OT_CUDA(cudaMemsetAsync(end, 0xff, sizeof(int) * n_route, s));
        k_model_bounds<<<g1(n, 256), 256, 0, s>>>(pairs, n, start, end);
        k_fit_models<<<n_route, LT, 0, s>>>(t->d_key, pairs, start, end, (int)n, out);
        count_launch(2);
        // empty models are filled from a copy of the fitted ones (no reader sees a half-filled model)
        LeafModel* fitted = nullptr;
        OT_CUDA(cudaMallocAsync(&fitted, sizeof(LeafModel) * n_route, s));
        OT_CUDA(cudaMemcpyAsync(fitted, out, sizeof(LeafModel) * n_route, cudaMemcpyDeviceToDevice, s));
        k_fill_empty<<<g1(n_route, 256), 256, 0, s>>>(fitted, out, n_route, (int)n);
        count_launch();
        cudaFreeAsync(fitted, s);
        OT_CUDA(cudaGetLastError());
        cudaFreeAsync(pairs, s);
        cudaFreeAsync(tmp, s);
        cudaFreeAsync(start, s);
        cudaFreeAsync(end, s);
        return OT_OK;
    };
    if (t->d_models) cudaFree(t->d_models);
    if (t->d_mids) cudaFree(t->d_mids);
    t->d_models = t->d_mids = nullptr;
    t->has_index = false;
    OT_CUDA(cudaMalloc(&t->d_models, sizeof(LeafModel) * M));
    ot_status st;
    if (three) {
        OT_CUDA(cudaMalloc(&t->d_mids, sizeof(LeafModel) * prm->n_mid_models));
        if ((st = fit_stage(nullptr, prm->n_mid_models, t->d_mids)) != OT_OK) return st;
        if ((st = fit_stage(t->d_mids, M, t->d_models)) != OT_OK) return st;
    } else {
        if ((st = fit_stage(nullptr, M, t->d_models)) != OT_OK) return st;
    }
    OT_CUDA(cudaStreamSynchronize(s));
    t->root = rm;
    if (!t->d_root) OT_CUDA(cudaMalloc(&t->d_root, sizeof(RootModel)));
    OT_CUDA(cudaMemcpy(t->d_root, &rm, sizeof(RootModel), cudaMemcpyHostToDevice));
    t->n_models = M;
    t->n_mids = three ? prm->n_mid_models : 0;
    t->has_index = true;
    t->final_loss = final_loss;
    return OT_OK;
}

} // namespace ot
