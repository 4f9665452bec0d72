// ot_prims.cu -- scan, compaction, unique and a stable LSD radix sort for the octree builder
// and the deterministic spreading.
#include <algorithm>

#include "ot_internal.h"

namespace ot {

std::atomic<uint64_t> g_launches{0};

ot_status cuda_status(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) return OT_ERR_OOM;
    return OT_ERR_CUDA;
}

int num_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// ------------------------------------------------------------------------------------------
// Exclusive scan (uint32): block-local scans, scan of block totals (recursive), add-back.
// ------------------------------------------------------------------------------------------
constexpr int SCAN_T = 512, SCAN_I = 8, SCAN_TILE = SCAN_T * SCAN_I;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t w = lane < nw ? s_warp[lane] : 0u;
        uint32_t ws = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, ws, o);
            if (lane >= o) ws += y;
        }
        if (lane < nw) s_warp[lane] = ws - w;
        if (lane == nw - 1) s_warp[32] = ws;
    }
    __syncthreads();
    uint32_t r = s_warp[warp] + x - v;
    *total = s_warp[32];
    __syncthreads();
    return r;
}

__global__ void k_scan_tiles(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n,
                             uint32_t* __restrict__ tile_total) {
    __shared__ uint32_t s_warp[33];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_I;
    uint32_t v[SCAN_I];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0u;
        sum += v[i];
    }
    uint32_t tot;
    uint32_t run = block_exclusive_scan(sum, s_warp, &tot);
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == 0 && tile_total) tile_total[blockIdx.x] = tot;
}

__global__ void k_scan_add(uint32_t* __restrict__ out, int64_t n, const uint32_t* __restrict__ tile_off) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    const uint32_t add = tile_off[blockIdx.x];
    for (int i = threadIdx.x; i < SCAN_TILE; i += blockDim.x)
        if (base + i < n) out[base + i] += add;
}

__global__ void k_total(const uint32_t* in_last, const uint32_t* scan_last, uint32_t* total) {
    *total = *in_last + *scan_last;
}

// Tile totals of every level of the recursive scan of n values.
static int64_t scan_tile_elems(int64_t n) {
    int64_t total = 0;
    for (int64_t m = n; m > SCAN_TILE; m = (m + SCAN_TILE - 1) / SCAN_TILE) total += (m + SCAN_TILE - 1) / SCAN_TILE;
    return total;
}

size_t scan_ws_bytes(int64_t n) { return (size_t)(scan_tile_elems(n) + 1) * sizeof(uint32_t) + 256; }

// The recursive scan with its tile totals in tmp (scan_tile_elems(n) uint32).
static ot_status scan_levels(const uint32_t* d_in, uint32_t* d_out, int64_t n, uint32_t* tmp, cudaStream_t s) {
    const int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nt == 1) {
        k_scan_tiles<<<1, SCAN_T, 0, s>>>(d_in, d_out, n, nullptr);
        count_launch();
        return OT_OK;
    }
    k_scan_tiles<<<(unsigned)nt, SCAN_T, 0, s>>>(d_in, d_out, n, tmp);
    count_launch();
    ot_status st = scan_levels(tmp, tmp, nt, tmp + nt, s);
    if (st != OT_OK) return st;
    k_scan_add<<<(unsigned)nt, 256, 0, s>>>(d_out, n, tmp);
    count_launch();
    return OT_OK;
}

ot_status scan_u32_ws(const uint32_t* d_in, uint32_t* d_out, int64_t n, uint32_t* d_total, void* ws, cudaStream_t s) {
    if (n <= 0) {
        if (d_total) OT_CUDA(cudaMemsetAsync(d_total, 0, sizeof(uint32_t), s));
        return OT_OK;
    }
    // the total needs the last input, which an in-place scan overwrites: keep it first
    uint32_t* last = static_cast<uint32_t*>(ws);
    if (d_total) OT_CUDA(cudaMemcpyAsync(last, d_in + n - 1, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    ot_status st = scan_levels(d_in, d_out, n, last + 1, s);
    if (st != OT_OK) return st;
    if (d_total) {
        k_total<<<1, 1, 0, s>>>(last, d_out + n - 1, d_total);
        count_launch();
    }
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

ot_status scan_u32(const uint32_t* d_in, uint32_t* d_out, int64_t n, uint32_t* d_total, cudaStream_t s) {
    void* ws = nullptr;
    OT_CUDA(cudaMallocAsync(&ws, scan_ws_bytes(n), s));
    ot_status st = scan_u32_ws(d_in, d_out, n, d_total, ws, s);
    cudaFreeAsync(ws, s);
    return st;
}

// ------------------------------------------------------------------------------------------
// Stable LSD radix sort of uint64 keys, 8-bit digits.  A tile is RT threads x RI rounds; in
// round r thread t owns element r*RT + t, so (round, warp, lane) order is input order and the
// scatter ranks each element after every earlier element of the tile with the same digit.
// ------------------------------------------------------------------------------------------
constexpr int RT = 256, RI = 16, RTILE = RT * RI, RW = RT / 32;

// d_n (nullable): the element count in device memory, at most n (tiles past it stay empty).
__global__ void k_radix_hist(const uint64_t* __restrict__ in, int64_t n, int shift, uint32_t mask,
                             uint32_t* __restrict__ hist, int ntiles, const uint32_t* __restrict__ d_n) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    if (d_n) n = min(n, (int64_t)*d_n);
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RTILE;
#pragma unroll
    for (int r = 0; r < RI; ++r) {
        int64_t i = base + r * RT + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(uint32_t)(in[i] >> shift) & mask], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void k_radix_scatter(const uint64_t* __restrict__ in, uint64_t* __restrict__ out, int64_t n, int shift,
                                uint32_t mask, const uint32_t* __restrict__ offs, int ntiles,
                                const uint32_t* __restrict__ d_n) {
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_w[RW][256];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (d_n) n = min(n, (int64_t)*d_n);
    if ((int64_t)blockIdx.x * RTILE >= n) return;  // block-uniform
    const unsigned lt = (1u << lane) - 1u;
    s_base[tid] = offs[(int64_t)tid * ntiles + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * RTILE;
    for (int r = 0; r < RI; ++r) {
#pragma unroll
        for (int w = 0; w < RW; ++w) s_w[w][tid] = 0;
        __syncthreads();
        const int64_t i = base + r * RT + tid;
        const bool valid = i < n;
        uint64_t v = valid ? in[i] : 0ULL;
        uint32_t d = valid ? ((uint32_t)(v >> shift) & mask) : 256u;
        unsigned grp = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(grp & lt);
        if (valid && rank == 0) s_w[warp][d] = __popc(grp);
        __syncthreads();
        {  // digit tid: exclusive prefix over the warps of this round
            uint32_t run = s_base[tid];
#pragma unroll
            for (int w = 0; w < RW; ++w) {
                uint32_t c = s_w[w][tid];
                s_w[w][tid] = run;
                run += c;
            }
            s_base[tid] = run;
        }
        __syncthreads();
        if (valid) out[s_w[warp][d] + rank] = v;
        __syncthreads();
    }
}

// Histograms and offsets (256 per tile each), then the scan's temporaries.
size_t radix_ws_bytes(int64_t n) {
    int64_t nt = (n + RTILE - 1) / RTILE;
    if (nt < 1) nt = 1;
    return (size_t)(2 * 256 * nt) * sizeof(uint32_t) + scan_ws_bytes(256 * nt) + 256;
}

static ot_status radix_passes(uint64_t* d_keys, uint64_t* d_tmp, int64_t n, int bit0, int bit1, uint32_t* hist,
                              uint32_t* offs, cudaStream_t s, const uint32_t* d_n = nullptr,
                              uint64_t** result = nullptr) {
    uint32_t* stmp = offs + 256 * ((n + RTILE - 1) / RTILE);
    const int nt = (int)((n + RTILE - 1) / RTILE);
    uint64_t* src = d_keys;
    uint64_t* dst = d_tmp;
    for (int sh = bit0; sh < bit1; sh += 8) {
        const int nb = std::min(8, bit1 - sh);
        const uint32_t mask = (1u << nb) - 1u;
        k_radix_hist<<<nt, RT, 0, s>>>(src, n, sh, mask, hist, nt, d_n);
        count_launch();
        ot_status st = scan_u32_ws(hist, offs, (int64_t)256 * nt, nullptr, stmp, s);
        if (st != OT_OK) return st;
        k_radix_scatter<<<nt, RT, 0, s>>>(src, dst, n, sh, mask, offs, nt, d_n);
        count_launch();
        std::swap(src, dst);
    }
    if (result)
        *result = src;  // the caller takes the sorted keys where the last pass left them
    else if (src != d_keys)
        OT_CUDA(cudaMemcpyAsync(d_keys, src, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

ot_status radix_sort_u64_dn(uint64_t* d_keys, uint64_t* d_tmp, int64_t n_max, const uint32_t* d_n, int bit0,
                            int bit1, void* ws, uint64_t** result, cudaStream_t s) {
    *result = d_keys;
    if (n_max <= 1 || bit1 <= bit0) return OT_OK;
    const int64_t nt = (n_max + RTILE - 1) / RTILE;
    uint32_t* hist = static_cast<uint32_t*>(ws);
    uint32_t* offs = hist + 256 * nt;
    return radix_passes(d_keys, d_tmp, n_max, bit0, bit1, hist, offs, s, d_n, result);
}

ot_status radix_sort_u64(uint64_t* d_keys, uint64_t* d_tmp, int64_t n, int bit0, int bit1, cudaStream_t s) {
    if (n <= 1 || bit1 <= bit0) return OT_OK;
    void* ws = nullptr;
    OT_CUDA(cudaMallocAsync(&ws, radix_ws_bytes(n), s));
    ot_status st = radix_sort_u64_ws(d_keys, d_tmp, n, bit0, bit1, ws, s);
    cudaFreeAsync(ws, s);
    return st;
}

ot_status radix_sort_u64_ws(uint64_t* d_keys, uint64_t* d_tmp, int64_t n, int bit0, int bit1, void* ws,
                            cudaStream_t s) {
    if (n <= 1 || bit1 <= bit0) return OT_OK;
    const int64_t nt = (n + RTILE - 1) / RTILE;
    uint32_t* hist = static_cast<uint32_t*>(ws);
    uint32_t* offs = hist + 256 * nt;
    return radix_passes(d_keys, d_tmp, n, bit0, bit1, hist, offs, s);
}

// ------------------------------------------------------------------------------------------
// Compaction and unique.
// ------------------------------------------------------------------------------------------
__global__ void k_compact(const uint64_t* __restrict__ in, const uint32_t* __restrict__ flag,
                          const uint32_t* __restrict__ pos, int64_t n, uint64_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) out[pos[i]] = in[i];
}

static unsigned grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    int64_t cap = (int64_t)num_sms() * 32;
    return (unsigned)std::max<int64_t>(1, std::min(g, cap));
}

ot_status compact_u64(const uint64_t* d_in, const uint32_t* d_flag, uint32_t* d_scan, int64_t n, uint64_t* d_out,
                      int64_t* h_count, cudaStream_t s) {
    if (n <= 0) {
        *h_count = 0;
        return OT_OK;
    }
    uint32_t* tot = nullptr;
    OT_CUDA(cudaMallocAsync(&tot, sizeof(uint32_t), s));
    ot_status st = scan_u32(d_flag, d_scan, n, tot, s);
    if (st != OT_OK) return st;
    k_compact<<<grid_for(n, 256), 256, 0, s>>>(d_in, d_flag, d_scan, n, d_out);
    count_launch();
    uint32_t h = 0;
    OT_CUDA(cudaMemcpyAsync(&h, tot, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    OT_CUDA(cudaFreeAsync(tot, s));
    OT_CUDA(cudaStreamSynchronize(s));
    *h_count = h;
    return OT_OK;
}

__global__ void k_head_flags(const uint64_t* __restrict__ k, int64_t n, uint32_t* __restrict__ flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || k[i] != k[i - 1]) ? 1u : 0u;
}

ot_status unique_u64(uint64_t* d_keys, int64_t n, int64_t* h_count, cudaStream_t s) {
    if (n <= 1) {
        *h_count = n;
        return OT_OK;
    }
    uint32_t *flag = nullptr, *pos = nullptr;
    uint64_t* tmp = nullptr;
    OT_CUDA(cudaMallocAsync(&flag, sizeof(uint32_t) * n, s));
    OT_CUDA(cudaMallocAsync(&pos, sizeof(uint32_t) * n, s));
    OT_CUDA(cudaMallocAsync(&tmp, sizeof(uint64_t) * n, s));
    k_head_flags<<<grid_for(n, 256), 256, 0, s>>>(d_keys, n, flag);
    count_launch();
    int64_t m = 0;
    ot_status st = compact_u64(d_keys, flag, pos, n, tmp, &m, s);
    if (st != OT_OK) return st;
    OT_CUDA(cudaMemcpyAsync(d_keys, tmp, sizeof(uint64_t) * m, cudaMemcpyDeviceToDevice, s));
    OT_CUDA(cudaFreeAsync(flag, s));
    OT_CUDA(cudaFreeAsync(pos, s));
    OT_CUDA(cudaFreeAsync(tmp, s));
    *h_count = m;
    return OT_OK;
}

} // namespace ot

// ------------------------------------------------------------------------------------------
// Allocation-free variants: every temporary lives in caller-provided scratch.
// ------------------------------------------------------------------------------------------
namespace ot {

int64_t scan_noalloc_elems(int64_t n) {
    int64_t total = 0;
    int64_t m = n;
    while (m > SCAN_TILE) {
        const int64_t nt = (m + SCAN_TILE - 1) / SCAN_TILE;
        total += nt;
        m = nt;
    }
    return total + 1;
}

// Exclusive scan with the tile totals of every level in tmp (scan_noalloc_elems(n) uint32).
ot_status scan_u32_noalloc(const uint32_t* d_in, uint32_t* d_out, int64_t n, uint32_t* tmp, cudaStream_t s) {
    if (n <= 0) return OT_OK;
    const int64_t nt = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nt == 1) {
        k_scan_tiles<<<1, SCAN_T, 0, s>>>(d_in, d_out, n, nullptr);
        count_launch();
    } else {
        uint32_t* tiles = tmp;
        k_scan_tiles<<<(unsigned)nt, SCAN_T, 0, s>>>(d_in, d_out, n, tiles);
        count_launch();
        ot_status st = scan_u32_noalloc(tiles, tiles, nt, tmp + nt, s);
        if (st != OT_OK) return st;
        k_scan_add<<<(unsigned)nt, 256, 0, s>>>(d_out, n, tiles);
        count_launch();
    }
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

size_t radix_noalloc_bytes(int64_t n) {
    int64_t nt = (n + RTILE - 1) / RTILE;
    if (nt < 1) nt = 1;
    return (size_t)(2 * 256 * nt + scan_noalloc_elems(256 * nt)) * sizeof(uint32_t) + 256;
}

ot_status radix_sort_u64_noalloc(uint64_t* d_keys, uint64_t* d_tmp, int64_t n, int bit0, int bit1, void* ws,
                                 cudaStream_t s) {
    if (n <= 1 || bit1 <= bit0) return OT_OK;
    const int nt = (int)((n + RTILE - 1) / RTILE);
    uint32_t* hist = static_cast<uint32_t*>(ws);
    uint32_t* offs = hist + 256 * (int64_t)nt;
    uint32_t* stmp = offs + 256 * (int64_t)nt;
    uint64_t* src = d_keys;
    uint64_t* dst = d_tmp;
    for (int sh = bit0; sh < bit1; sh += 8) {
        const int nb = std::min(8, bit1 - sh);
        const uint32_t mask = (1u << nb) - 1u;
        k_radix_hist<<<nt, RT, 0, s>>>(src, n, sh, mask, hist, nt, nullptr);
        count_launch();
        ot_status st = scan_u32_noalloc(hist, offs, (int64_t)256 * nt, stmp, s);
        if (st != OT_OK) return st;
        k_radix_scatter<<<nt, RT, 0, s>>>(src, dst, n, sh, mask, offs, nt, nullptr);
        count_launch();
        std::swap(src, dst);
    }
    if (src != d_keys) OT_CUDA(cudaMemcpyAsync(d_keys, src, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
    OT_CUDA(cudaGetLastError());
    return OT_OK;
}

} // namespace ot
