// ot_internal.h -- library-private declarations shared by the translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "octtrack.h"
#include "ot_common.cuh"

struct ot_octree {
    int device = 0;
    int64_t n = 0;
    int lmin = 0, lmax = 0;
    uint64_t* d_key = nullptr;
    uint8_t* d_level = nullptr;
    // level map: the leaf holding the anchor of every cell of level lmap_level
    uint32_t* d_lmap = nullptr;
    int lmap_level = 0;
    uint4* d_desc = nullptr;  // subtree descriptor of every level-map cell
    int periodic = 0;         // stencils and level-mates wrap around the unit cube
    uint8_t* d_lmap_lv = nullptr;  // level of leaf lmap[c]
    // the same table at the pyramid level min(lmax, 7), fixed for the octree's life (it is
    // d_lmap when the two levels agree): leaf ranges of the cells of the pyramid of means
    uint32_t* d_pmap = nullptr;
    int pyr_level = 0;
    // refined cells of the node levels pyr_level+1 .. lmax-1, by first leaf: level
    // pyr_level+1+k is d_nodes[node_off[k] .. node_off[k] + node_cnt[k])
    int* d_nodes = nullptr;
    int64_t node_off[ot::MAXLEVEL] = {};
    int64_t node_cnt[ot::MAXLEVEL] = {};
    // level-mate table (null until built): 8 value slots per leaf and octant of its cell, in
    // library memory (mates_owned) or the caller's
    uint32_t* d_mates = nullptr;
    bool mates_owned = false;
    // with the table: flags of the cell means it reads, closed under "a mean needs its
    // children's", one byte per entry of the means array (null without the table: every mean
    // is computed)
    uint8_t* d_need_flags = nullptr;
    // learned index
    bool has_index = false;
    ot::RootModel root{};
    ot::RootModel* d_root = nullptr;  // device copy read by the queries
    ot::LeafModel* d_models = nullptr;  // leaf models
    int n_models = 0;
    ot::LeafModel* d_mids = nullptr;    // middle stage (null: two-stage index)
    int n_mids = 0;
    float final_loss = 0.0f;
    // diagnostics: [0] error word (unsigned), [1..2] fallback counter (u64)
    unsigned* d_err = nullptr;
    unsigned long long* d_fallbacks = nullptr;
};

namespace ot {

extern std::atomic<uint64_t> g_launches;
inline void count_launch(uint64_t k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// status helpers
ot_status cuda_status(cudaError_t e);
#define OT_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return ot::cuda_status(e_); \
    } while (0)

int num_sms();

TreeView tree_view(const ot_octree* t);

// primitives (ot_prims.cu) -------------------------------------------------------------------
// Exclusive scan of n uint32 (in place allowed); returns the total in *d_total if non-null.
// Temporary storage is allocated stream-ordered and released before return.
ot_status scan_u32(const uint32_t* d_in, uint32_t* d_out, int64_t n, uint32_t* d_total, cudaStream_t s);
// The same scan with its temporaries in ws (scan_ws_bytes(n) bytes, 4-byte aligned): no allocation.
size_t scan_ws_bytes(int64_t n);
ot_status scan_u32_ws(const uint32_t* d_in, uint32_t* d_out, int64_t n, uint32_t* d_total, void* ws, cudaStream_t s);
// Stable LSD radix sort of n uint64 by bits [bit0, bit1) (8-bit digits).  d_tmp: n uint64
// scratch.  Result in d_keys.  Temporaries (histograms) are stream-ordered allocations.
ot_status radix_sort_u64(uint64_t* d_keys, uint64_t* d_tmp, int64_t n, int bit0, int bit1, cudaStream_t s);
// Workspace bytes of radix_sort_u64_ws / radix_sort_u64_dn (histograms, offsets and the
// scan's temporaries): with it those sorts allocate nothing.
size_t radix_ws_bytes(int64_t n);
// Sort of the first *d_n (device value, <= n_max) keys with workspace of radix_ws_bytes(n_max)
// bytes; *result is the buffer (d_keys or d_tmp) holding the sorted keys.
ot_status radix_sort_u64_dn(uint64_t* d_keys, uint64_t* d_tmp, int64_t n_max, const uint32_t* d_n, int bit0,
                            int bit1, void* ws, uint64_t** result, cudaStream_t s);
// Same sort with caller-provided workspace (no allocation): ws of radix_ws_bytes(n) bytes.
ot_status radix_sort_u64_ws(uint64_t* d_keys, uint64_t* d_tmp, int64_t n, int bit0, int bit1, void* ws,
                            cudaStream_t s);
// Compaction: out[j] = in[i] for the i with flag[i] != 0, in order; *h_count on the host
// (synchronises).  d_scan: n uint32 scratch.
ot_status compact_u64(const uint64_t* d_in, const uint32_t* d_flag, uint32_t* d_scan, int64_t n, uint64_t* d_out,
                      int64_t* h_count, cudaStream_t s);
// Sorted input -> unique values in place; *h_count on the host (synchronises).
ot_status unique_u64(uint64_t* d_keys, int64_t n, int64_t* h_count, cudaStream_t s);

// Allocation-free scan / radix sort: temporaries in caller scratch.
ot_status scan_u32_noalloc(const uint32_t* d_in, uint32_t* d_out, int64_t n, uint32_t* tmp, cudaStream_t s);
size_t radix_noalloc_bytes(int64_t n);
ot_status radix_sort_u64_noalloc(uint64_t* d_keys, uint64_t* d_tmp, int64_t n, int bit0, int bit1, void* ws,
                                 cudaStream_t s);

// builder (ot_build.cu) ------------------------------------------------------------------------
ot_status build_tree(const ot_sphere* h_spheres, int n, const ot_build_params* p, cudaStream_t s, ot_octree* t);
// Level map (level < 0: min(lmax, 7)) and the error word.
ot_status finish_tree(ot_octree* t, cudaStream_t s, int map_level = -1);
ot_status validate_leaves(const uint64_t* d_key, const uint8_t* d_level, int64_t n, int full, cudaStream_t s,
                          int* lmin, int* lmax);
ot_status leaf_centres(const ot_octree* t, double* d_xyz, cudaStream_t s);

// learned index (ot_learned.cu) ----------------------------------------------------------------
ot_status train_index(ot_octree* t, const ot_index_params* p, cudaStream_t s);
ot_status mlp_grad(const float* d_params, const float* d_x, const float* d_t, int64_t n, float* d_grad,
                   float* d_loss, cudaStream_t s);

// point kernels (ot_interp.cu) -------------------------------------------------------------------
ot_status launch_locate(const ot_octree* t, const double* x, const double* y, const double* z, int64_t n, int search,
                        int32_t* host, unsigned long long* n_miss, cudaStream_t s);
// Trilinear interpolation needs interp_ws_bytes(t, OT_TRILINEAR, sizeof(T)) bytes of workspace
// (the cell means of the field, 16-byte aligned); the delta kernels need none.
template <typename T>
ot_status launch_interp(const ot_octree* t, int kernel, const double* x, const double* y, const double* z, int64_t n,
                        const int32_t* host_in, int search, const T* field, T* u, int32_t* host_out, void* ws,
                        size_t ws_bytes, cudaStream_t s);
size_t interp_ws_bytes(const ot_octree* t, int kernel, size_t elem);

// pyramid of cell means over levels 0 .. lmap_level (ot_pyramid.cu) ---------------------------
// Level l occupies cells [pyramid_offset(l), pyramid_offset(l) + 8^l), 4 values per cell.
int64_t pyramid_offset(int l);
// Node means of levels pyr_level+1 .. lmax-1 follow the pyramid: node_levels arrays of n
// entries (4 values each), indexed by the refined cell's first leaf.
int node_levels(const ot_octree* t);
ot_status build_node_lists(ot_octree* t, cudaStream_t s);
// Flags of the means the level-mate table reads (need_flag_bytes(t) bytes, one per entry of
// the means array, set by the table builder), closed under "a mean needs its children's".
size_t need_flag_bytes(const ot_octree* t);
ot_status close_need_flags(ot_octree* t, uint8_t* need, cudaStream_t s);
size_t pyramid_bytes(const ot_octree* t, size_t elem);  // elem: sizeof the field type
template <typename T> ot_status launch_pyramid(const ot_octree* t, const T* field, T* pyr, cudaStream_t s);

// level-mate table (ot_mates.cu): fills t->d_mates (mates_bytes(t) bytes) on stream s -----
ot_status build_mates(ot_octree* t, cudaStream_t s);
size_t mates_bytes(const ot_octree* t);
bool mates_fit(const ot_octree* t);

// Morton order of points (ot_order.cu) ----------------------------------------------------------
size_t order_ws_bytes(int64_t n);
bool order_fits(int64_t n, int level);
ot_status launch_point_sort(const double* x, const double* y, const double* z, int64_t n, int level,
                            uint64_t* pairs, int* ib_out, cudaStream_t s);

// spreading (ot_spread.cu) ---------------------------------------------------------------------
size_t spread_ws_bytes(const ot_octree* t, int kernel, int64_t n);
template <typename T>
ot_status launch_spread(const ot_octree* t, int kernel, int mode, const double* x, const double* y, const double* z,
                        const T* F, const T* dV, int64_t n, T* f, void* ws, size_t ws_bytes, cudaStream_t s);
// Sorted spreading with every temporary in `scratch` (spread_noalloc_bytes(kernel, n) bytes).
size_t spread_noalloc_bytes(int kernel, int64_t n);
ot_status launch_spread_sorted_noalloc(const ot_octree* t, int kernel, const double* x, const double* y,
                                       const double* z, const float* F, const float* dV, int64_t n, float* f,
                                       void* scratch, cudaStream_t s);

} // namespace ot
