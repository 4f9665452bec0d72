// ot_tune.cu -- autotuner of the batched launch: times graph replays of the batch over a grid
// of launch shapes (threads per block, 32-point rows per work item, resident blocks per SM,
// point order; with the level-mate table, the trilinear launch's own rows and blocks per SM)
// and, optionally, of level-map levels (the staging depth of the top tree levels), and keeps
// the fastest.  Timing is by CUDA events on the caller's stream, after one warm-up replay.
#include <algorithm>
#include <vector>

#include "ot_internal.h"

namespace {

// Mean time of `reps` replays of a batch made with launch shape `lp`, or a negative value when
// the shape is rejected.
float time_shape(const ot_octree* t, const ot_group* groups, int n_groups, const float* d_field, int search,
                 const ot_launch& lp, int reps, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, ot_status* err) {
    ot_batch* b = nullptr;
    ot_status st = ot_batch_create(t, groups, n_groups, d_field, search, &lp, s, &b);
    if (st != OT_OK) {
        if (st != OT_ERR_ARG) *err = st;
        return -1.0f;
    }
    float ms = -1.0f;
    if ((st = ot_batch_run(b, s)) == OT_OK && cudaEventRecord(e0, s) == cudaSuccess) {
        for (int r = 0; r < reps && st == OT_OK; ++r) st = ot_batch_run(b, s);
        if (st == OT_OK && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
            cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
            ms /= (float)reps;
        else
            ms = -1.0f;
    }
    if (st != OT_OK) *err = st;
    ot_batch_destroy(b);
    return ms;
}

} // namespace

extern "C" ot_status ot_batch_autotune(ot_octree* t, const ot_group* groups, int n_groups, const float* d_field,
                                       int search, int tune_map_level, int reps, void* stream,
                                       ot_tune_result* out) {
    if (!t || !groups || !d_field || !out || n_groups < 1 || reps < 1) return OT_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int> levels;
    if (tune_map_level) {
        for (int L = std::max(0, std::min(t->lmax, 6)); L <= std::min(t->lmax, 8); ++L) levels.push_back(L);
    } else {
        levels.push_back(t->lmap_level);
    }
    const int blocks[] = {128, 256};
    const int tiles[] = {1, 2, 4, 8};
    const int per_sm[] = {0, 2};
    const int orders[] = {0, 8};  // caller's order, or Morton order of level-8 cells
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    OT_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return OT_ERR_CUDA;
    }
    ot_status err = OT_OK;
    ot_tune_result best{};
    best.ms = -1.0f;
    best.map_level = t->lmap_level;
    const int start_level = t->lmap_level;
    // with the level-mate table the delta-kernel and trilinear groups run as two launches: each
    // part is tuned on its own groups, then the pair is timed together
    std::vector<ot_group> delta_g, tri_g;
    for (int g = 0; g < n_groups; ++g) (groups[g].kernel == OT_TRILINEAR ? tri_g : delta_g).push_back(groups[g]);
    const bool split = t->d_mates != nullptr;
    const int tri_tiles[] = {2, 4, 8};
    const int tri_per_sm[] = {1, 2, 3, 4};
    for (int L : levels) {
        if (L != t->lmap_level && (err = ot_octree_set_map_level(t, L, stream)) != OT_OK) break;
        if (!split) {
            for (int k = 0; k < 2 * 4 * 2 * 2 && err == OT_OK; ++k) {
                const ot_launch lp{blocks[(k / 8) % 2], tiles[(k / 2) % 4], per_sm[k % 2], orders[k / 16], 0, 0};
                const float ms = time_shape(t, groups, n_groups, d_field, search, lp, reps, s, e0, e1, &err);
                if (err != OT_OK || ms < 0.0f) continue;
                ++best.tried;
                if (best.ms < 0.0f || ms < best.ms) {
                    best.ms = ms;
                    best.launch = lp;
                    best.map_level = L;
                }
            }
        } else {
            ot_launch lp{256, 4, 0, 0, 0, 0};
            float part_ms = -1.0f;
            for (int k = 0; !delta_g.empty() && k < 2 * 4 * 2 && err == OT_OK; ++k) {
                const ot_launch c{blocks[(k / 8) % 2], tiles[(k / 2) % 4], per_sm[k % 2], 0, 0, 0};
                const float ms = time_shape(t, delta_g.data(), (int)delta_g.size(), d_field, search, c, reps, s, e0,
                                            e1, &err);
                if (err != OT_OK || ms < 0.0f) continue;
                ++best.tried;
                if (part_ms < 0.0f || ms < part_ms) part_ms = ms, lp = c;
            }
            part_ms = -1.0f;
            ot_launch tri_best = lp;
            for (int k = 0; !tri_g.empty() && k < 3 * 4 * 2 && err == OT_OK; ++k) {
                ot_launch c = lp;
                c.tri_tile = tri_tiles[k % 3];
                // resident warps per SM of 8, 16, 24, 32 whatever the block size the delta
                // launch chose
                c.tri_blocks_per_sm = tri_per_sm[(k / 3) % 4] * (256 / lp.block);
                c.order_level = orders[k / 12];
                const float ms = time_shape(t, tri_g.data(), (int)tri_g.size(), d_field, search, c, reps, s, e0, e1,
                                            &err);
                if (err != OT_OK || ms < 0.0f) continue;
                ++best.tried;
                if (part_ms < 0.0f || ms < part_ms) part_ms = ms, tri_best = c;
            }
            if (err != OT_OK) break;
            const float ms = time_shape(t, groups, n_groups, d_field, search, tri_best, reps, s, e0, e1, &err);
            if (err == OT_OK && ms >= 0.0f && (best.ms < 0.0f || ms < best.ms)) {
                best.ms = ms;
                best.launch = tri_best;
                best.map_level = L;
            }
        }
        if (err != OT_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // leave the octree at the best level map (or where it started, on an error)
    const int final_level = (err == OT_OK && best.ms >= 0.0f) ? best.map_level : start_level;
    if (t->lmap_level != final_level) {
        const ot_status st = ot_octree_set_map_level(t, final_level, stream);
        if (err == OT_OK) err = st;
    }
    if (err != OT_OK) return err;
    if (best.ms < 0.0f) return OT_ERR_ARG;
    *out = best;
    return OT_OK;
}
