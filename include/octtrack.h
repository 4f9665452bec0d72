/*
 * octtrack.h -- C ABI of the GB300 octree Lagrangian-Eulerian coupling library.
 *
 * The library locates Lagrangian points (IBM markers and point particles) in a 2:1
 * balanced linear octree stored as a Morton-sorted array of leaves, interpolates a
 * cell-centred velocity field to them, and spreads marker forces back to the cells as the
 * exact adjoint of the interpolation.
 *
 * Conventions (every entry point):
 *   - Pointers prefixed d_ are device pointers owned and allocated by the caller; h_ are
 *     host pointers.  The library owns what it creates (octrees, indexes, batches) and
 *     frees it in the matching *_destroy call.
 *   - stream is a cudaStream_t (NULL = legacy default stream).  Calls are asynchronous on
 *     it unless stated otherwise; outputs are valid once the stream has reached them.
 *   - Arguments are validated on the host; a bad argument returns OT_ERR_ARG and launches
 *     nothing.  No C++ exception crosses this boundary.
 *   - Output order always equals input order.
 *   - Device-side findings (a point outside the unit cube, a stencil cell that is not a
 *     finest-level leaf, a bounded loop that reached its cap) never trap: they set bits
 *     of a per-octree error word that ot_last_error() reads after a stream sync.
 *
 * Geometry: one tree, the unit cube [0,1)^3.  Integer coordinates have 21 bits per axis
 * (MAXLEVEL = 21), so a Morton key (x bit b -> key bit 3b, y -> 3b+1, z -> 3b+2) fits in
 * 63 bits.  A leaf of level l at integer cell (i,j,k) covers [i,i+1)x[j,j+1)x[k,k+1)/2^l and
 * is stored by its anchor key morton(i<<(21-l), j<<(21-l), k<<(21-l)) and its level.
 * (The paper's Algorithm 1 uses p4est's 2-D MAXLEVEL = 30; 21 is the 3-D 64-bit value.)
 */
#ifndef OCTTRACK_H
#define OCTTRACK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ot_octree ot_octree;
typedef struct ot_batch ot_batch;

typedef enum {
    OT_OK = 0,
    OT_ERR_ARG = -1,        /* invalid argument (null pointer, size, enum value)          */
    OT_ERR_CUDA = -2,       /* a CUDA runtime call failed                                  */
    OT_ERR_OOM = -3,        /* device allocation failed                                    */
    OT_ERR_UNSORTED = -4,   /* leaves not strictly increasing / not aligned / not a tiling */
    OT_ERR_UNBALANCED = -5, /* leaves violate the requested 2:1 balance                    */
    OT_ERR_NOT_FOUND = -6,  /* reserved                                                    */
    OT_ERR_STENCIL = -7,    /* reserved for callers that turn error bits into a status     */
    OT_ERR_LIMIT = -8,      /* a size exceeds a documented limit                           */
    OT_ERR_NO_INDEX = -9    /* OT_LEARNED requested before ot_index_train                  */
} ot_status;

/* interpolation / spreading kernels */
enum { OT_TRILINEAR = 1, OT_PESKIN4 = 2, OT_ROMA3 = 3 };
/* host-cell search */
enum { OT_BINARY = 0, OT_LEARNED = 1 };
/* spreading modes */
enum { OT_SORTED = 0, OT_ATOMIC = 1 };
/* learned-index root model */
enum { OT_ROOT_LINEAR = 0, OT_ROOT_MLP = 1 };
/* bits of the device error word */
enum {
    OT_DEV_OUTSIDE = 1u,     /* a point outside [0,1)^3 or NaN (host = -1)                   */
    OT_DEV_STENCIL = 2u,     /* a delta-kernel stencil cell outside the domain or not a leaf
                                of the finest level: its weight was dropped                */
    OT_DEV_REFINED_CAP = 4u, /* reserved (never set: refined level-mates have no leaf cap)  */
    OT_DEV_WINDOW = 8u       /* a learned prediction missed; plain search answered instead  */
};

/* Limits. */
#define OT_MAX_LEAVES 2000000000LL /* leaf indices are int32 */
#define OT_MAX_SPHERES 4096
#define OT_MAX_LEVEL 20            /* lmax; keys need 3*lmax <= 63 bits and one spare level  */

/* A refinement sphere: cells whose closed box lies within `shell` of the sphere surface
 * |p - c| = r are refined (Sec. 3.1 refinement; Sec. 3.3 auxiliary IBM forest). */
typedef struct {
    double c[3];
    double r;
    double shell;
} ot_sphere;

typedef struct {
    int lmin, lmax;   /* 0 <= lmin <= lmax <= OT_MAX_LEVEL                                  */
    int balance_full; /* 1: face+edge+corner 2:1 balance; 0: face-only balance               */
} ot_build_params;

/* ---------------------------------------------------------------------------------------
 * Octree
 * -------------------------------------------------------------------------------------*/

/* Build the leaves on the device (Sec. 3.1: refine / balance; Sec. 3.3: refinement driven
 * only by proximity to the IBM surfaces): start from the uniform level lmin, split a cell
 * of level < lmax whenever the FP64 distance from its closed box to some sphere surface,
 * max(0, d_near - r, r - d_far), is <= shell; then add the fewest splits that make any two
 * adjacent leaves differ by at most one level.  Leaves come out Morton-sorted.
 * h_spheres: n host records (0 <= n <= OT_MAX_SPHERES).  Synchronises the stream (sizes
 * are read back).  *out receives a new octree; free it with ot_octree_destroy. */
ot_status ot_octree_build(const ot_sphere* h_spheres, int n, const ot_build_params* params, void* stream,
                          ot_octree** out);

/* Adopt caller leaves (copied): d_keys strictly increasing anchor keys, d_levels their
 * levels; they must tile the unit cube (OT_ERR_UNSORTED otherwise) and satisfy the 2:1
 * balance named by balance_full (OT_ERR_UNBALANCED otherwise).  Synchronises the stream. */
ot_status ot_octree_from_leaves(const uint64_t* d_keys, const uint8_t* d_levels, int64_t n, int balance_full,
                                void* stream, ot_octree** out);

/* Leaf count and level range. */
ot_status ot_octree_info(const ot_octree* t, int64_t* n_leaves, int* lmin, int* lmax);

/* Device pointers to the library-owned leaf arrays (valid until ot_octree_destroy). */
ot_status ot_octree_leaves(const ot_octree* t, int64_t* n, const uint64_t** d_keys, const uint8_t** d_levels);

/* Copy the leaves into caller buffers (d_keys: N uint64, d_levels: N uint8; either may be
 * NULL), asynchronously on stream. */
ot_status ot_octree_copy_leaves(const ot_octree* t, uint64_t* d_keys, uint8_t* d_levels, void* stream);

/* Level of the level map that every host search starts from (0 .. 8, capped at lmax): for
 * each cell of that level the map holds the leaf at the cell's anchor, so a point in a cell
 * covered by one leaf is located with one table read, and any other point is searched only
 * among its cell's leaves.  8^level * 4 bytes of device memory.  Octrees are created with
 * min(lmax, 7), or 8 when lmax > 10 (a level-map cell's subtree descriptor resolves leaves up
 * to 3 levels below it).  Synchronises the stream. */
ot_status ot_octree_set_map_level(ot_octree* t, int level, void* stream);
/* The current level-map level. */
ot_status ot_octree_get_map_level(const ot_octree* t, int* level);

/* Periodic unit cube (the turbulence box of Sec. 5.2): with periodic = 1, delta-kernel
 * stencils (interpolation and spreading) and trilinear level-mates wrap around the cube
 * (cell indices modulo the cells per axis) instead of dropping cells / taking the host's
 * index.  Batches made earlier on the octree keep the setting they were made with. */
ot_status ot_octree_set_periodic(ot_octree* t, int periodic);

/* Level-mate table (the trilinear level-mate rule of Sec. 2.3.2, resolved once per octree):
 * for every leaf h and octant o of its cell (bit d of o set when the point lies in the upper
 * half on axis d), the 8 level-mates c + {0, s_d} of the trilinear stencil, each as a value
 * slot -- the leaf whose value it takes (a leaf of the host's level, or the coarser leaf that
 * covers it) or its cell-mean entry when it is refined.  With the table built, trilinear
 * interpolation (ot_interpolate and batches created afterwards) finds its host leaf and reads
 * one 32-byte row instead of searching for the 7 level-mates; the results are bit-identical.
 * Built with it: the parent-block table of the delta kernels (Sec. 2.2 stencils on the finest
 * level; for every block of 8 finest leaves, the first leaves of the 27 blocks around it), with
 * which a marker's stencil takes one lookup instead of one per block, and the flags of the
 * cell means the level-mate table reads, so that the cell means recomputed for trilinear
 * interpolation are those only.  Both leave every result unchanged bit for bit.
 * enable = 1 builds (or rebuilds) them: 272 bytes of device memory per leaf plus one byte per
 * cell-mean entry; OT_ERR_LIMIT when the leaf count or the cell-mean count reaches 2^31,
 * OT_ERR_OOM when the memory is not there (the octree is then left without a table).
 * enable = 0 frees them.  Batches made while a table existed hold its pointer: recreate them
 * after rebuilding or freeing it.  The octree's
 * periodic setting is part of the table: ot_octree_set_periodic rebuilds it (on the legacy
 * default stream).  Synchronises the stream. */
ot_status ot_octree_build_mates(ot_octree* t, int enable, void* stream);
/* *bytes = the tables' size: 256 bytes per leaf (level-mate rows) + 128 bytes per 8 leaves
 * (parent-block rows). */
ot_status ot_octree_mates_bytes(const ot_octree* t, size_t* bytes);
/* Builds the table in caller memory (d_buffer: 16-byte aligned, at least ot_octree_mates_bytes
 * bytes; the caller keeps ownership and must keep it allocated and untouched while the octree
 * or a batch made on it is used).  A table the library held before is freed.  Lets a caller
 * that rebuilds octrees reuse one buffer instead of allocating a table per octree.  Errors as
 * ot_octree_build_mates (OT_ERR_ARG for a short or misaligned buffer).  Synchronises the
 * stream. */
ot_status ot_octree_build_mates_in(ot_octree* t, void* d_buffer, size_t bytes, void* stream);
/* *has = 1 when the level-mate table is built. */
ot_status ot_octree_has_mates(const ot_octree* t, int* has);

/* Leaf centres, FP64, written as 3 planes of N (x..., y..., z...). */
ot_status ot_octree_centres(const ot_octree* t, double* d_xyz, void* stream);

ot_status ot_octree_destroy(ot_octree* t);

/* ---------------------------------------------------------------------------------------
 * Learned index (not in the paper; a two-stage recursive model index after Kraska et al.,
 * SIGMOD 2018): a root model maps a key to one of n_leaf_models linear models; each leaf
 * model predicts the key's position in the leaf array and stores the maximum error of
 * that prediction over the stored keys.  A query searches only the error window, verifies
 * the answer and falls back to the plain binary search, so results are bit-identical to it.
 * -------------------------------------------------------------------------------------*/

typedef struct {
    int root;          /* OT_ROOT_LINEAR or OT_ROOT_MLP (1 -> 32 ReLU -> 1)                    */
    int n_leaf_models; /* 1 .. 1<<22; 4096 for the two-stage index                           */
    int n_mid_models;  /* 0: two-stage (root -> leaf models).  > 0: three-stage: the root picks
                          one of n_mid_models linear models, whose position estimate picks the
                          leaf model (integer scaling, monotone within a mid model)            */
    int epochs;        /* MLP root: training length; an epoch is min(N / batch, 512) Adam steps */
    int batch;         /* MLP root: minibatch size                                           */
    float lr;          /* MLP root: Adam step size                                           */
    uint64_t seed;     /* MLP root: minibatch sampling                                       */
    int steps;         /* MLP root: > 0 replaces epochs by this many Adam steps              */
    const float* h_init; /* MLP root: nullable; 97 host floats (w1, b1, w2, b2) to start from
                            instead of the spline initialisation (a warm start: retraining
                            after a re-adaptation from the previous tree's network)          */
} ot_index_params;

/* Train on the device over the octree's keys; replaces a previous index.  Synchronises. */
ot_status ot_index_train(ot_octree* t, const ot_index_params* params, void* stream);

/* The trained MLP root's 97 parameters (w1[32], b1[32], w2[32], b2) into host memory;
 * OT_ERR_NO_INDEX without an index or with a linear root. */
ot_status ot_index_get_root_params(const ot_octree* t, float* h_params);

/* Index statistics (host values): window length (mean over the stored keys, max over the
 * leaf models), number of empty models, learned-query fallbacks counted since the last reset,
 * and the mean number of halving probes a stored key's window takes (ceil(log2(window));
 * a plain binary search of the whole array takes ceil(log2(N))). */
typedef struct {
    double mean_window;
    int64_t max_window;
    int64_t empty_models;
    uint64_t fallbacks;
    float final_loss; /* MLP root: last minibatch loss (0 for a linear root) */
    double mean_probes;
} ot_index_stats;
ot_status ot_index_get_stats(const ot_octree* t, ot_index_stats* s, int reset_fallbacks);

/* Root network hooks for gradient checks: loss and gradient of the MSE loss of params
 * (97 floats: w1[32], b1[32], w2[32], b2) over n samples (d_x, d_t), on the device.
 * d_grad: 97 floats; d_loss: 1 float. */
ot_status ot_index_mlp_grad(const float* d_params, const float* d_x, const float* d_t, int64_t n, float* d_grad,
                            float* d_loss, void* stream);

/* ---------------------------------------------------------------------------------------
 * Locate / interpolate / spread
 * -------------------------------------------------------------------------------------*/

/* Host-cell search (Algorithm 1, Sec. 3.2): d_host[i] = the leaf whose half-open box holds
 * point i, i.e. the last leaf whose anchor key <= the point's key at MAXLEVEL, computed from
 * floor(x 2^21) in FP64 so that points on a face go to the upper cell.  A point outside
 * [0,1)^3 or NaN gets -1 and, when d_n_miss is not NULL, increments *d_n_miss.
 * search: OT_BINARY or OT_LEARNED (OT_ERR_NO_INDEX without a trained index). */
ot_status ot_locate(const ot_octree* t, const double* d_x, const double* d_y, const double* d_z, int64_t n,
                    int search, int32_t* d_host, unsigned long long* d_n_miss, void* stream);

/* Interpolation of a cell-centred field (float4 per leaf: x, y, z, unused) to n points.
 *   OT_TRILINEAR (Sec. 2.3.2): the host leaf (level l) and its 7 level-mates, the cells
 *     c + {0, s_d} per axis where s_d = sign of the offset from the host centre; a
 *     level-mate inside a coarser leaf takes that leaf's value, a refined one the
 *     volume-weighted mean of its leaves, one outside the cube the host's index on that axis.
 *     The refined means are rebuilt by each call from the field, in the caller's workspace:
 *     a dense pyramid of cell means over levels 0 .. L = min(lmax, 7) (16 * (8^(L+1) - 1) / 7
 *     bytes in FP32, 38 MB at L = 7) and, for levels L+1 .. lmax-1, one array of N means per
 *     level indexed by the refined cell's first leaf (16 N bytes per level in FP32).
 *   OT_PESKIN4 / OT_ROMA3 (Sec. 2.2, Eq. ibm_interpolate): u(X) = sum over the 4^3 / 3^3
 *     finest-level cells around X of phi(rx) phi(ry) phi(rz) u(cell); Peskin's 4-point or
 *     the paper's 3-point function.  Cells outside the cube or not finest-level leaves are
 *     dropped and flagged (OT_DEV_STENCIL).
 * d_u: 3 planes of n floats.  d_host_in: host leaves from ot_locate, or NULL to locate
 * here (search selects how); d_host_out (nullable) receives them.  For the delta kernels the
 * host is the finest cell holding X when that cell is a leaf, else a plain search result.
 * d_workspace: ot_interpolate_workspace_size bytes, 16-byte aligned (OT_ERR_ARG when short);
 * the delta kernels need none (NULL, 0).  Nothing is allocated: every temporary lives there. */
ot_status ot_interpolate(const ot_octree* t, int kernel, const double* d_x, const double* d_y, const double* d_z,
                         int64_t n, const int32_t* d_host_in, int search, const float* d_field, float* d_u,
                         int32_t* d_host_out, void* d_workspace, size_t ws_bytes, void* stream);

/* FP64 variant: d_field is N x 4 doubles, d_u 3 planes of n doubles; weights in FP64. */
ot_status ot_interpolate_f64(const ot_octree* t, int kernel, const double* d_x, const double* d_y,
                             const double* d_z, int64_t n, const int32_t* d_host_in, int search,
                             const double* d_field, double* d_u, int32_t* d_host_out, void* d_workspace,
                             size_t ws_bytes, void* stream);

/* *bytes = the workspace of ot_interpolate (fp64 = 0) or ot_interpolate_f64 (fp64 = 1) with
 * the given kernel on this octree: the cell means for OT_TRILINEAR, 0 for the delta kernels.
 * It does not depend on the point count. */
ot_status ot_interpolate_workspace_size(const ot_octree* t, int kernel, int fp64, size_t* bytes);

/* Workspace for OT_SORTED spreading of n markers with the given kernel: every temporary of
 * the sorted spreading (pairs, sort buffers, histograms, scan totals, marker records), so that
 * ot_spread allocates nothing. */
ot_status ot_spread_workspace_size(const ot_octree* t, int kernel, int64_t n, size_t* bytes);

/* Force spreading, the exact adjoint of the delta-kernel interpolation (Sec. 2.2, Eq. for
 * F(x)): f(cell) += sum_k F_k phi phi phi dV_k / h^3, h = 2^-lmax, dV_k = h^3 when d_dV is
 * NULL (the paper's literal form).  d_F: 3 planes of n floats; d_f: float4 per leaf,
 * ACCUMULATED (the caller zeroes it), component w untouched.
 *   OT_SORTED: one pair per (marker, overlapping 2x2x2 block of finest cells) is radix-sorted
 *     by block (stable); each block sums its 8 cells' contributions in marker order:
 *     bit-identical run to run and for any launch shape.
 *     Needs d_workspace of ot_spread_workspace_size bytes (16-byte aligned); nothing is
 *     allocated.
 *   OT_ATOMIC: float atomics; order varies run to run.  d_workspace may be NULL. */
ot_status ot_spread(const ot_octree* t, int kernel, int mode, const double* d_x, const double* d_y,
                    const double* d_z, const float* d_F, const float* d_dV, int64_t n, float* d_f,
                    void* d_workspace, size_t ws_bytes, void* stream);

/* FP64 variant: d_F 3 planes of n doubles, d_dV n doubles or NULL, d_f N x 4 doubles. */
ot_status ot_spread_f64(const ot_octree* t, int kernel, int mode, const double* d_x, const double* d_y,
                        const double* d_z, const double* d_F, const double* d_dV, int64_t n, double* d_f,
                        void* d_workspace, size_t ws_bytes, void* stream);

/* Size of the library's static device scratch used by ot_spread_noalloc: 64 MiB on every GPU
 * that loads the library, held until the process exits. */
#define OT_NOALLOC_SCRATCH_BYTES (64u << 20)

/* Sorted force spreading that allocates nothing (no counterpart in the paper: it exists for
 * callers that cannot call cudaMalloc, e.g. a solver whose memory pool already owns the
 * device, or code that must not risk an allocation's synchronisation or failure mid-step).
 * Same result as ot_spread(kernel, OT_SORTED, ...) for FP32: d_f is accumulated, d_dV may be
 * NULL.  The scratch is a fixed library array of OT_NOALLOC_SCRATCH_BYTES per device; it
 * holds about 446 bytes per marker for OT_PESKIN4 (at most 150,635 markers) and 132 bytes per
 * marker for OT_ROMA3 (at most 508,394); larger n returns OT_ERR_LIMIT and launches nothing.
 * The first call on a device (with that device current) looks up the scratch address; make
 * that first call before any stream capture.  The address is looked up again when the device's
 * context changed (after cudaDeviceReset, say): make the first call after such a change
 * outside a stream capture too.  All calls share the one array: calls whose
 * work overlaps on the GPU (different streams, or different threads without ordering) race
 * and give wrong results; order them on one stream.  The array keeps the last call's
 * contents; nothing in it needs clearing between calls. */
ot_status ot_spread_noalloc(const ot_octree* t, int kernel, const double* d_x, const double* d_y,
                            const double* d_z, const float* d_F, const float* d_dV, int64_t n, float* d_f,
                            void* stream);

/* Marker force of the direct-forcing step (Sec. 2.2): F_k = (U_k - u*_k) / dt, evaluated as
 * (U_k - u*_k) * (1 / dt) in FP32, for the interpolated velocities d_u (3 planes of n floats)
 * and the markers' prescribed velocities d_U (3 planes, or NULL for markers at rest, U = 0);
 * d_F: 3 planes of n floats (may alias neither input).  dt > 0.  Asynchronous on `stream`. */
ot_status ot_marker_force(const float* d_U, const float* d_u, int64_t n, float dt, float* d_F, void* stream);

/* ---------------------------------------------------------------------------------------
 * Multi-direct forcing (Sec. 2.2): n_iter rounds of
 *   u_k = I u (Eq. ibm_interpolate, the delta kernel `kernel`),  F_k = (U_k - u_k) / dt,
 *   F = S F_k (OT_SORTED spreading, marker volumes d_dV or h^3),  u += dt F / rho,  f += F.
 * The printed correction u = u* + F / rho is read with the time step, u* + dt F / rho (equal
 * in lattice units, dt = 1), applied to the velocity corrected so far.
 *   d_u: float4 per leaf; in: the unforced velocity u*, out: the corrected velocity.
 *   d_f: float4 per leaf; out: the total force of the rounds (overwritten).
 *   d_U: 3 planes of n floats, the markers' prescribed velocities.
 *   d_slip (nullable): n_iter + 1 floats, sqrt(sum_k |U_k - u_k|^2) before each round and
 *     after the last (summed with FP64 atomics: its last bits may vary run to run).
 *   d_workspace: ot_ibm_mdf_workspace_size bytes, 256-byte aligned.
 * Deterministic (d_slip aside).  Asynchronous on `stream`.
 * -------------------------------------------------------------------------------------*/
ot_status ot_ibm_mdf_workspace_size(const ot_octree* t, int kernel, int64_t n, int n_iter, size_t* bytes);
ot_status ot_ibm_mdf(const ot_octree* t, int kernel, const double* d_x, const double* d_y, const double* d_z,
                     const float* d_U, const float* d_dV, int64_t n, float rho, float dt, int n_iter, float* d_u,
                     float* d_f, float* d_slip, void* d_workspace, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------------------
 * Rigid bodies (Sec. 2.3): per-body linear and angular sums of a marker quantity v,
 *   d_lin[b] = scale sum_{k in b} v_k w_k,  d_ang[b] = scale sum_{k in b} (X_k - x_b) x v_k w_k,
 * w_k = d_dV[k] (or w when d_dV is NULL).  With v = u at the internal markers (interpolated,
 * e.g. trilinear, since the body interior need not be refined) and scale = rho_f: the internal
 * fluid's linear momentum P and angular momentum L (the printed sums swap the two names
 * against the text and omit rho_f); with v = F_k at the surface markers and scale = -1: the
 * IBM force -sum F_k dV_k and torque -sum (X_k - x_b) x F_k dV_k.  The markers of body b are
 * d_start[b] .. d_start[b+1]-1 (device int64, n_bodies + 1 entries); d_xb: n_bodies x 3 body
 * centres; d_lin, d_ang: n_bodies x 3 doubles.  FP64 sums in a fixed order (deterministic).
 * -------------------------------------------------------------------------------------*/
ot_status ot_body_sums(const double* d_x, const double* d_y, const double* d_z, const float* d_v, const float* d_dV,
                       float w, int64_t n, const int64_t* d_start, int n_bodies, const double* d_xb, double scale,
                       double* d_lin, double* d_ang, void* stream);

/* ---------------------------------------------------------------------------------------
 * Batched launch: every group of points (IBM markers with a delta kernel, point particles
 * with trilinear) located and interpolated by ONE persistent kernel, captured once in a
 * CUDA graph and replayed.
 * -------------------------------------------------------------------------------------*/

typedef struct {
    int kernel;           /* OT_TRILINEAR, OT_PESKIN4 or OT_ROMA3                          */
    const double *d_x, *d_y, *d_z;
    int64_t n;
    float* d_u;           /* 3 planes of n                                                 */
    int32_t* d_host;      /* nullable                                                      */
} ot_group;

/* Launch shape of the batched kernel (0 = library default). */
typedef struct {
    int block;       /* threads per block: 64 .. 256, multiple of 32 (default 256)          */
    int tile;        /* 32-point rows per work item taken from the queue: 1 .. 64 (default 4) */
    int blocks_per_sm; /* resident blocks per SM of every launch of the batch, capped by
                          occupancy (0: the occupancy max); 2 also selects the delta-kernel
                          code compiled for 2 blocks per SM (more registers per thread, no
                          spills) instead of 3.  With the octree's level-mate table built, the
                          delta-kernel groups and the trilinear groups run as two launches  */
    int order_level;   /* 0: points in the caller's order.  L in 1..21: each replay first sorts
                          every trilinear group of >= 64 points by the Morton key of their
                          level-L cells (on the device, inside the graph), interpolates them in
                          that order (a warp's points then share host leaves and level-mates)
                          and writes the results back in the caller's order; identical
                          results                                                           */
    int tri_tile;      /* with the level-mate table, the trilinear launch's rows per work item
                          (0: tile)                                                          */
    int tri_blocks_per_sm; /* with the level-mate table, the trilinear launch's resident blocks
                          per SM, capped by occupancy (0: 2, which measured fastest: its loads
                          are latency-bound and fewer warps keep more of each SM's cache
                          per warp)                                                          */
    int tri_records;   /* with the level-mate table: 0 (default): value records for the hot
                          leaves -- the leaves of level <= min(level-map level, hot level),
                          the hot level being the deepest at which the trilinear points, spread
                          evenly, would give every leaf at least 4 -- holding for each octant
                          of the leaf's cell its 8 level-mate values (96 bytes), rewritten from
                          the field at every replay; a point in a level-map cell inside a hot
                          leaf reads the cell's 8-byte entry and one record instead of the
                          level-mate row and 8 scattered values; identical results.  Costs
                          8 bytes per level-map cell and 768 bytes per hot leaf.  k > 0: the
                          same with the hot level capped at k (a smaller record set); -1: off */
} ot_launch;

/* Create a batch over groups (copied) reading d_field (float4 per leaf).  search selects
 * the host-cell search.  launch may be NULL.  Captures the graph on `stream`.  The graph
 * holds the octree's device pointers: the octree must outlive the batch, and a batch made
 * before ot_octree_set_map_level or ot_index_train on the same octree must be recreated.
 * A replay recomputes the pyramid of cell means of d_field (when some group is trilinear)
 * and then runs the batch kernel, so the field may change between replays. */
ot_status ot_batch_create(const ot_octree* t, const ot_group* groups, int n_groups, const float* d_field,
                          int search, const ot_launch* launch, void* stream, ot_batch** out);
ot_status ot_batch_run(ot_batch* b, void* stream);
ot_status ot_batch_destroy(ot_batch* b);

/* Autotuner of the batched launch (not in the paper): creates the batch for every launch
 * shape of {128, 256} threads x {1, 2, 4, 8} rows per work item x {occupancy max, 2} blocks
 * per SM x {caller's order, level-8 Morton order} and, when tune_map_level != 0, every
 * level-map level from min(lmax, 6) to min(lmax, 8); times `reps` graph replays of each (CUDA
 * events on `stream`, after one warm-up replay) and returns the fastest.  With the level-mate
 * table built the two launches are tuned one after the other: the delta-kernel groups alone
 * over threads x rows x blocks per SM (16 shapes), then the trilinear groups alone over
 * tri_tile {2, 4, 8} x tri_blocks_per_sm {1, 2, 3, 4} x (256 / threads) x order (24 shapes:
 * 8 to 32 resident warps per SM at the delta launch's block size), and the pair is
 * timed together.  The octree is left at the chosen level-map level (batches made earlier on
 * it must be recreated).  The groups' outputs are overwritten.  Synchronises the stream; takes
 * about (1 + reps) * 32 (or 41) * levels replays. */
typedef struct {
    ot_launch launch; /* fastest launch shape                                                */
    int map_level;    /* its level-map level                                                 */
    float ms;         /* mean time of one replay there                                       */
    int tried;        /* settings timed                                                      */
} ot_tune_result;
ot_status ot_batch_autotune(ot_octree* t, const ot_group* groups, int n_groups, const float* d_field, int search,
                            int tune_map_level, int reps, void* stream, ot_tune_result* out);

/* ---------------------------------------------------------------------------------------
 * Analytic field on the leaves (not in the paper; the synthetic stand-in for the fluid
 * solver's velocity): d_field[leaf] = (sum_m A_m cos(2 pi n_m . c + phi_m), 0) at each leaf
 * centre c, FP32.  h_wave: 3 x n_modes integer wave vectors (|component| <= 4096); h_amp:
 * 3 x n_modes amplitudes; h_phase: n_modes phases (radians).  n_modes <= 64.  The argument
 * is reduced modulo one turn exactly (integer fixed point, phase rounded to 2^-32 turns);
 * only the cosine is FP32.  Asynchronous on `stream`.
 * -------------------------------------------------------------------------------------*/
ot_status ot_field_fourier(const ot_octree* t, int n_modes, const int32_t* h_wave, const double* h_amp,
                           const double* h_phase, float* d_field, void* stream);

/* Mean-force removal in a periodic box (Sec. 5.2): subtracts from every leaf of d_field
 * (float4 per leaf) its volume-weighted mean over the unit cube, sum_c f_c 8^-level_c,
 * summed in FP64 in a fixed order (deterministic).  d_mean (nullable, device): the 3
 * subtracted components.  d_workspace: ot_field_mean_workspace_size bytes (24,600 bytes),
 * 8-byte aligned, for the block partials; nothing is allocated.  Asynchronous on `stream`. */
ot_status ot_field_mean_workspace_size(const ot_octree* t, size_t* bytes);
ot_status ot_field_subtract_mean(const ot_octree* t, float* d_field, double* d_mean, void* d_workspace,
                                 size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------------------
 * Morton order of a point set (not in the paper's API; its ranks keep their Lagrangian points
 * grouped by cell, Sec. 3.2): d_perm[i] = the index of the i-th point along the Z curve of
 * the cells of `level` (1..21; stable, so points of one cell keep their order; points outside
 * [0,1)^3 last).  Storing points in this order lets a warp's points share their host leaves
 * and level-mates.  n < 2^31 and 3 level + ceil(log2 n) <= 64.  d_workspace:
 * ot_points_order_workspace_size bytes, 16-byte aligned.  Asynchronous on `stream`.
 * -------------------------------------------------------------------------------------*/
ot_status ot_points_order_workspace_size(int64_t n, size_t* bytes);
ot_status ot_points_morton_order(const double* d_x, const double* d_y, const double* d_z, int64_t n, int level,
                                 int32_t* d_perm, void* d_workspace, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------------------
 * Point-particle advection (Sec. 2.3.2, Eq. PointParticle, gravity off): per particle
 *   a = f_p (u - v)/tau, f_p = 1 + 0.15 (re_coef |u - v|)^0.687 (re_coef = 0: f_p = 1),
 *   v += dt (3/2 a - 1/2 a_prev), x += dt (3/2 v_old - 1/2 v_prev); Euler when first != 0.
 * periodic != 0 wraps the new positions into [0, 1) per axis (x - floor(x)).
 * d_x: 3 planes of n doubles (positions, FP64); d_v, d_a_prev, d_v_prev: 3 planes of n
 * floats; d_u: 3 planes of n floats (interpolated fluid velocity).
 * -------------------------------------------------------------------------------------*/
ot_status ot_advect_ab2(double* d_x, float* d_v, float* d_a_prev, float* d_v_prev, const float* d_u, int64_t n,
                        float tau, float re_coef, float dt, int first, int periodic, void* stream);

/* ---------------------------------------------------------------------------------------
 * Diagnostics
 * -------------------------------------------------------------------------------------*/

/* Device error word of the octree (OT_DEV_* bits) accumulated since the last clear.
 * Synchronises the stream.  clear != 0 zeroes it afterwards. */
ot_status ot_last_error(const ot_octree* t, unsigned* bits, int clear, void* stream);

/* Kernels this library has launched since load (a process-wide counter). */
uint64_t ot_launch_count(void);

const char* ot_status_string(ot_status s);

#ifdef __cplusplus
}
#endif
#endif /* OCTTRACK_H */
