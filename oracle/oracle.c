/*
 * oracle.c -- plain FP64 CPU oracle for the octree Lagrangian-Eulerian coupling path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls this
 * file; only the test-suite, the smoke check and the CPU-baseline leg of the benchmark do.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * Every routine is the plain definition of the quantity it computes, written for a reader
 * who checks it against the paper by eye: no blocking, fusion or reordering.  OpenMP only
 * splits independent points across host cores.  Compile with -ffp-contract=off so that no
 * multiply-add is fused behind the reader's back (the refinement test must round exactly
 * as written).
 *
 * Conventions shared with the CUDA path by *specification only* (restated, not shared code):
 *   MAXLEVEL = 21: integer octree coordinates have 21 bits per axis, so a 3-D Morton key
 *   fits in 63 bits.  (The paper's Algorithm 1 quotes p4est's 2-D value 30.)
 *   Morton key: bit b of x goes to key bit 3b, of y to 3b+1, of z to 3b+2.
 *   A leaf at level l with integer cell coordinates (i,j,k) covers the half-open box
 *   [i,i+1)x[j,j+1)x[k,k+1) * 2^-l and has the anchor key morton(i<<(21-l), ...).
 *
 * Parity status:
 *   or_morton, or_unmorton ............ pinned (closed-form keys, round trip)
 *   or_octree_build ................... pinned (independent dense builder, partition, balance)
 *   or_locate_ub / brute .............. pinned (agreement with each other and with a dense-grid
 *                                       painting of the leaves; faces, corners, NaN)
 *   or_phi_peskin4, or_phi_roma3 ...... pinned (closed-form values, moment conditions)
 *   or_interp_delta, or_spread_delta .. pinned (linear exactness, adjoint identity, conservation)
 *   or_interp_trilinear ............... pinned for same-level and refined level-mates (linear
 *                                       exactness, textbook trilinear on uniform trees);
 *                                       parity unpinned for hanging (coarser) and out-of-domain
 *                                       level-mates beyond constant-field reproduction
 *   or_mlp_loss_grad .................. pinned (central finite differences)
 *   or_advect_ab2 ..................... pinned (closed-form relaxation of a constant field;
 *                                       periodic wrap: exact crossings of each face, the
 *                                       x >= 1 fix-up, state other than x unchanged)
 *   periodic variants (_p) ............ pinned (uniform periodic trees against independent
 *                                       numpy sums over wrapped indices and scipy trilinear on
 *                                       a wrap-padded grid; spread conservation at the walls)
 *   or_field_mean ..................... pinned (constant field; zero after subtraction)
 *   or_body_sums ...................... pinned (uniform translation gives P = rho V u; a rigid
 *                                       rotation gives L = rho I Omega with I from the tensor
 *                                       form; torque of a force through the centre vanishes)
 *   or_ibm_mdf ........................ pinned (slip recursion s' = s - A s / rho against a
 *                                       brute-force interpolation-spreading matrix A, monotone
 *                                       slip decrease, force conservation, zero-slip fixed point)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXLEVEL 21

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------------------ */
/* Morton (Z-order) keys -- the ordering of p4est's linear octree (Sec. 3.1, 3.2).        */
/* ------------------------------------------------------------------------------------ */

uint64_t or_morton(uint32_t x, uint32_t y, uint32_t z) {
    uint64_t key = 0;
    for (int b = 0; b < OR_MAXLEVEL; ++b) {
        key |= (uint64_t)((x >> b) & 1u) << (3 * b);
        key |= (uint64_t)((y >> b) & 1u) << (3 * b + 1);
        key |= (uint64_t)((z >> b) & 1u) << (3 * b + 2);
    }
    return key;
}

void or_unmorton(uint64_t key, uint32_t *x, uint32_t *y, uint32_t *z) {
    uint32_t a = 0, b = 0, c = 0;
    for (int bit = 0; bit < OR_MAXLEVEL; ++bit) {
        a |= (uint32_t)((key >> (3 * bit)) & 1u) << bit;
        b |= (uint32_t)((key >> (3 * bit + 1)) & 1u) << bit;
        c |= (uint32_t)((key >> (3 * bit + 2)) & 1u) << bit;
    }
    *x = a;
    *y = b;
    *z = c;
}

/* Number of MAXLEVEL cells along one axis of a level-l cell. */
static uint32_t cell_len(int level) { return 1u << (OR_MAXLEVEL - level); }

/* Number of MAXLEVEL keys covered by a level-l leaf: 8^(21-l). */
static uint64_t key_span(int level) { return (uint64_t)1 << (3 * (OR_MAXLEVEL - level)); }

/* First index i with keys[i] > q (keys sorted ascending). */
int64_t or_upper_bound(const uint64_t *keys, int64_t n, uint64_t q) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (keys[mid] <= q)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

/* First index i with keys[i] >= q. */
static int64_t lower_bound(const uint64_t *keys, int64_t n, uint64_t q) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (keys[mid] < q)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

/* Leaf whose key range holds the MAXLEVEL key q: the last key <= q (leaves partition the
 * domain, so that leaf contains q). */
static int64_t leaf_of_key(const uint64_t *keys, int64_t n, uint64_t q) {
    return or_upper_bound(keys, n, q) - 1;
}

/* ------------------------------------------------------------------------------------ */
/* Octree build: refinement by distance to sphere surfaces (Sec. 3.1 item 1, Sec. 3.3),   */
/* then 2:1 balance (Sec. 3.1 item 2).                                                    */
/* ------------------------------------------------------------------------------------ */

/* Distance from the closed box [lo, lo+h]^3 to a sphere surface |p - c| = r:
 *   max(0, d_near - r, r - d_far), d_near/d_far = min/max distance from c to the box.
 * Evaluated in this exact operation order (x, then y, then z). */
static int box_near_surface(const double lo[3], double h, const double *sph) {
    double near2 = 0.0, far2 = 0.0;
    for (int d = 0; d < 3; ++d) {
        double c = sph[d];
        double hi = lo[d] + h;
        double below = lo[d] - c; /* > 0 when c lies below the box */
        double above = c - hi;    /* > 0 when c lies above the box */
        double e = 0.0;
        if (below > e) e = below;
        if (above > e) e = above;
        near2 = near2 + e * e;
        double f0 = fabs(c - lo[d]);
        double f1 = fabs(c - hi);
        double f = f0 > f1 ? f0 : f1;
        far2 = far2 + f * f;
    }
    double r = sph[3], w = sph[4];
    double dist = 0.0;
    double t0 = sqrt(near2) - r;
    double t1 = r - sqrt(far2);
    if (t0 > dist) dist = t0;
    if (t1 > dist) dist = t1;
    return dist <= w;
}

typedef struct {
    uint64_t *key;
    uint8_t *level;
    int64_t n, cap;
} leafvec;

static void lv_push(leafvec *v, uint64_t key, uint8_t level) {
    if (v->n == v->cap) {
        v->cap = v->cap ? 2 * v->cap : 1024;
        v->key = (uint64_t *)realloc(v->key, (size_t)v->cap * sizeof(uint64_t));
        v->level = (uint8_t *)realloc(v->level, (size_t)v->cap);
    }
    v->key[v->n] = key;
    v->level[v->n] = level;
    v->n++;
}

typedef struct {
    const double *spheres; /* n x 5: cx, cy, cz, r, w */
    int nsph, lmax;
    leafvec *out;
} build_ctx;

static int cell_refines(const build_ctx *cx, uint32_t i, uint32_t j, uint32_t k, int l) {
    double h = ldexp(1.0, -l);
    double lo[3] = {i * h, j * h, k * h};
    for (int s = 0; s < cx->nsph; ++s)
        if (box_near_surface(lo, h, cx->spheres + 5 * s)) return 1;
    return 0;
}

/* Depth-first refinement; children visited in Morton order, so leaves come out sorted. */
static void refine_rec(const build_ctx *cx, uint32_t i, uint32_t j, uint32_t k, int l) {
    if (l < cx->lmax && cell_refines(cx, i, j, k, l)) {
        for (int c = 0; c < 8; ++c)
            refine_rec(cx, 2 * i + (c & 1), 2 * j + ((c >> 1) & 1), 2 * k + ((c >> 2) & 1), l + 1);
    } else {
        lv_push(cx->out, or_morton(i << (OR_MAXLEVEL - l), j << (OR_MAXLEVEL - l), k << (OR_MAXLEVEL - l)),
                (uint8_t)l);
    }
}

/* One ripple sweep: every leaf B looks at its neighbour cells n at B's own level; if the
 * leaf A holding n is two or more levels coarser than B, A must be split.  Returns the
 * number of leaves marked. */
static int64_t mark_unbalanced(const uint64_t *key, const uint8_t *level, int64_t n, int full, uint8_t *mark) {
    int64_t nmarked = 0;
    memset(mark, 0, (size_t)n);
#pragma omp parallel for schedule(dynamic, 4096) reduction(+ : nmarked)
    for (int64_t b = 0; b < n; ++b) {
        int lb = level[b];
        uint32_t x, y, z;
        or_unmorton(key[b], &x, &y, &z);
        int64_t ci = x >> (OR_MAXLEVEL - lb), cj = y >> (OR_MAXLEVEL - lb), ck = z >> (OR_MAXLEVEL - lb);
        int64_t ncell = (int64_t)1 << lb;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int nz = (dx != 0) + (dy != 0) + (dz != 0);
                    if (nz == 0) continue;
                    if (!full && nz != 1) continue; /* face neighbours only */
                    int64_t ni = ci + dx, nj = cj + dy, nk = ck + dz;
                    if (ni < 0 || nj < 0 || nk < 0 || ni >= ncell || nj >= ncell || nk >= ncell) continue;
                    uint64_t q = or_morton((uint32_t)(ni << (OR_MAXLEVEL - lb)), (uint32_t)(nj << (OR_MAXLEVEL - lb)),
                                           (uint32_t)(nk << (OR_MAXLEVEL - lb)));
                    int64_t a = leaf_of_key(key, n, q);
                    if ((int)level[a] + 2 <= lb) {
                        if (!mark[a]) {
                            mark[a] = 1; /* benign race: every writer stores 1 */
                            nmarked++;   /* may over-count; only "> 0" is used */
                        }
                    }
                }
    }
    return nmarked;
}

/* Build the leaves of the linear octree.  spheres: n x (cx, cy, cz, r, w).  full = 1 for
 * face+edge+corner balance, 0 for face-only.  Returns the leaf count; *keys and *levels are
 * malloc'ed arrays the caller frees with or_free(). */
int64_t or_octree_build(const double *spheres, int nsph, int lmin, int lmax, int full, uint64_t **keys_out,
                        uint8_t **levels_out) {
    /* refine each level-lmin root cell on its own (independent subtrees), then concatenate
     * the subtrees in Morton order of their roots */
    int64_t nroot = (int64_t)1 << (3 * lmin);
    leafvec *sub = (leafvec *)calloc((size_t)nroot, sizeof(leafvec));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t m = 0; m < nroot; ++m) {
        build_ctx cx = {spheres, nsph, lmax, &sub[m]};
        uint32_t x, y, z;
        /* cell m of level lmin in Morton order: its anchor at MAXLEVEL is m << 3(21-lmin) */
        or_unmorton((uint64_t)m << (3 * (OR_MAXLEVEL - lmin)), &x, &y, &z);
        refine_rec(&cx, x >> (OR_MAXLEVEL - lmin), y >> (OR_MAXLEVEL - lmin), z >> (OR_MAXLEVEL - lmin), lmin);
    }
    leafvec v = {0, 0, 0, 0};
    for (int64_t m = 0; m < nroot; ++m) v.n += sub[m].n;
    v.cap = v.n;
    v.key = (uint64_t *)malloc((size_t)v.n * sizeof(uint64_t));
    v.level = (uint8_t *)malloc((size_t)v.n);
    int64_t at = 0;
    for (int64_t m = 0; m < nroot; ++m) {
        memcpy(v.key + at, sub[m].key, (size_t)sub[m].n * sizeof(uint64_t));
        memcpy(v.level + at, sub[m].level, (size_t)sub[m].n);
        at += sub[m].n;
        free(sub[m].key);
        free(sub[m].level);
    }
    free(sub);
    /* ripple until no leaf needs splitting */
    for (;;) {
        uint8_t *mark = (uint8_t *)malloc((size_t)v.n);
        int64_t nm = mark_unbalanced(v.key, v.level, v.n, full, mark);
        if (nm == 0) {
            free(mark);
            break;
        }
        leafvec w = {0, 0, 0, 0};
        for (int64_t a = 0; a < v.n; ++a) {
            if (!mark[a]) {
                lv_push(&w, v.key[a], v.level[a]);
                continue;
            }
            int l = v.level[a] + 1;
            uint32_t x, y, z;
            or_unmorton(v.key[a], &x, &y, &z);
            for (int c = 0; c < 8; ++c) {
                uint32_t cxk = x + (uint32_t)(c & 1) * cell_len(l);
                uint32_t cyk = y + (uint32_t)((c >> 1) & 1) * cell_len(l);
                uint32_t czk = z + (uint32_t)((c >> 2) & 1) * cell_len(l);
                lv_push(&w, or_morton(cxk, cyk, czk), (uint8_t)l);
            }
        }
        free(mark);
        free(v.key);
        free(v.level);
        v = w;
    }
    *keys_out = v.key;
    *levels_out = v.level;
    return v.n;
}

void or_free(void *p) { free(p); }

/* Count balance violations: pairs (B, A) with A holding a neighbour cell of B and
 * level(A) <= level(B) - 2.  Same neighbour definition as the build. */
int64_t or_count_unbalanced(const uint64_t *key, const uint8_t *level, int64_t n, int full) {
    uint8_t *mark = (uint8_t *)malloc((size_t)n);
    int64_t c = mark_unbalanced(key, level, n, full, mark);
    int64_t exact = 0;
    for (int64_t i = 0; i < n; ++i) exact += mark[i];
    free(mark);
    return c ? exact : 0;
}

/* Leaf centres in the unit cube: ((anchor + half a cell) / 2^21) per axis; out is n x 3. */
void or_leaf_centres(const uint64_t *key, const uint8_t *level, int64_t n, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < n; ++a) {
        uint32_t x, y, z;
        or_unmorton(key[a], &x, &y, &z);
        double half = 0.5 * (double)cell_len(level[a]);
        double s = ldexp(1.0, -OR_MAXLEVEL);
        out[3 * a + 0] = ((double)x + half) * s;
        out[3 * a + 1] = ((double)y + half) * s;
        out[3 * a + 2] = ((double)z + half) * s;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Host-cell search (Algorithm 1, Sec. 3.2).                                               */
/* ------------------------------------------------------------------------------------ */

/* Integer MAXLEVEL coordinates of a point; 0 when the point is outside [0,1)^3 or NaN. */
static int point_coords(double x, double y, double z, uint32_t q[3]) {
    double p[3] = {x, y, z};
    for (int d = 0; d < 3; ++d) {
        if (!(p[d] >= 0.0 && p[d] < 1.0)) return 0;
        q[d] = (uint32_t)floor(p[d] * 2097152.0); /* 2^21: exact scaling, floor semantics */
    }
    return 1;
}

/* Host of a point: the leaf whose half-open box holds it (Sec. 3.2, the host cell that
 * Algorithm 1 identifies).  Leaves tile the cube and the MAXLEVEL descendants of a level-l leaf
 * are the contiguous keys [anchor, anchor + 8^(21-l)), so that leaf is the last one whose
 * anchor key is <= the key of the point's MAXLEVEL cell. */
void or_locate_ub(const uint64_t *key, const uint8_t *level, int64_t n, const double *x, const double *y,
                  const double *z, int64_t np, int32_t *host) {
    (void)level;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < np; ++p) {
        uint32_t q[3];
        if (!point_coords(x[p], y[p], z[p], q)) {
            host[p] = -1;
            continue;
        }
        host[p] = (int32_t)leaf_of_key(key, n, or_morton(q[0], q[1], q[2]));
    }
}

/* Naive scan over every leaf (the O(N_p N_cell) method of Sec. 3.2): the leaf whose box
 * holds the point.  For tiny trees only. */
void or_locate_brute(const uint64_t *key, const uint8_t *level, int64_t n, const double *x, const double *y,
                     const double *z, int64_t np, int32_t *host) {
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < np; ++p) {
        double pt[3] = {x[p], y[p], z[p]};
        int32_t found = -1;
        for (int64_t a = 0; a < n && found < 0; ++a) {
            uint32_t c[3];
            or_unmorton(key[a], &c[0], &c[1], &c[2]);
            double h = ldexp(1.0, -level[a]);
            int in = 1;
            for (int d = 0; d < 3; ++d) {
                double lo = ldexp((double)c[d], -OR_MAXLEVEL);
                if (!(pt[d] >= lo && pt[d] < lo + h)) in = 0;
            }
            if (in) found = (int32_t)a;
        }
        host[p] = found;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Discrete delta kernels (Sec. 2.2).  Argument r is in grid units (x / dx).              */
/* ------------------------------------------------------------------------------------ */

/* Peskin's 4-point function (Peskin, Acta Numerica 2002). */
double or_phi_peskin4(double r) {
    double a = fabs(r);
    if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
    if (a <= 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
    return 0.0;
}

/* The paper's 3-point function (Sec. 2.2; the Roma et al. kernel). */
double or_phi_roma3(double r) {
    double a = fabs(r);
    if (a <= 0.5) return (1.0 + sqrt(1.0 - 3.0 * a * a)) / 3.0;
    if (a <= 1.5) return (5.0 - 3.0 * a - sqrt(-2.0 + 6.0 * a - 3.0 * a * a)) / 6.0;
    return 0.0;
}

/* Stencil of one axis for a point at fine-grid coordinate s = X 2^lmax - 0.5 (cell c has its
 * centre at s = c).  Peskin-4: cells floor(s)-1 .. floor(s)+2.  Roma-3: the nearest centre
 * floor(s+0.5) and its two neighbours. */
static int stencil_first(int kernel, double s) {
    if (kernel == 2) return (int)floor(s) - 1;
    return (int)floor(s + 0.5) - 1;
}
static int stencil_width(int kernel) { return kernel == 2 ? 4 : 3; }
static double phi(int kernel, double r) { return kernel == 2 ? or_phi_peskin4(r) : or_phi_roma3(r); }

/* Leaf index of the finest-level cell (i,j,k), or -1 when the cell is outside the domain or
 * is not a leaf of level lmax (IBM operations live on the finest level only, Sec. 2.4). */
/* Periodic domain (Sec. 5.2's turbulence box): cell indices wrap modulo the cells per axis. */
static int64_t wrap_index(int64_t i, int64_t nc) { return ((i % nc) + nc) % nc; }

static int64_t fine_leaf_p(const uint64_t *key, const uint8_t *level, int64_t n, int lmax, int64_t i, int64_t j,
                           int64_t k, int periodic) {
    int64_t nc = (int64_t)1 << lmax;
    if (periodic) {
        i = wrap_index(i, nc);
        j = wrap_index(j, nc);
        k = wrap_index(k, nc);
    }
    if (i < 0 || j < 0 || k < 0 || i >= nc || j >= nc || k >= nc) return -1;
    uint64_t q = or_morton((uint32_t)(i << (OR_MAXLEVEL - lmax)), (uint32_t)(j << (OR_MAXLEVEL - lmax)),
                           (uint32_t)(k << (OR_MAXLEVEL - lmax)));
    int64_t a = leaf_of_key(key, n, q);
    if (level[a] != lmax) return -1;
    return a;
}

/* IBM interpolation, Eq. (ibm_interpolate):  u*(X_k) = sum_x u*(x) W(x - X_k) dx^3 with
 * W = prod_d phi(./dx)/dx, i.e. u*(X_k) = sum over the stencil of phi(rx) phi(ry) phi(rz) u(cell).
 * kernel: 2 = Peskin-4, 3 = Roma-3.  field: N x 4 (x, y, z, unused).  u: 3 planes of np.
 * Stencil cells that are outside the domain or not finest-level leaves are skipped and
 * counted in *n_bad (returned). */
int64_t or_interp_delta_p(const uint64_t *key, const uint8_t *level, int64_t n, int lmax, int kernel,
                          const double *field, const double *x, const double *y, const double *z, int64_t np,
                          double *u, int periodic) {
    int64_t nbad = 0;
    int wdt = stencil_width(kernel);
    double scale = ldexp(1.0, lmax);
#pragma omp parallel for schedule(static) reduction(+ : nbad)
    for (int64_t p = 0; p < np; ++p) {
        double s[3] = {x[p] * scale - 0.5, y[p] * scale - 0.5, z[p] * scale - 0.5};
        int i0[3];
        for (int d = 0; d < 3; ++d) i0[d] = stencil_first(kernel, s[d]);
        double acc[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < wdt; ++c)
            for (int b = 0; b < wdt; ++b)
                for (int a = 0; a < wdt; ++a) {
                    int64_t leaf = fine_leaf_p(key, level, n, lmax, i0[0] + a, i0[1] + b, i0[2] + c, periodic);
                    if (leaf < 0) {
                        nbad++;
                        continue;
                    }
                    double w = phi(kernel, s[0] - (i0[0] + a)) * phi(kernel, s[1] - (i0[1] + b)) *
                               phi(kernel, s[2] - (i0[2] + c));
                    for (int d = 0; d < 3; ++d) acc[d] += w * field[4 * leaf + d];
                }
        for (int d = 0; d < 3; ++d) u[d * np + p] = acc[d];
    }
    return nbad;
}

/* IBM spreading, the adjoint of or_interp_delta:
 *   f(x) += sum_k F_k W(x - X_k) dV_k = sum_k F_k phi phi phi dV_k / dx^3,
 * with dV_k = dx^3 when dV is NULL (the paper's literal form, Eq. for F(x)).
 * F: 3 planes of np.  f: N x 4, accumulated (component 3 untouched).  Sequential over
 * markers.  Returns the number of skipped stencil cells. */
int64_t or_spread_delta_p(const uint64_t *key, const uint8_t *level, int64_t n, int lmax, int kernel,
                          const double *x, const double *y, const double *z, const double *F, const double *dV,
                          int64_t np, double *f, int periodic) {
    int64_t nbad = 0;
    int wdt = stencil_width(kernel);
    double scale = ldexp(1.0, lmax);
    double h3 = ldexp(1.0, -3 * lmax);
    for (int64_t p = 0; p < np; ++p) {
        double s[3] = {x[p] * scale - 0.5, y[p] * scale - 0.5, z[p] * scale - 0.5};
        int i0[3];
        for (int d = 0; d < 3; ++d) i0[d] = stencil_first(kernel, s[d]);
        double vol = dV ? dV[p] / h3 : 1.0;
        for (int c = 0; c < wdt; ++c)
            for (int b = 0; b < wdt; ++b)
                for (int a = 0; a < wdt; ++a) {
                    int64_t leaf = fine_leaf_p(key, level, n, lmax, i0[0] + a, i0[1] + b, i0[2] + c, periodic);
                    if (leaf < 0) {
                        nbad++;
                        continue;
                    }
                    double w = phi(kernel, s[0] - (i0[0] + a)) * phi(kernel, s[1] - (i0[1] + b)) *
                               phi(kernel, s[2] - (i0[2] + c));
                    for (int d = 0; d < 3; ++d) f[4 * leaf + d] += F[d * np + p] * w * vol;
                }
    }
    return nbad;
}

int64_t or_interp_delta(const uint64_t *key, const uint8_t *level, int64_t n, int lmax, int kernel,
                        const double *field, const double *x, const double *y, const double *z, int64_t np,
                        double *u) {
    return or_interp_delta_p(key, level, n, lmax, kernel, field, x, y, z, np, u, 0);
}

int64_t or_spread_delta(const uint64_t *key, const uint8_t *level, int64_t n, int lmax, int kernel,
                        const double *x, const double *y, const double *z, const double *F, const double *dV,
                        int64_t np, double *f) {
    return or_spread_delta_p(key, level, n, lmax, kernel, x, y, z, F, dV, np, f, 0);
}

/* Volume-weighted mean of a cell field over the unit cube, sum_c f_c 8^-level_c (the mean
 * force removed in a periodic box, Sec. 5.2), and its subtraction from every cell. */
void or_field_mean(const uint8_t *level, int64_t n, const double *f, double mean[3]) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t c = 0; c < n; ++c)
        for (int d = 0; d < 3; ++d) acc[d] += f[4 * c + d] * ldexp(1.0, -3 * level[c]);
    for (int d = 0; d < 3; ++d) mean[d] = acc[d];
}

/* Multi-direct forcing (Sec. 2.2): n_iter rounds, each
 *   u_k = I u                      (interpolation to the markers, Eq. ibm_interpolate)
 *   F_k = (U_k - u_k) / dt         (marker force)
 *   F   = S F_k                    (spreading, with the marker volumes dV or dx^3)
 *   u  += dt F / rho,  f += F      (velocity correction; f is the total force of the step)
 * The printed correction u = u* + F/rho omits the time step; it is read as u* + dt F/rho (the
 * dimensionally consistent form, identical in lattice units dt = 1), applied to the velocity
 * corrected so far (the iterated form of multi-direct forcing).  u_star: N x 4 (component 3
 * copied); u_out, f_out: N x 4.  slip (nullable): n_iter + 1 values of sqrt(sum_k |U_k - u_k|^2),
 * before each round and after the last.  Returns the skipped stencil cells of the first
 * interpolation. */
int64_t or_ibm_mdf(const uint64_t *key, const uint8_t *level, int64_t n, int lmax, int kernel,
                   const double *u_star, const double *x, const double *y, const double *z, const double *U,
                   const double *dV, int64_t nm, double rho, double dt, int n_iter, double *u_out, double *f_out,
                   double *slip) {
    double *uk = (double *)malloc(sizeof(double) * 3 * (size_t)(nm > 0 ? nm : 1));
    double *Fk = (double *)malloc(sizeof(double) * 3 * (size_t)(nm > 0 ? nm : 1));
    double *F = (double *)malloc(sizeof(double) * 4 * (size_t)(n > 0 ? n : 1));
    memcpy(u_out, u_star, sizeof(double) * 4 * (size_t)n);
    memset(f_out, 0, sizeof(double) * 4 * (size_t)n);
    int64_t nbad = 0;
    for (int it = 0; it <= n_iter; ++it) {
        int64_t b = or_interp_delta(key, level, n, lmax, kernel, u_out, x, y, z, nm, uk);
        if (it == 0) nbad = b;
        double s2 = 0.0;
        for (int64_t k = 0; k < nm; ++k)
            for (int d = 0; d < 3; ++d) {
                double e = U[d * nm + k] - uk[d * nm + k];
                s2 += e * e;
                Fk[d * nm + k] = e / dt;
            }
        if (slip) slip[it] = sqrt(s2);
        if (it == n_iter) break;
        memset(F, 0, sizeof(double) * 4 * (size_t)n);
        or_spread_delta(key, level, n, lmax, kernel, x, y, z, Fk, dV, nm, F);
        for (int64_t c = 0; c < n; ++c)
            for (int d = 0; d < 3; ++d) {
                u_out[4 * c + d] += dt * F[4 * c + d] / rho;
                f_out[4 * c + d] += F[4 * c + d];
            }
    }
    free(uk);
    free(Fk);
    free(F);
    return nbad;
}

/* Per-body linear and angular sums of a marker quantity (Sec. 2.3, rigid bodies):
 *   lin_b = scale * sum_{k in b} v_k w_k,   ang_b = scale * sum_{k in b} (X_k - x_b) x v_k w_k,
 * with w_k = dV[k] (or w when dV is NULL).  With v = u at the internal markers and
 * scale = rho_f these are the internal fluid's linear momentum P and angular momentum L; with
 * v = F_k at the surface markers and scale = -1, the IBM force and torque -sum F_k dV_k and
 * -sum (X_k - x_b) x F_k dV_k.  The printed formulas swap the names P and L against the
 * text (linear momentum P, angular momentum L) and drop rho_f from the discrete sums; read
 * with the text and the integrals.  Markers of body b are start[b] .. start[b+1]-1.
 * v: 3 planes of n; xb: nb x 3; lin, ang: nb x 3. */
void or_body_sums(const double *x, const double *y, const double *z, const double *v, const double *dV, double w,
                  int64_t n, const int64_t *start, int nb, const double *xb, double scale, double *lin,
                  double *ang) {
    for (int b = 0; b < nb; ++b) {
        double l[3] = {0.0, 0.0, 0.0}, a[3] = {0.0, 0.0, 0.0};
        for (int64_t k = start[b]; k < start[b + 1]; ++k) {
            double wk = dV ? dV[k] : w;
            double vv[3] = {v[k] * wk, v[n + k] * wk, v[2 * n + k] * wk};
            double r[3] = {x[k] - xb[3 * b], y[k] - xb[3 * b + 1], z[k] - xb[3 * b + 2]};
            for (int d = 0; d < 3; ++d) l[d] += vv[d];
            a[0] += r[1] * vv[2] - r[2] * vv[1];
            a[1] += r[2] * vv[0] - r[0] * vv[2];
            a[2] += r[0] * vv[1] - r[1] * vv[0];
        }
        for (int d = 0; d < 3; ++d) {
            lin[3 * b + d] = scale * l[d];
            ang[3 * b + d] = scale * a[d];
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* Point-particle trilinear interpolation (Sec. 2.3.2).  The paper names the scheme only;  */
/* this is the reading of "host leaf and its 7 level-mates":                               */
/*   host leaf at level l, cell coords c; t_d = x_d 2^l - (c_d + 1/2) in [-1/2, 1/2);      */
/*   s_d = +1 if t_d >= 0 else -1; level-mates are the cells c + {0, s_d} per axis at       */
/*   level l; trilinear weights prod (1-|t_d|) or |t_d|.  Value of a level-mate cell m:     */
/*     a leaf of level l           -> its value;                                           */
/*     inside a coarser leaf       -> that leaf's value (hanging neighbour);               */
/*     refined                     -> volume-weighted mean of the leaves inside it          */
/*                                    (the coalescence average of Sec. 2.1.1);              */
/*     outside [0,1)^3 on an axis  -> the host's index on that axis (constant extrapolation). */
/* ------------------------------------------------------------------------------------ */

static void levelmate_value(const uint64_t *key, const uint8_t *level, int64_t n, const double *field, int l,
                            int64_t i, int64_t j, int64_t k, double out[3]) {
    uint64_t anchor = or_morton((uint32_t)(i << (OR_MAXLEVEL - l)), (uint32_t)(j << (OR_MAXLEVEL - l)),
                                (uint32_t)(k << (OR_MAXLEVEL - l)));
    int64_t a = leaf_of_key(key, n, anchor);
    if (level[a] <= l) {
        for (int d = 0; d < 3; ++d) out[d] = field[4 * a + d];
        return;
    }
    /* refined: leaves with keys in [anchor, anchor + 8^(21-l)) */
    uint64_t end = anchor + key_span(l);
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t b = a; b < n && key[b] < end; ++b) {
        double vol = ldexp(1.0, -3 * (level[b] - l)); /* fraction of the level-l cell */
        for (int d = 0; d < 3; ++d) acc[d] += vol * field[4 * b + d];
    }
    for (int d = 0; d < 3; ++d) out[d] = acc[d];
}

/* host: leaf of each point (from a locate), -1 entries give NaN.  u: 3 planes of np. */
void or_interp_trilinear_p(const uint64_t *key, const uint8_t *level, int64_t n, const double *field,
                           const double *x, const double *y, const double *z, const int32_t *host, int64_t np,
                           double *u, int periodic) {
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < np; ++p) {
        if (host[p] < 0) {
            for (int d = 0; d < 3; ++d) u[d * np + p] = NAN;
            continue;
        }
        int64_t h = host[p];
        int l = level[h];
        uint32_t a[3];
        or_unmorton(key[h], &a[0], &a[1], &a[2]);
        double pt[3] = {x[p], y[p], z[p]};
        int64_t c[3], sgn[3];
        double t[3];
        int64_t ncell = (int64_t)1 << l;
        for (int d = 0; d < 3; ++d) {
            c[d] = a[d] >> (OR_MAXLEVEL - l);
            t[d] = pt[d] * ldexp(1.0, l) - ((double)c[d] + 0.5);
            sgn[d] = t[d] >= 0.0 ? 1 : -1;
        }
        double acc[3] = {0.0, 0.0, 0.0};
        for (int corner = 0; corner < 8; ++corner) {
            int64_t m[3];
            double w = 1.0;
            for (int d = 0; d < 3; ++d) {
                int off = (corner >> d) & 1;
                m[d] = c[d] + off * sgn[d];
                if (m[d] < 0 || m[d] >= ncell) m[d] = periodic ? wrap_index(m[d], ncell) : c[d];
                w *= off ? fabs(t[d]) : 1.0 - fabs(t[d]);
            }
            double v[3];
            levelmate_value(key, level, n, field, l, m[0], m[1], m[2], v);
            for (int d = 0; d < 3; ++d) acc[d] += w * v[d];
        }
        for (int d = 0; d < 3; ++d) u[d * np + p] = acc[d];
    }
}

/* ------------------------------------------------------------------------------------ */
/* Learned-index root network: 1 -> 32 (ReLU) -> 1, MSE loss.  Parameter layout (97):      */
/*   w1[0..31], b1[0..31], w2[0..31], b2.                                                 */
/* ------------------------------------------------------------------------------------ */

#define OR_MLP_H 32

double or_mlp_forward1(const double *prm, double xin) {
    const double *w1 = prm, *b1 = prm + OR_MLP_H, *w2 = prm + 2 * OR_MLP_H, b2 = prm[3 * OR_MLP_H];
    double y = b2;
    for (int k = 0; k < OR_MLP_H; ++k) {
        double zk = w1[k] * xin + b1[k];
        double hk = zk > 0.0 ? zk : 0.0;
        y += w2[k] * hk;
    }
    return y;
}

/* loss = (1/B) sum_i (y_i - t_i)^2 and its gradient by the chain rule (ReLU'(0) = 0). */
double or_mlp_loss_grad(const double *prm, const double *xin, const double *tgt, int64_t nb, double *grad) {
    const double *w1 = prm, *b1 = prm + OR_MLP_H, *w2 = prm + 2 * OR_MLP_H;
    memset(grad, 0, sizeof(double) * (3 * OR_MLP_H + 1));
    double loss = 0.0;
    for (int64_t i = 0; i < nb; ++i) {
        double y = or_mlp_forward1(prm, xin[i]);
        double e = y - tgt[i];
        loss += e * e;
        double g = 2.0 * e / (double)nb; /* dL/dy_i */
        grad[3 * OR_MLP_H] += g;
        for (int k = 0; k < OR_MLP_H; ++k) {
            double zk = w1[k] * xin[i] + b1[k];
            double hk = zk > 0.0 ? zk : 0.0;
            grad[2 * OR_MLP_H + k] += g * hk;
            double dz = zk > 0.0 ? g * w2[k] : 0.0;
            grad[k] += dz * xin[i];
            grad[OR_MLP_H + k] += dz;
        }
    }
    return loss / (double)nb;
}

/* ------------------------------------------------------------------------------------ */
/* Point-particle advection (Sec. 2.3.2, Eq. PointParticle with gravity off):              */
/*   a = f_p (u(x_p) - v) / tau,  f_p = 1 + 0.15 Re_p^0.687,  Re_p = re_coef |u - v|       */
/*   (re_coef = 2 r_p / nu; re_coef = 0 gives Stokes drag, f_p = 1),                        */
/*   v_{n+1} = v_n + dt (3/2 a_n - 1/2 a_{n-1}),  x_{n+1} = x_n + dt (3/2 v_n - 1/2 v_{n-1}); */
/*   the first step (no history) is explicit Euler; periodic != 0 wraps positions into [0,1). */
/* State planes of np each: x[3], v[3], a_prev[3], v_prev[3]; u: 3 planes.                  */
/* ------------------------------------------------------------------------------------ */

void or_advect_ab2(double *x, double *v, double *a_prev, double *v_prev, const double *u, int64_t np,
                   double tau, double re_coef, double dt, int first, int periodic) {
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < np; ++p) {
        double rel[3], mag2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            rel[d] = u[d * np + p] - v[d * np + p];
            mag2 += rel[d] * rel[d];
        }
        double fp = 1.0;
        if (re_coef > 0.0) fp = 1.0 + 0.15 * pow(re_coef * sqrt(mag2), 0.687);
        for (int d = 0; d < 3; ++d) {
            double vn = v[d * np + p];
            double an = fp * rel[d] / tau;
            double am = first ? an : a_prev[d * np + p];
            double vm = first ? vn : v_prev[d * np + p];
            v[d * np + p] = vn + dt * (1.5 * an - 0.5 * am);
            double xn = x[d * np + p] + dt * (1.5 * vn - 0.5 * vm);
            if (periodic) { /* wrap into [0, 1) */
                xn = xn - floor(xn);
                if (xn >= 1.0) xn = 0.0;
            }
            x[d * np + p] = xn;
            a_prev[d * np + p] = an;
            v_prev[d * np + p] = vn;
        }
    }
}

/* Vectorised delta-kernel evaluation for tests: kernel 2 = Peskin-4, 3 = Roma-3. */
void or_phi_array(int kernel, const double *r, int64_t n, double *out) {
    for (int64_t i = 0; i < n; ++i) out[i] = phi(kernel, r[i]);
}

void or_interp_trilinear(const uint64_t *key, const uint8_t *level, int64_t n, const double *field,
                         const double *x, const double *y, const double *z, const int32_t *host, int64_t np,
                         double *u) {
    or_interp_trilinear_p(key, level, n, field, x, y, z, host, np, u, 0);
}
