/*
 * sg.h -- C ABI of libsg, a CUDA (sm_103a) implementation of the contiguous
 * sparse-grid storage of "Contiguous Storage of Grid Data for Heterogeneous
 * Computing" (Gu & Hu) and of the level-set sweeps run over it.
 *
 * Storage ("MeshWithGridDataPackages", Listing 1; "Array Storage and Access"):
 *   - a background mesh of dims[0] x dims[1] x dims[2] coarse cells of size
 *     lc = 4h starting at lo; cell index c = I + nx (J + ny K);
 *   - cells cut by the band own a 4x4x4 data package; package ids 0 and 1 are
 *     the far-field inside (value -F) and outside (+F) packages, active
 *     packages follow from id 2 in increasing cell index ("Indexing");
 *   - every field is one contiguous float array [P][64], data index
 *     d = i + 4j + 16k inside a package (structure of arrays);
 *   - cell_pkg[nc] (int32) maps a cell to its package; pkg_cell[P] (int32,
 *     -1 for the far packages) and pkg_type[P] (uint8: 0 far inside,
 *     1 far outside, 2 core, 3 inner) are the per-package meta data;
 *   - nbr[P][27] (int32) holds the packages of the 3x3x3 cell neighbourhood,
 *     entry (di+1) + 3(dj+1) + 9(dk+1) ("Neighbourhood"); cells outside the
 *     domain are the outside far package; far packages are their own
 *     neighbours ("Initialization Process", step 5).
 *
 * Conventions for every call:
 *   - all work is queued on the grid's CUDA stream and the call returns a
 *     launch-time status; only sg_tag_allocate and sg_status_sync block;
 *   - device-side problems set a sticky error word, reported by
 *     sg_status_sync;
 *   - no C++ exception crosses this interface;
 *   - state order: sg_create -> sg_tag_allocate -> sg_init_sdf -> the sweeps
 *     and the probe; a call out of order returns SG_ERR_STATE;
 *   - the grid owns every array it allocates; particle arrays belong to the
 *     caller;
 *   - a failed call leaves the grid in its previous state and records a
 *     message for sg_last_error.
 */
#ifndef SG_H
#define SG_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SG_API __attribute__((visibility("default")))
#else
#define SG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sg_grid sg_grid;
typedef int32_t sg_status;

enum {
    SG_OK = 0,
    SG_ERR_INVALID = 1,  /* bad argument (null pointer, size, kind, mode) */
    SG_ERR_OOM = 2,      /* the allocator returned NULL */
    SG_ERR_CUDA = 3,     /* a CUDA runtime call failed */
    SG_ERR_STATE = 4,    /* call out of order (e.g. a sweep before init) */
    SG_ERR_CAPACITY = 5, /* sizes beyond the supported range */
    SG_ERR_TIMEOUT = 6,  /* a bounded device wait gave up */
    SG_ERR_DEVICE = 7,   /* a kernel reported an inconsistency */
    SG_ERR_IO = 8        /* a file could not be written */
};

enum {
    SG_SHAPE_SPHERE = 0,
    SG_SHAPE_PLANE = 1,
    SG_SHAPE_TORUS = 2,
    SG_SHAPE_PRISM = 3,
    SG_SHAPE_ROUNDED_BOX = 4,
    SG_SHAPE_SHELL = 5
};

/* Analytic body, in a local frame: a world point x maps to q = R^T (x - centre)
 * with R = rot (row-major, local to world).  Parameters p per kind:
 *   sphere: p0 radius; plane: q_z = 0; torus: p0 major (about local z), p1
 *   minor; prism: triangle (p0,p1),(p2,p3),(p4,p5) extruded over q_z in
 *   [p6, p7]; rounded box: half extents p0..p2, rounding p3; shell: the
 *   solid between the spheres of radii p0 < p1 (the shelled sphere of the
 *   paper's "Performance Evaluation").
 * Host struct, copied by value. */
typedef struct {
    int32_t kind;
    int32_t pad;
    double centre[3];
    double rot[9];
    double p[8];
} sg_shape;

/* Grid description (host struct, copied).
 *   lo, dims, h     background mesh of dims coarse cells of 4h from lo;
 *   id_order        package ids in linear cell order (0, "sorted by spatial
 *                   location" with x fastest) or in the Morton order of the
 *                   cells (1: bit interleave of I, J, K, I lowest);
 *   far_value       F of the far packages (-F inside, +F outside); <= 0: 16h;
 *   kernel_support  support of the Wendland C2 kernel of the integrals, a
 *                   length (0: 2h; at most 3h, so that every tap with a
 *                   non-zero weight lies in the 5^3 stencil);
 *   heaviside_eps   half width of the smoothed Heaviside, a length (0: h).
 * The surrogate integrals are defined for the defaults (2h, h) only. */
typedef struct {
    double lo[3];
    int32_t dims[3];
    int32_t id_order;
    double h;
    double far_value;
    double kernel_support;
    double heaviside_eps;
} sg_grid_desc;

/* Optional device-memory hook.  alloc returns device memory of at least
 * `bytes` usable on `stream` (NULL on failure); free releases it.  With a
 * NULL allocator the library uses cudaMallocAsync / cudaFreeAsync. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*free)(void *ptr, size_t bytes, void *stream, void *ctx);
    void *ctx;
} sg_allocator;

enum {
    SG_FIELD_PHI = 0,  /* level set phi */
    SG_FIELD_GX = 1,   /* gradient of phi */
    SG_FIELD_GY = 2,
    SG_FIELD_GZ = 3,
    SG_FIELD_W = 4,    /* kernel weight integral */
    SG_FIELD_GWX = 5,  /* h * gradient of W */
    SG_FIELD_GWY = 6,
    SG_FIELD_GWZ = 7,
    SG_FIELD_LAP = 8,  /* 7-point Laplacian of phi */
    SG_FIELD_S0 = 9,   /* smoothed sign of the last sg_reinit call */
    SG_N_FLOAT_FIELDS = 10,
    SG_FIELD_CELL_PKG = 100, /* int32 [nx*ny*nz] */
    SG_FIELD_PKG_CELL = 101, /* int32 [P] */
    SG_FIELD_PKG_TYPE = 102, /* uint8 [P] */
    SG_FIELD_NBR = 103       /* int32 [P*27] */
};

/* Morton-order the particles inside sg_probe (see sg_probe). */
#define SG_PROBE_MORTON 1

/* Create an empty grid on `stream` (a cudaStream_t; NULL = legacy default).
 * Errors: SG_ERR_INVALID (null pointers, h <= 0, a dimension < 1),
 * SG_ERR_CAPACITY (more than 2^31 - 1 cells or 4*dims >= 2^21). */
SG_API sg_status sg_create(const sg_grid_desc *desc, const sg_allocator *alloc, void *stream, sg_grid **out);

/* Release every array the grid owns (stream-ordered), then the handle. */
SG_API sg_status sg_destroy(sg_grid *g);

/* Band tagging and package allocation ("Initialization Process", steps 1-3
 * and 5; "Indexing"; "Neighbourhood").  A cell is core when the distance
 * from its centre lo + (4I + 2)h to the surface is below lc (1 - 2^-10)
 * (float-float evaluation), inner when it is not core and one of its 26
 * neighbours is core; ids follow the cell index.  Fills cell_pkg, pkg_cell,
 * pkg_type and nbr and writes P (including the 2 far packages) to
 * *n_packages.  Synchronises the stream (P sizes the package arrays).
 * May be called again to re-tag; previous field contents are discarded (the
 * field buffers are kept and reused when large enough, so a grid re-tagged
 * with a package count it has seen before allocates nothing). */
SG_API sg_status sg_tag_allocate(sg_grid *g, const sg_shape *shape, int64_t *n_packages);

/* Multi-resolution tagging (Sec. "Multi-resolution Level-set", and step 1
 * of "Initialization Process": for successive layers only the cells covered
 * by the coarse core cells are evaluated).  `coarse` is the layer below g:
 * same lo, half the dims, exactly twice the spacing, tagged and initialised.
 * A cell of g inside a coarse core cell is classified by its own distance
 * exactly as sg_tag_allocate does; any other cell is far, inside when its
 * coarse cell is far inside or an inner cell whose phi (data point 0) is
 * negative.  Such a cell lies at least 1.13 cells of g from the surface, so
 * the result equals sg_tag_allocate on g bit for bit, with distances
 * evaluated only under coarse core cells.  n_packages as sg_tag_allocate;
 * evaluated (may be NULL) receives the number of cells whose distance was
 * evaluated.  Synchronises like sg_tag_allocate.
 * Errors: SG_ERR_INVALID (null or mismatched coarse layer, bad shape),
 * SG_ERR_STATE (coarse layer without phi), SG_ERR_OOM, SG_ERR_CAPACITY. */
SG_API sg_status sg_tag_allocate_from(sg_grid *g, const sg_grid *coarse, const sg_shape *shape, int64_t *n_packages,
                                      int64_t *evaluated);

/* The number of layers of a multi-resolution stack ending at `finest` (the
 * paper computes it in advance): 1 + the number of halvings of the
 * background mesh that keep every dimension even before halving and at
 * least min_dims after it.  Host-only arithmetic; 0 for NULL or
 * min_dims < 1.  Layer k (0 coarsest) has spacing h 2^(L-1-k) and dims
 * dims / 2^(L-1-k) over the same domain. */
SG_API int32_t sg_multires_layers(const sg_grid_desc *finest, int32_t min_dims);

/* Level-set values ("Initialization Process", step 4): phi at the
 * cell-centred data points lo + (4I + i + 0.5) h, evaluated in float-float
 * and rounded once; far packages hold -F and +F.  Requires a tagged grid. */
SG_API sg_status sg_init_sdf(sg_grid *g, const sg_shape *shape);

/* Regularised central difference (Listing 5) on every active package:
 * g_a = ((phi(+e_a) - phi(0)) + (phi(0) - phi(-e_a))) / (2h); neighbours
 * through the index shift of Listing 2.  Far packages keep g = 0.
 * Writes SG_FIELD_GX/GY/GZ.  Requires phi. */
SG_API sg_status sg_gradient(sg_grid *g);

/* Consistency (sign) correction (Sec. "Consistency Correction"): the sign
 * of phi is trusted only where |phi| < trust h (trust h rounded to float),
 * close to the surface, and carried from there to the rest of the domain by
 * two diffusion steps, each a Jacobi flood over face neighbours in which an
 * unknown entry takes the sign of the sum of its labelled neighbours'
 * signs, run until a sweep changes nothing:
 *   1. over the data points of the active packages, from the trusted
 *      points; then phi <- sign |phi| wherever a sign was found;
 *   2. over the background cells: core cells blocked, inner cells start
 *      with the sign their package's points share; a far cell takes the
 *      far package of its label (0 inside, 1 outside) and the neighbour
 *      and face tables are rebuilt to match.
 * (The paper names the cell step first; here it runs second because every
 * data point within h of the surface lies in a core cell, so the cells have
 * no trusted sign before the points.)  For a grid whose magnitudes are
 * distances this restores every sign a leaky surface got wrong outside the
 * trusted band.  out (host, may be NULL): [4] = points flipped, far cells
 * moved, point sweeps, cell sweeps (each count ends with the first sweep
 * that changes nothing).  Derived fields (g, W, ...) are stale
 * afterwards.  Blocks until done (it reads convergence flags).
 * Errors: SG_ERR_INVALID (trust <= 0 or not finite), SG_ERR_STATE (no phi),
 * SG_ERR_OOM, SG_ERR_TIMEOUT (a flood that does not settle, which cannot
 * happen for valid tables, or a grid-barrier wait of a persistent flood
 * that gave up after its bounded number of polls; phi and the tables are
 * then unchanged). */
SG_API sg_status sg_consistency_correct(sg_grid *g, float trust, int64_t *out);

/* Testing hooks of sg_consistency_correct (out as there, may be NULL):
 *   SG_DEBUG_CC_ABSENT_POINTS / _CELLS: one CTA is counted at every grid
 *     barrier of the point (cell) flood and never arrives, so that flood's
 *     first barrier cannot complete: every CTA gives up after its 2^21 polls
 *     (at least 67 ms; 0.54 s measured on a B300) and the call returns
 *     SG_ERR_TIMEOUT with phi and the tables unchanged (the corrections are
 *     applied only after both floods settled) and the grid usable;
 *   SG_DEBUG_CC_PER_SWEEP: the floods run as one launch per sweep with the
 *     host reading the flags (the path of devices without cooperative
 *     launch) instead of one persistent launch each.
 * Errors: as sg_consistency_correct; SG_ERR_INVALID (unknown flags, or an
 * absent CTA with SG_DEBUG_CC_PER_SWEEP); SG_ERR_DEVICE (an absent CTA on a
 * device without cooperative launch, where the floods do not wait on one
 * another). */
#define SG_DEBUG_CC_ABSENT_POINTS 1
#define SG_DEBUG_CC_ABSENT_CELLS 2
#define SG_DEBUG_CC_PER_SWEEP 4
SG_API sg_status sg_debug_consistency(sg_grid *g, float trust, int32_t flags, int64_t *out);
/* sg_debug_consistency with SG_DEBUG_CC_ABSENT_POINTS | SG_DEBUG_CC_ABSENT_CELLS. */
SG_API sg_status sg_debug_consistency_absent_cta(sg_grid *g, float trust);

/* Testing hook, process-wide: with on != 0 the probe, the exact kernel
 * integrals and the relaxation steps recorded afterwards take their 64-bit
 * address kernels, which otherwise serve only stores too large for 32-bit
 * byte offsets (2^24 packages and more for the probe and the integrals,
 * 2^21 for the relaxation's table, 2^30 particles for the probe).  Results
 * are the same bit for bit either way. */
SG_API void sg_debug_wide_offsets(int32_t on);

/* The "sequential" benchmark of "Performance Evaluation": a small change to
 * every active value, phi <- phi + delta on every active package (far
 * packages untouched).  Requires phi. */
SG_API sg_status sg_sequential_update(sg_grid *g, float delta);

/* 7-point Laplacian sum_a (phi(+e_a) - 2 phi + phi(-e_a)) / h^2 on every
 * active package (the stencil benchmark of "Performance Evaluation").
 * Writes SG_FIELD_LAP.  Requires phi. */
SG_API sg_status sg_laplacian(sg_grid *g);

/* Reinitialisation: `iterations` Jacobi sweeps of
 * phi <- phi - dt S0 (sqrt(G) - 1), dt = cfl h, S0 = phi0 / sqrt(phi0^2 + h^2)
 * with phi0 = phi at entry, and the Godunov sum G over the axes of
 * max(max(D-,0)^2, min(D+,0)^2) where phi0 > 0 and
 * max(min(D-,0)^2, max(D+,0)^2) where phi0 < 0 (no change where phi0 = 0).
 * Far packages are fixed.  Not in the paper (Sussman, Smereka & Osher 1994;
 * Rouy & Tourin 1992).  Errors: SG_ERR_INVALID for iterations < 0 or
 * cfl <= 0.  Requires phi. */
SG_API sg_status sg_reinit(sg_grid *g, int32_t iterations, float cfl);

/* Kernel integrals ("Integral with SPH Smoothing Kernel and Grid-Particle
 * Coupling"), mode 0 (exact): with the Wendland C2 kernel w(q) of support
 * 2h and the smoothed Heaviside H of half width h, over the offsets s of
 * the 5^3 stencil (taps with |s| >= 2 weigh zero):
 *   W  = sum_s w(|s|) H(-phi(x+sh)) / sum_s w(|s|)
 *   G^ = h grad W = sum_s w'(|s|) (-s/|s|) H(-phi(x+sh)) / sum_s w(|s|).
 * Far packages: W = 1 inside, 0 outside, G^ = 0.  Writes SG_FIELD_W and
 * SG_FIELD_GWX/GWY/GWZ.  Mode 0 takes mlp = NULL; mode 1 (surrogate with
 * exact fallback, see SG_SUR_*) takes an sg_mlp*: one pass classifies every
 * point and writes the trivial and fallback values and a list of network
 * points, a second runs the network over the list in 128-row tensor-core
 * tiles (a product that never completes within its bounded wait sets the
 * device error word: sg_status_sync returns SG_ERR_TIMEOUT).  The grid
 * keeps the list's buffer (4 bytes per data point) for later calls.
 * Errors: SG_ERR_INVALID for an unknown mode or a missing or extra network;
 * SG_ERR_CAPACITY for mode 1 on 2^24 or more packages (the surrogate path
 * indexes points and gathers in 32 bits).  Requires phi. */
SG_API sg_status sg_kernel_integrals(sg_grid *g, int32_t mode, const void *mlp);

/* Particle probe ("Grid-Particle Coupling"): trilinear interpolation of phi,
 * grad phi, W and G^ at n particles.  x, y, z are device arrays of n floats;
 * the eight outputs are device arrays of n floats in input order (any may
 * be NULL to skip it).  The lattice coordinate u = (x - lo)/h - 1/2 of the
 * float position is formed in float-float (x (1/h) - (lo/h + 1/2), about 44
 * bits), so i0 = floor(u) is the exact decision unless u lies within about
 * 1e-10 of an integer, and t = u - i0 is correct to float rounding; i0 is
 * clamped to +-2^24 (far outside any domain).  Home cell floor(i0/4) (the
 * outside far package when outside the domain),
 * corners reached through the home package's neighbourhood.  The normal is
 * grad/|grad| (0 where |grad| = 0).  Fields not yet computed read as 0.
 * With SG_PROBE_MORTON the particles are walked in Morton order (stable
 * sort by the bit interleave of k_a = clamp(i0_a + 1, 0, 4 dims_a + 1), x in
 * the lowest bit) and results are written back in input order; an input
 * whose sampled adjacent pairs (one in 128) are already in that order is
 * walked as it is.  The walk only affects speed: the results are the same
 * for any order.
 * Errors: SG_ERR_INVALID (n < 0, null positions), SG_ERR_CAPACITY
 * (n >= 2^31).  Requires phi. */
SG_API sg_status sg_probe(sg_grid *g, int64_t n, const float *x, const float *y, const float *z, float *phi, float *nx,
                   float *ny, float *nz, float *W, float *Gx, float *Gy, float *Gz, int32_t flags);

/* Morton keys (as in sg_probe) and the stable sorted order of n particles:
 * keys[n] (uint64) and order[n] (int32, order[r] = input index of rank r),
 * device arrays owned by the caller.  Requires a tagged grid. */
SG_API sg_status sg_morton_order(sg_grid *g, int64_t n, const float *x, const float *y, const float *z, uint64_t *keys,
                          int32_t *order);

/* ------------------------------------------------------------------------ */
/* Batches: many bodies, one launch per sweep.                               */
/* ------------------------------------------------------------------------ */
typedef struct sg_batch sg_batch;

/* How a batch run is scheduled.  pkgs_per_item: packages each half-warp
 * takes per work item (1, 2, 4 or 8; a CTA takes 16 times that, for the
 * face stencils and the integrals alike); depth: packages whose loads a
 * half-warp has in flight at once (1 or 2, at most pkgs_per_item).  The
 * sweeps are those of sg_gradient, sg_reinit(reinit_iterations, cfl) and
 * sg_kernel_integrals(integrals_mode, m): integrals_mode 0 is the exact sum,
 * 1 the surrogate with fallback, whose network m is bound by
 * sg_batch_set_surrogate. */
typedef struct {
    int32_t pkgs_per_item;
    int32_t depth;
    int32_t reinit_iterations;
    float cfl;
    int32_t integrals_mode;
    int32_t reserved;
} sg_batch_plan;

/* Concatenate the packages of n initialised grids (same device) into one
 * global store: body i owns package ids [base_i, base_i + P_i) with its own
 * far packages and neighbour ids shifted by base_i.  phi is copied from the
 * grids (they may be destroyed afterwards); device memory comes from the
 * first grid's allocator; work runs on `stream`.  Not in the paper (the
 * batched, persistent launch of many bodies is this library's).
 * Errors: SG_ERR_INVALID (null, n < 1, grids on different devices),
 * SG_ERR_STATE (a grid without phi), SG_ERR_CAPACITY, SG_ERR_OOM. */
SG_API sg_status sg_batch_create(sg_grid *const *grids, int32_t n, void *stream, sg_batch **out);
SG_API sg_status sg_batch_destroy(sg_batch *b);

/* Restore every body's phi to its value at batch creation. */
SG_API sg_status sg_batch_reset(sg_batch *b);

/* One run: gradient of phi, smoothed sign, reinit sweeps, kernel integrals
 * over all bodies, each sweep one persistent kernel that takes work items
 * from an atomic counter.  The sequence of a plan is captured into a CUDA
 * graph on its first run and replayed afterwards.  Per body the results
 * equal those of the single-grid calls bit for bit.
 * Errors: SG_ERR_INVALID (bad plan), SG_ERR_CAPACITY (more than 1020
 * sweeps, or surrogate integrals on a store of 2^24 or more packages),
 * SG_ERR_CUDA. */
SG_API sg_status sg_batch_run(sg_batch *b, const sg_batch_plan *plan);

/* Time runs of every (pkgs_per_item, depth) pair for the plan's sweeps
 * (`reps` runs each, after one warm-up), write the fastest pair into *plan
 * and, when times_ms is not NULL, the mean time of each of the 7 candidates
 * (1,1) (2,1) (2,2) (4,1) (4,2) (8,1) (8,2) in that order.  Leaves phi reset. */
SG_API sg_status sg_batch_autotune(sg_batch *b, sg_batch_plan *plan, int32_t reps, float *times_ms);

/* The autotuner with a cache file (not in the paper; the batched launch and
 * its autotuner are this library's).  The key names the GPU (name, SM count,
 * compute capability), the plan's reinit_iterations and integrals_mode, and
 * the batch's package count rounded down to a power of two.  When the file
 * `path` has an entry for the key, its (pkgs_per_item, depth) go into *plan
 * without a run and *hit (if not NULL) is 1; otherwise the call is
 * sg_batch_autotune(b, plan, reps, NULL), whose choice is appended to the
 * file, and *hit is 0.  A missing file is an empty cache.  The file holds
 * one line "<key> <pkgs_per_item> <depth>" per tuning; the last line of a
 * key wins; lines that do not parse, or name no candidate, are ignored.
 * Appends of one short line each are safe between processes sharing the
 * file.  Errors: those of sg_batch_autotune, SG_ERR_INVALID (null, reps <
 * 1), SG_ERR_IO (the choice could not be appended; *plan holds it anyway). */
SG_API sg_status sg_batch_autotune_cached(sg_batch *b, sg_batch_plan *plan, int32_t reps, const char *path,
                                          int32_t *hit);

/* The cache key of (b, plan) as sg_batch_autotune_cached forms it, into
 * key[0 .. cap).  Errors: SG_ERR_INVALID, SG_ERR_CUDA, SG_ERR_CAPACITY (cap
 * too small). */
SG_API sg_status sg_batch_autotune_key(const sg_batch *b, const sg_batch_plan *plan, char *key, int32_t cap);

/* Host-only access to a cache file (no device needed).  lookup: *found = 1
 * and the entry's values when the file has a valid line for `key` (the last
 * one), else *found = 0 (also when the file does not exist).  store: append
 * "<key> <pkgs_per_item> <depth>"; `key` must be 1..399 characters without
 * blanks and the pair one of the seven candidates.  Errors: SG_ERR_INVALID,
 * SG_ERR_IO (store only). */
SG_API sg_status sg_autotune_cache_lookup(const char *path, const char *key, int32_t *pkgs_per_item, int32_t *depth,
                                          int32_t *found);
SG_API sg_status sg_autotune_cache_store(const char *path, const char *key, int32_t pkgs_per_item, int32_t depth);

/* Borrow body `body`'s slice of a batch field (SG_FIELD_PHI, _GX.._GZ, _W,
 * _GWX.._GWZ, _S0: [P_body][64] floats; SG_FIELD_NBR: [P_body][27] global
 * ids; SG_FIELD_CELL_PKG: [nx*ny*nz] global ids of the body's background
 * cells). */
SG_API sg_status sg_batch_get_field(sg_batch *b, int32_t body, int32_t field, void **dev_ptr, int64_t *n_elems);
SG_API int64_t sg_batch_n_packages(const sg_batch *b);
SG_API const char *sg_batch_last_error(const sg_batch *b);

struct sg_mlp; /* the surrogate network, declared with its calls below */

/* Bind the network used by plans with integrals_mode 1 (NULL unbinds).
 * The batch borrows it: it must outlive every run that uses it.  Its packed
 * weights are read at each replay, so later sg_mlp_set_params or training
 * steps take effect.  Rebinding waits for the batch's stream and drops the
 * graphs captured with the previous network. */
SG_API sg_status sg_batch_set_surrogate(sg_batch *b, const struct sg_mlp *m);

/* Particle relaxation over a batch, the application of the grid-particle
 * coupling (Sec. "Grid-Particle Coupling": the interpolated kernel integral
 * acts as a surface force on particles).  Each step probes every particle as
 * sg_probe does (trilinear phi, g, W, G of its body, n = g / |g|) and moves
 * it by
 *     x <- x - step h clip(phi / h, -1, 1) n
 * (h its body's spacing), which pulls particles onto the zero level set.
 * Particles are stored body after body; the walk is the storage order, so
 * particles sorted by Morton key per body (sg_morton_order) give local
 * gathers. */
typedef struct {
    int64_t n;              /* particles of all bodies */
    const int64_t *offsets; /* host [n_bodies + 1]: body i owns particles [offsets[i], offsets[i+1]); offsets[0] = 0,
                               offsets[n_bodies] = n, non-decreasing */
    float *x, *y, *z;       /* device [n], updated in place (caller-owned) */
    float *out[8];          /* device [n] or NULL each: phi, nx, ny, nz, W, Gx, Gy, Gz probed by the last step, before
                               its move; must not alias the positions */
    int32_t steps;          /* relaxation steps (0: positions unchanged) */
    float step;             /* displacement per step in units of h, e.g. 0.1 */
    int32_t sweeps;         /* 1: first run the plan's sweeps (as sg_batch_run); 0: probe the fields as they are */
    int32_t reserved;
} sg_relax;

/* Run [the plan's sweeps +] `steps` relaxation steps, all captured as one
 * CUDA graph on the first call with these arguments and replayed while they
 * stay the same (pointers, sizes, offsets, plan).  `plan` may be NULL when
 * sweeps = 0.  Asynchronous on the batch's stream.  Not in the paper as an
 * API (the paper states the coupling; the batched relaxation is this
 * library's).
 * Errors: SG_ERR_INVALID (null arrays, bad offsets, bad plan, steps < 0),
 * SG_ERR_CAPACITY (2^31 or more particle tiles of 256; surrogate sweeps on a
 * store of 2^24 or more packages), SG_ERR_OOM, SG_ERR_CUDA. */
SG_API sg_status sg_batch_relax(sg_batch *b, const sg_batch_plan *plan, const sg_relax *r);

/* ------------------------------------------------------------------------ */
/* Kernel-integral surrogate (not in the paper): a 27 -> 64 -> 64 -> 4       */
/* multilayer perceptron with SiLU hidden activations, BF16 weights and      */
/* activations, FP32 accumulation (tcgen05 tensor cores, accumulators in     */
/* tensor memory) and FP32 master weights.  It stands in for the kernel      */
/* integral of "Integral with SPH Smoothing Kernel and Grid-Particle         */
/* Coupling" at the points the classes below leave to it.                    */
/* ------------------------------------------------------------------------ */
typedef struct sg_mlp sg_mlp;

/* Parameter vector (FP32, host): W1[64][27], b1[64], W2[64][64], b2[64],
 * W3[4][64], b3[4] (row = output unit).  Inputs are bf16 rows of 32 values:
 * 27 inputs then 5 zeros.  The surrogate integrals feed the network the 27
 * values v = clip(sign phi(x + s h) / h, -1, 1) of a point in its canonical
 * frame: sign = -1 where phi(x) < 0; axes reversed where the central
 * difference sign (phi(x + h e_a) - phi(x - h e_a)) is negative; axes
 * ordered by decreasing |difference| (equal magnitudes keep the lower axis
 * first); input n' = (s'x+1) + 3 (s'y+1) + 9 (s'z+1) at the canonical
 * offset s'.  Outputs (W', G'x, G'y, G'z) in that frame are carried back:
 * W = W' (1 - W' where sign = -1), component k of G' belongs to the k-th
 * ordered axis, negated where that axis was reversed or sign = -1.  The
 * tap weights depend on |s| alone and H(-z) = 1 - H(z), so this is a
 * symmetry of the exact integrals; the network learns one 48th of their
 * input space. */
#define SG_MLP_NPARAM 6212
#define SG_MLP_ROW 32

/* Create a network on the current device from `params` (copied); work runs
 * on `stream`.  Errors: SG_ERR_INVALID, SG_ERR_OOM, SG_ERR_CUDA. */
SG_API sg_status sg_mlp_create(const float *params, void *stream, sg_mlp **out);
SG_API sg_status sg_mlp_destroy(sg_mlp *m);
/* Replace the parameters (copied; Adam moments and step count reset). */
SG_API sg_status sg_mlp_set_params(sg_mlp *m, const float *params);
/* Read the FP32 master parameters back (synchronises the stream).  Returns
 * SG_ERR_TIMEOUT when a tensor-core product of an earlier call on this
 * network never signalled completion (each wait is bounded; the kernel then
 * frees its tensor memory and returns). */
SG_API sg_status sg_mlp_get_params(sg_mlp *m, float *params);
/* y[n][4] = network(x[n][SG_MLP_ROW]) on the rows as given; device arrays
 * owned by the caller (16-byte aligned). */
SG_API sg_status sg_mlp_forward(sg_mlp *m, int64_t n, const void *x_bf16, float *y);
/* Gradient of L = mean over rows and the 4 outputs of (y - t)^2 with respect
 * to every parameter, written to grad[SG_MLP_NPARAM] (device, FP32); rows
 * idx[0..n) of x and t (idx NULL: rows 0..n); *loss (device, may be NULL)
 * receives L.  Uses the BF16 copy of the current parameters.  Each CTA of
 * 128 rows forms its partial gradient; the partials are summed in CTA order,
 * so the result does not depend on scheduling. */
SG_API sg_status sg_mlp_loss_grad(sg_mlp *m, int64_t n, const void *x_bf16, const float *t, const int32_t *idx,
                                  float *grad, float *loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) with
 * learning rate lr on the batch of rows idx[0..batch) (or 0..batch); the
 * gradient is formed as by sg_mlp_loss_grad, so training is reproducible. */
SG_API sg_status sg_mlp_train_step(sg_mlp *m, int64_t batch, const void *x_bf16, const float *t,
                                   const int32_t *idx, float lr, float *loss);
SG_API const char *sg_mlp_last_error(const sg_mlp *m);

/* Classes of a data point for sg_kernel_integrals mode 1, decided on the
 * real values of the grid's float phi (the same decisions as an exact
 * evaluation; the curvature test is exact up to its float-float sum):
 *   SG_SUR_TRIVIAL_IN / _OUT: every one of the 27 taps has -phi_s >= h
 *     (resp. phi_s >= h), where the smoothed Heaviside saturates: W = 1 / 0,
 *     G = 0;
 *   SG_SUR_FALLBACK: |phi| < h, or |kappa| h > 0.1 with kappa the 7-point
 *     Laplacian of phi: the exact 27-tap sum of mode 0, bit for bit;
 *   SG_SUR_NETWORK: the network on the point's canonical inputs. */
enum { SG_SUR_TRIVIAL_IN = 0, SG_SUR_TRIVIAL_OUT = 1, SG_SUR_FALLBACK = 2, SG_SUR_NETWORK = 3 };

/* Class of every data point: cls[P*64] (device, caller-owned); far packages
 * get 255.  Requires phi. */
SG_API sg_status sg_surrogate_classify(sg_grid *g, uint8_t *cls);

/* Training samples of a grid whose exact integrals (mode 0) are current:
 * every SG_SUR_NETWORK point whose SplitMix64 hash of (seed, point index)
 * falls below `keep` (a fraction in [0, 1]), in point order: x rows of
 * SG_MLP_ROW bf16 canonical inputs and t rows of the exact (W, Gx, Gy, Gz)
 * carried into the point's canonical frame.  At most cap rows are written;
 * *count receives the number of points selected (synchronises). */
SG_API sg_status sg_surrogate_samples(sg_grid *g, uint64_t seed, float keep, int64_t cap, void *x_bf16, float *t,
                                      int64_t *count);

/* Points per class (SG_SUR_* order) of the last mode-1 sg_kernel_integrals
 * call on this grid (synchronises). */
SG_API sg_status sg_surrogate_stats(sg_grid *g, int64_t counts[4]);

/* Checkpoint restore (the paper's "Data Transfer": registered variables
 * synchronised to the host for output, and back).  A checkpoint is the
 * tagging's tables and the fields, read through sg_get_field; sg_restore
 * puts the tables back into a grid created with the same description:
 * P packages (far included), cell_pkg[nx ny nz], pkg_cell[P], pkg_type[P],
 * nbr[P][27] and optionally phi[P][64], all host arrays, copied (the call
 * synchronises).  The face table is rebuilt from nbr and every table is
 * checked as sg_check_tables does; the grid is then tagged (state 1), or
 * ready for the sweeps and the probe when phi is given.  Other fields
 * (gradient, integrals) are written through sg_get_field afterwards.  The
 * grid's earlier fields are dropped.
 * Errors: SG_ERR_INVALID (P < 2, a null table, or tables that are not
 * consistent: the grid is then untagged), SG_ERR_CAPACITY, SG_ERR_OOM. */
SG_API sg_status sg_restore(sg_grid *g, int64_t P, const int32_t *cell_pkg, const int32_t *pkg_cell,
                            const uint8_t *pkg_type, const int32_t *nbr, const float *phi);

/* Allocation-free variant of sg_morton_order.  The paper has no counterpart;
 * this entry point exists for callers that cannot let a library allocate
 * device memory: applications that hand (nearly) all of the device memory to
 * their own pool at start-up, as particle codes sized to fill the GPU do, and
 * loops that cannot afford the device-wide synchronisation that cudaMalloc and
 * cudaFree may cause.  It takes the grid description instead of a grid (the
 * keys depend only on lo, h and dims), reads x, y, z and writes keys (may be
 * NULL) and order exactly as sg_morton_order does, with the same caller-owned
 * device arrays, and calls no allocator at all.
 *
 * Its scratch is one static device array of the library, sized for
 * SG_NOALLOC_MAX_PARTICLES particles (about 6 MiB); every GPU that loads the
 * library holds it until the process exits.  The first call on a device looks
 * up the array's device address with that device current, so make that first
 * call before any stream capture.  All calls share the array and the sort
 * writes every scratch byte before reading it, so no state carries over from
 * one call to the next; but calls that overlap on the GPU (different streams,
 * or threads that do not order their streams) race on the array: serialise
 * them.  Work is queued on `stream` (a cudaStream_t; NULL = legacy default).
 * The arrays must be device memory of the current device (checked with
 * cudaPointerGetAttributes: anything else is SG_ERR_INVALID before any
 * launch).
 * Errors: SG_ERR_INVALID (null pointers, n < 0, h <= 0, a dimension < 1, an
 * array not on the current device), SG_ERR_CAPACITY (n >
 * SG_NOALLOC_MAX_PARTICLES, 4*dims >= 2^21, or more than 64 devices),
 * SG_ERR_CUDA (address lookup or launch failed). */
#define SG_NOALLOC_MAX_PARTICLES 262144
SG_API sg_status sg_morton_order_noalloc(const sg_grid_desc *desc, int64_t n, const float *x, const float *y,
                                         const float *z, uint64_t *keys, int32_t *order, void *stream);

/* Borrow the device pointer and element count of a field; valid until the
 * grid is destroyed or re-tagged.  A float field not written since the last
 * tagging reads as zeros on first request (W: 1 in the inside far package). */
SG_API sg_status sg_get_field(sg_grid *g, int32_t field, void **dev_ptr, int64_t *n_elems);

/* Number of packages P (including the far packages); 0 before tagging. */
SG_API int64_t sg_n_packages(const sg_grid *g);

/* Change the stream used by later calls. */
SG_API sg_status sg_set_stream(sg_grid *g, void *stream);

/* Synchronise the grid's stream and return the sticky device error status
 * (SG_OK, SG_ERR_DEVICE or SG_ERR_TIMEOUT) or SG_ERR_CUDA.  The word stays
 * set until sg_clear_error. */
SG_API sg_status sg_status_sync(sg_grid *g);

/* Check the tables of a tagged grid on the device (asynchronous; the result
 * is the sticky word read by sg_status_sync): every package and neighbour
 * id in range, far packages their own neighbours (Sec. "Neighbourhood"),
 * each active package its own centre entry and its cell's package, every
 * neighbour entry the package of that neighbour cell (the outside far
 * package beyond the domain), the face rows copies of the neighbour rows,
 * every cell's package naming it back.  Every read is bounds-checked before
 * use, so tables edited through sg_get_field pointers can be checked before
 * a sweep reads them.  Sets SG_ERR_DEVICE on any inconsistency.
 * Errors: SG_ERR_STATE (not tagged). */
SG_API sg_status sg_check_tables(sg_grid *g);

/* Reset the sticky device error word (queued on the grid's stream). */
SG_API sg_status sg_clear_error(sg_grid *g);

/* Message of the last failed call on this grid ("" if none). */
SG_API const char *sg_last_error(const sg_grid *g);

/* Library version string. */
SG_API const char *sg_version(void);

/* Number of CUDA kernels this process has launched through the library so
 * far (all grids, all devices); for accounting launches in a timed region. */
SG_API int64_t sg_kernel_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* SG_H */
