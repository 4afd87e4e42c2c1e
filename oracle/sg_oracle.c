/*
 * sg_oracle.c -- plain FP64 CPU oracle of the sparse narrow-band level-set grid.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls this code;
 * it is loaded by the tests, by the smoke check and by the benchmark's CPU
 * baseline.  It shares no source with the CUDA library.
 *
 * Every routine is a literal loop over cells, packages or data points in
 * double precision, following the paper ("Contiguous Storage of Grid Data for
 * Heterogeneous Computing", Gu & Hu) where it defines the step, and the
 * readings listed in the design notes where it is silent:
 *
 *   storage, far packages 0/1 ............ "Array Storage and Access"
 *   package / cell / data index .......... "Indexing"
 *   27-entry neighbourhood, index shift .. "Neighbourhood", Listing 2
 *   core / inner tagging, sorting ........ "Initialization Process", steps 1-3
 *   level-set values, neighbourhood ...... "Initialization Process", steps 4-5
 *   regularised central difference ....... "Small Feature Cleaning", Listing 5
 *   kernel integral, trilinear probe ..... "Integral with SPH Smoothing Kernel
 *                                           and Grid-Particle Coupling"
 *   Godunov reinitialisation ............. not in the paper; Sussman, Smereka &
 *                                           Osher (1994) with the Godunov
 *                                           Hamiltonian of Rouy & Tourin (1992)
 *   Wendland C2 kernel ................... Wendland (1995)
 *   Morton order ......................... bit interleave of fine indices
 *
 * Package size is 4 per axis; the in-package data index is d = i + 4j + 16k.
 * Background cell index is c = I + nx (J + ny K).  Package ids 0 and 1 are the
 * far-field inside (negative) and outside (positive) packages; active packages
 * follow from id 2 in increasing cell index.
 *
 * Compile with -O2 -fopenmp -ffp-contract=off (no fused multiply-add, no
 * fast-math) so that every float and double operation is a single IEEE op.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PKG 4
#define PKG3 64

typedef struct {
    int32_t kind; /* 0 sphere, 1 plane, 2 torus, 3 prism, 4 rounded box, 5 shell */
    int32_t pad;
    double centre[3];
    double rot[9]; /* row-major, local -> world */
    double p[8];
} or_shape;

typedef struct {
    double lo[3];
    int32_t dims[3];
    int32_t id_order; /* package ids: 0 in linear cell order, 1 in Morton order of the cells */
    double h;         /* fine spacing; coarse cell lc = 4h */
    double far_value; /* F: far packages hold -F (inside) and +F (outside) */
    double support;   /* kernel support (a length; 0: 2h) */
    double eps;       /* Heaviside half width (a length; 0: h) */
} or_grid;

/* ------------------------------------------------------------------------- */
/* threads                                                                    */
/* ------------------------------------------------------------------------- */
void or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int or_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Signed distance functions (negative inside), exact for each primitive.     */
/* ------------------------------------------------------------------------- */
static void to_local(const or_shape *s, double x, double y, double z, double q[3]) {
    double d0 = x - s->centre[0], d1 = y - s->centre[1], d2 = z - s->centre[2];
    for (int i = 0; i < 3; ++i) q[i] = s->rot[0 * 3 + i] * d0 + s->rot[1 * 3 + i] * d1 + s->rot[2 * 3 + i] * d2;
}

static double clamp01(double t) { return t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t); }

/* squared distance from (px,py) to the segment a-b */
static double seg_dist2(double px, double py, double ax, double ay, double bx, double by) {
    double ex = bx - ax, ey = by - ay, wx = px - ax, wy = py - ay;
    double t = clamp01((wx * ex + wy * ey) / (ex * ex + ey * ey));
    double dx = wx - t * ex, dy = wy - t * ey;
    return dx * dx + dy * dy;
}

/* exact signed distance to a filled triangle in the plane */
static double triangle_sdf(double px, double py, const double *t) {
    double d2 = seg_dist2(px, py, t[0], t[1], t[2], t[3]);
    double e2 = seg_dist2(px, py, t[2], t[3], t[4], t[5]);
    double f2 = seg_dist2(px, py, t[4], t[5], t[0], t[1]);
    if (e2 < d2) d2 = e2;
    if (f2 < d2) d2 = f2;
    double orient = (t[2] - t[0]) * (t[5] - t[1]) - (t[3] - t[1]) * (t[4] - t[0]);
    double c0 = (t[2] - t[0]) * (py - t[1]) - (t[3] - t[1]) * (px - t[0]);
    double c1 = (t[4] - t[2]) * (py - t[3]) - (t[5] - t[3]) * (px - t[2]);
    double c2 = (t[0] - t[4]) * (py - t[5]) - (t[1] - t[5]) * (px - t[4]);
    int inside = (orient > 0.0) ? (c0 > 0.0 && c1 > 0.0 && c2 > 0.0) : (c0 < 0.0 && c1 < 0.0 && c2 < 0.0);
    return inside ? -sqrt(d2) : sqrt(d2);
}

double or_sdf(const or_shape *s, double x, double y, double z) {
    double q[3];
    to_local(s, x, y, z, q);
    switch (s->kind) {
    case 0: /* sphere */
        return sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]) - s->p[0];
    case 1: /* plane q_z = 0 */
        return q[2];
    case 2: { /* torus about local z */
        double a = sqrt(q[0] * q[0] + q[1] * q[1]) - s->p[0];
        return sqrt(a * a + q[2] * q[2]) - s->p[1];
    }
    case 3: { /* triangle extruded over [p6, p7] */
        double w0 = triangle_sdf(q[0], q[1], s->p);
        double zc = 0.5 * (s->p[6] + s->p[7]), hz = 0.5 * (s->p[7] - s->p[6]);
        double w1 = fabs(q[2] - zc) - hz;
        double in = w0 > w1 ? w0 : w1;
        if (in > 0.0) in = 0.0;
        double a = w0 > 0.0 ? w0 : 0.0, b = w1 > 0.0 ? w1 : 0.0;
        return in + sqrt(a * a + b * b);
    }
    case 4: { /* box with half extents p0..p2 rounded by p3 */
        double r = s->p[3], o = 0.0, m = -INFINITY;
        for (int i = 0; i < 3; ++i) {
            double d = fabs(q[i]) - (s->p[i] - r);
            if (d > 0.0) o += d * d;
            if (d > m) m = d;
        }
        return sqrt(o) + (m < 0.0 ? m : 0.0) - r;
    }
    case 5: { /* shell between the spheres of radii p0 < p1 */
        double r = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
        return fabs(r - 0.5 * (s->p[0] + s->p[1])) - 0.5 * (s->p[1] - s->p[0]);
    }
    default:
        return NAN;
    }
}

void or_sdf_many(const or_shape *s, int64_t n, const double *x, const double *y, const double *z, double *out) {
    for (int64_t i = 0; i < n; ++i) out[i] = or_sdf(s, x[i], y[i], z[i]);
}

/* ------------------------------------------------------------------------- */
/* Tagging and package allocation ("Initialization Process", steps 1-3, 5)    */
/* ------------------------------------------------------------------------- */
/*
 * cell_type[c]: 0 far inside, 1 far outside, 2 core, 3 inner.
 * Core: |d(cell centre)| < lc (1 - 2^-10), the strict "distance less than the
 *       cell size" test with the threshold moved off exact lattice ties.
 * Inner: not core and one of the 26 neighbouring cells is core.
 * Package ids: 2 + number of active cells with a smaller cell index, which is
 *       the "sorted by spatial location" order with cells in linear order;
 *       with id_order 1, 2 + the rank of the cell in the Morton order of the
 *       active cells (bit interleave of I, J, K, I lowest).
 * Far cells map to package 0 when d < 0 and to package 1 otherwise.
 * Returns P, the package count including the two far packages.
 * near_ties receives the number of cells with ||d| - T| < 1e-9 lc, where
 * float-float evaluation might decide differently.
 */
static int64_t tag_inner_and_ids(const or_grid *g, int32_t *cell_pkg, uint8_t *cell_type);

typedef struct {
    uint64_t key;
    int64_t cell;
} or_cellkey;

static int cmp_cellkey(const void *pa, const void *pb) {
    const or_cellkey *a = (const or_cellkey *)pa, *b = (const or_cellkey *)pb;
    return a->key < b->key ? -1 : (a->key > b->key ? 1 : 0);
}

int64_t or_tag(const or_grid *g, const or_shape *s, int32_t *cell_pkg, uint8_t *cell_type, int64_t *near_ties) {
    const int64_t nx = g->dims[0], ny = g->dims[1], nz = g->dims[2];
    const int64_t nc = nx * ny * nz;
    const double lc = 4.0 * g->h;
    const double T = lc * (1.0 - ldexp(1.0, -10));
    double *d = (double *)malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1));
    int64_t ties = 0;
#pragma omp parallel for schedule(static) reduction(+ : ties)
    for (int64_t c = 0; c < nc; ++c) {
        int64_t I = c % nx, J = (c / nx) % ny, K = c / (nx * ny);
        double x = g->lo[0] + (4.0 * (double)I + 2.0) * g->h;
        double y = g->lo[1] + (4.0 * (double)J + 2.0) * g->h;
        double z = g->lo[2] + (4.0 * (double)K + 2.0) * g->h;
        d[c] = or_sdf(s, x, y, z);
        cell_type[c] = fabs(d[c]) < T ? 2 : (d[c] < 0.0 ? 0 : 1);
        if (fabs(fabs(d[c]) - T) < 1e-9 * lc) ties++;
    }
    free(d);
    if (near_ties) *near_ties = ties;
    return tag_inner_and_ids(g, cell_pkg, cell_type);
}

/* Steps 2-3 of the tagging on classified cells: inner cells and package ids. */
static int64_t tag_inner_and_ids(const or_grid *g, int32_t *cell_pkg, uint8_t *cell_type) {
    const int64_t nx = g->dims[0], ny = g->dims[1], nz = g->dims[2];
    const int64_t nc = nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c) {
        if (cell_type[c] == 2) continue;
        int64_t I = c % nx, J = (c / nx) % ny, K = c / (nx * ny);
        int found = 0;
        for (int dk = -1; dk <= 1 && !found; ++dk)
            for (int dj = -1; dj <= 1 && !found; ++dj)
                for (int di = -1; di <= 1 && !found; ++di) {
                    int64_t a = I + di, b = J + dj, e = K + dk;
                    if (a < 0 || b < 0 || e < 0 || a >= nx || b >= ny || e >= nz) continue;
                    if (cell_type[a + nx * (b + ny * e)] == 2) found = 1;
                }
        if (found) cell_type[c] = 3;
    }
    int64_t next = 2;
    for (int64_t c = 0; c < nc; ++c) {
        if (cell_type[c] >= 2)
            cell_pkg[c] = (int32_t)next++;
        else
            cell_pkg[c] = cell_type[c]; /* 0 inside, 1 outside */
    }
    if (g->id_order == 1) {
        /* ids in the Morton order of the active cells instead: sort them by
           the bit interleave of (I, J, K), I in the lowest bit */
        const int64_t n = next - 2;
        or_cellkey *a = (or_cellkey *)malloc(sizeof(or_cellkey) * (size_t)(n > 0 ? n : 1));
        int64_t m = 0;
        for (int64_t c = 0; c < nc; ++c) {
            if (cell_pkg[c] < 2) continue;
            const uint64_t IJK[3] = {(uint64_t)(c % nx), (uint64_t)((c / nx) % ny), (uint64_t)(c / (nx * ny))};
            uint64_t key = 0;
            for (int b = 0; b < 21; ++b)
                for (int ax = 0; ax < 3; ++ax) key |= ((IJK[ax] >> b) & 1ull) << (3 * b + ax);
            a[m].key = key;
            a[m].cell = c;
            ++m;
        }
        qsort(a, (size_t)n, sizeof(or_cellkey), cmp_cellkey);
        for (int64_t r = 0; r < n; ++r) cell_pkg[a[r].cell] = (int32_t)(2 + r);
        free(a);
    }
    return next;
}

/*
 * Tagging of a finer layer from its coarser one ("Multi-resolution
 * Level-set", step 1 of "Initialization Process": for successive layers only
 * the cells covered by the coarse core cells are evaluated).  The coarse
 * layer gc has the same lo, half the dims and twice the spacing.  A fine
 * cell inside a coarse core cell is classified by its own distance as in
 * or_tag; any other fine cell is far, inside when its coarse cell is far
 * inside or is an inner cell whose level set (data point 0) is negative.
 * evaluated receives the number of distance evaluations.
 */
int64_t or_tag_from(const or_grid *g, const or_shape *s, const or_grid *gc, const int32_t *c_cell_pkg,
                    const uint8_t *c_pkg_type, const double *c_phi, int32_t *cell_pkg, uint8_t *cell_type,
                    int64_t *near_ties, int64_t *evaluated) {
    const int64_t nx = g->dims[0], ny = g->dims[1], nz = g->dims[2];
    const int64_t nc = nx * ny * nz, cnx = gc->dims[0], cny = gc->dims[1];
    const double lc = 4.0 * g->h;
    const double T = lc * (1.0 - ldexp(1.0, -10));
    int64_t ties = 0, evals = 0;
#pragma omp parallel for schedule(static) reduction(+ : ties, evals)
    for (int64_t c = 0; c < nc; ++c) {
        int64_t I = c % nx, J = (c / nx) % ny, K = c / (nx * ny);
        const int64_t pc = c_cell_pkg[(I / 2) + cnx * ((J / 2) + cny * (K / 2))];
        if (pc >= 2 && c_pkg_type[pc] == 2) {
            double x = g->lo[0] + (4.0 * (double)I + 2.0) * g->h;
            double y = g->lo[1] + (4.0 * (double)J + 2.0) * g->h;
            double z = g->lo[2] + (4.0 * (double)K + 2.0) * g->h;
            const double d = or_sdf(s, x, y, z);
            cell_type[c] = fabs(d) < T ? 2 : (d < 0.0 ? 0 : 1);
            if (fabs(fabs(d) - T) < 1e-9 * lc) ties++;
            evals++;
        } else {
            const int inside = pc < 2 ? pc == 0 : c_phi[pc * PKG3] < 0.0;
            cell_type[c] = inside ? 0 : 1;
        }
    }
    if (near_ties) *near_ties = ties;
    if (evaluated) *evaluated = evals;
    return tag_inner_and_ids(g, cell_pkg, cell_type);
}

/*
 * Per-package meta data and neighbourhood ("Initialization Process", step 5;
 * "Neighbourhood"): nbr[p][n] with n = (di+1) + 3(dj+1) + 9(dk+1) is the
 * package of cell (I+di, J+dj, K+dk); cells outside the domain map to the
 * outside far package 1.  The far packages are their own neighbours.
 * pkg_cell of the far packages is -1.
 */
void or_tables(const or_grid *g, const int32_t *cell_pkg, const uint8_t *cell_type, int64_t P, int32_t *pkg_cell,
               uint8_t *pkg_type, int32_t *nbr) {
    const int64_t nx = g->dims[0], ny = g->dims[1], nz = g->dims[2];
    const int64_t nc = nx * ny * nz;
    for (int f = 0; f < 2; ++f) {
        pkg_cell[f] = -1;
        pkg_type[f] = (uint8_t)f;
        for (int n = 0; n < 27; ++n) nbr[f * 27 + n] = f;
    }
    for (int64_t c = 0; c < nc; ++c) {
        int32_t p = cell_pkg[c];
        if (p < 2) continue;
        pkg_cell[p] = (int32_t)c;
        pkg_type[p] = cell_type[c];
    }
#pragma omp parallel for schedule(static)
    for (int64_t p = 2; p < P; ++p) {
        int64_t c = pkg_cell[p];
        int64_t I = c % nx, J = (c / nx) % ny, K = c / (nx * ny);
        for (int dk = -1; dk <= 1; ++dk)
            for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di) {
                    int64_t a = I + di, b = J + dj, e = K + dk;
                    int n = (di + 1) + 3 * (dj + 1) + 9 * (dk + 1);
                    if (a < 0 || b < 0 || e < 0 || a >= nx || b >= ny || e >= nz)
                        nbr[p * 27 + n] = 1;
                    else
                        nbr[p * 27 + n] = cell_pkg[a + nx * (b + ny * e)];
                }
    }
}

/* ------------------------------------------------------------------------- */
/* Index shift (Listing 2): a shift s per axis in [-4, 7] relative to the     */
/* package origin selects neighbour n = (s + 4) / 4 and data s + 4 - 4n.      */
/* Returns the flat index package * 64 + data index.                          */
/* ------------------------------------------------------------------------- */
static inline int64_t shift_index(const int32_t *nb, int sx, int sy, int sz) {
    int nx = (sx + PKG) / PKG, ny = (sy + PKG) / PKG, nz = (sz + PKG) / PKG;
    int64_t pkg = nb[nx + 3 * ny + 9 * nz];
    int dx = sx + PKG - nx * PKG, dy = sy + PKG - ny * PKG, dz = sz + PKG - nz * PKG;
    return pkg * PKG3 + dx + PKG * dy + PKG * PKG * dz;
}

/* ------------------------------------------------------------------------- */
/* Level-set values ("Initialization Process", step 4), cell-centred data:   */
/* x = lo + (4 I + i + 0.5) h.  Far packages hold -F and +F.                  */
/* ------------------------------------------------------------------------- */
void or_init_sdf(const or_grid *g, const or_shape *s, int64_t P, const int32_t *pkg_cell, double *phi) {
    const int64_t nx = g->dims[0], ny = g->dims[1];
    for (int d = 0; d < PKG3; ++d) {
        phi[d] = -g->far_value;
        phi[PKG3 + d] = g->far_value;
    }
#pragma omp parallel for schedule(static)
    for (int64_t p = 2; p < P; ++p) {
        int64_t c = pkg_cell[p];
        int64_t I = c % nx, J = (c / nx) % ny, K = c / (nx * ny);
        for (int k = 0; k < PKG; ++k)
            for (int j = 0; j < PKG; ++j)
                for (int i = 0; i < PKG; ++i) {
                    double x = g->lo[0] + ((double)(4 * I + i) + 0.5) * g->h;
                    double y = g->lo[1] + ((double)(4 * J + j) + 0.5) * g->h;
                    double z = g->lo[2] + ((double)(4 * K + k) + 0.5) * g->h;
                    phi[p * PKG3 + i + PKG * j + PKG * PKG * k] = or_sdf(s, x, y, z);
                }
    }
}

/* ------------------------------------------------------------------------- */
/* Regularised central difference (Listing 5), three axes, divided by h:      */
/* p = phi(+e) - phi(0), m = phi(0) - phi(-e), grad = (p + m) / (2h).         */
/* Far packages keep a zero gradient.                                         */
/* ------------------------------------------------------------------------- */
void or_gradient(const or_grid *g, int64_t P, const int32_t *nbr, const double *phi, double *gx, double *gy,
                 double *gz) {
    double *out[3] = {gx, gy, gz};
    for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 2 * PKG3; ++d) out[a][d] = 0.0;
    const double inv2h = 1.0 / (2.0 * g->h);
#pragma omp parallel for schedule(static)
    for (int64_t p = 2; p < P; ++p) {
        const int32_t *nb = nbr + p * 27;
        for (int k = 0; k < PKG; ++k)
            for (int j = 0; j < PKG; ++j)
                for (int i = 0; i < PKG; ++i) {
                    double c = phi[shift_index(nb, i, j, k)];
                    for (int a = 0; a < 3; ++a) {
                        int ex = a == 0, ey = a == 1, ez = a == 2;
                        double pl = phi[shift_index(nb, i + ex, j + ey, k + ez)] - c;
                        double mi = c - phi[shift_index(nb, i - ex, j - ey, k - ez)];
                        out[a][p * PKG3 + i + PKG * j + PKG * PKG * k] = (pl + mi) * inv2h;
                    }
                }
    }
}

/* "Sequential" access of the paper's benchmark: phi <- phi + delta on every  */
/* active value, in float as the device stores it.                            */
void or_sequential(int64_t P, float *phi, float delta) {
    for (int64_t i = 2 * PKG3; i < P * PKG3; ++i) phi[i] = phi[i] + delta;
}

/* 7-point Laplacian: sum over axes of (phi(+e) - 2 phi(0) + phi(-e)) / h^2.  */
void or_laplacian(const or_grid *g, int64_t P, const int32_t *nbr, const double *phi, double *lap) {
    for (int d = 0; d < 2 * PKG3; ++d) lap[d] = 0.0;
    const double inv_h2 = 1.0 / (g->h * g->h);
#pragma omp parallel for schedule(static)
    for (int64_t p = 2; p < P; ++p) {
        const int32_t *nb = nbr + p * 27;
        for (int k = 0; k < PKG; ++k)
            for (int j = 0; j < PKG; ++j)
                for (int i = 0; i < PKG; ++i) {
                    double c = phi[shift_index(nb, i, j, k)];
                    double s = 0.0;
                    for (int a = 0; a < 3; ++a) {
                        int ex = a == 0, ey = a == 1, ez = a == 2;
                        s += phi[shift_index(nb, i + ex, j + ey, k + ez)] - 2.0 * c +
                             phi[shift_index(nb, i - ex, j - ey, k - ez)];
                    }
                    lap[p * PKG3 + i + PKG * j + PKG * PKG * k] = s * inv_h2;
                }
    }
}

/* ------------------------------------------------------------------------- */
/* Reinitialisation (Sussman, Smereka & Osher 1994; Godunov Hamiltonian).     */
/*   S0 = phi0 / sqrt(phi0^2 + h^2) from phi0 = phi at entry,                 */
/*   a = D^- phi, b = D^+ phi per axis,                                       */
/*   phi0 > 0: G = sum max(max(a,0)^2, min(b,0)^2)                            */
/*   phi0 < 0: G = sum max(min(a,0)^2, max(b,0)^2)                            */
/*   phi_new = phi - dt S0 (sqrt(G) - 1), dt = cfl h; phi0 = 0: unchanged.    */
/* Jacobi sweeps; far packages are never changed.                             */
/* ------------------------------------------------------------------------- */
void or_reinit_s0(const or_grid *g, int64_t P, const double *phi0, double *s0) {
    const double h2 = g->h * g->h;
    for (int64_t i = 0; i < P * PKG3; ++i) s0[i] = phi0[i] / sqrt(phi0[i] * phi0[i] + h2);
}

void or_reinit_step(const or_grid *g, int64_t P, const int32_t *nbr, const double *phi0, const double *s0,
                    const double *phi_in, double *phi_out, double dt) {
    const double inv_h = 1.0 / g->h;
    for (int d = 0; d < 2 * PKG3; ++d) phi_out[d] = phi_in[d];
#pragma omp parallel for schedule(static)
    for (int64_t p = 2; p < P; ++p) {
        const int32_t *nb = nbr + p * 27;
        for (int k = 0; k < PKG; ++k)
            for (int j = 0; j < PKG; ++j)
                for (int i = 0; i < PKG; ++i) {
                    int64_t at = p * PKG3 + i + PKG * j + PKG * PKG * k;
                    double c = phi_in[at];
                    double G = 0.0;
                    for (int ax = 0; ax < 3; ++ax) {
                        int ex = ax == 0, ey = ax == 1, ez = ax == 2;
                        double a = (c - phi_in[shift_index(nb, i - ex, j - ey, k - ez)]) * inv_h;
                        double b = (phi_in[shift_index(nb, i + ex, j + ey, k + ez)] - c) * inv_h;
                        double u, v;
                        if (phi0[at] > 0.0) {
                            u = a > 0.0 ? a : 0.0;
                            v = b < 0.0 ? b : 0.0;
                        } else {
                            u = a < 0.0 ? a : 0.0;
                            v = b > 0.0 ? b : 0.0;
                        }
                        G += (u * u > v * v) ? u * u : v * v;
                    }
                    if (phi0[at] == 0.0)
                        phi_out[at] = c;
                    else
                        phi_out[at] = c - dt * s0[at] * (sqrt(G) - 1.0);
                }
    }
}

void or_reinit(const or_grid *g, int64_t P, const int32_t *nbr, double *phi, int32_t iterations, double cfl) {
    size_t n = (size_t)(P * PKG3);
    double *phi0 = (double *)malloc(n * sizeof(double));
    double *s0 = (double *)malloc(n * sizeof(double));
    double *tmp = (double *)malloc(n * sizeof(double));
    memcpy(phi0, phi, n * sizeof(double));
    or_reinit_s0(g, P, phi0, s0);
    double *a = phi, *b = tmp;
    for (int32_t it = 0; it < iterations; ++it) {
        or_reinit_step(g, P, nbr, phi0, s0, a, b, cfl * g->h);
        double *t = a;
        a = b;
        b = t;
    }
    if (a != phi) memcpy(phi, a, n * sizeof(double));
    free(phi0);
    free(s0);
    free(tmp);
}

/* ------------------------------------------------------------------------- */
/* Kernel integrals ("Integral with SPH Smoothing Kernel"):                   */
/*   Wendland C2, support 2h:  w(q) = (1 - q/2)^4 (1 + 2q) for q < 2, else 0  */
/*                             w'(q) = -5 q (1 - q/2)^3                       */
/*   smoothed Heaviside, eps = h: H(z) = 0 (z < -eps), 1 (z > eps),           */
/*                             1/2 (1 + z/eps + sin(pi z / eps) / pi) between */
/*   W  = sum_s w(|s|) H(-phi(x + s h)) / sum_s w(|s|)                        */
/*   G^ = h grad W = sum_s w'(|s|) (-s/|s|) H(-phi(x + s h)) / sum_s w(|s|)   */
/* summed over all 125 offsets s in {-2..2}^3 (taps at |s| >= 2 weigh 0).     */
/* Far packages: W = 1 inside, 0 outside; G^ = 0.                             */
/* ------------------------------------------------------------------------- */
/* Wendland C2 of support R (in units of h): (1 - q/R)^4 (1 + 4 q/R) for
   q < R, else 0, and its derivative -20 (q / R^2) (1 - q/R)^3. */
double or_wendland_r(double q, double R) {
    if (q >= R) return 0.0;
    double t = 1.0 - q / R;
    return t * t * t * t * (1.0 + 4.0 * q / R);
}
double or_wendland_r_dq(double q, double R) {
    if (q >= R) return 0.0;
    double t = 1.0 - q / R;
    return -20.0 * q / (R * R) * t * t * t;
}
double or_wendland(double q) {
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return t * t * t * t * (1.0 + 2.0 * q);
}

double or_wendland_dq(double q) {
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return -5.0 * q * t * t * t;
}

double or_heaviside(double z, double eps) {
    if (z < -eps) return 0.0;
    if (z > eps) return 1.0;
    return 0.5 * (1.0 + z / eps + sin(M_PI * z / eps) / M_PI);
}

void or_kernel_integrals(const or_grid *g, int64_t P, const int32_t *nbr, const double *phi, double *W, double *Gx,
                         double *Gy, double *Gz) {
    /* support R h (R <= 3, so that every tap lies in the 5^3 stencil) and Heaviside half width eps */
    const double R = g->support > 0.0 ? g->support / g->h : 2.0;
    const double eps = g->eps > 0.0 ? g->eps : g->h;
    for (int d = 0; d < PKG3; ++d) {
        W[d] = 1.0;
        W[PKG3 + d] = 0.0;
        Gx[d] = Gy[d] = Gz[d] = 0.0;
        Gx[PKG3 + d] = Gy[PKG3 + d] = Gz[PKG3 + d] = 0.0;
    }
#pragma omp parallel for schedule(static)
    for (int64_t p = 2; p < P; ++p) {
        const int32_t *nb = nbr + p * 27;
        for (int k = 0; k < PKG; ++k)
            for (int j = 0; j < PKG; ++j)
                for (int i = 0; i < PKG; ++i) {
                    double num = 0.0, den = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
                    for (int sz = -2; sz <= 2; ++sz)
                        for (int sy = -2; sy <= 2; ++sy)
                            for (int sx = -2; sx <= 2; ++sx) {
                                double q = sqrt((double)(sx * sx + sy * sy + sz * sz));
                                double w = or_wendland_r(q, R);
                                double H = or_heaviside(-phi[shift_index(nb, i + sx, j + sy, k + sz)], eps);
                                num += w * H;
                                den += w;
                                if (q > 0.0) {
                                    double dw = or_wendland_r_dq(q, R) * H / q;
                                    gx += dw * (double)(-sx);
                                    gy += dw * (double)(-sy);
                                    gz += dw * (double)(-sz);
                                }
                            }
                    int64_t at = p * PKG3 + i + PKG * j + PKG * PKG * k;
                    W[at] = num / den;
                    Gx[at] = gx / den;
                    Gy[at] = gy / den;
                    Gz[at] = gz / den;
                }
    }
}

/* ------------------------------------------------------------------------- */
/* Particle probe ("Grid-Particle Coupling"): trilinear interpolation.        */
/* The fine lattice coordinate of a float32 position x is the plain           */
/* definition in double precision: u = (x - lo) / h - 1/2, i0 = floor(u),     */
/* t = u - i0 (u clamped to +-2^40 so that far-away particles stay           */
/* representable).  Home cell I = floor(i0 / 4), local l0 = i0 - 4I.  Corners */
/* l0 + {0,1} are reached from the home package by the index shift; a home    */
/* cell outside the domain is the outside far package.                        */
/* Outputs (in input order): phi, normal n = g/|g| (0 when |g| = 0), W, G^.   */
/* ------------------------------------------------------------------------- */
static double lattice_u(const or_grid *g, int a, float x) {
    double u = ((double)x - g->lo[a]) / g->h - 0.5;
    const double lim = 1099511627776.0; /* 2^40 */
    if (u < -lim) u = -lim;
    if (u > lim) u = lim;
    return u;
}

static void lattice(const or_grid *g, int a, float x, int64_t *i0, double *t) {
    const double u = lattice_u(g, a, x);
    const double f = floor(u);
    *i0 = (int64_t)f;
    *t = u - f;
}

/* Particles with some lattice coordinate u within tol of an integer: their  */
/* cell decision rests on the last bits of the arithmetic (the counterpart of */
/* the tagging threshold test).  mask (optional) receives bit a set where     */
/* axis a is tied; returns the number of particles with any tied axis.        */
int64_t or_lattice_ties(const or_grid *g, int64_t n, const float *x, const float *y, const float *z, double tol,
                        uint8_t *mask) {
    int64_t ties = 0;
#pragma omp parallel for schedule(static) reduction(+ : ties)
    for (int64_t q = 0; q < n; ++q) {
        const float p[3] = {x[q], y[q], z[q]};
        uint8_t tie = 0;
        for (int a = 0; a < 3; ++a) {
            const double u = lattice_u(g, a, p[a]);
            if (fabs(u - nearbyint(u)) < tol) tie |= (uint8_t)(1u << a);
        }
        if (mask) mask[q] = tie;
        ties += tie != 0;
    }
    return ties;
}

void or_probe(const or_grid *g, const int32_t *cell_pkg, const int32_t *nbr, const double *const fields[8], int64_t n,
              const float *x, const float *y, const float *z, double *const out[8]) {
    /* fields: phi, gx, gy, gz, W, Gx, Gy, Gz (package-major, 64 per package)
       out:    phi, nx, ny, nz, W, Gx, Gy, Gz */
    const int64_t nx = g->dims[0], ny = g->dims[1], nz = g->dims[2];
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) {
        int64_t i0[3];
        double t[3];
        lattice(g, 0, x[q], &i0[0], &t[0]);
        lattice(g, 1, y[q], &i0[1], &t[1]);
        lattice(g, 2, z[q], &i0[2], &t[2]);
        int64_t I[3];
        int l0[3];
        for (int a = 0; a < 3; ++a) {
            I[a] = i0[a] >= 0 ? i0[a] / 4 : -((-i0[a] + 3) / 4);
            l0[a] = (int)(i0[a] - 4 * I[a]);
        }
        int64_t home = 1;
        if (I[0] >= 0 && I[1] >= 0 && I[2] >= 0 && I[0] < nx && I[1] < ny && I[2] < nz)
            home = cell_pkg[I[0] + nx * (I[1] + ny * I[2])];
        const int32_t *nb = nbr + home * 27;
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int c = 0; c < 8; ++c) {
            int a0 = c & 1, a1 = (c >> 1) & 1, a2 = (c >> 2) & 1;
            double w = (a0 ? t[0] : 1.0 - t[0]) * (a1 ? t[1] : 1.0 - t[1]) * (a2 ? t[2] : 1.0 - t[2]);
            int64_t at = shift_index(nb, l0[0] + a0, l0[1] + a1, l0[2] + a2);
            for (int f = 0; f < 8; ++f) acc[f] += w * fields[f][at];
        }
        double gn = sqrt(acc[1] * acc[1] + acc[2] * acc[2] + acc[3] * acc[3]);
        out[0][q] = acc[0];
        for (int a = 0; a < 3; ++a) out[1 + a][q] = gn > 0.0 ? acc[1 + a] / gn : 0.0;
        for (int f = 4; f < 8; ++f) out[f][q] = acc[f];
    }
}

/* ------------------------------------------------------------------------- */
/* Consistency (sign) correction ("Consistency Correction"): the sign of phi  */
/* is trusted only at data points with |phi| < tau, close to the surface,     */
/* and carried from there to the rest of the domain by two diffusion steps,  */
/* one over the data points of the packages and one over the background      */
/* cells.  Each is a Jacobi flood over face neighbours: an unknown entry      */
/* takes the sign of the sum of its labelled neighbours' signs, until nothing */
/* changes.                                                                   */
/*  - points: the trusted points start with their sign; the flood runs over  */
/*    active packages only; then phi <- sign * |phi| where a sign is known;   */
/*  - cells: core cells (the surface passes through them) are blocked; an    */
/*    inner cell starts with the sign its package's points share; far cells  */
/*    take their flooded label (package 0 inside, 1 outside) and the         */
/*    neighbour table follows.                                               */
/* The point step runs first: every point within h of the surface lies in a  */
/* core cell, so the cells have no trusted sign until the points have one.   */
/* changed[0] counts points whose sign flipped, changed[1] far cells moved, */
/* changed[2] and changed[3] the point and cell sweeps, each up to and       */
/* including the first sweep that labels nothing.                            */
/* ------------------------------------------------------------------------- */
#define CC_BLOCK 2
static int face_step(const or_grid *g, int64_t c, int f, int64_t *out) {
    const int64_t nx = g->dims[0], ny = g->dims[1], nz = g->dims[2];
    int64_t I = c % nx, J = (c / nx) % ny, K = c / (nx * ny);
    int a = f >> 1, d = (f & 1) ? 1 : -1;
    if (a == 0) I += d;
    if (a == 1) J += d;
    if (a == 2) K += d;
    if (I < 0 || J < 0 || K < 0 || I >= nx || J >= ny || K >= nz) return 0;
    *out = I + nx * (J + ny * K);
    return 1;
}

void or_consistency_correct(const or_grid *g, int64_t P, int32_t *cell_pkg, const int32_t *pkg_cell,
                            const uint8_t *pkg_type, int32_t *nbr, double *phi, double tau, int64_t changed[4]) {
    const int64_t nx = g->dims[0], ny = g->dims[1], nz = g->dims[2], nc = nx * ny * nz;
    changed[0] = changed[1] = changed[2] = changed[3] = 0;
    /* points: trusted seeds */
    const int64_t np = P * PKG3;
    int8_t *sg = (int8_t *)calloc((size_t)np, 1), *sn = (int8_t *)calloc((size_t)np, 1);
    for (int64_t q = 2 * PKG3; q < np; ++q) {
        const double v = phi[q];
        if (fabs(v) < tau) sg[q] = v > 0.0 ? 1 : (v < 0.0 ? -1 : 0);
    }
    /* points: flood over the face neighbours inside active packages */
    for (;;) {
        int64_t moved = 0;
        ++changed[2];
        memcpy(sn, sg, (size_t)np);
        for (int64_t p = 2; p < P; ++p) {
            const int32_t *nb = nbr + p * 27;
            for (int e = 0; e < PKG3; ++e) {
                if (sg[p * PKG3 + e]) continue;
                const int i = e % 4, j = (e / 4) % 4, k = e / 16;
                int sum = 0;
                for (int f = 0; f < 6; ++f) {
                    const int a = f >> 1, d = (f & 1) ? 1 : -1;
                    const int64_t at = shift_index(nb, i + (a == 0) * d, j + (a == 1) * d, k + (a == 2) * d);
                    if (at / PKG3 >= 2) sum += sg[at];
                }
                if (sum != 0) {
                    sn[p * PKG3 + e] = sum > 0 ? 1 : -1;
                    ++moved;
                }
            }
        }
        int8_t *t = sg;
        sg = sn;
        sn = t;
        if (!moved) break;
    }
    for (int64_t q = 2 * PKG3; q < np; ++q) {
        const double v = phi[q];
        if ((sg[q] > 0 && v < 0.0) || (sg[q] < 0 && v > 0.0)) {
            phi[q] = -v;
            ++changed[0];
        }
    }
    /* cells: seeds from the inner packages' point signs */
    int8_t *lab = (int8_t *)calloc((size_t)nc, 1), *nxt = (int8_t *)calloc((size_t)nc, 1);
    for (int64_t c = 0; c < nc; ++c) {
        const int64_t p = cell_pkg[c];
        if (p < 2) continue;
        if (pkg_type[p] == 2) {
            lab[c] = CC_BLOCK;
            continue;
        }
        int pos = 0, neg = 0;
        for (int e = 0; e < PKG3; ++e) {
            pos |= sg[p * PKG3 + e] > 0;
            neg |= sg[p * PKG3 + e] < 0;
        }
        lab[c] = (pos && neg) ? CC_BLOCK : (pos ? 1 : (neg ? -1 : 0));
    }
    /* cells: flood */
    for (;;) {
        int64_t moved = 0;
        ++changed[3];
        memcpy(nxt, lab, (size_t)nc);
        for (int64_t c = 0; c < nc; ++c) {
            if (lab[c] != 0) continue;
            int sum = 0;
            for (int f = 0; f < 6; ++f) {
                int64_t o;
                if (face_step(g, c, f, &o) && (lab[o] == 1 || lab[o] == -1)) sum += lab[o];
            }
            if (sum != 0) {
                nxt[c] = sum > 0 ? 1 : -1;
                ++moved;
            }
        }
        int8_t *t = lab;
        lab = nxt;
        nxt = t;
        if (!moved) break;
    }
    /* far cells follow their label; neighbour entries naming far packages follow the cells */
    for (int64_t c = 0; c < nc; ++c) {
        if (cell_pkg[c] >= 2 || (lab[c] != 1 && lab[c] != -1)) continue;
        const int32_t want = lab[c] < 0 ? 0 : 1;
        if (cell_pkg[c] != want) {
            cell_pkg[c] = want;
            ++changed[1];
        }
    }
    for (int64_t p = 2; p < P; ++p) {
        const int64_t c = pkg_cell[p];
        const int64_t I = c % nx, J = (c / nx) % ny, K = c / (nx * ny);
        for (int n = 0; n < 27; ++n) {
            const int64_t i = I + n % 3 - 1, j = J + (n / 3) % 3 - 1, k = K + n / 9 - 1;
            if (nbr[p * 27 + n] >= 2 || i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) continue;
            nbr[p * 27 + n] = cell_pkg[i + nx * (j + ny * k)];
        }
    }
    free(lab);
    free(nxt);
    free(sg);
    free(sn);
}

/* ------------------------------------------------------------------------- */
/* Particle relaxation: the coupling of Sec. "Grid-Particle Coupling" used as */
/* a surface force.  Each step probes every particle (or_probe above) and     */
/* then moves it by -step h clip(phi/h, -1, 1) n, the position being stored   */
/* in float32 after each step.  out holds the probe of the last step.         */
/* ------------------------------------------------------------------------- */
void or_relax(const or_grid *g, const int32_t *cell_pkg, const int32_t *nbr, const double *const fields[8], int64_t n,
              float *x, float *y, float *z, int32_t steps, double step, double *const out[8]) {
    const double h = g->h;
    for (int32_t k = 0; k < steps; ++k) {
        or_probe(g, cell_pkg, nbr, fields, n, x, y, z, out);
#pragma omp parallel for schedule(static)
        for (int64_t q = 0; q < n; ++q) {
            double s = out[0][q] / h;
            if (s < -1.0) s = -1.0;
            if (s > 1.0) s = 1.0;
            const double m = step * h * s;
            x[q] = (float)((double)x[q] - m * out[1][q]);
            y[q] = (float)((double)y[q] - m * out[2][q]);
            z[q] = (float)((double)z[q] - m * out[3][q]);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Morton order of particles: key = interleave of k_a = clamp(i0_a + 1, 0,    */
/* 4 dims_a + 1) (at most 21 bits per axis), x in the lowest bit; order =     */
/* stable sort by (key, input index).                                         */
/* ------------------------------------------------------------------------- */
void or_morton_keys(const or_grid *g, int64_t n, const float *x, const float *y, const float *z, uint64_t *keys) {
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) {
        const float *src[3] = {x, y, z};
        uint64_t k[3];
        for (int a = 0; a < 3; ++a) {
            int64_t i0;
            double t;
            lattice(g, a, src[a][q], &i0, &t);
            int64_t v = i0 + 1, vmax = 4 * (int64_t)g->dims[a] + 1;
            if (v < 0) v = 0;
            if (v > vmax) v = vmax;
            k[a] = (uint64_t)v;
        }
        uint64_t key = 0;
        for (int b = 0; b < 21; ++b)
            for (int a = 0; a < 3; ++a) key |= ((k[a] >> b) & 1ull) << (3 * b + a);
        keys[q] = key;
    }
}

typedef struct {
    uint64_t key;
    int64_t idx;
} or_kv;

static int kv_cmp(const void *pa, const void *pb) {
    const or_kv *a = (const or_kv *)pa, *b = (const or_kv *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

void or_morton_order(int64_t n, const uint64_t *keys, int64_t *order) {
    or_kv *kv = (or_kv *)malloc(sizeof(or_kv) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        kv[i].key = keys[i];
        kv[i].idx = i;
    }
    qsort(kv, (size_t)n, sizeof(or_kv), kv_cmp);
    for (int64_t i = 0; i < n; ++i) order[i] = kv[i].idx;
    free(kv);
}

/* ------------------------------------------------------------------------- */
/* Kernel-integral surrogate: a 27 -> 64 -> 64 -> 4 multilayer perceptron     */
/* with SiLU hidden activations (not in the paper; the learned stand-in for   */
/* the kernel integral).  Inputs: v_n = clip(phi(x + s h) / h, -1, 1) for the */
/* 27 offsets s in {-1,0,1}^3, n = (sx+1) + 3 (sy+1) + 9 (sz+1).  Outputs:   */
/* (W, Gx, Gy, Gz).  Parameters, one flat vector:                            */
/*   W1[64][27], b1[64], W2[64][64], b2[64], W3[4][64], b3[4]  (6212 values) */
/* Loss: mean over the batch and the 4 outputs of (y - t)^2.                 */
/* Adam (Kingma & Ba 2015) with bias correction.                             */
/* ------------------------------------------------------------------------- */
#define MLP_IN 27
#define MLP_H 64
#define MLP_OUT 4
#define MLP_NPARAM (MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_OUT * MLP_H + MLP_OUT)

int64_t or_mlp_nparam(void) { return MLP_NPARAM; }

static double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

/* Forward pass of n samples; y[n][4].  Hidden pre-activations are returned
 * when z1, z2 ([n][64]) are not NULL. */
void or_mlp_forward(const double *par, int64_t n, const double *x, double *y, double *z1, double *z2) {
    const double *W1 = par, *b1 = W1 + MLP_H * MLP_IN, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H;
    const double *W3 = b2 + MLP_H, *b3 = W3 + MLP_OUT * MLP_H;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < n; ++s) {
        double a1[MLP_H], a2[MLP_H];
        for (int o = 0; o < MLP_H; ++o) {
            double z = b1[o];
            for (int i = 0; i < MLP_IN; ++i) z += W1[o * MLP_IN + i] * x[s * MLP_IN + i];
            if (z1) z1[s * MLP_H + o] = z;
            a1[o] = z * sigmoid(z);
        }
        for (int o = 0; o < MLP_H; ++o) {
            double z = b2[o];
            for (int i = 0; i < MLP_H; ++i) z += W2[o * MLP_H + i] * a1[i];
            if (z2) z2[s * MLP_H + o] = z;
            a2[o] = z * sigmoid(z);
        }
        for (int o = 0; o < MLP_OUT; ++o) {
            double z = b3[o];
            for (int i = 0; i < MLP_H; ++i) z += W3[o * MLP_H + i] * a2[i];
            y[s * MLP_OUT + o] = z;
        }
    }
}

/* Loss and its gradient with respect to every parameter (grad[6212]). */
double or_mlp_loss_grad(const double *par, int64_t n, const double *x, const double *t, double *grad) {
    const double *W2 = par + MLP_H * MLP_IN + MLP_H, *W3 = W2 + MLP_H * MLP_H + MLP_H;
    double *z1 = (double *)malloc(sizeof(double) * (size_t)(n * MLP_H));
    double *z2 = (double *)malloc(sizeof(double) * (size_t)(n * MLP_H));
    double *y = (double *)malloc(sizeof(double) * (size_t)(n * MLP_OUT));
    or_mlp_forward(par, n, x, y, z1, z2);
    for (int64_t k = 0; k < MLP_NPARAM; ++k) grad[k] = 0.0;
    double *gW1 = grad, *gb1 = gW1 + MLP_H * MLP_IN, *gW2 = gb1 + MLP_H, *gb2 = gW2 + MLP_H * MLP_H;
    double *gW3 = gb2 + MLP_H, *gb3 = gW3 + MLP_OUT * MLP_H;
    double loss = 0.0;
    const double scale = 1.0 / (double)(n * MLP_OUT);
    for (int64_t s = 0; s < n; ++s) {
        double a1[MLP_H], a2[MLP_H], dy[MLP_OUT], dz2[MLP_H], dz1[MLP_H];
        for (int o = 0; o < MLP_H; ++o) a1[o] = z1[s * MLP_H + o] * sigmoid(z1[s * MLP_H + o]);
        for (int o = 0; o < MLP_H; ++o) a2[o] = z2[s * MLP_H + o] * sigmoid(z2[s * MLP_H + o]);
        for (int o = 0; o < MLP_OUT; ++o) {
            double e = y[s * MLP_OUT + o] - t[s * MLP_OUT + o];
            loss += e * e * scale;
            dy[o] = 2.0 * e * scale;
            gb3[o] += dy[o];
            for (int i = 0; i < MLP_H; ++i) gW3[o * MLP_H + i] += dy[o] * a2[i];
        }
        for (int i = 0; i < MLP_H; ++i) {
            double d = 0.0;
            for (int o = 0; o < MLP_OUT; ++o) d += dy[o] * W3[o * MLP_H + i];
            double z = z2[s * MLP_H + i], sg = sigmoid(z);
            dz2[i] = d * sg * (1.0 + z * (1.0 - sg)); /* SiLU'(z) */
            gb2[i] += dz2[i];
            for (int j = 0; j < MLP_H; ++j) gW2[i * MLP_H + j] += dz2[i] * a1[j];
        }
        for (int j = 0; j < MLP_H; ++j) {
            double d = 0.0;
            for (int i = 0; i < MLP_H; ++i) d += dz2[i] * W2[i * MLP_H + j];
            double z = z1[s * MLP_H + j], sg = sigmoid(z);
            dz1[j] = d * sg * (1.0 + z * (1.0 - sg));
            gb1[j] += dz1[j];
            for (int i = 0; i < MLP_IN; ++i) gW1[j * MLP_IN + i] += dz1[j] * x[s * MLP_IN + i];
        }
    }
    free(z1);
    free(z2);
    free(y);
    return loss;
}

/* One Adam step (step >= 1) on par with moments m, v. */
void or_adam_step(double *par, const double *grad, double *m, double *v, int64_t n, double lr, double beta1,
                  double beta2, double eps, int64_t step) {
    const double c1 = 1.0 - pow(beta1, (double)step), c2 = 1.0 - pow(beta2, (double)step);
    for (int64_t k = 0; k < n; ++k) {
        m[k] = beta1 * m[k] + (1.0 - beta1) * grad[k];
        v[k] = beta2 * v[k] + (1.0 - beta2) * grad[k] * grad[k];
        par[k] -= lr * (m[k] / c1) / (sqrt(v[k] / c2) + eps);
    }
}

/* Surrogate inputs of every data point of the active packages: x[P][64][27]
 * (far packages left untouched). */
void or_surrogate_inputs(const or_grid *g, int64_t P, const int32_t *nbr, const double *phi, double *x) {
    const double inv_h = 1.0 / g->h;
#pragma omp parallel for schedule(static)
    for (int64_t p = 2; p < P; ++p) {
        const int32_t *nb = nbr + p * 27;
        for (int d = 0; d < PKG3; ++d) {
            int i = d & 3, j = (d >> 2) & 3, k = d >> 4;
            for (int sz = -1; sz <= 1; ++sz)
                for (int sy = -1; sy <= 1; ++sy)
                    for (int sx = -1; sx <= 1; ++sx) {
                        double v = phi[shift_index(nb, i + sx, j + sy, k + sz)] * inv_h;
                        if (v < -1.0) v = -1.0;
                        if (v > 1.0) v = 1.0;
                        x[(p * PKG3 + d) * 27 + (sx + 1) + 3 * (sy + 1) + 9 * (sz + 1)] = v;
                    }
        }
    }
}

/* Canonical frame of a surrogate input (not in the paper; it follows from    */
/* the definitions of W and G^).  The tap weights depend on |s| alone and H   */
/* is antisymmetric, H(-z) = 1 - H(z), so negating phi maps (W, G^) to         */
/* (1 - W, -G^) and a signed permutation T of the axes maps G^ to T G^.  The   */
/* frame of a point: sign = -1 when phi(x) < 0 (else 1); g_a = sign (phi(x +   */
/* h e_a) - phi(x - h e_a)), exact in double; axis a reversed when g_a < 0;    */
/* axes ordered by decreasing |g_a|, equal magnitudes keeping the lower axis   */
/* first: canonical axis k is original axis p[k].  The canonical input at      */
/* canonical offset s' is sign phi(x + s h) / h (clipped to [-1, 1]) with      */
/* s[p[k]] = (reversed p[k] ? -1 : 1) s'[k].  code = (sign < 0) | reversed    */
/* axes << 1 | index of (p[0], p[1], p[2]) among the six permutations in      */
/* lexicographic order << 4.  x receives 27 canonical inputs per point.       */
void or_surrogate_canonical(const or_grid *g, int64_t P, const int32_t *nbr, const float *phi, double *x,
                            int32_t *code) {
    static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    const double h = g->h;
#pragma omp parallel for schedule(static)
    for (int64_t p = 2; p < P; ++p) {
        const int32_t *nb = nbr + p * 27;
        for (int d = 0; d < PKG3; ++d) {
            const int i = d & 3, j = (d >> 2) & 3, k = d >> 4;
            double f[27];
            for (int n = 0; n < 27; ++n)
                f[n] = (double)phi[shift_index(nb, i + n % 3 - 1, j + (n / 3) % 3 - 1, k + n / 9 - 1)];
            const double sign = f[13] < 0.0 ? -1.0 : 1.0;
            const double ga[3] = {sign * (f[14] - f[12]), sign * (f[16] - f[10]), sign * (f[22] - f[4])};
            int rev = 0;
            for (int a = 0; a < 3; ++a)
                if (ga[a] < 0.0) rev |= 1 << a;
            int pi = 0;
            for (int c = 0; c < 6; ++c) { /* the ordering with no later axis strictly larger than an earlier one */
                const int *q = perms[c];
                int good = 1;
                for (int u = 0; u < 3; ++u)
                    for (int w = u + 1; w < 3; ++w) {
                        const double mu = fabs(ga[q[u]]), mw = fabs(ga[q[w]]);
                        if (mw > mu || (mw == mu && q[w] < q[u])) good = 0;
                    }
                if (good) {
                    pi = c;
                    break;
                }
            }
            const int *q = perms[pi];
            for (int m = 0; m < 27; ++m) {
                const int sp[3] = {m % 3 - 1, (m / 3) % 3 - 1, m / 9 - 1};
                int so[3];
                for (int kk = 0; kk < 3; ++kk) so[q[kk]] = ((rev >> q[kk]) & 1 ? -1 : 1) * sp[kk];
                const int n = (so[0] + 1) + 3 * (so[1] + 1) + 9 * (so[2] + 1);
                double v = sign * f[n] / h;
                if (v < -1.0) v = -1.0;
                if (v > 1.0) v = 1.0;
                x[(p * PKG3 + d) * 27 + m] = v;
            }
            code[p * PKG3 + d] = (sign < 0.0 ? 1 : 0) | (rev << 1) | (pi << 4);
        }
    }
}

/* Classes of the surrogate integral (a reading: the network stands in for    */
/* the kernel integral of "Integral with SPH Smoothing Kernel and Grid-       */
/* Particle Coupling"), decided on the real values of the float field phi:    */
/*   0  every one of the 27 taps is inside at or beyond the Heaviside's half  */
/*      width (-phi_s / h >= 1), where it saturates: W = 1 and G^ = 0;        */
/*   1  every tap outside (phi_s / h >= 1): W = 0, G^ = 0;                     */
/*   2  fallback: |phi / h| < 1 at the point, or |kappa| h > 0.1 with kappa    */
/*      the 7-point Laplacian (phi_+x + phi_-x + ... - 6 phi) / h^2;           */
/*   3  network.                                                              */
/* Comparisons are taken in double precision on the float values widened;    */
/* the tap and |phi| tests are exact, the curvature test is exact up to       */
/* the rounding of the Laplacian's sum, and *ties counts points whose         */
/* |kappa| h lies within 1e-9 (relative) of 0.1.  Far packages get 255.       */
void or_surrogate_class(const or_grid *g, int64_t P, const int32_t *nbr, const float *phi, uint8_t *cls,
                        int64_t *ties) {
    const double h = g->h;
    int64_t nt = 0;
    for (int d = 0; d < 2 * PKG3; ++d) cls[d] = 255;
#pragma omp parallel for schedule(static) reduction(+ : nt)
    for (int64_t p = 2; p < P; ++p) {
        const int32_t *nb = nbr + p * 27;
        for (int d = 0; d < PKG3; ++d) {
            int i = d & 3, j = (d >> 2) & 3, k = d >> 4;
            int all_in = 1, all_out = 1;
            for (int n = 0; n < 27; ++n) {
                int sx = n % 3 - 1, sy = (n / 3) % 3 - 1, sz = n / 9 - 1;
                double f = (double)phi[shift_index(nb, i + sx, j + sy, k + sz)];
                all_in &= -f >= h; /* -phi_s / h >= 1 with h > 0, compared without rounding */
                all_out &= f >= h;
            }
            uint8_t c;
            if (all_in)
                c = 0;
            else if (all_out)
                c = 1;
            else {
                double v = (double)phi[shift_index(nb, i, j, k)];
                double a = (double)phi[shift_index(nb, i + 1, j, k)] + (double)phi[shift_index(nb, i - 1, j, k)] +
                           (double)phi[shift_index(nb, i, j + 1, k)] + (double)phi[shift_index(nb, i, j - 1, k)] +
                           (double)phi[shift_index(nb, i, j, k + 1)] + (double)phi[shift_index(nb, i, j, k - 1)] -
                           6.0 * v;
                double kap = a / (h * h);
                double kh = fabs(kap) * h;
                if (fabs(kh - 0.1) < 1e-10) ++nt;
                if (fabs(v) < h || kh > 0.1) /* |phi / h| < 1, compared without rounding */
                    c = 2;
                else
                    c = 3;
            }
            cls[p * PKG3 + d] = c;
        }
    }
    if (ties) *ties = nt;
}
