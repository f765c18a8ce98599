/*
 * eam_oracle.c -- plain, serial, FP64 reference of the EAM molecular-dynamics
 * timestep of "Breaking the Molecular Dynamics Timescale Barrier Using a
 * Wafer-Scale System" (arXiv 2405.07898).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library; the two meet
 * only in the seeded input generators.
 *
 * Everything here is the plain definition, written for checking by eye:
 *   - cubic splines through uniform knots by the textbook tridiagonal
 *     (Thomas) solve for the knot second derivatives;
 *   - periodic wrap and minimum image (Section "Periodic Boundary Conditions");
 *   - cell bins by a stable counting sort and a 27-cell stencil neighbour list
 *     filtered by r^2 < r_list^2 (Section "Neighbor list": the squared distance
 *     is compared, no square root), plus an O(N^2) all-pairs list;
 *   - electron density, Eq. 2; potential energy, Eq. 3; force, Eq. 4;
 *   - velocity-Verlet (kick-drift-kick) integration, whose half-step
 *     velocities are exactly the leap-frog velocities of Eq. 5.
 * Readings of points the paper leaves open (listed in the design notes):
 *   - the density sum excludes j = i;
 *   - all cutoff tests are strict (r^2 < r_cut^2, r^2 < r_list^2);
 *   - splines are C2 cubics on uniform knots; outside the knot range a
 *     spline continues linearly with its end slope;
 *   - the neighbour list is rebuilt when 10 steps have passed since the last
 *     build or when some atom has moved more than skin/2 since then.
 *
 * Compile with -ffp-contract=off: every product and sum is rounded as written.
 * The per-atom loops of the evaluation and the integrator carry OpenMP
 * pragmas; the parity build ignores them (no -fopenmp: one thread, the sums
 * in the order written).  A second build with -fopenmp is used only to time
 * the oracle on all host cores; there the per-atom results are the same and
 * only the sums over atoms (energies, virial, largest displacement) are
 * taken in another order.  The list build stays serial in both.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* 1 eV/(Angstrom amu) in Angstrom/fs^2 (CODATA 2018 e and u). */
static const double ORC_ACCEL = 9.648533215665e-3;

/* ------------------------------------------------------------------------ */
/* cubic splines on uniform knots                                           */

typedef struct {
    int32_t n;
    double x0, dx;
    const double *y;
    int32_t bc_lo, bc_hi; /* 0 = natural (S'' = 0), 1 = clamped (S' given) */
    double d_lo, d_hi;
} orc_knots;

typedef struct {
    int32_t n;      /* knots */
    double x0, h;   /* first knot, spacing */
    double *coef;   /* (n-1) rows: S_k(t) = a + b t + c t^2 + d t^3, t = x - x_k */
} orc_spline;

/* Second derivatives M_k of the interpolating cubic, then the per-interval
 * polynomial.  For uniform spacing h the continuity of S' at interior knots
 * gives  M_{k-1} + 4 M_k + M_{k+1} = 6/h^2 (y_{k+1} - 2 y_k + y_{k-1});
 * a natural end sets M = 0, a clamped end with slope s gives
 * 2 M_0 + M_1 = 6/h ((y_1 - y_0)/h - s)  and
 * M_{n-2} + 2 M_{n-1} = 6/h (s - (y_{n-1} - y_{n-2})/h). */
int orc_spline_coeffs(int32_t n, double h, const double *y, int32_t bc_lo, double d_lo,
                      int32_t bc_hi, double d_hi, double *coef)
{
    if (n < 2 || !(h > 0.0)) return -1;
    double *sub = calloc((size_t)n, sizeof(double));
    double *dia = calloc((size_t)n, sizeof(double));
    double *sup = calloc((size_t)n, sizeof(double));
    double *rhs = calloc((size_t)n, sizeof(double));
    double *M = calloc((size_t)n, sizeof(double));
    if (!sub || !dia || !sup || !rhs || !M) {
        free(sub); free(dia); free(sup); free(rhs); free(M);
        return -2;
    }
    if (bc_lo == 1) {
        dia[0] = 2.0; sup[0] = 1.0;
        rhs[0] = 6.0 / h * ((y[1] - y[0]) / h - d_lo);
    } else {
        dia[0] = 1.0; sup[0] = 0.0; rhs[0] = 0.0;
    }
    for (int32_t k = 1; k < n - 1; ++k) {
        sub[k] = 1.0; dia[k] = 4.0; sup[k] = 1.0;
        rhs[k] = 6.0 / (h * h) * (y[k + 1] - 2.0 * y[k] + y[k - 1]);
    }
    if (bc_hi == 1) {
        sub[n - 1] = 1.0; dia[n - 1] = 2.0;
        rhs[n - 1] = 6.0 / h * (d_hi - (y[n - 1] - y[n - 2]) / h);
    } else {
        sub[n - 1] = 0.0; dia[n - 1] = 1.0; rhs[n - 1] = 0.0;
    }
    /* Thomas algorithm: forward elimination, back substitution */
    for (int32_t k = 1; k < n; ++k) {
        double w = sub[k] / dia[k - 1];
        dia[k] = dia[k] - w * sup[k - 1];
        rhs[k] = rhs[k] - w * rhs[k - 1];
    }
    M[n - 1] = rhs[n - 1] / dia[n - 1];
    for (int32_t k = n - 2; k >= 0; --k)
        M[k] = (rhs[k] - sup[k] * M[k + 1]) / dia[k];

    for (int32_t k = 0; k < n - 1; ++k) {
        double *c = coef + 4 * (size_t)k;
        c[0] = y[k];
        c[1] = (y[k + 1] - y[k]) / h - h * (2.0 * M[k] + M[k + 1]) / 6.0;
        c[2] = M[k] / 2.0;
        c[3] = (M[k + 1] - M[k]) / (6.0 * h);
    }
    free(sub); free(dia); free(sup); free(rhs); free(M);
    return 0;
}

/* Value, first and second derivative at x.  Interval k = floor((x-x0)/h),
 * capped to the last interval; beyond either end the spline continues along
 * its end tangent. */
double orc_spline_eval(int32_t n, double x0, double h, const double *coef, double x,
                       double *dy, double *d2y)
{
    double x_end = x0 + (double)(n - 1) * h;
    double val, der, der2;
    if (x < x0) {
        const double *c = coef;
        val = c[0] + c[1] * (x - x0);
        der = c[1];
        der2 = 0.0;
    } else if (x > x_end) {
        const double *c = coef + 4 * (size_t)(n - 2);
        double t = h;
        double y_end = c[0] + t * (c[1] + t * (c[2] + t * c[3]));
        double s_end = c[1] + t * (2.0 * c[2] + t * 3.0 * c[3]);
        val = y_end + s_end * (x - x_end);
        der = s_end;
        der2 = 0.0;
    } else {
        int64_t k = (int64_t)floor((x - x0) / h);
        if (k > n - 2) k = n - 2;
        const double *c = coef + 4 * (size_t)k;
        double t = x - (x0 + (double)k * h);
        val = c[0] + t * (c[1] + t * (c[2] + t * c[3]));
        der = c[1] + t * (2.0 * c[2] + t * 3.0 * c[3]);
        der2 = 2.0 * c[2] + 6.0 * c[3] * t;
    }
    if (dy) *dy = der;
    if (d2y) *d2y = der2;
    return val;
}

static double spl(const orc_spline *s, double x, double *dy, double *d2y)
{
    return orc_spline_eval(s->n, s->x0, s->h, s->coef, x, dy, d2y);
}

/* ------------------------------------------------------------------------ */
/* the potential: per-type F and f, per-type-pair phi (Eq. 3)               */

typedef struct {
    int32_t ntypes;
    double *mass;
    orc_spline *F, *f, *phi; /* F[t], f[t], phi[pair index of (a <= b)] */
    double r_cut, skin;
} orc_pot;

static int32_t pair_index(int32_t ntypes, int32_t a, int32_t b)
{
    if (a > b) { int32_t t = a; a = b; b = t; }
    return a * ntypes - a * (a - 1) / 2 + (b - a);
}

static int build_one(orc_spline *s, const orc_knots *k)
{
    s->n = k->n;
    s->x0 = k->x0;
    s->h = k->dx;
    s->coef = malloc(sizeof(double) * 4 * (size_t)(k->n > 1 ? k->n - 1 : 1));
    if (!s->coef) return -2;
    return orc_spline_coeffs(k->n, k->dx, k->y, k->bc_lo, k->d_lo, k->bc_hi, k->d_hi, s->coef);
}

void orc_pot_destroy(orc_pot *p);

orc_pot *orc_pot_create(int32_t ntypes, const double *mass, const orc_knots *F,
                        const orc_knots *f, const orc_knots *phi, double r_cut, double skin)
{
    if (ntypes < 1) return NULL;
    int32_t npair = ntypes * (ntypes + 1) / 2;
    orc_pot *p = calloc(1, sizeof(orc_pot));
    if (!p) return NULL;
    p->ntypes = ntypes;
    p->r_cut = r_cut;
    p->skin = skin;
    p->mass = malloc(sizeof(double) * (size_t)ntypes);
    p->F = calloc((size_t)ntypes, sizeof(orc_spline));
    p->f = calloc((size_t)ntypes, sizeof(orc_spline));
    p->phi = calloc((size_t)npair, sizeof(orc_spline));
    if (!p->mass || !p->F || !p->f || !p->phi) { orc_pot_destroy(p); return NULL; }
    memcpy(p->mass, mass, sizeof(double) * (size_t)ntypes);
    int bad = 0;
    for (int32_t t = 0; t < ntypes; ++t) {
        bad |= build_one(&p->F[t], &F[t]);
        bad |= build_one(&p->f[t], &f[t]);
    }
    for (int32_t q = 0; q < npair; ++q) bad |= build_one(&p->phi[q], &phi[q]);
    if (bad) { orc_pot_destroy(p); return NULL; }
    return p;
}

void orc_pot_destroy(orc_pot *p)
{
    if (!p) return;
    int32_t npair = p->ntypes * (p->ntypes + 1) / 2;
    for (int32_t t = 0; t < p->ntypes; ++t) {
        if (p->F) free(p->F[t].coef);
        if (p->f) free(p->f[t].coef);
    }
    for (int32_t q = 0; q < npair && p->phi; ++q) free(p->phi[q].coef);
    free(p->F); free(p->f); free(p->phi); free(p->mass);
    free(p);
}

/* ------------------------------------------------------------------------ */
/* geometry: periodic axes (Section "Periodic Boundary Conditions") and open */
/* axes (the open, non-periodic boundaries of the thin-slab workloads,       */
/* Section "How Performance Was Measured").  `open` holds one bit per axis   */
/* (1: x, 2: y, 4: z) that is open; on an open axis the box is the extent of */
/* the cell grid, positions are not wrapped and displacements are plain      */
/* differences.                                                              */

static int is_open(int open, int d) { return (open >> d) & 1; }

/* Periodic image of each coordinate on the periodic axes: a coordinate
 * already in [0, L) is kept as it is, any other becomes x - L floor(x / L). */
void orc_wrap(int64_t n, const double box[3], int open, double *pos)
{
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            if (is_open(open, d)) continue;
            double x = pos[3 * i + d];
            if (x >= 0.0 && x < box[d]) continue;
            double q = floor(x / box[d]);
            pos[3 * i + d] = x - box[d] * q;
        }
}

/* Displacement x_j - x_i along one axis: the minimum image on a periodic
 * axis (|raw| < 1.5 L), the difference on an open one. */
static double min_image(double xj, double xi, double L, int open_axis)
{
    double d = xj - xi;
    if (open_axis) return d;
    if (d > 0.5 * L) d = d - L;
    else if (d < -0.5 * L) d = d + L;
    return d;
}

/* Squared distance, summed in the fixed order (dx^2 + dy^2) + dz^2. */
static double dist2(const double *xi, const double *xj, const double box[3], int open, double d[3])
{
    d[0] = min_image(xj[0], xi[0], box[0], is_open(open, 0));
    d[1] = min_image(xj[1], xi[1], box[1], is_open(open, 1));
    d[2] = min_image(xj[2], xi[2], box[2], is_open(open, 2));
    return (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
}

/* Cells per axis n_d = floor(L_d / r_list); a periodic axis needs n_d >= 3
 * (the 27-cell stencil may not meet its own image), an open axis n_d >= 1. */
int orc_cell_dims(const double box[3], int open, double r_list, int32_t ncell[3])
{
    for (int d = 0; d < 3; ++d) {
        double q = floor(box[d] / r_list);
        ncell[d] = (int32_t)q;
        if (ncell[d] < (is_open(open, d) ? 1 : 3)) return -1;
    }
    return 0;
}

/* Cell of a position: c_d = floor(x_d * (n_d / L_d)) clamped to [0, n_d - 1]
 * (on an open axis, atoms outside the box go to the edge cells). */
static int64_t cell_of(const double *x, const double box[3], const int32_t ncell[3])
{
    int64_t c[3];
    for (int d = 0; d < 3; ++d) {
        double s = (double)ncell[d] / box[d];
        double q = floor(x[d] * s);
        int64_t cd = (int64_t)q;
        if (cd < 0) cd = 0;
        if (cd > ncell[d] - 1) cd = ncell[d] - 1;
        c[d] = cd;
    }
    return (c[2] * ncell[1] + c[1]) * ncell[0] + c[0];
}

/* Stable counting sort of atoms into cells: cell_start[c] .. cell_start[c+1]
 * index cell_atoms, which lists the atoms of cell c in ascending index. */
int orc_cells(int64_t n, const double box[3], int open, double r_list, const double *pos,
              int32_t *cell_start, int32_t *cell_atoms)
{
    int32_t nc[3];
    if (orc_cell_dims(box, open, r_list, nc)) return -1;
    int64_t ncells = (int64_t)nc[0] * nc[1] * nc[2];
    int64_t *cursor = calloc((size_t)ncells, sizeof(int64_t));
    int64_t *cell = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!cursor || !cell) { free(cursor); free(cell); return -2; }
    for (int64_t c = 0; c <= ncells; ++c) cell_start[c] = 0;
    for (int64_t i = 0; i < n; ++i) {
        cell[i] = cell_of(pos + 3 * i, box, nc);
        cell_start[cell[i] + 1] += 1;
    }
    for (int64_t c = 0; c < ncells; ++c) cell_start[c + 1] += cell_start[c];
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = cell[i];
        cell_atoms[cell_start[c] + cursor[c]] = (int32_t)i;
        cursor[c] += 1;
    }
    free(cursor);
    free(cell);
    return 0;
}

/* Neighbour list (Section "Neighbor list"): for each atom, the atoms j != i
 * of the 27 surrounding cells (cells beyond an open edge do not exist) whose
 * squared minimum-image distance is below r_list^2.  CSR output: offsets[n+1], js[offsets[i] .. offsets[i+1]).
 * Returns the total number of entries (which may exceed cap: then only the
 * count is meaningful), or a negative error code. */
int64_t orc_list_cells(int64_t n, const double box[3], int open, double r_list, const double *pos,
                       int64_t *offsets, int32_t *js, int64_t cap)
{
    int32_t nc[3];
    if (orc_cell_dims(box, open, r_list, nc)) return -1;
    int64_t ncells = (int64_t)nc[0] * nc[1] * nc[2];
    int32_t *start = malloc(sizeof(int32_t) * (size_t)(ncells + 1));
    int32_t *atoms = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!start || !atoms) { free(start); free(atoms); return -2; }
    orc_cells(n, box, open, r_list, pos, start, atoms);
    double rl2 = r_list * r_list;
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        offsets[i] = m;
        const double *xi = pos + 3 * i;
        int64_t c = cell_of(xi, box, nc);
        int64_t cx = c % nc[0], cy = (c / nc[0]) % nc[1], cz = c / ((int64_t)nc[0] * nc[1]);
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t ex = cx + dx, ey = cy + dy, ez = cz + dz;
                    if ((ex < 0 || ex >= nc[0]) && is_open(open, 0)) continue;
                    if ((ey < 0 || ey >= nc[1]) && is_open(open, 1)) continue;
                    if ((ez < 0 || ez >= nc[2]) && is_open(open, 2)) continue;
                    ex = (ex + nc[0]) % nc[0];
                    ey = (ey + nc[1]) % nc[1];
                    ez = (ez + nc[2]) % nc[2];
                    int64_t e = (ez * nc[1] + ey) * nc[0] + ex;
                    for (int32_t q = start[e]; q < start[e + 1]; ++q) {
                        int32_t j = atoms[q];
                        if (j == i) continue;
                        double d[3];
                        if (dist2(xi, pos + 3 * (int64_t)j, box, open, d) < rl2) {
                            if (m < cap) js[m] = j;
                            m += 1;
                        }
                    }
                }
    }
    offsets[n] = m;
    free(start);
    free(atoms);
    return m;
}

/* The same list by testing every pair (the definition, O(N^2)). */
int64_t orc_list_brute(int64_t n, const double box[3], int open, double r_list, const double *pos,
                       int64_t *offsets, int32_t *js, int64_t cap)
{
    double rl2 = r_list * r_list;
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        offsets[i] = m;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3];
            if (dist2(pos + 3 * i, pos + 3 * j, box, open, d) < rl2) {
                if (m < cap) js[m] = (int32_t)j;
                m += 1;
            }
        }
    }
    offsets[n] = m;
    return m;
}

/* ------------------------------------------------------------------------ */
/* EAM density, energy, force and virial (Eqs. 2-4)                          */

/* Electron density at atom i (Eq. 2, j != i, r < r_cut), the embedding
 * derivative F'_i(rho_i), and the embedding energy sum of Eq. 3. */
static double density_pass(const orc_pot *p, int64_t n, const double box[3], int open, const double *pos,
                           const int32_t *types, const int64_t *off, const int32_t *js,
                           double *rho, double *Fp)
{
    double rc2 = p->r_cut * p->r_cut;
    double e_embed = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : e_embed)
    for (int64_t i = 0; i < n; ++i) {
        double r_i = 0.0;
        for (int64_t q = off[i]; q < off[i + 1]; ++q) {
            int64_t j = js[q];
            double d[3];
            double r2 = dist2(pos + 3 * i, pos + 3 * j, box, open, d);
            if (r2 < rc2) r_i += spl(&p->f[types[j]], sqrt(r2), NULL, NULL);
        }
        double dF;
        double Fi = spl(&p->F[types[i]], r_i, &dF, NULL);
        rho[i] = r_i;
        Fp[i] = dF;
        e_embed += Fi;
    }
    return e_embed;
}

/* Forces F_i = -dU/dx_i: with d = x_j - x_i and r = |d|,
 *   s_ij = phi'_{ij}(r) + F'_i f'_{t_j}(r) + F'_j f'_{t_i}(r),
 *   F_i  = sum_j s_ij d / r                                    (Eq. 4),
 * the pair energy (1/2) sum_{i != j} phi_ij(r_ij)               (Eq. 3),
 * and the virial W_ab = -(1/2) sum_i sum_j s_ij d_a d_b / r, stored
 * xx, yy, zz, xy, xz, yz. */
static double force_pass(const orc_pot *p, int64_t n, const double box[3], int open, const double *pos,
                         const int32_t *types, const int64_t *off, const int32_t *js,
                         const double *Fp, double *force, double virial[6])
{
    double rc2 = p->r_cut * p->r_cut;
    double e_pair = 0.0;
    for (int k = 0; k < 6; ++k) virial[k] = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : e_pair, virial[0:6])
    for (int64_t i = 0; i < n; ++i) {
        double fi[3] = {0.0, 0.0, 0.0};
        int32_t ti = types[i];
        for (int64_t q = off[i]; q < off[i + 1]; ++q) {
            int64_t j = js[q];
            int32_t tj = types[j];
            double d[3];
            double r2 = dist2(pos + 3 * i, pos + 3 * j, box, open, d);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2);
            double dphi, dfj, dfi;
            double phi = spl(&p->phi[pair_index(p->ntypes, ti, tj)], r, &dphi, NULL);
            spl(&p->f[tj], r, &dfj, NULL);
            spl(&p->f[ti], r, &dfi, NULL);
            double s = dphi + Fp[i] * dfj + Fp[j] * dfi;
            for (int a = 0; a < 3; ++a) fi[a] += s * d[a] / r;
            e_pair += 0.5 * phi;
            virial[0] += -0.5 * s * d[0] * d[0] / r;
            virial[1] += -0.5 * s * d[1] * d[1] / r;
            virial[2] += -0.5 * s * d[2] * d[2] / r;
            virial[3] += -0.5 * s * d[0] * d[1] / r;
            virial[4] += -0.5 * s * d[0] * d[2] / r;
            virial[5] += -0.5 * s * d[1] * d[2] / r;
        }
        for (int a = 0; a < 3; ++a) force[3 * i + a] = fi[a];
    }
    return e_pair;
}

/* The two passes of orc_eam_eval separately (the same functions): the
 * density pass alone -- rho_i and F'_i of every atom of the list (Eq. 2);
 * returns the embedding energy sum -- and the force pass with F' given for
 * every atom (Eq. 4); returns the pair energy.  Used to check a spatial
 * decomposition whose ranks exchange F' of their boundary atoms between the
 * two passes. */
double orc_density(const orc_pot *p, int64_t n, const double box[3], int open, const double *pos,
                   const int32_t *types, const int64_t *off, const int32_t *js, double *rho, double *Fp)
{
    return density_pass(p, n, box, open, pos, types, off, js, rho, Fp);
}

double orc_force_given_fp(const orc_pot *p, int64_t n, const double box[3], int open, const double *pos,
                          const int32_t *types, const int64_t *off, const int32_t *js, const double *Fp,
                          double *force, double virial[6])
{
    return force_pass(p, n, box, open, pos, types, off, js, Fp, force, virial);
}

/* Density, forces, energies and virial for positions `pos` and a
 * neighbour list built for them (or for positions within skin/2 of them).
 * Any output pointer may be NULL except force. */
int orc_eam_eval(const orc_pot *p, int64_t n, const double box[3], int open, const double *pos,
                 const int32_t *types, const int64_t *off, const int32_t *js,
                 double *rho, double *Fp, double *force, double energy[2], double virial[6])
{
    double *rho_w = rho ? rho : malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *Fp_w = Fp ? Fp : malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double vir_w[6];
    if (!rho_w || !Fp_w) return -2;
    double e_embed = density_pass(p, n, box, open, pos, types, off, js, rho_w, Fp_w);
    double e_pair = force_pass(p, n, box, open, pos, types, off, js, Fp_w, force, vir_w);
    if (energy) { energy[0] = e_embed; energy[1] = e_pair; }
    if (virial) memcpy(virial, vir_w, sizeof(vir_w));
    if (!rho) free(rho_w);
    if (!Fp) free(Fp_w);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* molecular dynamics: velocity Verlet (Eq. 1 integrated as in Eq. 5)        */

typedef struct {
    const orc_pot *pot;
    int64_t n;
    double box[3];
    int open;
    double *pos, *vel, *force, *rho, *Fp, *x_ref;
    int32_t *types;
    int64_t *off;
    int32_t *js;
    int64_t cap;
    int64_t step, rebuilds;
    int32_t since_build;
    double energy[2], virial[6];
} orc_sys;

void orc_sys_destroy(orc_sys *s);

static int rebuild(orc_sys *s)
{
    double r_list = s->pot->r_cut + s->pot->skin;
    orc_wrap(s->n, s->box, s->open, s->pos);
    for (;;) {
        int64_t m = orc_list_cells(s->n, s->box, s->open, r_list, s->pos, s->off, s->js, s->cap);
        if (m < 0) return (int)m;
        if (m <= s->cap) break;
        free(s->js);
        s->cap = m + m / 4 + 16;
        s->js = malloc(sizeof(int32_t) * (size_t)s->cap);
        if (!s->js) return -2;
    }
    memcpy(s->x_ref, s->pos, sizeof(double) * 3 * (size_t)s->n);
    s->since_build = 0;
    s->rebuilds += 1;
    return 0;
}

static int evaluate(orc_sys *s)
{
    return orc_eam_eval(s->pot, s->n, s->box, s->open, s->pos, s->types, s->off, s->js, s->rho, s->Fp,
                        s->force, s->energy, s->virial);
}

orc_sys *orc_sys_create(const orc_pot *pot, int64_t n, const double box[3], int open, const double *pos,
                        const double *vel, const int32_t *types)
{
    orc_sys *s = calloc(1, sizeof(orc_sys));
    if (!s) return NULL;
    size_t nn = (size_t)(n > 0 ? n : 1);
    s->pot = pot;
    s->n = n;
    s->open = open;
    memcpy(s->box, box, sizeof(s->box));
    s->pos = malloc(sizeof(double) * 3 * nn);
    s->vel = calloc(3 * nn, sizeof(double));
    s->force = calloc(3 * nn, sizeof(double));
    s->rho = calloc(nn, sizeof(double));
    s->Fp = calloc(nn, sizeof(double));
    s->x_ref = malloc(sizeof(double) * 3 * nn);
    s->types = malloc(sizeof(int32_t) * nn);
    s->off = malloc(sizeof(int64_t) * (nn + 1));
    s->cap = 64 * (int64_t)nn;
    s->js = malloc(sizeof(int32_t) * (size_t)s->cap);
    if (!s->pos || !s->vel || !s->force || !s->rho || !s->Fp || !s->x_ref || !s->types ||
        !s->off || !s->js) {
        orc_sys_destroy(s);
        return NULL;
    }
    memcpy(s->pos, pos, sizeof(double) * 3 * (size_t)n);
    if (vel) memcpy(s->vel, vel, sizeof(double) * 3 * (size_t)n);
    memcpy(s->types, types, sizeof(int32_t) * (size_t)n);
    if (rebuild(s) || evaluate(s)) { orc_sys_destroy(s); return NULL; }
    s->rebuilds = 0;
    return s;
}

void orc_sys_destroy(orc_sys *s)
{
    if (!s) return;
    free(s->pos); free(s->vel); free(s->force); free(s->rho); free(s->Fp);
    free(s->x_ref); free(s->types); free(s->off); free(s->js);
    free(s);
}

/* nsteps of kick (dt/2) - drift (dt) - [rebuild] - force - kick (dt/2).
 * The half-step velocity after the first kick is the leap-frog v^{k+1/2}
 * of Eq. 5 and the drift is its position update. */
int orc_sys_step(orc_sys *s, int64_t nsteps, double dt, int32_t rebuild_every)
{
    double half_skin2 = 0.25 * s->pot->skin * s->pot->skin;
    for (int64_t it = 0; it < nsteps; ++it) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < s->n; ++i) {
            double m = s->pot->mass[s->types[i]];
            for (int a = 0; a < 3; ++a) {
                double acc = s->force[3 * i + a] / m * ORC_ACCEL;
                s->vel[3 * i + a] += acc * (0.5 * dt);
                s->pos[3 * i + a] += s->vel[3 * i + a] * dt;
            }
        }
        s->step += 1;
        s->since_build += 1;
        double worst = 0.0;
#pragma omp parallel for schedule(static) reduction(max : worst)
        for (int64_t i = 0; i < s->n; ++i) {
            double dx = s->pos[3 * i] - s->x_ref[3 * i];
            double dy = s->pos[3 * i + 1] - s->x_ref[3 * i + 1];
            double dz = s->pos[3 * i + 2] - s->x_ref[3 * i + 2];
            double d2 = dx * dx + dy * dy + dz * dz;
            if (d2 > worst) worst = d2;
        }
        if (s->since_build >= rebuild_every || worst > half_skin2) {
            int rc = rebuild(s);
            if (rc) return rc;
        }
        int rc = evaluate(s);
        if (rc) return rc;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < s->n; ++i) {
            double m = s->pot->mass[s->types[i]];
            for (int a = 0; a < 3; ++a) {
                double acc = s->force[3 * i + a] / m * ORC_ACCEL;
                s->vel[3 * i + a] += acc * (0.5 * dt);
            }
        }
    }
    return 0;
}

/* Potential energy (Eq. 3) and kinetic energy sum_i m v^2 / 2 in eV. */
void orc_sys_energy(const orc_sys *s, double *pe, double *ke)
{
    double k = 0.0;
    for (int64_t i = 0; i < s->n; ++i) {
        double m = s->pot->mass[s->types[i]];
        double v2 = s->vel[3 * i] * s->vel[3 * i] + s->vel[3 * i + 1] * s->vel[3 * i + 1] +
                    s->vel[3 * i + 2] * s->vel[3 * i + 2];
        k += 0.5 * m * v2 / ORC_ACCEL;
    }
    if (pe) *pe = s->energy[0] + s->energy[1];
    if (ke) *ke = k;
}

void orc_sys_virial(const orc_sys *s, double w[6]) { memcpy(w, s->virial, sizeof(s->virial)); }

/* Copies of the current state; any pointer may be NULL. */
void orc_sys_get(const orc_sys *s, double *pos, double *vel, double *force, double *rho,
                 double *Fp, int64_t counters[2])
{
    size_t n3 = sizeof(double) * 3 * (size_t)s->n;
    if (pos) memcpy(pos, s->pos, n3);
    if (vel) memcpy(vel, s->vel, n3);
    if (force) memcpy(force, s->force, n3);
    if (rho) memcpy(rho, s->rho, sizeof(double) * (size_t)s->n);
    if (Fp) memcpy(Fp, s->Fp, sizeof(double) * (size_t)s->n);
    if (counters) { counters[0] = s->step; counters[1] = s->rebuilds; }
}

/* ------------------------------------------------------------------------ */
/* differentiation: force-matching loss and its gradient                    */
/*
 * Loss of one configuration (single atom type):
 *   L = (E - E_ref)^2 / N + w sum_i |F_i - F_ref,i|^2,
 * with E of Eq. 3 and F of Eq. 4.  Every spline is linear in its per-interval
 * coefficients (a, b, c, d), so dL/d(coefficients) is accumulated here and the
 * knot gradient follows as M^T times it (orc_spline_basis gives M).
 *
 * With A = 2 (E - E_ref) / N, g_i = F_i - F_ref,i, and for the position
 * perturbation dx = g:  dr_ij = (x_j - x_i)/r . (g_j - g_i),
 * drho_i = sum_j f'(r_ij) dr_ij.  Since F = -dE/dx,
 *   dL = A dE/dtheta - 2 w D_g[dE/dtheta]  (D_g: derivative along dx = g),
 * where
 *   dE/dtheta(phi) = 1/2 sum_{i != j} B(r_ij)       D_g = 1/2 sum B'(r_ij) dr_ij
 *   dE/dtheta(F)   = sum_i B(rho_i)                  D_g = sum_i B'(rho_i) drho_i
 *   dE/dtheta(f)   = sum_i F'(rho_i) sum_j B(r_ij)
 *            D_g = sum_i [F''(rho_i) drho_i sum_j B(r_ij) + F'(rho_i) sum_j B'(r_ij) dr_ij]
 * and for a coefficient row (a, b, c, d) of the interval holding x, B = (1, t,
 * t^2, t^3) and B' = (0, 1, 2t, 3t^2), t = x - x_k.
 */

/* Interval and local coordinate of x on a spline (beyond the ends: the end
 * interval; then the coefficient derivative rows below are those of the
 * linear continuation, which depends on the end interval only). */
static int64_t seg_of(const orc_spline *s, double x, double *t)
{
    int64_t k;
    if (x < s->x0) k = 0;
    else {
        k = (int64_t)floor((x - s->x0) / s->h);
        if (k > s->n - 2) k = s->n - 2;
    }
    *t = x - (s->x0 + (double)k * s->h);
    return k;
}

/* d(value)/d(a,b,c,d) and d(derivative)/d(a,b,c,d) at x, following
 * orc_spline_eval: inside the table the cubic; outside, the tangent line at
 * the end knot (value y_end + s_end (x - x_end), slope s_end). */
static void coef_rows(const orc_spline *s, double x, int64_t *k, double bv[4], double bd[4])
{
    double t;
    double x_end = s->x0 + (double)(s->n - 1) * s->h;
    *k = seg_of(s, x, &t);
    if (x < s->x0) {
        /* y_0 + b_0 (x - x0): a and b of interval 0 */
        bv[0] = 1.0; bv[1] = x - s->x0; bv[2] = 0.0; bv[3] = 0.0;
        bd[0] = 0.0; bd[1] = 1.0; bd[2] = 0.0; bd[3] = 0.0;
    } else if (x > x_end) {
        double hh = s->h, e = x - x_end;
        /* y_end = a + b h + c h^2 + d h^3, s_end = b + 2 c h + 3 d h^2 */
        bv[0] = 1.0; bv[1] = hh + e; bv[2] = hh * hh + 2.0 * hh * e; bv[3] = hh * hh * hh + 3.0 * hh * hh * e;
        bd[0] = 0.0; bd[1] = 1.0; bd[2] = 2.0 * hh; bd[3] = 3.0 * hh * hh;
    } else {
        bv[0] = 1.0; bv[1] = t; bv[2] = t * t; bv[3] = t * t * t;
        bd[0] = 0.0; bd[1] = 1.0; bd[2] = 2.0 * t; bd[3] = 3.0 * t * t;
    }
}

/* M: coefficients of the spline through unit knot vectors (end slopes 0):
 * column q holds the 4(n-1) coefficients for y = e_q; row-major
 * M[(4k + c) * n + q]. */
int orc_spline_basis(int32_t n, double h, int32_t bc_lo, int32_t bc_hi, double *M)
{
    double *y = calloc((size_t)n, sizeof(double));
    double *c = malloc(sizeof(double) * 4 * (size_t)(n - 1));
    if (!y || !c) { free(y); free(c); return -2; }
    for (int32_t q = 0; q < n; ++q) {
        for (int32_t k = 0; k < n; ++k) y[k] = (k == q) ? 1.0 : 0.0;
        int rc = orc_spline_coeffs(n, h, y, bc_lo, 0.0, bc_hi, 0.0, c);
        if (rc) { free(y); free(c); return rc; }
        for (int32_t r = 0; r < 4 * (n - 1); ++r) M[(size_t)r * n + q] = c[r];
    }
    free(y);
    free(c);
    return 0;
}

/* Loss of one configuration and dL/d(coefficients) of phi, f and F (arrays
 * of 4(n-1) each, accumulated into: the caller zeroes them).  Returns the
 * energy and forces through e_out / f_out when given. */
int orc_force_match(const orc_pot *p, int64_t n, const double box[3], int open, const double *pos,
                    double e_ref, const double *f_ref, double w, double *loss,
                    double *g_phi, double *g_f, double *g_F, double *e_out, double *f_out)
{
    if (p->ntypes != 1) return -1;
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *wp = malloc(sizeof(double) * 3 * nn);
    int32_t *types = calloc(nn, sizeof(int32_t));
    int64_t *off = malloc(sizeof(int64_t) * (nn + 1));
    double *rho = malloc(sizeof(double) * nn), *Fp = malloc(sizeof(double) * nn);
    double *force = malloc(sizeof(double) * 3 * nn), *g = malloc(sizeof(double) * 3 * nn);
    double *drho = calloc(nn, sizeof(double));
    int64_t cap = 64 * (int64_t)nn;
    int32_t *js = malloc(sizeof(int32_t) * (size_t)cap);
    int status = 0;
    if (!wp || !types || !off || !rho || !Fp || !force || !g || !drho || !js) {
        status = -2;
        goto done;
    }
    memcpy(wp, pos, sizeof(double) * 3 * (size_t)n);
    orc_wrap(n, box, open, wp);
    int64_t m = orc_list_cells(n, box, open, p->r_cut + p->skin, wp, off, js, cap);
    if (m < 0 || m > cap) {
        status = -3;
        goto done;
    }
    double energy[2], vir[6];
    orc_eam_eval(p, n, box, open, wp, types, off, js, rho, Fp, force, energy, vir);
    double E = energy[0] + energy[1];
    double A = 2.0 * (E - e_ref) / (double)n;
    double sq = 0.0;
    for (int64_t i = 0; i < 3 * n; ++i) {
        g[i] = force[i] - f_ref[i];
        sq += g[i] * g[i];
    }
    *loss = (E - e_ref) * (E - e_ref) / (double)n + w * sq;
    double rc2 = p->r_cut * p->r_cut;
    const orc_spline *sphi = &p->phi[0], *sf = &p->f[0], *sF = &p->F[0];
    /* drho_i = sum_j f'(r_ij) dr_ij */
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t q = off[i]; q < off[i + 1]; ++q) {
            int64_t j = js[q];
            double d[3];
            double r2 = dist2(wp + 3 * i, wp + 3 * j, box, open, d);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2), df;
            spl(sf, r, &df, NULL);
            double dr = (d[0] * (g[3 * j] - g[3 * i]) + d[1] * (g[3 * j + 1] - g[3 * i + 1]) +
                         d[2] * (g[3 * j + 2] - g[3 * i + 2])) / r;
            drho[i] += df * dr;
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        double dF, d2F, bv[4], bd[4];
        int64_t k;
        spl(sF, rho[i], &dF, &d2F);
        /* F: A B(rho_i) - 2w B'(rho_i) drho_i */
        coef_rows(sF, rho[i], &k, bv, bd);
        for (int c = 0; c < 4; ++c) g_F[4 * k + c] += A * bv[c] - 2.0 * w * bd[c] * drho[i];
        for (int64_t q = off[i]; q < off[i + 1]; ++q) {
            int64_t j = js[q];
            double d[3];
            double r2 = dist2(wp + 3 * i, wp + 3 * j, box, open, d);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2);
            double dr = (d[0] * (g[3 * j] - g[3 * i]) + d[1] * (g[3 * j + 1] - g[3 * i + 1]) +
                         d[2] * (g[3 * j + 2] - g[3 * i + 2])) / r;
            /* phi: (1/2) A B(r) - w B'(r) dr */
            coef_rows(sphi, r, &k, bv, bd);
            for (int c = 0; c < 4; ++c) g_phi[4 * k + c] += 0.5 * A * bv[c] - w * bd[c] * dr;
            /* f (density contributed by j at i):
               A F'_i B(r) - 2w [F''_i drho_i B(r) + F'_i B'(r) dr] */
            coef_rows(sf, r, &k, bv, bd);
            for (int c = 0; c < 4; ++c)
                g_f[4 * k + c] += A * dF * bv[c] - 2.0 * w * (d2F * drho[i] * bv[c] + dF * bd[c] * dr);
        }
    }
    if (e_out) *e_out = E;
    if (f_out) memcpy(f_out, force, sizeof(double) * 3 * (size_t)n);
done:
    free(wp); free(types); free(off); free(rho); free(Fp); free(force); free(g); free(drho); free(js);
    return status;
}
