/*
 * FP64 CPU oracle for short-range Lennard-Jones 12-6 molecular dynamics.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this
 * file; only the tests, the smoke check and the benchmark's CPU-baseline leg
 * use it.  It shares no code, header, table or constant with the CUDA
 * library.  It is deliberately plain and slow: every loop is written in the
 * order the method states it, so a reader can check it against the paper
 * (tinyMD, Machado et al., arXiv 2009.07400) by eye.
 *
 * What it follows:
 *   - Sec. 3.2, Eq. 1: positions and velocities come from integrating
 *     F = m a.  The integrator is velocity Verlet (kick-drift-kick).
 *   - Sec. 3.2, Eq. 2: the 12-6 pair force, evaluated in the operation order
 *     of the potential kernel in Sec. 4.2:
 *         sr2 = 1/rsq; sr6 = sr2*sr2*sr2*sigma^6;
 *         f = 48*sr6*(sr6-0.5)*sr2*epsilon;  F_i += f * del,
 *     with del = x_i - x_j and the strict cutoff test rsq < rc^2.
 *   - Sec. 3.2 (commented potential beside Eq. 2): V = 4 eps [(s/r)^12 -
 *     (s/r)^6], truncated at rc and not shifted.
 *   - Sec. 3.2, Fig. 1: Verlet lists with a buffer ("skin"), built from cell
 *     lists whose cell side is >= r = rc + skin, scanning the neighbour
 *     cells; half lists store each pair once (Newton's third law).
 *   - Sec. 3.2: periodic boundaries in every direction, realised here as the
 *     minimum-image convention on one box (valid while L >= 2 (rc+skin)).
 *   - Sec. 6: reneighbouring every 20 steps, dt = 0.005, rc = 2.5, skin 0.3.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - the minimum image uses one branch per component,
 *       if dx > L/2: dx -= L  else if dx < -L/2: dx += L;
 *   - r^2 is ((dx*dx + dy*dy) + dz*dz), each operation rounded (compiled
 *     with -ffp-contract=off), compared strictly with (rc+skin)^2;
 *   - wrapping into the box at a rebuild is one conditional +/-L per
 *     component; an atom that rounds onto x == L keeps that coordinate and
 *     is put in the last cell;
 *   - cells per dimension nc = floor(L / (rc+skin)), side s = L / nc,
 *     cell coordinate c = (int)(x / s) clamped to nc-1, linear id
 *     (cx*nc_y + cy)*nc_z + cz;
 *   - binning is a stable counting sort (atoms of a cell in ascending id);
 *   - when nc < 3 the 27 neighbour cells are de-duplicated;
 *   - a half list keeps pair (i,j) in row i iff j's nearest image lies in
 *     i's upper half-space: del = x_i - x_j (minimum image) has del.z < 0,
 *     or del.z == 0 and del.y < 0, or both zero and del.x < 0, or del == 0
 *     and j > i (del of the pair seen from j is exactly -del, so each pair
 *     is kept once, and every row holds about half of its neighbours);
 *   - rebuild after the drift of step n iff n % rebuild_every == 0, plus an
 *     initial build at step 0; rebuild_every == 0 instead rebuilds after any
 *     drift that leaves some atom more than skin/2 from where it was at the
 *     last build (the condition under which a list built with the skin still
 *     holds every pair inside rc, Sec. 3.2, Fig. 1);
 *   - KE = 1/2 m sum v^2, W = sum over pairs of f*r^2 (= sum r_ij . F_ij).
 *
 * Spring-dashpot contact (Sec. 3.2, Eq. 3; potential = 1): spheres of
 * diameter sigma, for |x_ij| < sigma (strict)
 *     F_i += K xi + gamma xi_dot,   xi = xhat (sigma - r),
 *     xi_dot = -xhat (xhat . v_ij),  xhat = x_ij / r,  r = |x_ij|,
 * with x_ij = x_i - x_j (minimum image) and v_ij = v_i - v_j.  Readings:
 * v_ij is the relative velocity of i to j; in velocity Verlet the force
 * after the drift uses the half-step velocities (the latest ones), i.e. the
 * integrator stays explicit; the elastic energy is 1/2 K (sigma - r)^2 per
 * overlapping pair; W = sum over pairs of x_ij . F_ij (dashpot included).
 * The list radius is cutoff + skin, so cutoff >= sigma.
 *
 * Parity unpinned: none of the functions here.  Each is pinned by a test
 * against closed forms, textbook lattice sums, brute force, conservation
 * laws or finite differences (tests/test_oracle_*.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* Physical and algorithmic parameters of one system. */
typedef struct {
    double epsilon, sigma, mass, cutoff, skin, dt;
    int32_t rebuild_every;
    int32_t half;
    int32_t potential;      /* 0: Lennard-Jones (Eq. 2); 1: spring-dashpot (Eq. 3) */
    int32_t pad_;
    double k_spring, gamma; /* Eq. 3: K and the dissipation constant; sigma is the diameter */
} orc_params;

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads for the following parallel loops (timing runs only). */
void orc_set_num_threads(int k)
{
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}

/* ---------------------------------------------------------------------------
 * Geometry
 * ------------------------------------------------------------------------- */

/* Cell grid of Sec. 3.2 / Fig. 1: side >= r = rc + skin.  Returns -1 when the
 * box is smaller than 2 r in some dimension (minimum image would be wrong). */
int orc_cell_grid(const double L[3], double r, int32_t nc[3], double s[3])
{
    for (int d = 0; d < 3; d++) {
        if (!(L[d] >= 2.0 * r)) return -1;
        nc[d] = (int32_t)floor(L[d] / r);
        s[d] = L[d] / (double)nc[d];
    }
    return 0;
}

/* Wrap every coordinate into [0, L] with one conditional shift. */
void orc_wrap(int64_t n, const double L[3], double *x)
{
    for (int64_t i = 0; i < n; i++)
        for (int d = 0; d < 3; d++) {
            double c = x[3 * i + d];
            if (c < 0.0) c = c + L[d];
            else if (c >= L[d]) c = c - L[d];
            x[3 * i + d] = c;
        }
}

static int32_t cell_coord(double c, double s, int32_t nc)
{
    int32_t k = (int32_t)(c / s);
    if (k >= nc) k = nc - 1;
    if (k < 0) k = 0;
    return k;
}

/* Stable counting sort of atoms into cells.
 * cell_of[n], cell_start[ncell+1], cell_atoms[n]. */
void orc_bin(int64_t n, const double *x, const int32_t nc[3], const double s[3],
             int32_t *cell_of, int32_t *cell_start, int32_t *cell_atoms)
{
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    for (int64_t c = 0; c <= ncell; c++) cell_start[c] = 0;
    for (int64_t i = 0; i < n; i++) {
        int32_t cx = cell_coord(x[3 * i + 0], s[0], nc[0]);
        int32_t cy = cell_coord(x[3 * i + 1], s[1], nc[1]);
        int32_t cz = cell_coord(x[3 * i + 2], s[2], nc[2]);
        cell_of[i] = (cx * nc[1] + cy) * nc[2] + cz;
        cell_start[cell_of[i] + 1] += 1;           /* histogram */
    }
    for (int64_t c = 0; c < ncell; c++)            /* exclusive scan */
        cell_start[c + 1] += cell_start[c];
    int32_t *cursor = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncell > 0 ? ncell : 1));
    for (int64_t c = 0; c < ncell; c++) cursor[c] = cell_start[c];
    for (int64_t i = 0; i < n; i++)                /* stable scatter */
        cell_atoms[cursor[cell_of[i]]++] = (int32_t)i;
    free(cursor);
}

/* Minimum-image displacement component. */
static double min_image(double dx, double L)
{
    double h = 0.5 * L;
    if (dx > h) dx = dx - L;
    else if (dx < -h) dx = dx + L;
    return dx;
}

static void displacement(const double *x, int64_t i, int64_t j, const double L[3], double del[3])
{
    for (int d = 0; d < 3; d++)
        del[d] = min_image(x[3 * i + d] - x[3 * j + d], L[d]);
}

/* Half-list ownership of the pair (i, j) with displacement del = x_i - x_j
 * (minimum image): j's image in i's upper half-space (header comment). */
static int half_owner(const double del[3], int64_t i, int64_t j)
{
    if (del[2] != 0.0) return del[2] < 0.0;
    if (del[1] != 0.0) return del[1] < 0.0;
    if (del[0] != 0.0) return del[0] < 0.0;
    return j > i;
}

static double norm2(const double del[3])
{
    double a = del[0] * del[0];
    double b = del[1] * del[1];
    double c = del[2] * del[2];
    return (a + b) + c;
}

/* ---------------------------------------------------------------------------
 * Verlet lists (Sec. 3.2, Fig. 1).  Row-major output: row i holds counts[i]
 * ids in list[i*cap ...].  Entries beyond cap are counted but not stored.
 * Return value: the largest count seen (caller compares with cap).
 * ------------------------------------------------------------------------- */

int32_t orc_neighbors_brute(int64_t n, const double *x, const double L[3], double r,
                            int32_t half, int32_t cap, int32_t *counts, int32_t *list)
{
    double r2 = r * r;
    int32_t maxc = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(max : maxc)
    for (int64_t i = 0; i < n; i++) {
        int32_t k = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double del[3];
            displacement(x, i, j, L, del);
            if (norm2(del) < r2) {
                if (half && !half_owner(del, i, j)) continue;
                if (k < cap) list[i * cap + k] = (int32_t)j;
                k++;
            }
        }
        counts[i] = k;
        if (k > maxc) maxc = k;
    }
    return maxc;
}

/* Distinct neighbour cells (including the cell itself) of cell (cx,cy,cz);
 * with nc < 3 several of the 27 offsets name the same cell, which is kept
 * once.  Returns how many were written to out[27]. */
static int neighbour_cells(int32_t cx, int32_t cy, int32_t cz, const int32_t nc[3], int64_t out[27])
{
    int m = 0;
    for (int ox = -1; ox <= 1; ox++)
        for (int oy = -1; oy <= 1; oy++)
            for (int oz = -1; oz <= 1; oz++) {
                int32_t a = (cx + ox + nc[0]) % nc[0];
                int32_t b = (cy + oy + nc[1]) % nc[1];
                int32_t c = (cz + oz + nc[2]) % nc[2];
                int64_t id = ((int64_t)a * nc[1] + b) * nc[2] + c;
                int seen = 0;
                for (int q = 0; q < m; q++)
                    if (out[q] == id) seen = 1;
                if (!seen) out[m++] = id;
            }
    return m;
}

int32_t orc_neighbors_cells(int64_t n, const double *x, const double L[3], const int32_t nc[3],
                            const int32_t *cell_of, const int32_t *cell_start,
                            const int32_t *cell_atoms, double r, int32_t half, int32_t cap,
                            int32_t *counts, int32_t *list)
{
    double r2 = r * r;
    int32_t maxc = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(max : maxc)
    for (int64_t i = 0; i < n; i++) {
        int32_t ci = cell_of[i];
        int32_t cz = ci % nc[2];
        int32_t cy = (ci / nc[2]) % nc[1];
        int32_t cx = ci / (nc[2] * nc[1]);
        int64_t cells[27];
        int m = neighbour_cells(cx, cy, cz, nc, cells);
        int32_t k = 0;
        for (int q = 0; q < m; q++) {
            for (int32_t t = cell_start[cells[q]]; t < cell_start[cells[q] + 1]; t++) {
                int64_t j = cell_atoms[t];
                if (j == i) continue;
                double del[3];
                displacement(x, i, j, L, del);
                if (norm2(del) < r2) {
                    if (half && !half_owner(del, i, j)) continue;
                    if (k < cap) list[i * cap + k] = (int32_t)j;
                    k++;
                }
            }
        }
        counts[i] = k;
        if (k > maxc) maxc = k;
    }
    return maxc;
}

/* Full Verlet rows of the m atoms ids[] only (the criterion and candidate
 * order of orc_neighbors_cells), for checks on systems too large to list
 * whole: counts[q] and list[q * cap ...] for atom ids[q]; returns the
 * longest row. */
int32_t orc_neighbors_sample(int64_t n, const double *x, const double L[3], const int32_t nc[3],
                             const int32_t *cell_of, const int32_t *cell_start,
                             const int32_t *cell_atoms, double r, int64_t m, const int64_t *ids,
                             int32_t cap, int32_t *counts, int32_t *list)
{
    double r2 = r * r;
    int32_t maxc = 0;
    (void)n;
#pragma omp parallel for schedule(dynamic, 16) reduction(max : maxc)
    for (int64_t q = 0; q < m; q++) {
        int64_t i = ids[q];
        int32_t ci = cell_of[i];
        int32_t cz = ci % nc[2];
        int32_t cy = (ci / nc[2]) % nc[1];
        int32_t cx = ci / (nc[2] * nc[1]);
        int64_t cells[27];
        int mc = neighbour_cells(cx, cy, cz, nc, cells);
        int32_t k = 0;
        for (int c = 0; c < mc; c++)
            for (int32_t t = cell_start[cells[c]]; t < cell_start[cells[c] + 1]; t++) {
                int64_t j = cell_atoms[t];
                if (j == i) continue;
                double del[3];
                displacement(x, i, j, L, del);
                if (norm2(del) < r2) {
                    if (k < cap) list[q * cap + k] = (int32_t)j;
                    k++;
                }
            }
        counts[q] = k;
        if (k > maxc) maxc = k;
    }
    return maxc;
}

/* ---------------------------------------------------------------------------
 * Pair terms (Sec. 3.2 Eq. 2 in the operation order of the Sec. 4.2 kernel).
 * ------------------------------------------------------------------------- */

/* Scalar f with F_i = f * del for one pair at squared distance rsq. */
static double lj_f(double rsq, double epsilon, double sigma6)
{
    double sr2 = 1.0 / rsq;
    double sr6 = sr2 * sr2 * sr2 * sigma6;
    return 48.0 * sr6 * (sr6 - 0.5) * sr2 * epsilon;
}

/* Pair energy 4 eps [(s/r)^12 - (s/r)^6], unshifted. */
static double lj_v(double rsq, double epsilon, double sigma6)
{
    double sr2 = 1.0 / rsq;
    double sr6 = sr2 * sr2 * sr2 * sigma6;
    return 4.0 * epsilon * sr6 * (sr6 - 1.0);
}

static double pow6(double a) { double a2 = a * a; return a2 * a2 * a2; }

/* Forces over a Verlet list.  Full list: row i sums over its entries.
 * Half list: each stored pair updates i (+) and j (-). */
void orc_forces_list(int64_t n, const double *x, const double L[3], int32_t cap,
                     const int32_t *counts, const int32_t *list, const orc_params *p, double *F)
{
    double rc2 = p->cutoff * p->cutoff;
    double sigma6 = pow6(p->sigma);
    if (!p->half) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++) {
            double fi[3] = {0.0, 0.0, 0.0};
            for (int32_t k = 0; k < counts[i]; k++) {
                int64_t j = list[i * cap + k];
                double del[3];
                displacement(x, i, j, L, del);
                double rsq = norm2(del);
                if (rsq < rc2) {
                    double f = lj_f(rsq, p->epsilon, sigma6);
                    for (int d = 0; d < 3; d++) fi[d] += f * del[d];
                }
            }
            for (int d = 0; d < 3; d++) F[3 * i + d] = fi[d];
        }
        return;
    }
    for (int64_t t = 0; t < 3 * n; t++) F[t] = 0.0;
    for (int64_t i = 0; i < n; i++)
        for (int32_t k = 0; k < counts[i]; k++) {
            int64_t j = list[i * cap + k];
            double del[3];
            displacement(x, i, j, L, del);
            double rsq = norm2(del);
            if (rsq < rc2) {
                double f = lj_f(rsq, p->epsilon, sigma6);
                for (int d = 0; d < 3; d++) {
                    F[3 * i + d] += f * del[d];
                    F[3 * j + d] -= f * del[d];
                }
            }
        }
}

/* The plain definition: F_i = sum over all j != i within rc (minimum image). */
void orc_forces_brute(int64_t n, const double *x, const double L[3], const orc_params *p, double *F)
{
    double rc2 = p->cutoff * p->cutoff;
    double sigma6 = pow6(p->sigma);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        double fi[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double del[3];
            displacement(x, i, j, L, del);
            double rsq = norm2(del);
            if (rsq < rc2) {
                double f = lj_f(rsq, p->epsilon, sigma6);
                for (int d = 0; d < 3; d++) fi[d] += f * del[d];
            }
        }
        for (int d = 0; d < 3; d++) F[3 * i + d] = fi[d];
    }
}

/* Forces on a subset of atoms only (sampled parity at sizes too large for a
 * full oracle pass): plain definition restricted to candidates found through
 * the cell list of a binned configuration. */
void orc_forces_sample(int64_t n, const double *x, const double L[3], const int32_t nc[3],
                       const int32_t *cell_of, const int32_t *cell_start, const int32_t *cell_atoms,
                       const orc_params *p, int64_t m, const int64_t *ids, double *F)
{
    double rc2 = p->cutoff * p->cutoff;
    double sigma6 = pow6(p->sigma);
    (void)n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < m; q++) {
        int64_t i = ids[q];
        int32_t ci = cell_of[i];
        int32_t cz = ci % nc[2];
        int32_t cy = (ci / nc[2]) % nc[1];
        int32_t cx = ci / (nc[2] * nc[1]);
        int64_t cells[27];
        int mc = neighbour_cells(cx, cy, cz, nc, cells);
        double fi[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < mc; c++)
            for (int32_t t = cell_start[cells[c]]; t < cell_start[cells[c] + 1]; t++) {
                int64_t j = cell_atoms[t];
                if (j == i) continue;
                double del[3];
                displacement(x, i, j, L, del);
                double rsq = norm2(del);
                if (rsq < rc2) {
                    double f = lj_f(rsq, p->epsilon, sigma6);
                    for (int d = 0; d < 3; d++) fi[d] += f * del[d];
                }
            }
        for (int d = 0; d < 3; d++) F[3 * q + d] = fi[d];
    }
}

/* Potential energy and pair virial over a Verlet list, each pair once.
 * For a full list a pair appears in both rows; it is taken from row i with
 * j > i.  Per-atom energies (half of each pair to each atom) are written to
 * pe_atom when it is not NULL. */
void orc_energy_list(int64_t n, const double *x, const double L[3], int32_t cap,
                     const int32_t *counts, const int32_t *list, const orc_params *p,
                     double *pe, double *virial, double *pe_atom)
{
    double rc2 = p->cutoff * p->cutoff;
    double sigma6 = pow6(p->sigma);
    double e = 0.0, w = 0.0;
    if (pe_atom)
        for (int64_t i = 0; i < n; i++) pe_atom[i] = 0.0;
    for (int64_t i = 0; i < n; i++)
        for (int32_t k = 0; k < counts[i]; k++) {
            int64_t j = list[i * cap + k];
            if (!p->half && j < i) continue;
            double del[3];
            displacement(x, i, j, L, del);
            double rsq = norm2(del);
            if (rsq < rc2) {
                double v = lj_v(rsq, p->epsilon, sigma6);
                e += v;
                w += lj_f(rsq, p->epsilon, sigma6) * rsq;
                if (pe_atom) {
                    pe_atom[i] += 0.5 * v;
                    pe_atom[j] += 0.5 * v;
                }
            }
        }
    *pe = e;
    *virial = w;
}

/* Per-atom split of the potential energy and pair virial over a list (each
 * pair's V and f r^2 shared half and half by its two atoms); the sums of the
 * two arrays are the totals of orc_energy_list. */
void orc_energy_atoms(int64_t n, const double *x, const double L[3], int32_t cap,
                      const int32_t *counts, const int32_t *list, const orc_params *p,
                      double *pe_atom, double *w_atom)
{
    double rc2 = p->cutoff * p->cutoff;
    double sigma6 = pow6(p->sigma);
    for (int64_t i = 0; i < n; i++) {
        pe_atom[i] = 0.0;
        w_atom[i] = 0.0;
    }
    for (int64_t i = 0; i < n; i++)
        for (int32_t k = 0; k < counts[i]; k++) {
            int64_t j = list[i * cap + k];
            if (!p->half && j < i) continue;
            double del[3];
            displacement(x, i, j, L, del);
            double rsq = norm2(del);
            if (rsq < rc2) {
                double v = lj_v(rsq, p->epsilon, sigma6);
                double w = lj_f(rsq, p->epsilon, sigma6) * rsq;
                pe_atom[i] += 0.5 * v;
                pe_atom[j] += 0.5 * v;
                w_atom[i] += 0.5 * w;
                w_atom[j] += 0.5 * w;
            }
        }
}

/* Eq. 3 for one pair: adds the force on i to fi, returns 1 if in contact
 * (and then the pair's elastic energy and x_ij . F_ij through pe, w). */
static int sd_pair(const double del[3], const double vij[3], const orc_params *p, double fi[3],
                   double *pe, double *w)
{
    double rsq = norm2(del);
    if (!(rsq < p->sigma * p->sigma)) return 0;
    double r = sqrt(rsq);
    double xhat[3] = {del[0] / r, del[1] / r, del[2] / r};
    double vn = xhat[0] * vij[0] + xhat[1] * vij[1] + xhat[2] * vij[2];
    double overlap = p->sigma - r;
    double f[3];
    for (int d = 0; d < 3; d++) {
        double xi = xhat[d] * overlap;
        double xi_dot = -xhat[d] * vn;
        f[d] = p->k_spring * xi + p->gamma * xi_dot;
        fi[d] += f[d];
    }
    *pe = 0.5 * p->k_spring * overlap * overlap;
    *w = del[0] * f[0] + del[1] * f[1] + del[2] * f[2];
    return 1;
}

/* Spring-dashpot forces over a full list (each row holds every j within
 * the list radius of i). */
void orc_forces_sd_list(int64_t n, const double *x, const double *v, const double L[3],
                        int32_t cap, const int32_t *counts, const int32_t *list,
                        const orc_params *p, double *F)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double fi[3] = {0.0, 0.0, 0.0};
        for (int32_t k = 0; k < counts[i]; k++) {
            int64_t j = list[i * cap + k];
            double del[3], vij[3], pe, w;
            displacement(x, i, j, L, del);
            for (int d = 0; d < 3; d++) vij[d] = v[3 * i + d] - v[3 * j + d];
            sd_pair(del, vij, p, fi, &pe, &w);
        }
        for (int d = 0; d < 3; d++) F[3 * i + d] = fi[d];
    }
}

/* The plain definition of Eq. 3: every j != i (minimum image). */
void orc_forces_sd_brute(int64_t n, const double *x, const double *v, const double L[3],
                         const orc_params *p, double *F)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        double fi[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double del[3], vij[3], pe, w;
            displacement(x, i, j, L, del);
            for (int d = 0; d < 3; d++) vij[d] = v[3 * i + d] - v[3 * j + d];
            sd_pair(del, vij, p, fi, &pe, &w);
        }
        for (int d = 0; d < 3; d++) F[3 * i + d] = fi[d];
    }
}

/* Elastic energy and virial over a full list (each pair counted from both
 * sides, halved); per-atom values (half of each pair) when pe_atom != NULL. */
void orc_energy_sd_list(int64_t n, const double *x, const double *v, const double L[3],
                        int32_t cap, const int32_t *counts, const int32_t *list,
                        const orc_params *p, double *pe_out, double *w_out, double *pe_atom)
{
    double pe_t = 0.0, w_t = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double pi = 0.0;
        for (int32_t k = 0; k < counts[i]; k++) {
            int64_t j = list[i * cap + k];
            double del[3], vij[3], pe, w, fi[3] = {0.0, 0.0, 0.0};
            displacement(x, i, j, L, del);
            for (int d = 0; d < 3; d++) vij[d] = v[3 * i + d] - v[3 * j + d];
            if (sd_pair(del, vij, p, fi, &pe, &w)) {
                pi += 0.5 * pe;
                w_t += 0.5 * w;
            }
        }
        pe_t += pi;
        if (pe_atom) pe_atom[i] = pi;
    }
    *pe_out = pe_t;
    *w_out = w_t;
}

double orc_kinetic(int64_t n, const double *v, double mass)
{
    double s = 0.0;
    for (int64_t t = 0; t < 3 * n; t++) s += v[t] * v[t];
    return 0.5 * mass * s;
}

/* Thermodynamic outputs of one (PE, KE, W) record of an n-atom periodic box
 * of volume vol: the temperature with the centre-of-mass momentum removed,
 * T = 2 KE / (3n - 3), and the virial pressure P = (n T + W / 3) / vol.  Not
 * printed in the paper (its outputs are forces and energies); these are the
 * textbook definitions for a pair potential in a periodic box.  n = 1 has
 * no free degree: T = P = 0. */
void orc_thermo(double pe, double ke, double w, int64_t n, double vol, double out[6])
{
    const double t = n > 1 ? 2.0 * ke / (3.0 * (double)n - 3.0) : 0.0;
    out[0] = pe;
    out[1] = ke;
    out[2] = pe + ke;
    out[3] = w;
    out[4] = t;
    out[5] = n > 1 ? ((double)n * t + w / 3.0) / vol : 0.0;
}

/* ---------------------------------------------------------------------------
 * Velocity Verlet with the fixed rebuild schedule (Sec. 3.2 Eq. 1, Sec. 6).
 * ------------------------------------------------------------------------- */

typedef struct {
    int64_t n;
    double L[3];
    orc_params p;
    int32_t nc[3];
    double s[3];
    int32_t cap;
    int32_t *cell_of, *cell_start, *cell_atoms, *counts, *list;
} orc_sim;

static void sim_free(orc_sim *S)
{
    free(S->cell_of); free(S->cell_start); free(S->cell_atoms);
    free(S->counts); free(S->list);
}

/* Wrap, bin and build the list; grows cap until every row fits. */
static int sim_rebuild(orc_sim *S, double *x)
{
    orc_wrap(S->n, S->L, x);
    orc_bin(S->n, x, S->nc, S->s, S->cell_of, S->cell_start, S->cell_atoms);
    for (;;) {
        double r = S->p.cutoff + S->p.skin;
        int32_t m = orc_neighbors_cells(S->n, x, S->L, S->nc, S->cell_of, S->cell_start,
                                        S->cell_atoms, r, S->p.half, S->cap, S->counts, S->list);
        if (m <= S->cap) return 0;
        S->cap = m + 16;
        free(S->list);
        S->list = (int32_t *)malloc(sizeof(int32_t) * (size_t)S->n * (size_t)S->cap);
        if (!S->list) return -2;
    }
}

static int sim_init(orc_sim *S, int64_t n, const double L[3], const orc_params *p)
{
    memset(S, 0, sizeof(*S));
    S->n = n;
    S->p = *p;
    for (int d = 0; d < 3; d++) S->L[d] = L[d];
    if (orc_cell_grid(L, p->cutoff + p->skin, S->nc, S->s) != 0) return -1;
    int64_t ncell = (int64_t)S->nc[0] * S->nc[1] * S->nc[2];
    S->cap = 64;
    S->cell_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    S->cell_start = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncell + 1));
    S->cell_atoms = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    S->counts = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    S->list = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (size_t)S->cap);
    if (!S->cell_of || !S->cell_start || !S->cell_atoms || !S->counts || !S->list) {
        sim_free(S);
        return -2;
    }
    return 0;
}

/* Runs nsteps velocity-Verlet steps starting after step `step0` (so the
 * first step taken is step0+1).  x, v are updated in place; F holds the
 * forces of the final positions.  When energies is not NULL it receives
 * (PE, KE, W) after every step, 3*nsteps doubles.  Positions are wrapped
 * only at rebuilds.  Returns 0, -1 (box too small) or -2 (out of memory). */
int orc_vv_run(int64_t n, const double L[3], const orc_params *p, double *x, double *v,
               double *F, int64_t step0, int64_t nsteps, double *energies)
{
    orc_sim S;
    int rc = sim_init(&S, n, L, p);
    if (rc) return rc;
    if ((rc = sim_rebuild(&S, x))) { sim_free(&S); return rc; }
    /* displacement trigger: positions at the last build */
    double *xref = NULL;
    if (p->rebuild_every == 0) {
        xref = (double *)malloc(sizeof(double) * 3 * (size_t)n);
        if (!xref) { sim_free(&S); return -2; }
        memcpy(xref, x, sizeof(double) * 3 * (size_t)n);
    }
    const int sd = p->potential == 1;
    if (sd) orc_forces_sd_list(n, x, v, S.L, S.cap, S.counts, S.list, p, F);
    else orc_forces_list(n, x, S.L, S.cap, S.counts, S.list, p, F);
    double half_dt_m = 0.5 * p->dt / p->mass;
    for (int64_t q = 1; q <= nsteps; q++) {
        int64_t step = step0 + q;
        for (int64_t t = 0; t < 3 * n; t++) {
            v[t] += half_dt_m * F[t];
            x[t] += p->dt * v[t];
        }
        int rebuild = 0;
        if (p->rebuild_every > 0) {
            rebuild = step % p->rebuild_every == 0;
        } else {
            double h = 0.5 * p->skin, m2 = 0.0;
            for (int64_t i = 0; i < n; i++) {
                double d2 = 0.0;
                for (int k = 0; k < 3; k++) {
                    double d = x[3 * i + k] - xref[3 * i + k];
                    d2 += d * d;
                }
                if (d2 > m2) m2 = d2;
            }
            rebuild = m2 > h * h;
        }
        if (rebuild) {
            if ((rc = sim_rebuild(&S, x))) { sim_free(&S); free(xref); return rc; }
            if (xref) memcpy(xref, x, sizeof(double) * 3 * (size_t)n);
        }
        /* Eq. 3's dashpot reads the half-step velocities held in v here */
        if (sd) orc_forces_sd_list(n, x, v, S.L, S.cap, S.counts, S.list, p, F);
        else orc_forces_list(n, x, S.L, S.cap, S.counts, S.list, p, F);
        for (int64_t t = 0; t < 3 * n; t++) v[t] += half_dt_m * F[t];
        if (energies) {
            double pe, w;
            if (sd) orc_energy_sd_list(n, x, v, S.L, S.cap, S.counts, S.list, p, &pe, &w, NULL);
            else orc_energy_list(n, x, S.L, S.cap, S.counts, S.list, p, &pe, &w, NULL);
            energies[3 * (q - 1) + 0] = pe;
            energies[3 * (q - 1) + 1] = orc_kinetic(n, v, p->mass);
            energies[3 * (q - 1) + 2] = w;
        }
    }
    sim_free(&S);
    free(xref);
    return 0;
}
