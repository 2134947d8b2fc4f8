/*
 * FP64 CPU oracle gradient of an MD trajectory loss (test infrastructure).
 *
 * TEST INFRASTRUCTURE ONLY: called from the tests and nowhere in the product
 * path; shares no code with the CUDA library.
 *
 * The paper (tinyMD) integrates Newton's equation (Sec. 3.2, Eq. 1) with the
 * LJ force of Sec. 3.2, Eq. 2; it does not differentiate trajectories.  This
 * file differentiates that same forward map, written out plainly:
 *
 *   forward step n -> n+1 (velocity Verlet, c = dt / (2 m)):
 *       vh      = v_n + c F(x_n)
 *       x_{n+1} = x_n + dt vh
 *       v_{n+1} = vh  + c F(x_{n+1})
 *   loss     = (1/W) sum_{n=S-W+1..S} PE(x_n)
 *
 *   reverse (adjoints ax = dLoss/dx, av = dLoss/dv, theta = (eps, sigma)):
 *       ax += dPE/dx(x_n)/W = -F(x_n)/W   and  g_theta += dPE/dtheta(x_n)/W
 *                                           when n is in the loss window
 *       av_h  = av;  ax += c J(x_{n+1}) av;  g_theta += c dF/dtheta(x_{n+1}) . av
 *       av_h += dt ax
 *       av    = av_h;  ax += c J(x_n) av_h;  g_theta += c dF/dtheta(x_n) . av_h
 *   where J = dF/dx is symmetric, so J^T u = J u.
 *
 * Pair derivatives (f is the scalar with F_i = sum_j f(r^2) d_ij, d = x_i - x_j):
 *   f      = 48 eps sr6 (sr6 - 1/2) sr2,          sr2 = 1/r^2, sr6 = sigma^6 sr2^3
 *   f'     = df/d(r^2) = 48 eps sr2^2 sr6 (2 - 7 sr6)
 *   (J u)_i = sum_j [ f (u_i - u_j) + 2 f' d (d . (u_i - u_j)) ]
 *   df/deps = f / eps,   df/dsigma = 144 eps sr2 sr6 (4 sr6 - 1) / sigma
 *   V      = 4 eps sr6 (sr6 - 1),  dV/deps = V / eps,
 *   dV/dsigma = 24 eps sr6 (2 sr6 - 1) / sigma
 * The cutoff rc is an absolute length held fixed; pairs crossing it are a
 * measure-zero set whose jump the gradient ignores.
 *
 * Parity unpinned: none.  Pinned by central finite differences of the
 * oracle's own forward loss (tests/test_oracle_adjoint.py) and by finite
 * differences of the oracle forces for the J u product.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double epsilon, sigma, mass, cutoff, skin, dt;
    int32_t rebuild_every;
    int32_t half;
    int32_t potential;      /* the adjoint covers Lennard-Jones (potential 0) only */
    int32_t pad_;
    double k_spring, gamma;
} orc_params;

/* From md_oracle.c */
int orc_cell_grid(const double L[3], double r, int32_t nc[3], double s[3]);
void orc_wrap(int64_t n, const double L[3], double *x);
void orc_bin(int64_t n, const double *x, const int32_t nc[3], const double s[3],
             int32_t *cell_of, int32_t *cell_start, int32_t *cell_atoms);
int32_t orc_neighbors_cells(int64_t n, const double *x, const double L[3], const int32_t nc[3],
                            const int32_t *cell_of, const int32_t *cell_start,
                            const int32_t *cell_atoms, double r, int32_t half, int32_t cap,
                            int32_t *counts, int32_t *list);
void orc_forces_list(int64_t n, const double *x, const double L[3], int32_t cap,
                     const int32_t *counts, const int32_t *list, const orc_params *p, double *F);
void orc_energy_list(int64_t n, const double *x, const double L[3], int32_t cap,
                     const int32_t *counts, const int32_t *list, const orc_params *p,
                     double *pe, double *virial, double *pe_atom);

static double mi(double dx, double L)
{
    double h = 0.5 * L;
    if (dx > h) dx = dx - L;
    else if (dx < -h) dx = dx + L;
    return dx;
}

/* A Verlet list (half: every pair once) owned by the adjoint. */
typedef struct {
    int64_t n;
    int32_t cap, nc[3];
    double s[3];
    int32_t *cell_of, *cell_start, *cell_atoms, *counts, *list;
} alist;

static int alist_init(alist *A, int64_t n, const double L[3], const orc_params *p)
{
    memset(A, 0, sizeof(*A));
    A->n = n;
    if (orc_cell_grid(L, p->cutoff + p->skin, A->nc, A->s)) return -1;
    int64_t ncell = (int64_t)A->nc[0] * A->nc[1] * A->nc[2];
    A->cap = 64;
    A->cell_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    A->cell_start = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncell + 1));
    A->cell_atoms = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    A->counts = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    A->list = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (size_t)A->cap);
    return (A->cell_of && A->cell_start && A->cell_atoms && A->counts && A->list) ? 0 : -2;
}

static void alist_free(alist *A)
{
    free(A->cell_of); free(A->cell_start); free(A->cell_atoms); free(A->counts); free(A->list);
}

/* Builds a half list for the (already wrapped) positions x. */
static int alist_build(alist *A, const double *x, const double L[3], const orc_params *p)
{
    orc_bin(A->n, x, A->nc, A->s, A->cell_of, A->cell_start, A->cell_atoms);
    for (;;) {
        int32_t m = orc_neighbors_cells(A->n, x, L, A->nc, A->cell_of, A->cell_start, A->cell_atoms,
                                        p->cutoff + p->skin, 1, A->cap, A->counts, A->list);
        if (m <= A->cap) return 0;
        A->cap = m + 16;
        free(A->list);
        A->list = (int32_t *)malloc(sizeof(int32_t) * (size_t)A->n * (size_t)A->cap);
        if (!A->list) return -2;
    }
}

/* out += scale * J(x) u over the pairs of a half list. */
static void pair_jvp(const alist *A, const double *x, const double L[3], const orc_params *p,
                     const double *u, double scale, double *out)
{
    double rc2 = p->cutoff * p->cutoff;
    double s2 = p->sigma * p->sigma;
    double sigma6 = s2 * s2 * s2;
    for (int64_t i = 0; i < A->n; i++)
        for (int32_t k = 0; k < A->counts[i]; k++) {
            int64_t j = A->list[i * A->cap + k];
            double d[3], du[3];
            for (int c = 0; c < 3; c++) {
                d[c] = mi(x[3 * i + c] - x[3 * j + c], L[c]);
                du[c] = u[3 * i + c] - u[3 * j + c];
            }
            double rsq = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
            if (!(rsq < rc2)) continue;
            double sr2 = 1.0 / rsq;
            double sr6 = sr2 * sr2 * sr2 * sigma6;
            double f = 48.0 * sr6 * (sr6 - 0.5) * sr2 * p->epsilon;
            double fp = 48.0 * p->epsilon * sr2 * sr2 * sr6 * (2.0 - 7.0 * sr6);
            double ddu = d[0] * du[0] + d[1] * du[1] + d[2] * du[2];
            for (int c = 0; c < 3; c++) {
                double t = f * du[c] + 2.0 * fp * d[c] * ddu;
                out[3 * i + c] += scale * t;
                out[3 * j + c] -= scale * t;
            }
        }
}

/* g[0] += scale * sum_i u_i . dF_i/deps, g[1] += scale * sum_i u_i . dF_i/dsigma */
static void pair_dforce_dtheta(const alist *A, const double *x, const double L[3],
                               const orc_params *p, const double *u, double scale, double g[2])
{
    double rc2 = p->cutoff * p->cutoff;
    double s2 = p->sigma * p->sigma;
    double sigma6 = s2 * s2 * s2;
    double ge = 0.0, gs = 0.0;
    for (int64_t i = 0; i < A->n; i++)
        for (int32_t k = 0; k < A->counts[i]; k++) {
            int64_t j = A->list[i * A->cap + k];
            double d[3], ddu = 0.0;
            for (int c = 0; c < 3; c++) d[c] = mi(x[3 * i + c] - x[3 * j + c], L[c]);
            double rsq = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
            if (!(rsq < rc2)) continue;
            for (int c = 0; c < 3; c++) ddu += d[c] * (u[3 * i + c] - u[3 * j + c]);
            double sr2 = 1.0 / rsq;
            double sr6 = sr2 * sr2 * sr2 * sigma6;
            double f = 48.0 * sr6 * (sr6 - 0.5) * sr2 * p->epsilon;
            ge += (f / p->epsilon) * ddu;
            gs += (144.0 * p->epsilon * sr2 * sr6 * (4.0 * sr6 - 1.0) / p->sigma) * ddu;
        }
    g[0] += scale * ge;
    g[1] += scale * gs;
}

/* g[0] += scale * dPE/deps, g[1] += scale * dPE/dsigma */
static void pair_dpe_dtheta(const alist *A, const double *x, const double L[3],
                            const orc_params *p, double scale, double g[2])
{
    double rc2 = p->cutoff * p->cutoff;
    double s2 = p->sigma * p->sigma;
    double sigma6 = s2 * s2 * s2;
    double ge = 0.0, gs = 0.0;
    for (int64_t i = 0; i < A->n; i++)
        for (int32_t k = 0; k < A->counts[i]; k++) {
            int64_t j = A->list[i * A->cap + k];
            double d[3];
            for (int c = 0; c < 3; c++) d[c] = mi(x[3 * i + c] - x[3 * j + c], L[c]);
            double rsq = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
            if (!(rsq < rc2)) continue;
            double sr2 = 1.0 / rsq;
            double sr6 = sr2 * sr2 * sr2 * sigma6;
            ge += 4.0 * sr6 * (sr6 - 1.0);
            gs += 24.0 * p->epsilon * sr6 * (2.0 * sr6 - 1.0) / p->sigma;
        }
    g[0] += scale * ge;
    g[1] += scale * gs;
}

/* J(x) u for tests: out = J u (out is overwritten). */
int orc_jvp(int64_t n, const double L[3], const orc_params *p, const double *x, const double *u,
            double *out)
{
    alist A;
    double *xw = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    if (!xw) return -2;
    memcpy(xw, x, sizeof(double) * 3 * (size_t)n);
    orc_wrap(n, L, xw);
    int rc = alist_init(&A, n, L, p);
    if (!rc) rc = alist_build(&A, xw, L, p);
    if (!rc) {
        memset(out, 0, sizeof(double) * 3 * (size_t)n);
        pair_jvp(&A, xw, L, p, u, 1.0, out);
    }
    alist_free(&A);
    free(xw);
    return rc;
}

/* Forward loss only (no storage); used by finite-difference pins. */
int orc_traj_loss(int64_t n, const double L[3], const orc_params *p, const double *x0,
                  const double *v0, int64_t nsteps, int64_t window, double *loss);

/* Loss and its gradient with respect to eps, sigma, x0 and v0.  Every
 * intermediate x_n is stored (this is the plain version: no checkpoints).
 * g_x0 / g_v0 may be NULL. */
int orc_adjoint(int64_t n, const double L[3], const orc_params *p, const double *x0,
                const double *v0, int64_t nsteps, int64_t window, double *loss,
                double *g_eps, double *g_sigma, double *g_x0, double *g_v0)
{
    size_t n3 = 3 * (size_t)n;
    orc_params ph = *p;
    ph.half = 1;
    double *X = (double *)malloc(sizeof(double) * n3 * (size_t)(nsteps + 1));
    double *v = (double *)malloc(sizeof(double) * n3);
    double *F = (double *)malloc(sizeof(double) * n3);
    double *ax = (double *)calloc(n3, sizeof(double));
    double *av = (double *)calloc(n3, sizeof(double));
    alist A;
    int rc = alist_init(&A, n, L, &ph);
    if (!X || !v || !F || !ax || !av || rc) {
        rc = rc ? rc : -2;
        goto done;
    }
    double c = 0.5 * p->dt / p->mass;
    int64_t every = p->rebuild_every > 0 ? p->rebuild_every : 1;

    /* Forward: store x_n (wrapped at rebuild steps). */
    memcpy(X, x0, sizeof(double) * n3);
    memcpy(v, v0, sizeof(double) * n3);
    orc_wrap(n, L, X);
    if ((rc = alist_build(&A, X, L, &ph))) goto done;
    orc_forces_list(n, X, L, A.cap, A.counts, A.list, &ph, F);
    double acc = 0.0;
    for (int64_t s = 1; s <= nsteps; s++) {
        double *xp = X + n3 * (size_t)(s - 1), *xn = X + n3 * (size_t)s;
        for (size_t t = 0; t < n3; t++) {
            v[t] += c * F[t];
            xn[t] = xp[t] + p->dt * v[t];
        }
        if (s % every == 0) {
            orc_wrap(n, L, xn);
            if ((rc = alist_build(&A, xn, L, &ph))) goto done;
        }
        orc_forces_list(n, xn, L, A.cap, A.counts, A.list, &ph, F);
        for (size_t t = 0; t < n3; t++) v[t] += c * F[t];
        if (s > nsteps - window) {
            double pe, w;
            orc_energy_list(n, xn, L, A.cap, A.counts, A.list, &ph, &pe, &w, NULL);
            acc += pe;
        }
    }
    *loss = acc / (double)window;

    /* Reverse sweep.  The list for x_s is the one built at the last rebuild
     * step r(s) = every * floor(s / every); it is rebuilt from the stored
     * (wrapped) X_r whenever the sweep enters a new block. */
    double g[2] = {0.0, 0.0};
    int64_t cur_block = -1;
    for (int64_t s = nsteps; s >= 1; s--) {
        double *xn = X + n3 * (size_t)s, *xp = X + n3 * (size_t)(s - 1);
        int64_t b = s / every;
        if (b != cur_block) {
            if ((rc = alist_build(&A, X + n3 * (size_t)(b * every), L, &ph))) goto done;
            cur_block = b;
        }
        if (s > nsteps - window) {                 /* loss term at x_s */
            orc_forces_list(n, xn, L, A.cap, A.counts, A.list, &ph, F);
            for (size_t t = 0; t < n3; t++) ax[t] -= F[t] / (double)window;
            pair_dpe_dtheta(&A, xn, L, &ph, 1.0 / (double)window, g);
        }
        /* v_s = vh + c F(x_s) */
        pair_jvp(&A, xn, L, &ph, av, c, ax);
        pair_dforce_dtheta(&A, xn, L, &ph, av, c, g);
        /* x_s = x_{s-1} + dt vh  (the wrap is a translation: derivative 1) */
        for (size_t t = 0; t < n3; t++) av[t] += p->dt * ax[t];
        /* vh = v_{s-1} + c F(x_{s-1}); x_{s-1} may belong to the previous block */
        int64_t bp = (s - 1) / every;
        if (bp != cur_block) {
            if ((rc = alist_build(&A, X + n3 * (size_t)(bp * every), L, &ph))) goto done;
            cur_block = bp;
        }
        pair_jvp(&A, xp, L, &ph, av, c, ax);
        pair_dforce_dtheta(&A, xp, L, &ph, av, c, g);
    }
    *g_eps = g[0];
    *g_sigma = g[1];
    if (g_x0) memcpy(g_x0, ax, sizeof(double) * n3);
    if (g_v0) memcpy(g_v0, av, sizeof(double) * n3);
    rc = 0;
done:
    alist_free(&A);
    free(X); free(v); free(F); free(ax); free(av);
    return rc;
}

/* ---------------------------------------------------------------------------
 * Forward loss, optionally recording or replaying the discrete structure of a
 * trajectory: the Verlet list of every rebuild and, for every force
 * evaluation, which listed pairs were inside rc.  Replaying the structure of
 * an unperturbed run gives the smooth branch of the loss through that run;
 * the unshifted cutoff makes the raw loss jump by V(rc)/W whenever a
 * perturbation moves a cutoff crossing to another step.
 * ------------------------------------------------------------------------- */

typedef struct {
    int64_t n, nsteps, every, nblocks;
    int32_t *cap;              /* per block */
    int32_t **counts, **list;  /* per block */
    uint8_t **mask;            /* per step s = 0..nsteps: one byte per list slot */
} orc_trace;

void orc_trace_free(orc_trace *T)
{
    if (!T) return;
    for (int64_t b = 0; b < T->nblocks; b++) {
        free(T->counts[b]);
        free(T->list[b]);
    }
    for (int64_t s = 0; s <= T->nsteps; s++) free(T->mask[s]);
    free(T->cap); free(T->counts); free(T->list); free(T->mask);
    free(T);
}

static orc_trace *trace_new(int64_t n, int64_t nsteps, int64_t every)
{
    orc_trace *T = (orc_trace *)calloc(1, sizeof(orc_trace));
    if (!T) return NULL;
    T->n = n;
    T->nsteps = nsteps;
    T->every = every;
    T->nblocks = nsteps / every + 1;
    T->cap = (int32_t *)calloc((size_t)T->nblocks, sizeof(int32_t));
    T->counts = (int32_t **)calloc((size_t)T->nblocks, sizeof(int32_t *));
    T->list = (int32_t **)calloc((size_t)T->nblocks, sizeof(int32_t *));
    T->mask = (uint8_t **)calloc((size_t)(nsteps + 1), sizeof(uint8_t *));
    if (!T->cap || !T->counts || !T->list || !T->mask) {
        orc_trace_free(T);
        return NULL;
    }
    return T;
}

/* Forces (and, when pe != NULL, the energy) of x over a half list.  mode 0:
 * plain cutoff test; 1: plain test, recorded into m; 2: replay m. */
static void masked_pass(int64_t n, const double *x, const double L[3], int32_t cap,
                        const int32_t *counts, const int32_t *list, const orc_params *p,
                        int mode, uint8_t *m, double *F, double *pe)
{
    double rc2 = p->cutoff * p->cutoff;
    double s2 = p->sigma * p->sigma;
    double sigma6 = s2 * s2 * s2;
    double e = 0.0;
    memset(F, 0, sizeof(double) * 3 * (size_t)n);
    for (int64_t i = 0; i < n; i++)
        for (int32_t k = 0; k < counts[i]; k++) {
            int64_t j = list[i * cap + k];
            double d[3];
            for (int c = 0; c < 3; c++) d[c] = mi(x[3 * i + c] - x[3 * j + c], L[c]);
            double rsq = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
            int in = (mode == 2) ? m[i * cap + k] : (rsq < rc2);
            if (mode == 1) m[i * cap + k] = (uint8_t)in;
            if (!in) continue;
            double sr2 = 1.0 / rsq;
            double sr6 = sr2 * sr2 * sr2 * sigma6;
            double f = 48.0 * sr6 * (sr6 - 0.5) * sr2 * p->epsilon;
            for (int c = 0; c < 3; c++) {
                F[3 * i + c] += f * d[c];
                F[3 * j + c] -= f * d[c];
            }
            e += 4.0 * p->epsilon * sr6 * (sr6 - 1.0);
        }
    if (pe) *pe = e;
}

/* mode 0: plain; 1: record into *trace (allocated here); 2: replay *trace. */
int orc_traj_loss_ex(int64_t n, const double L[3], const orc_params *p, const double *x0,
                     const double *v0, int64_t nsteps, int64_t window, double *loss,
                     int mode, orc_trace **trace)
{
    size_t n3 = 3 * (size_t)n;
    orc_params ph = *p;
    ph.half = 1;
    int64_t every = p->rebuild_every > 0 ? p->rebuild_every : 1;
    double *x = (double *)malloc(sizeof(double) * n3);
    double *v = (double *)malloc(sizeof(double) * n3);
    double *F = (double *)malloc(sizeof(double) * n3);
    orc_trace *T = NULL;
    alist A;
    int rc = alist_init(&A, n, L, &ph);
    if (!x || !v || !F || rc) {
        rc = rc ? rc : -2;
        goto done;
    }
    if (mode == 1) {
        T = trace_new(n, nsteps, every);
        if (!T) { rc = -2; goto done; }
    } else if (mode == 2) {
        T = *trace;
        if (!T || T->n != n || T->nsteps != nsteps || T->every != every) { rc = -3; goto done; }
    }
    memcpy(x, x0, sizeof(double) * n3);
    memcpy(v, v0, sizeof(double) * n3);
    double c = 0.5 * p->dt / p->mass;
    double acc = 0.0;
    int32_t cap = 0, *counts = NULL, *list = NULL;
    for (int64_t s = 0; s <= nsteps; s++) {
        if (s > 0)
            for (size_t t = 0; t < n3; t++) {
                v[t] += c * F[t];
                x[t] += p->dt * v[t];
            }
        if (s % every == 0) {
            int64_t b = s / every;
            orc_wrap(n, L, x);
            if (mode == 2) {
                cap = T->cap[b]; counts = T->counts[b]; list = T->list[b];
            } else {
                if ((rc = alist_build(&A, x, L, &ph))) goto done;
                cap = A.cap; counts = A.counts; list = A.list;
                if (mode == 1) {
                    T->cap[b] = cap;
                    T->counts[b] = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
                    T->list[b] = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (size_t)cap);
                    if (!T->counts[b] || !T->list[b]) { rc = -2; goto done; }
                    memcpy(T->counts[b], counts, sizeof(int32_t) * (size_t)n);
                    memcpy(T->list[b], list, sizeof(int32_t) * (size_t)n * (size_t)cap);
                }
            }
        }
        uint8_t *m = NULL;
        if (mode == 1) {
            T->mask[s] = (uint8_t *)calloc((size_t)n * (size_t)cap, 1);
            if (!T->mask[s]) { rc = -2; goto done; }
        }
        if (mode) m = T->mask[s];
        double pe = 0.0;
        int want = s > nsteps - window;
        masked_pass(n, x, L, cap, counts, list, &ph, mode, m, F, want ? &pe : NULL);
        if (s > 0) {
            for (size_t t = 0; t < n3; t++) v[t] += c * F[t];
            if (want) acc += pe;
        }
    }
    *loss = acc / (double)window;
    if (mode == 1) { *trace = T; T = NULL; }
    rc = 0;
done:
    if (mode == 1 && T) orc_trace_free(T);
    alist_free(&A);
    free(x); free(v); free(F);
    return rc;
}

int orc_traj_loss(int64_t n, const double L[3], const orc_params *p, const double *x0,
                  const double *v0, int64_t nsteps, int64_t window, double *loss)
{
    return orc_traj_loss_ex(n, L, p, x0, v0, nsteps, window, loss, 0, NULL);
}
