/*
 * md.h — C ABI of the GB300 short-range Lennard-Jones MD hot path.
 *
 * The operations follow tinyMD (Machado et al., arXiv 2009.07400):
 *   - Sec. 3.2, Eq. 1: positions and velocities are advanced by integrating
 *     F = m a (here: velocity Verlet, kick-drift-kick);
 *   - Sec. 3.2, Eq. 2: the 12-6 pair force, in the operation order of the
 *     potential kernel shown in Sec. 4.2 (sr2 = 1/r^2, sr6 = sr2^3 sigma^6,
 *     f = 48 eps sr6 (sr6 - 1/2) sr2, F_i += f (x_i - x_j)), strict cutoff
 *     test r^2 < rc^2;
 *   - Sec. 3.2, Fig. 1: Verlet lists with a buffer (skin) built from cell
 *     lists whose side is >= rc + skin; full or half lists (Sec. 3.2 and the
 *     half_nb specialisation of Sec. 4.2);
 *   - Sec. 3.2: periodic boundaries in all directions;
 *   - Sec. 4.2: neighbour-major list layout on GPUs (the k-th neighbours of
 *     consecutive atoms are contiguous);
 *   - Sec. 6: cells and lists rebuilt every 20 steps, dt = 0.005, rc = 2.5,
 *     skin 0.3, FP64.
 *
 * Conventions shared by every call:
 *   - A context owns all device memory it uses; it is created on the CUDA
 *     device that is current at md_create*, and every later call must be
 *     made with that device current.  A context is not thread-safe.
 *   - Host arrays passed in are copied; the caller keeps ownership.  Output
 *     arrays are caller-allocated.  Positions, velocities and forces cross
 *     the ABI as n x 3 row-major double arrays in the caller's atom order
 *     (the library reorders atoms internally by cell and maps back).
 *   - Work is enqueued on the context's stream.  Calls that return data to
 *     the host (md_energy, md_get_*) synchronise that stream; md_run
 *     synchronises once at its end to check the device error word.
 *   - Every call returns MD_OK (0) or a negative MD_ERR_* code; the text of
 *     the last error is available from md_last_error.  After MD_ERR_CUDA the
 *     context should be destroyed.
 *   - No global state: several contexts may coexist.
 */
#ifndef MD_GB300_H
#define MD_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MD_OK 0
#define MD_ERR_INVAL (-1)          /* bad argument (null pointer, n <= 0, bad phase ...) */
#define MD_ERR_BOX_TOO_SMALL (-2)  /* some L < 2 (rc + skin): minimum image would be wrong */
#define MD_ERR_NOMEM (-3)          /* device or host allocation failed */
#define MD_ERR_CUDA (-4)           /* a CUDA call failed */
#define MD_ERR_NL_OVERFLOW (-5)    /* list capacity could not be grown enough */
#define MD_ERR_TIMEOUT (-6)        /* a bounded device wait gave up */
#define MD_ERR_NONFINITE (-7)      /* a position/velocity/force is NaN or Inf */
#define MD_ERR_BADPOS (-8)         /* an atom moved more than one box length since the last wrap */
#define MD_ERR_STATE (-9)          /* call not valid in the current state */

#define MD_FP64 0   /* every arithmetic step in FP64 */
#define MD_MIXED 1  /* FP32 pair arithmetic with Kahan sums; FP64 integration and reductions */
#define MD_DW 2     /* pair arithmetic (Eq. 2) in double word: each quantity an unevaluated
                       sum of two FP32 numbers (~48 significant bits), on the FP32 pipe;
                       forces agree with FP64 to ~1e-13; FP64 integration and reductions.
                       Positions relative to the cell centre are split into a high part
                       on a power-of-two grid and a low part at each binning and step;
                       an atom that moves more than a cell side beyond its cell between
                       binnings stops the run with MD_ERR_BADPOS.  The exponent range is
                       FP32's: pairs closer than ~2e-3 sigma overflow the pair terms
                       (MD_ERR_NONFINITE at the next binning).  Full per-atom lists
                       only (MD_LIST_FULL).  md_adjoint runs the
                       forward and, by default, the reverse pair terms in double
                       word (md_set_adjoint_precision).                             */

/* Verlet-list layouts (md_params.list_type).  All hold every pair with
 * r^2 < (rc + skin)^2 at the build (Sec. 3.2, Fig. 1); md_get_neighbors
 * returns the same exact per-atom rows for every type. */
#define MD_LIST_FULL 0    /* one row per atom with all its neighbours (Sec. 4.2 GPU layout) */
#define MD_LIST_HALF 1    /* each pair once (Sec. 3.2 "half of the particle pairs") */
#define MD_LIST_GROUP2 2  /* one row per group of 2 atoms of a cell: the union of the
                             members' rows (a superset, built with an FP32 test whose
                             margin covers the FP64 criterion); mixed path only */
#define MD_LIST_GROUP4 4  /* the same for groups of 4 atoms */

/* Orthorhombic periodic box with origin 0: [0,lx) x [0,ly) x [0,lz). */
typedef struct {
    double lx, ly, lz;
} md_box;

/* Physical and algorithmic parameters (LJ reduced units). */
typedef struct {
    double epsilon;          /* well depth (V(2^(1/6) sigma) = -epsilon)            */
    double sigma;            /* distance of the zero of V                           */
    double mass;             /* atom mass                                           */
    double cutoff;           /* rc, an absolute length; pairs with r^2 < rc^2 act   */
    double skin;             /* Verlet buffer; list radius rs = rc + skin (strict)  */
    double dt;               /* time step                                           */
    int32_t rebuild_every;   /* > 0: rebuild cells + list after the drift of step n
                                when n % rebuild_every == 0 (plus once at start),
                                the schedule of Sec. 6.  0: rebuild after any drift
                                that moved some atom more than skin/2 (less 1e-5)
                                since the last binning, so every list holds all
                                pairs inside rc; checked on the device each step,
                                the rebuild is a conditional node of the captured
                                step graph (no host round trip)                   */
    int32_t precision;       /* MD_FP64, MD_MIXED or MD_DW                          */
    int32_t list_type;       /* MD_LIST_FULL, MD_LIST_HALF (pair (i,j) stored
                                with i iff j's nearest image is in i's upper
                                half-space: del = x_i - x_j has del.z < 0, ties
                                by del.y, del.x, then id_j > id_i),
                                MD_LIST_GROUP2 or MD_LIST_GROUP4 (mixed path:
                                consecutive atoms of a cell, in the library's
                                cell order, share one row; each gathered
                                neighbour position serves every member)     */
    int32_t threads_per_atom;/* 1, 2, 4 or 8 lanes per atom in the full-list force
                                kernels; 0 = a default from the atom count and
                                precision (md_autotune's choices measured on
                                GB300; md_autotune itself times the candidates) */
} md_params;

/* Read-only facts about a context. */
typedef struct {
    int64_t n;               /* total atoms over all replicas                       */
    int32_t nrep;            /* replicas                                            */
    int32_t precision, list_type, threads_per_atom;
    int32_t list_capacity;   /* entries per row the list can hold (per group for
                                the group list types)                           */
    int32_t max_neighbors;   /* largest row of the last build (group rows for the
                                group list types)                               */
    int64_t ncells;          /* cells over all replicas                             */
    int64_t step;            /* steps taken by md_run / md_integrate(2)             */
    int64_t kernel_launches; /* kernels this context launched (graph nodes counted) */
    int64_t rebuilds;        /* list builds done                                    */
    int32_t cell_split;      /* 1: the list build scans half-size cells (see
                                md_set_cell_split)                              */
} md_info;

/* Per-phase device time of md_profile (Force / Neigh / Other, the
 * breakdown of the paper's Fig. 4 and 5).  "force" is the force kernel alone
 * (with its fused velocity-Verlet epilogue on full lists); "neigh" is binning
 * plus list build; "other" is everything else (first drift, energies, the
 * half-list force clear and integration). */
typedef struct {
    double force_ms, neigh_ms, other_ms;
    int64_t force_launches, neigh_launches, other_launches;
    int64_t steps;
    double mean_neighbors;   /* list entries per atom of the list in use at the
                                end: sum of its row lengths / atoms            */
    int64_t rows;            /* rows of that list (atoms, or groups)            */
} md_phase_times;

typedef struct md_ctx md_ctx;

/* Creates a context for one periodic system of n atoms.
 *   box, params: copied.  pos, vel: host, n x 3 doubles (caller order).
 *   stream: a cudaStream_t to enqueue on, or NULL for a stream owned by the
 *   context.  The initial state is binned, a list is built and forces are
 *   computed before md_create returns.
 * At most 67,108,863 atoms per context (26-bit list indices) and 1023 cells
 * per box edge.
 * Errors: MD_ERR_INVAL, MD_ERR_BOX_TOO_SMALL, MD_ERR_NONFINITE, MD_ERR_NOMEM,
 *   MD_ERR_CUDA.  On error *out is NULL. */
int md_create(const md_box *box, const md_params *params, int64_t n, const double *pos,
              const double *vel, void *stream, md_ctx **out);

/* Creates one context holding nrep independent periodic replicas (same
 * params, own boxes) that every call advances together: replica r owns
 * counts[r] atoms, stored consecutively in pos/vel (host, sum(counts) x 3).
 * Same errors as md_create. */
int md_create_batch(int32_t nrep, const md_box *boxes, const md_params *params,
                    const int64_t *counts, const double *pos, const double *vel, void *stream,
                    md_ctx **out);

/* As md_create, with pos and vel in device memory of the current device
 * (n x 3 doubles, row major, caller order), e.g. the data pointers of CUDA
 * tensors; nothing is copied through the host.  They are read on `stream`
 * (the context's stream), so the caller orders their producer before the
 * call; they may be freed once md_create_device has returned.  Non-finite
 * values are detected on the device and reported as MD_ERR_NONFINITE.
 * Errors: as md_create, and MD_ERR_INVAL if pos or vel is not device memory
 * of the current device. */
int md_create_device(const md_box *box, const md_params *params, int64_t n, const double *pos,
                     const double *vel, void *stream, md_ctx **out);

void md_destroy(md_ctx *ctx);

/* Text of the last error of ctx (or of the last failed md_create* when ctx is
 * NULL); never NULL. */
const char *md_last_error(const md_ctx *ctx);

/* Replaces positions and velocities (host, n x 3, caller order) and
 * re-establishes cells, list and forces.  Used for restarts.  The values are
 * checked on the device as they are uploaded.
 * Errors: MD_ERR_NONFINITE (a NaN or Inf; the context holds no valid state
 * until the next successful md_set_state*), MD_ERR_BADPOS, MD_ERR_CUDA. */
int md_set_state(md_ctx *ctx, const double *pos, const double *vel);

/* md_set_state with pos and vel in device memory (the conventions of
 * md_create_device). */
int md_set_state_device(md_ctx *ctx, const double *pos, const double *vel);

/* Cell binning (Sec. 3.2, Fig. 1): wraps every position into the box with
 * one conditional +/-L per component, assigns cell (int)(x/s) (clamped to
 * nc-1) with nc = floor(L/(rc+skin)), s = L/nc, and counting-sorts atoms by
 * (cell, caller id).  Errors: MD_ERR_BADPOS, MD_ERR_NONFINITE, MD_ERR_CUDA. */
int md_bin_cells(md_ctx *ctx);

/* Verlet list build (Sec. 3.2, Fig. 1): for every atom, every atom j != i of
 * the 27 neighbour cells (each periodic image once) with
 * ((dx*dx + dy*dy) + dz*dz) < (rc+skin)^2 in FP64, dx the minimum-image
 * difference, each operation rounded.  Bins first if atoms moved since the
 * last md_bin_cells.  Grows the capacity on overflow.
 * Errors: MD_ERR_NL_OVERFLOW, MD_ERR_NOMEM, MD_ERR_CUDA. */
int md_build_neighbors(md_ctx *ctx);

/* LJ forces over the current list (Sec. 3.2 Eq. 2; Sec. 4.2 kernel order). */
int md_compute_forces(md_ctx *ctx);

/* Velocity Verlet half steps (Sec. 3.2, Eq. 1) with the stored forces:
 *   phase 1: v += dt/(2m) F; x += dt v      phase 2: v += dt/(2m) F
 * Errors: MD_ERR_INVAL (phase not 1 or 2). */
int md_integrate(md_ctx *ctx, int32_t phase);

/* Potential energy (truncated, unshifted 4 eps [(s/r)^12 - (s/r)^6], pairs
 * with r < rc once), kinetic energy 1/2 m sum v^2 and pair virial
 * sum_pairs r_ij . F_ij of the current state, reduced in FP64.  Each output
 * is a host array of nrep doubles (any may be NULL).  Synchronises. */
int md_energy(md_ctx *ctx, double *pe, double *ke, double *virial);

/* Thermodynamic outputs of one replica at one time. */
typedef struct {
    double pe, ke;           /* as md_energy                                        */
    double etot;             /* pe + ke                                             */
    double virial;           /* W = sum_pairs r_ij . F_ij                           */
    double temperature;      /* T = 2 KE / (3N - 3) (momentum removed; 0 if N = 1)  */
    double pressure;         /* P = (N T + W / 3) / V (0 if N = 1)                  */
} md_thermo_rec;

/* Temperature, pressure and total energy from (PE, KE, W) records, computed
 * on the device.  energies: host, nrec x nrep x 3 doubles in the layout of
 * md_run's energy log; or NULL with nrec = 1 for the current state (as
 * md_energy).  out: host, nrec x nrep records.  Synchronises.  Not in the
 * paper, whose outputs are the Eq. 2 forces and energies; the formulas are
 * the standard ones for a periodic LJ system.
 * Errors: MD_ERR_INVAL, MD_ERR_NOMEM, MD_ERR_CUDA. */
int md_thermo(md_ctx *ctx, const double *energies, int64_t nrec, md_thermo_rec *out);

/* Advances nsteps velocity-Verlet steps with the rebuild schedule; the
 * per-step work is replayed from CUDA graphs.  When energies is not NULL and
 * energy_every > 0, (PE, KE, W) of every replica after steps s0 + k *
 * energy_every (k = 1 .. nsteps / energy_every, s0 = steps taken before this
 * call) is written to energies (host, (nsteps / energy_every) x nrep x 3
 * doubles).  Synchronises once at the end.
 * Errors: MD_ERR_NL_OVERFLOW, MD_ERR_NONFINITE, MD_ERR_BADPOS, MD_ERR_CUDA. */
int md_run(md_ctx *ctx, int64_t nsteps, int32_t energy_every, double *energies);

/* Copies of the state in caller order (host, n x 3 doubles).  Synchronise. */
int md_get_positions(md_ctx *ctx, double *pos);
int md_get_velocities(md_ctx *ctx, double *vel);
int md_get_forces(md_ctx *ctx, double *force);

/* Device-memory getters: write positions, velocities or forces (n x 3
 * doubles, caller order, the values the host getters return) to `out`,
 * device memory of the current device, asynchronously on the context's
 * stream (no synchronisation; the caller orders its readers after it).
 * Errors: MD_ERR_INVAL (null, or out is not device memory), MD_ERR_CUDA. */
int md_get_positions_device(md_ctx *ctx, double *out);
int md_get_velocities_device(md_ctx *ctx, double *out);
int md_get_forces_device(md_ctx *ctx, double *out);

/* The cells of the last binning, per replica in order: cell_start (host,
 * ncells + nrep int32: each replica's exclusive prefix sums including its
 * end) and cell_atoms (host, n int32 caller ids, ascending within a cell;
 * ids are local to their replica).  Synchronises. */
int md_get_cells(md_ctx *ctx, int32_t *cell_start, int32_t *cell_atoms);

/* The current Verlet list in caller ids (local to the replica): counts (host,
 * n int32) and rows (host, n x cap int32; row i holds counts[i] ids).
 * Returns MD_ERR_INVAL if some row exceeds cap.  Synchronises. */
int md_get_neighbors(md_ctx *ctx, int32_t *counts, int32_t *rows, int32_t cap);

int md_get_info(md_ctx *ctx, md_info *info);

/* Sets the step counter (md_info.step) that the fixed rebuild schedule
 * counts with, e.g. to resume a run from a saved state: md_set_state with the
 * saved positions and velocities, then md_set_step with the saved step.
 * Errors: MD_ERR_INVAL (step < 0). */
int md_set_step(md_ctx *ctx, int64_t step);

/* Reallocates the list for `cap` entries per atom (rounded up to a multiple
 * of 4) and rebuilds it now, growing past `cap` if the current state needs
 * more.  Later rebuilds grow it again whenever a row overflows.
 * Errors: MD_ERR_INVAL (cap < 4), MD_ERR_NOMEM, MD_ERR_NL_OVERFLOW. */
int md_set_capacity(md_ctx *ctx, int32_t cap);

/* Runs nsteps like md_run (same kernels, same schedule) but launches them
 * one by one with a CUDA event pair around each phase on the context stream,
 * and reports the device time per phase.  Synchronises. */
int md_profile(md_ctx *ctx, int64_t nsteps, md_phase_times *out);

/* Changes epsilon and sigma (both > 0) and selects the Lennard-Jones force
 * (the default); forces are recomputed on next use. */
int md_set_lj(md_ctx *ctx, double epsilon, double sigma);

/* Switches the context to the spring-dashpot contact model of Sec. 3.2,
 * Eq. 3 (a second pair force on the same cells and lists): spheres of
 * diameter params.sigma touch when r = |x_ij| < sigma and then
 *     F_i += K xi + gamma xi_dot,  xi = xhat (sigma - r),
 *     xi_dot = -xhat (xhat . v_ij),  x_ij = x_i - x_j,  v_ij = v_i - v_j.
 * The force after a drift reads the half-step velocities (the latest).  PE
 * reported by md_energy is the elastic 1/2 K (sigma - r)^2 per contact, W the
 * sum of x_ij . F_ij.  Full lists are used (a half-list context switches and
 * rebuilds); md_set_lj switches back to Lennard-Jones.  K = gamma = 0 is the
 * paper's static setting (no force).
 * Errors: MD_ERR_INVAL (negative or non-finite K or gamma, cutoff < sigma),
 * MD_ERR_CUDA. */
int md_set_spring_dashpot(md_ctx *ctx, double k_spring, double gamma);

/* Differentiable rollout (not in the paper; it differentiates the Sec. 3.2
 * Eq. 1 / Eq. 2 forward map).  From the current state (x0, v0) of a
 * single-system context, runs nsteps velocity-Verlet steps with the rebuild
 * schedule counted from this call (rebuild at step 0 and whenever
 * step % rebuild_every == 0) and returns
 *     loss = (1/window) * sum_{n = nsteps-window+1 .. nsteps} PE(x_n)
 * and its gradient with respect to epsilon, sigma (rc held fixed), x0 and v0
 * by a hand-written reverse sweep: states are checkpointed every ckpt_every
 * steps and each block is recomputed bit-exactly (same list, same kernels)
 * before it is reversed.  g_x0 / g_v0: host, n x 3 doubles in caller order
 * (each may be NULL).  The context is left at (x0, v0).  Work memory
 * (nsteps/ckpt_every + 1 checkpoints of 84 B per atom, ckpt_every recomputed
 * snapshots of 48 B per atom, and the adjoint state) stays with the context
 * for later calls, grown when a call needs more, and is freed by md_destroy;
 * if growing it fails the whole workspace is released and MD_ERR_NOMEM
 * returned.
 * Errors: MD_ERR_INVAL (nrep != 1; rebuild_every == 0; spring-dashpot model; window not in
 * [1, nsteps]; ckpt_every not dividing both rebuild_every and nsteps),
 * MD_ERR_NOMEM, MD_ERR_CUDA and those of md_run. */
int md_adjoint(md_ctx *ctx, int64_t nsteps, int64_t window, int32_t ckpt_every, double *loss,
               double *g_eps, double *g_sigma, double *g_x0, double *g_v0);

/* md_adjoint with g_x0 and g_v0 in device memory of the current device (n x
 * 3 doubles, caller order; each may be NULL), written on the context's
 * stream; loss, g_eps and g_sigma stay host scalars.  Synchronises like
 * md_adjoint.  Errors: those of md_adjoint, and MD_ERR_INVAL if g_x0 or g_v0
 * is not device memory. */
int md_adjoint_device(md_ctx *ctx, int64_t nsteps, int64_t window, int32_t ckpt_every,
                      double *loss, double *g_eps, double *g_sigma, double *g_x0, double *g_v0);

/* Precision of the pair terms of md_adjoint's reverse sweep (the Jacobian-
 * vector products and the parameter derivatives): MD_MIXED evaluates them in
 * FP32 from the cell-relative FP32 positions (the default of a mixed
 * context), MD_FP64 in FP64 from the FP64 positions (the default of an FP64
 * context), MD_DW in double word from the split positions (the default of an
 * MD_DW context, and only there).  The forward run keeps the context's
 * precision, so a mixed context with MD_FP64 here differentiates its own
 * mixed trajectory with FP64 pair terms.  Not in the paper.
 * Errors: MD_ERR_INVAL (another value; MD_DW on a context of another
 * precision). */
int md_set_adjoint_precision(md_ctx *ctx, int32_t precision);

/* Force-kernel studies: variants of the mixed full-list force pass that the
 * library measured and did not adopt, kept runnable so those measurements can
 * be repeated on the current state and list (not part of the method).  Runs
 * one warm-up and `reps` timed launches of variant
 *   0  the library's kernel (16-byte FP32 cell-relative gathers, offsets
 *      selected in registers; Sec. 4.2's AoS layout),
 *   1  SoA gathers (three float arrays), 2  AoSoA gathers (blocks of four
 *      atoms, x0..x3 y0..y3 z0..z3: Sec. 4.2's clustered layout), both with
 *      the library's arithmetic in its order (bitwise the same forces),
 *   3  the 4x4x4-cell neighbourhood of each 2x2x2-cell tile staged in shared
 *      memory in the tile's frame (one block per tile), 4  the same staged by
 *      TMA bulk copies (one per cell: cells are contiguous ranges of the
 *      position array) completing on an mbarrier (bitwise variant 3's forces),
 *   5  the library's gathers through the texture path (tex1Dfetch on a
 *      texture object over the positions), 6  half of them (the pairs of a
 *      list chunk alternate between the two paths), both bitwise the
 *      library's forces,
 * with forces only (no integration), CUDA events on the context's stream;
 * *us = mean device time per launch in microseconds; forces (may be NULL):
 * host, n x 3 doubles in caller order.  Needs a single-system mixed LJ
 * context with full per-atom lists.
 * Errors: MD_ERR_INVAL, MD_ERR_STATE (wrong kind of context; variants 3, 4:
 * a neighbourhood above 3008 atoms; variants 5, 6: more atoms than a linear
 * texture holds), MD_ERR_TIMEOUT (variant 4: a bulk copy
 * did not complete within ~10 ms; the kernel returns), MD_ERR_NOMEM,
 * MD_ERR_CUDA. */
int md_study_force_variant(md_ctx *ctx, int32_t variant, int32_t reps, double *us, double *forces);

/* Chooses threads_per_atom and the list type by timing each candidate for
 * `steps` steps on the context's own state (which it restores), then the
 * winner with the other cell split (md_set_cell_split), keeps the fastest and
 * reports it in *chosen (may be NULL; the split in md_info.cell_split).
 * MD_DW contexts try full lists with 1, 2, 4 and 8 lanes per atom.
 * Results are cached per (precision, atoms-per-replica bucket) for the life
 * of the process. */
int md_autotune(md_ctx *ctx, int32_t steps, md_params *chosen);

/* Cell size of the list build (Sec. 3.2, Fig. 1: cells of side at least
 * rc + skin; smaller cells with a wider stencil also find every pair).
 * split = 1: the binning orders each cell's atoms by octant, i.e. by the
 * half-size cells, and the build scans, in each of the 27 neighbour cells,
 * only the octants that can hold a pair within rc + skin of the atom: the far
 * half of a face-adjacent cell lies at least s beyond the near side of the
 * atom's own cell (s >= rc + skin), so it is skipped for atoms on that near
 * side (with a margin of 1e-3 s for the FP32 half decisions).  The lists hold
 * the same pairs with either split (only the order of a cell's entries, and
 * so the rounding of the force sums, changes).  split = 0: whole cells.
 * Default: 0 (on the 1M-atom LJ liquid split cells take 61 against 37 us of
 * neighbour work per step: lanes of a warp keep different octants, and the
 * warp scans the union of their runs).  A change rebins, rebuilds the list
 * and recomputes the forces of the current state.
 * The cell arrays grow to 8 entries per cell the first time cells are split.
 * Not in the paper as an option; its cells are the split = 0 ones.
 * Errors: MD_ERR_INVAL (split not 0 or 1; split = 1 on boxes of 2^28 or more
 * cells, whose keys would not fit 31 bits), MD_ERR_NOMEM, MD_ERR_CUDA. */
int md_set_cell_split(md_ctx *ctx, int32_t split);

/* Allocation-free FP64 totals: out3[0] = sum pe_atom, out3[1] = 1/2 mass
 * sum |v|^2, out3[2] = sum w_atom, for callers that cannot allocate device
 * memory where they need these totals (an external engine that reserved the
 * whole GPU for its own pool, a fixed device-memory budget, or a loop that
 * must not call cudaMalloc because it can synchronise the device).  The
 * paper has no counterpart; this is a service of the library.
 *   pe_atom, w_atom: device, n doubles; vel: device, n x 3 doubles (row
 *   major, 24 bytes per atom: not a buffer of 4-double padded vectors such
 *   as the library's own internal state); out3: device, 3 doubles; stream:
 *   cudaStream_t or NULL.
 * Sums are taken in a fixed order (deterministic).  The only scratch is a
 * fixed 192 KiB array in the library's device data, so n may be at most
 * 33,554,432; larger n returns MD_ERR_INVAL with a message from
 * md_last_error(NULL).  No call allocates or frees device memory.  The
 * array has its own address in every CUDA context that loads the library;
 * the first call in a context (a device's primary context, or a driver-API
 * context made current by the caller) looks that address up and caches it
 * under the context's id: make that first call before any stream capture.
 * All calls in a context share the array: calls that overlap on the GPU
 * (other streams, other threads) race and must be serialised by the
 * caller.  Every call writes the scratch it reads, so nothing is left over
 * from an earlier call.  A non-sticky CUDA error left pending on the
 * calling thread by earlier work is cleared before the launches.
 * Errors: MD_ERR_INVAL, MD_ERR_CUDA. */
int md_energy_sums_static(int64_t n, const double *pe_atom, const double *w_atom,
                          const double *vel, double mass, double *out3, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MD_GB300_H */
