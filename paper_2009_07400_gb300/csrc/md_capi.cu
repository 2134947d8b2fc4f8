// Host runtime and C ABI (include/md.h) of the GB300 LJ MD hot path.
//
// A context owns the device state of one or more periodic replicas laid out
// back to back (structure of arrays, atoms sorted by (replica, cell, id) at
// every binning).  md_run turns a span of steps into a list of operations --
//     KD                 first half-kick + drift (from stored forces)
//     REBUILD            bin + build, after the drift of step n % every == 0
//     F(n)               forces at x_n fused with the rest of velocity Verlet
// -- cut at every rebuild into segments, and replays each segment from a
// CUDA graph cached under (buffer parities, operation string).  A steady
// 20-step cycle is one graph launch.
//
// Failure handling: kernels set bits in a device error word and every later
// kernel returns at once while it is set, so the state freezes at the first
// failure.  md_run synchronises once at its end; a list overflow is repaired
// by growing the capacity and resuming at the rebuild that overflowed.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/md.h"
#include "md_internal.cuh"

using namespace mdk;

namespace {

thread_local std::string g_create_error;

struct Op {
    // COND: the displacement-triggered rebuild check of step n (a graph
    // conditional node whose body bins and rebuilds)
    enum Kind { KD, REBUILD, FORCE, COND } kind;
    int64_t step;   // step n the op belongs to
    bool last;      // FORCE: last step of the run (store F, no next drift)
    bool energy;    // FORCE: log (PE, KE, W) of step n
};

struct GraphRec {
    cudaGraphExec_t exec;
    int launches;
    int xp_after, vp_after, pb_after;
};

}  // namespace

struct md_ctx {
    int64_t n = 0;
    int32_t nrep = 0;
    md_params p{};
    LJ lj{};
    std::vector<Rep> reps_h;
    std::vector<int64_t> counts_h;
    int64_t ncells = 0;     // cells over all replicas
    int64_t nids = 0;       // cell ids (tile padding included): sizes of cell arrays
    int64_t nchunks = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int device = 0;
    int tpa = 1;
    int32_t split = 0;      // cells split into octants for the list build (keys 8 per cell)
    int adj_prec = -1;      // md_set_adjoint_precision: pair terms of the reverse
                            // sweep in MD_FP64 / MD_MIXED; -1 = the context's

    Rep *reps_d = nullptr;
    int32_t *rep_of_d = nullptr;
    dvec4 *x[2] = {nullptr, nullptr}, *v[2] = {nullptr, nullptr};
    int32_t *id[2] = {nullptr, nullptr};
    float4 *p32[2] = {nullptr, nullptr};
    float4 *p32_ref = nullptr;      // displacement trigger: p32 at the last binning
    float4 *plo[2] = {nullptr, nullptr};   // double-word path: low parts of the split
                                    // positions, same parity as p32 (else null)
    float4 *vlo[2] = {nullptr, nullptr};   // contact model, double-word path: low parts
    float4 *v32[2] = {nullptr, nullptr};   // contact model, mixed path: FP32 velocity
                                    // copies, same parity as p32
    bool v32_fresh = false;         // v32[pb] == fl32(v) (else regenerated before a force)
    cudaStream_t side = nullptr;    // displacement trigger: captures the conditional bodies
    bool disp = false;              // md_params.rebuild_every == 0
    float disp2_thr = 0.f;
    float4 *f32 = nullptr;
    dvec4 *f64 = nullptr;
    int32_t *cell_key = nullptr, *cell_count = nullptr, *cell_start = nullptr, *perm = nullptr;
    int32_t *scan_tmp = nullptr;
    int64_t scan_len = 0;
    int64_t key_cap = 0;    // binning keys the cell arrays hold (nids, or 8 nids once split)
    int32_t *nb = nullptr, *nb_count = nullptr;
    int32_t cap = 0;
    // list shared by groups of gsz atoms (list types 2 and 4): group table,
    // per-cell group counts and their prefix sums, rows, row lengths; sized
    // for gsz when allocated (ngmax = ceil(n / gsz) + cell ids)
    int32_t *grp = nullptr, *gcnt = nullptr, *gcell_start = nullptr, *gnb = nullptr,
            *gnb_count = nullptr;
    uint8_t *gmask = nullptr;       // member bits per entry (laid out like gnb)
    uint16_t *gpair = nullptr;      // member pairs per group
    int64_t ngmax = 0;
    int32_t gcap = 0, gsz = 0;
    double expect_row = 0;          // expected full-list row at the densest replica
    float4 *offtab_d = nullptr;     // per replica: o s for the 64 cell-offset codes
    float *pe_atom = nullptr, *w_atom = nullptr;
    double *pe64 = nullptr, *w64 = nullptr, *ke64 = nullptr;
    DevStatus *status = nullptr;
    int64_t *chunk_rep_d = nullptr, *chunk_first_d = nullptr;
    double *partials_d = nullptr, *eout_d = nullptr;
    double *elog_d = nullptr;
    int64_t elog_cap = 0;
    double *io_d = nullptr;
    double *ctr_d = nullptr;

    // buffer parities: x (flips at binning and at each fused FP64 step), v and
    // id (flip at binning), p32 (flips at each fused step)
    int xp = 0, vp = 0, pb = 0;
    bool moved_since_bin = true, list_valid = false, forces_valid = false;
    int64_t step = 0, launches = 0, rebuilds = 0, builds_enqueued = 0;
    int32_t last_max = 0;
    std::string err;
    std::map<std::string, GraphRec> graphs;
    // md_adjoint's workspace, kept between calls (grow-only): checkpoints
    // (nck x n), the block's recomputed snapshots (ckpt x n), adjoint state
    struct {
        int64_t nck = 0, ckpt = 0;
        dvec4 *ck_x = nullptr, *ck_v = nullptr, *blk_x = nullptr, *xbar = nullptr, *wbar = nullptr;
        float4 *blk_p = nullptr, *ck_p = nullptr, *wbar32 = nullptr;
        float4 *ck_plo = nullptr;   // double-word path: the low parts beside ck_p
        float4 *blk_plo = nullptr, *wbar_lo = nullptr;   // double-word pair terms
        int32_t *ck_id = nullptr;
        double *ge = nullptr, *gs = nullptr, *g2 = nullptr;
    } adj;
};

namespace {

int fail(md_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    else g_create_error = msg;
    return code;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(c, MD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

Dev view(const md_ctx *c)
{
    Dev d{};
    d.n = c->n;
    d.ncells = c->nids;
    d.split = c->split;
    d.nrep = c->nrep;
    d.cap = c->cap;
    d.reps = c->reps_d;
    d.rep_of = c->rep_of_d;
    d.x = c->x[c->xp];
    d.v = c->v[c->vp];
    d.x_alt = c->x[1 - c->xp];
    d.x_nxt = c->x[1 - c->xp];
    d.v_alt = c->v[1 - c->vp];
    d.id = c->id[c->vp];
    d.id_alt = c->id[1 - c->vp];
    d.p32 = c->p32[c->pb];
    d.p32_nxt = c->p32[1 - c->pb];
    d.p32_ref = c->p32_ref;
    d.plo = c->plo[c->pb];
    d.plo_nxt = c->plo[1 - c->pb];
    d.disp2_thr = c->disp2_thr;
    d.f32 = c->f32;
    d.f64 = c->f64;
    d.cell_key = c->cell_key;
    d.cell_count = c->cell_count;
    d.cell_start = c->cell_start;
    d.perm = c->perm;
    d.nb = c->nb;
    d.nb_count = c->nb_count;
    d.pe_atom = c->pe_atom;
    d.w_atom = c->w_atom;
    d.pe_atom64 = c->pe64;
    d.w_atom64 = c->w64;
    d.ke_atom64 = c->ke64;
    d.status = c->status;
    d.ctr = c->ctr_d;
    d.grp = c->grp;
    d.gcnt = c->gcnt;
    d.gcell_start = c->gcell_start;
    d.gnb = c->gnb;
    d.gnb_count = c->gnb_count;
    d.gmask = c->gmask;
    d.gpair = c->gpair;
    d.ngmax = c->ngmax;
    d.gcap = c->gcap;
    d.offtab = c->offtab_d;
    if (c->lj.pot == 1 && (c->p.precision == MD_MIXED || c->p.precision == MD_DW)) {
        // contact model: velocity copies (and, double word, their low parts)
        d.v32 = c->v32[c->pb];
        d.v32_nxt = c->v32[1 - c->pb];
        d.vlo = c->vlo[c->pb];
        d.vlo_nxt = c->vlo[1 - c->pb];
    }
    return d;
}

// Host-side fault injection for tests: with MD_FAIL_ALLOC=k in the
// environment, the k-th device allocation of the process (counting from 0)
// fails as if the device were out of memory.  Nothing is injected on the GPU.
bool injected_alloc_failure()
{
    static const long fail_at = [] {
        const char *s = std::getenv("MD_FAIL_ALLOC");
        return s ? std::strtol(s, nullptr, 10) : -1L;
    }();
    static std::atomic<long> count{0};
    return fail_at >= 0 && count.fetch_add(1) == fail_at;
}

template <typename T>
int dalloc(md_ctx *c, T **p, size_t count)
{
    if (count == 0) count = 1;
    if (injected_alloc_failure()) {
        *p = nullptr;
        return fail(c, MD_ERR_NOMEM, "cudaMalloc: injected allocation failure (MD_FAIL_ALLOC)");
    }
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(c, MD_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return MD_OK;
}

void free_all(md_ctx *c)
{
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
    c->graphs.clear();
    void *ptrs[] = {c->reps_d, c->rep_of_d, c->x[0], c->x[1], c->v[0], c->v[1], c->id[0],
                    c->id[1], c->p32[0], c->p32[1], c->f32, c->f64, c->cell_key, c->cell_count,
                    c->cell_start, c->perm, c->scan_tmp, c->nb, c->nb_count, c->pe_atom,
                    c->w_atom, c->pe64, c->w64, c->ke64, c->status, c->chunk_rep_d,
                    c->chunk_first_d, c->partials_d, c->eout_d, c->elog_d, c->io_d, c->ctr_d,
                    c->p32_ref, c->v32[0], c->v32[1], c->adj.ck_x, c->adj.ck_v, c->adj.blk_x,
                    c->adj.xbar, c->adj.wbar, c->adj.blk_p, c->adj.ck_p, c->adj.wbar32, c->adj.ck_plo,
                    c->adj.blk_plo, c->adj.wbar_lo,
                    c->adj.ck_id, c->adj.ge, c->adj.gs, c->adj.g2, c->grp, c->gcnt,
                    c->gcell_start, c->gnb, c->gnb_count, c->offtab_d, c->gmask, c->gpair,
                    c->plo[0], c->plo[1], c->vlo[0], c->vlo[1]};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (c->own_stream && c->st) cudaStreamDestroy(c->st);
    if (c->side) cudaStreamDestroy(c->side);
}

bool is_mixed(const md_ctx *c) { return c->p.precision == MD_MIXED; }
// double-word pair arithmetic (FP32 pipe); state handled as on the mixed path
bool is_dw(const md_ctx *c) { return c->p.precision == MD_DW; }
// the FP64 path gathers x itself: its fused step writes the next x into the
// other buffer; the mixed and double-word paths update x in place
bool x_flips(const md_ctx *c) { return c->p.precision == MD_FP64; }
bool is_half(const md_ctx *c) { return c->p.list_type == MD_LIST_HALF; }
// group size of a list shared by groups of atoms (list types 2 and 4), else 0
int list_g(const md_ctx *c)
{
    return (c->p.list_type == MD_LIST_GROUP2 || c->p.list_type == MD_LIST_GROUP4) ? c->p.list_type : 0;
}
bool is_sd(const md_ctx *c) { return c->lj.pot == 1; }
bool batched(const md_ctx *c) { return c->nrep > 1; }
// the contact model's mixed and double-word paths keep velocity copies (v32,
// and on the double-word path their low parts)
bool uses_v32(const md_ctx *c)
{
    return c->lj.pot == 1 && (c->p.precision == MD_MIXED || c->p.precision == MD_DW);
}

int32_t round4(int64_t v) { return (int32_t)((v + 3) / 4 * 4); }

int alloc_list(md_ctx *c, int32_t cap)
{
    if (c->nb) cudaFree(c->nb);
    c->nb = nullptr;
    c->cap = round4(cap);
    int rc = dalloc(c, &c->nb, (size_t)c->n * (size_t)c->cap);
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
    c->graphs.clear();
    return rc;
}

// Group table for groups of g atoms of a cell: table, per-cell counts and
// their prefix sums, and the per-group row lengths and member-pair masks of a
// group list (ngmax = ceil(n / g) + cell ids).
int alloc_group_table(md_ctx *c, int g)
{
    if (c->gsz == g) return MD_OK;
    int32_t **arrs[] = {&c->grp, &c->gcnt, &c->gcell_start, &c->gnb_count};
    for (int32_t **a : arrs) {
        if (*a) cudaFree(*a);
        *a = nullptr;
    }
    if (c->gpair) cudaFree(c->gpair);
    c->gpair = nullptr;
    c->gsz = 0;
    c->ngmax = (c->n + g - 1) / g + c->nids;
    int rc;
    if ((rc = dalloc(c, &c->grp, (size_t)c->ngmax)) || (rc = dalloc(c, &c->gnb_count, (size_t)c->ngmax)) ||
        (rc = dalloc(c, &c->gpair, (size_t)c->ngmax)) ||
        (rc = dalloc(c, &c->gcnt, (size_t)c->nids)) || (rc = dalloc(c, &c->gcell_start, (size_t)c->nids + 1)))
        return rc;
    c->gsz = g;
    // group rows were laid out for the old ngmax
    if (c->gnb) cudaFree(c->gnb);
    if (c->gmask) cudaFree(c->gmask);
    c->gnb = nullptr;
    c->gmask = nullptr;
    return MD_OK;
}

// Group-list rows for groups of g atoms with `cap` entries per group row
// (rounded up to a multiple of 16).
int alloc_group(md_ctx *c, int g, int32_t cap)
{
    int rc = alloc_group_table(c, g);
    if (rc) return rc;
    if (c->gnb) cudaFree(c->gnb);
    if (c->gmask) cudaFree(c->gmask);
    c->gnb = nullptr;
    c->gmask = nullptr;
    c->gcap = (int32_t)((std::max<int64_t>(cap, 16) + 15) / 16 * 16);
    rc = dalloc(c, &c->gnb, (size_t)c->ngmax * (size_t)c->gcap);
    if (!rc) rc = dalloc(c, &c->gmask, (size_t)c->ngmax * (size_t)c->gcap);
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
    c->graphs.clear();
    return rc;
}

// Initial group-row capacity: the union of G rows of ~rho (4/3) pi rs^3
// entries measured 1.34x (G = 2) and 1.78x (G = 4) one row on LJ liquids;
// with margin.
int32_t group_cap0(const md_ctx *c, int g)
{
    return (int32_t)(c->expect_row * (g == 4 ? 2.4 : 1.8)) + 32;
}

// Capacity of the list type in use, and growing it after an overflow.
int32_t active_cap(const md_ctx *c) { return list_g(c) ? c->gcap : c->cap; }
int realloc_active(md_ctx *c, int32_t cap)
{
    return list_g(c) ? alloc_group(c, list_g(c), cap) : alloc_list(c, cap);
}

// ---------------------------------------------------------------------------
// Enqueue helpers (used both directly and under stream capture).
// ---------------------------------------------------------------------------
int enq_bin(md_ctx *c, int *nl)
{
    Dev d = view(c);
    if (launch_bin(d, c->scan_tmp, c->scan_len, c->st, nl) != 0)
        return fail(c, MD_ERR_CUDA, "binning launch failed");
    if (d.v32) c->v32_fresh = true;   // the gather writes v32 in the new order
    if (c->disp) {
        // the reordered state is copied back: buffer roles never change
        if (launch_copy_back(d, c->st, nl) != 0) return fail(c, MD_ERR_CUDA, "copy-back launch failed");
        CK(cudaMemsetAsync(&c->status->need_rebuild, 0, sizeof(int32_t), c->st));
    } else {
        c->xp = 1 - c->xp;  // reordered state now lives in the other buffers
        c->vp = 1 - c->vp;
    }
    c->moved_since_bin = false;
    c->list_valid = false;
    c->forces_valid = false;
    return MD_OK;
}

// The list build of the context's list type on stream st (group lists: the
// group table of the current binning first).
int launch_list_build(md_ctx *c, const Dev &d, cudaStream_t st, int *nl)
{
    if (list_g(c)) {
        if (launch_group_table(d, list_g(c), c->nids, c->scan_tmp, c->scan_len, st, nl) != 0) return -1;
        return launch_build_group(d, c->lj, list_g(c), st, nl);
    }
    return launch_build(d, c->lj, is_half(c), c->nids, st, nl);
}

int enq_build(md_ctx *c, int *nl)
{
    CK(cudaMemsetAsync(&c->status->max_count, 0, sizeof(int32_t), c->st));
    Dev d = view(c);
    if (launch_list_build(c, d, c->st, nl) != 0)
        return fail(c, MD_ERR_CUDA, "list build launch failed");
    c->list_valid = true;
    c->builds_enqueued++;
    return MD_OK;
}

int enq_energy(md_ctx *c, bool ke_from_v, double *out3, int *nl)
{
    Dev d = view(c);
    if (launch_energy(d, c->lj, c->p.precision, ke_from_v, c->chunk_rep_d, c->chunk_first_d,
                      c->nchunks, c->partials_d, out3, out3 ? nullptr : c->elog_d, c->st,
                      nl) != 0)
        return fail(c, MD_ERR_CUDA, "energy launch failed");
    return MD_OK;
}

// Forces at the current positions followed by `epi` (EPI_F / EPI_FK /
// EPI_FKKD); with `energy`, per-atom PE/W (and KE of the full-step v).
// ev (optional): an event pair recorded around the force kernel alone.
int enq_force(md_ctx *c, int epi, bool energy, int *nl, cudaEvent_t *ev = nullptr)
{
    Dev d = view(c);
    if (is_sd(c) && (is_mixed(c) || is_dw(c))) {
        // contact model, mixed and double-word paths: one fused kernel; the
        // velocity copies are regenerated only when something other than the
        // fused step or a binning changed v since they were made
        if (ev) CK(cudaEventRecord(ev[0], c->st));
        if (!c->v32_fresh) {
            if (is_dw(c) ? launch_velocity_dw(d, c->st, nl) : launch_velocity_f32(d, c->st, nl))
                return fail(c, MD_ERR_CUDA, "velocity copy launch failed");
            c->v32_fresh = true;
        }
        if (is_dw(c) ? launch_force_sd_dw(d, c->lj, epi, energy, c->st, nl)
                     : launch_force_sd(d, c->lj, true, epi, energy, c->st, nl))
            return fail(c, MD_ERR_CUDA, "force launch failed");
        if (ev) CK(cudaEventRecord(ev[1], c->st));
        if (epi == EPI_FKKD) c->pb = 1 - c->pb;      // next p32 and v32 written
        else if (epi == EPI_FK) c->v32_fresh = false;
    } else if (is_half(c) || is_sd(c)) {
        // force store, then the velocity-Verlet update in its own kernel
        if (ev) CK(cudaEventRecord(ev[0], c->st));
        if (is_sd(c)) {
            if (launch_force_sd(d, c->lj, false, EPI_F, energy, c->st, nl))
                return fail(c, MD_ERR_CUDA, "force launch failed");
        } else {
            if (is_mixed(c)) CK(cudaMemsetAsync(c->f32, 0, sizeof(float4) * c->n, c->st));
            else CK(cudaMemsetAsync(c->f64, 0, sizeof(dvec4) * c->n, c->st));
            if (ev) CK(cudaEventRecord(ev[0], c->st));
            if (launch_force(d, c->lj, c->p.precision, true, 1, EPI_F, energy, batched(c), c->st, nl))
                return fail(c, MD_ERR_CUDA, "force launch failed");
        }
        if (ev) CK(cudaEventRecord(ev[1], c->st));
        if (epi == EPI_FK) {
            if (launch_integrate(d, c->lj, c->p.precision, 2, batched(c), c->st, nl))
                return fail(c, MD_ERR_CUDA, "integrate launch failed");
        } else if (epi == EPI_FKKD) {
            if (launch_integrate(d, c->lj, c->p.precision, energy ? 4 : 3, batched(c), c->st, nl))
                return fail(c, MD_ERR_CUDA, "integrate launch failed");
        }
    } else {
        if (ev) CK(cudaEventRecord(ev[0], c->st));
        const int rc = list_g(c) ? launch_force_group(d, c->lj, list_g(c), epi, energy, batched(c), c->st, nl)
                       : is_dw(c) ? launch_force_dw(d, c->lj, c->tpa, epi, energy, batched(c), c->st, nl)
                                  : launch_force(d, c->lj, c->p.precision, false, c->tpa, epi, energy,
                                                 batched(c), c->st, nl);
        if (rc) return fail(c, MD_ERR_CUDA, "force launch failed");
        if (ev) CK(cudaEventRecord(ev[1], c->st));
        if (epi == EPI_FKKD) {
            c->pb = 1 - c->pb;
            if (x_flips(c)) c->xp = 1 - c->xp;
        }
    }
    if (epi == EPI_FKKD) c->moved_since_bin = true;
    c->forces_valid = (epi != EPI_FKKD);
    return MD_OK;
}

// Under stream capture: a one-thread kernel that sets a graph conditional
// when some atom moved past the trigger distance, then an IF node whose body
// bins (copying the state back) and rebuilds the list.  Buffer parities are
// the same whether or not the body runs.
int enq_cond_rebuild(md_ctx *c, int *nl)
{
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(c->st, &cs, nullptr, &g, &deps, nullptr, &nd));
    if (cs != cudaStreamCaptureStatusActive)
        return fail(c, MD_ERR_STATE, "conditional rebuild outside a graph capture");
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
    const Dev d = view(c);
    if (launch_rebuild_check(d, h, c->st, nl)) return fail(c, MD_ERR_CUDA, "check launch failed");
    CK(cudaStreamGetCaptureInfo(c->st, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
    CK(cudaStreamUpdateCaptureDependencies(c->st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    CK(cudaStreamBeginCaptureToGraph(c->side, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    int bl = 0, rc = MD_OK;
    if (launch_bin(d, c->scan_tmp, c->scan_len, c->side, &bl) != 0 ||
        launch_copy_back(d, c->side, &bl) != 0 || launch_list_build(c, d, c->side, &bl) != 0)
        rc = fail(c, MD_ERR_CUDA, "rebuild body launch failed");
    cudaGraph_t out = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->side, &out);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(c, MD_ERR_CUDA, std::string("body capture: ") + cudaGetErrorString(e));
    // counted as launches only when the body runs; the host does not know
    return MD_OK;
}

int enq_op(md_ctx *c, const Op &op, int *nl)
{
    int rc = MD_OK;
    if (op.kind == Op::KD) {
        Dev d = view(c);
        if (launch_integrate(d, c->lj, c->p.precision, 1, batched(c), c->st, nl))
            return fail(c, MD_ERR_CUDA, "integrate launch failed");
        c->moved_since_bin = true;
        c->forces_valid = false;
        c->v32_fresh = false;
    } else if (op.kind == Op::REBUILD) {
        if ((rc = enq_bin(c, nl))) return rc;
        if ((rc = enq_build(c, nl))) return rc;
    } else if (op.kind == Op::COND) {
        if ((rc = enq_cond_rebuild(c, nl))) return rc;
    } else {
        const int epi = op.last ? EPI_FK : EPI_FKKD;
        // For FK with energy on half lists the KE is of the final v: the
        // phase-2 kick then the energy pass reading v (ke_from_v).
        if ((rc = enq_force(c, epi, op.energy, nl))) return rc;
        if (op.energy) {
            if ((rc = enq_energy(c, op.last, nullptr, nl))) return rc;
        }
    }
    return rc;
}

std::string key_of(const md_ctx *c, const std::vector<Op> &ops)
{
    std::string k = std::to_string(c->xp) + std::to_string(c->vp) + std::to_string(c->pb) +
                    (uses_v32(c) && c->v32_fresh ? "f" : "") + ":";
    for (const Op &o : ops) {
        if (o.kind == Op::KD) k += 'K';
        else if (o.kind == Op::REBUILD) k += 'R';
        else if (o.kind == Op::COND) k += 'C';
        else k += o.last ? (o.energy ? 'L' : 'l') : (o.energy ? 'E' : 'e');
    }
    return k;
}

// Runs one segment of ops through a cached CUDA graph.
int run_segment(md_ctx *c, const std::vector<Op> &ops)
{
    const std::string key = key_of(c, ops);
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
        const int xp0 = c->xp, vp0 = c->vp, pb0 = c->pb;
        const bool mv = c->moved_since_bin, lv = c->list_valid, fv = c->forces_valid,
                   vf = c->v32_fresh;
        const int64_t be = c->builds_enqueued;
        CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
        int nl = 0, rc = MD_OK;
        for (const Op &op : ops)
            if ((rc = enq_op(c, op, &nl))) break;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->st, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return fail(c, MD_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
        GraphRec rec{};
        e = cudaGraphInstantiate(&rec.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(c, MD_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
        rec.launches = nl;
        rec.xp_after = c->xp;
        rec.vp_after = c->vp;
        rec.pb_after = c->pb;
        it = c->graphs.emplace(key, rec).first;
        // capture changed the host bookkeeping; rewind, the replay re-applies it
        c->xp = xp0; c->vp = vp0; c->pb = pb0;
        c->moved_since_bin = mv; c->list_valid = lv; c->forces_valid = fv;
        c->v32_fresh = vf;
        c->builds_enqueued = be;
    }
    CK(cudaGraphLaunch(it->second.exec, c->st));
    c->launches += it->second.launches;
    c->xp = it->second.xp_after;
    c->vp = it->second.vp_after;
    c->pb = it->second.pb_after;
    for (const Op &op : ops) {
        if (op.kind == Op::REBUILD) {
            c->builds_enqueued++;
            c->rebuilds++;
            c->moved_since_bin = false;
            c->list_valid = true;
            if (uses_v32(c)) c->v32_fresh = true;
        } else if (op.kind == Op::KD) {
            c->moved_since_bin = true;
            c->forces_valid = false;
            c->v32_fresh = false;
        } else if (op.kind == Op::COND) {
            c->list_valid = true;   // valid under the displacement criterion
        } else {
            c->forces_valid = op.last;
            if (uses_v32(c)) c->v32_fresh = !op.last;   // fused contact step: next v32 written
            if (!op.last) c->moved_since_bin = true;
        }
    }
    return MD_OK;
}

int read_status(md_ctx *c, DevStatus *s)
{
    CK(cudaMemcpyAsync(s, c->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return MD_OK;
}

int check_flags(md_ctx *c, const DevStatus &s)
{
    if (s.flags & FLAG_NONFINITE) return fail(c, MD_ERR_NONFINITE, "non-finite position or velocity");
    if (s.flags & FLAG_BADPOS) return fail(c, MD_ERR_BADPOS, "an atom moved more than one box length between wraps");
    if (s.flags & FLAG_BOUNDS) return fail(c, MD_ERR_STATE, "a device bounds check failed (debug build)");
    if (s.flags & FLAG_DWRANGE)
        return fail(c, MD_ERR_BADPOS, "double-word path: an atom moved more than a cell side beyond "
                                      "its cell since the last binning");
    return MD_OK;
}

int grow_list(md_ctx *c, int32_t seen_max)
{
    int64_t want = std::max<int64_t>((int64_t)(seen_max * 1.2) + 8, (int64_t)active_cap(c) * 3 / 2);
    if (want > (int64_t)1 << 16) return fail(c, MD_ERR_NL_OVERFLOW, "neighbour list capacity limit reached");
    int rc = realloc_active(c, (int32_t)want);
    if (rc) return fail(c, MD_ERR_NL_OVERFLOW, "cannot grow the neighbour list: " + c->err);
    return MD_OK;
}

// Bin + build with overflow repair (direct launches, synchronising).
int rebuild_now(md_ctx *c, bool bin)
{
    for (int attempt = 0; attempt < 8; attempt++) {
        int nl = 0, rc;
        if (bin && (rc = enq_bin(c, &nl))) return rc;
        bin = false;
        if ((rc = enq_build(c, &nl))) return rc;
        c->launches += nl;
        c->rebuilds++;
        DevStatus s;
        if ((rc = read_status(c, &s))) return rc;
        if ((rc = check_flags(c, s))) return rc;
        c->last_max = s.max_count;
        if (!(s.flags & FLAG_NL_OVERFLOW)) return MD_OK;
        CK(cudaMemsetAsync(&c->status->flags, 0, sizeof(int32_t), c->st));
        if ((rc = grow_list(c, s.max_count))) return rc;
    }
    return fail(c, MD_ERR_NL_OVERFLOW, "neighbour list kept overflowing");
}

int ensure_list(md_ctx *c)
{
    if (c->list_valid && !c->moved_since_bin) return MD_OK;
    return rebuild_now(c, true);
}

int ensure_forces(md_ctx *c)
{
    if (c->forces_valid) return MD_OK;
    int rc = ensure_list(c);
    if (rc) return rc;
    int nl = 0;
    if ((rc = enq_force(c, EPI_F, false, &nl))) return rc;
    c->launches += nl;
    return MD_OK;
}

// A rebuild planned by run_span: its step and the buffer parities right
// after its binning (the state a resume after an overflow starts from).
struct PlannedRebuild {
    int64_t step;
    int xp_after_bin, vp_after_bin, pb;
};

// Plans steps (first .. last) and executes them; `kd` = the drift to x_first
// is still to be done.
int run_span(md_ctx *c, int64_t s0, int64_t first, int64_t last, bool kd, int32_t energy_every,
             std::vector<PlannedRebuild> *rebuilds)
{
    const int64_t every = c->p.rebuild_every;
    std::vector<Op> seg;
    if (c->disp) {
        // every step: conditional rebuild, then the fused force step; graphs
        // of up to kDispSeg steps (the same shapes recur and are replayed)
        constexpr int64_t kDispSeg = 20;
        if (kd) seg.push_back({Op::KD, first, false, false});
        for (int64_t nstep = first; nstep <= last; nstep++) {
            const bool en = energy_every > 0 && ((nstep - s0) % energy_every) == 0;
            seg.push_back({Op::COND, nstep, false, false});
            seg.push_back({Op::FORCE, nstep, nstep == last, en});
            if ((nstep - first + 1) % kDispSeg == 0 || nstep == last) {
                int rc = run_segment(c, seg);
                if (rc) return rc;
                seg.clear();
            }
        }
        return MD_OK;
    }
    if (kd) seg.push_back({Op::KD, first, false, false});
    for (int64_t nstep = first; nstep <= last; nstep++) {
        const bool rebuild = (nstep % every) == 0;
        if (rebuild) {
            if (!seg.empty()) {
                int rc = run_segment(c, seg);
                if (rc) return rc;
                seg.clear();
            }
            seg.push_back({Op::REBUILD, nstep, false, false});
            rebuilds->push_back({nstep, 1 - c->xp, 1 - c->vp, c->pb});
        }
        // energies are logged every energy_every steps counted from the run's start
        const bool en = energy_every > 0 && ((nstep - s0) % energy_every) == 0;
        seg.push_back({Op::FORCE, nstep, nstep == last, en});
    }
    if (!seg.empty()) return run_segment(c, seg);
    return MD_OK;
}

int make_context(md_ctx *c, const md_box *boxes, const md_params *p, const int64_t *counts,
                 int32_t nrep, const double *pos, const double *vel, void *stream, bool on_device);
int set_state(md_ctx *c, const double *pos, const double *vel, bool on_device);
int gather_to(md_ctx *c, int what, double *dst);
bool is_device_pointer(const void *p);

// LJ constants of c->p (the same expressions as the FP64 definition).
void set_lj_constants(md_ctx *c)
{
    const md_params &q = c->p;
    const double rs = q.cutoff + q.skin;
    LJ &lj = c->lj;
    lj.rc2 = q.cutoff * q.cutoff;
    lj.rs2 = rs * rs;
    const double s2 = q.sigma * q.sigma;
    lj.sigma6 = s2 * s2 * s2;
    lj.sigma = q.sigma;
    lj.c48e = 48.0 * q.epsilon;
    lj.c24e = 24.0 * q.epsilon;
    lj.c4e = 4.0 * q.epsilon;
    lj.eps = q.epsilon;
    lj.rc2f = (float)lj.rc2;
    lj.sigma6f = (float)lj.sigma6;
    lj.c48ef = (float)lj.c48e;
    lj.c24ef = (float)lj.c24e;
    lj.c4ef = (float)lj.c4e;
    lj.half_dt_m = 0.5 * q.dt / q.mass;
    lj.dt = q.dt;
    lj.mass = q.mass;
    // double-word constants: high part fl32(c), low part fl32(c - high)
    auto split2 = [](double v, float out[2]) {
        out[0] = (float)v;
        out[1] = (float)(v - (double)out[0]);
    };
    split2(lj.rc2, lj.dw_rc2);
    const double s6 = lj.sigma6, s12 = lj.sigma6 * lj.sigma6;
    split2(48.0 * q.epsilon * s12, lj.dw_a12);
    split2(24.0 * q.epsilon * s6, lj.dw_a6);
    split2(4.0 * q.epsilon * s12, lj.dw_b12);
    split2(4.0 * q.epsilon * s6, lj.dw_b6);
    {
        const double e = q.epsilon, sg = q.sigma, s5 = s6 / sg, s11 = s12 / sg;
        const double adj[10] = {192.0 * e * s6, 672.0 * e * s12, 48.0 * s12, 24.0 * s6,
                                576.0 * e * s11, 144.0 * e * s5, 2.0 * s12, 2.0 * s6,
                                24.0 * e * s11, 12.0 * e * s5};
        for (int k = 0; k < 10; k++) split2(adj[k], lj.dw_adj[k]);
    }
    lj.rs2f_lo = (float)(lj.rs2 * (1.0 - 2.5e-4));
    lj.rs2f_hi = (float)(lj.rs2 * (1.0 + 2.5e-4));
    // spring-dashpot constants (pot, sd_k, sd_g are set by md_set_spring_dashpot)
    lj.sigmaf = (float)q.sigma;
    lj.sd_sig2 = q.sigma * q.sigma;
    lj.sd_sig2f = (float)lj.sd_sig2;
    lj.sd_kf = (float)lj.sd_k;
    lj.sd_gf = (float)lj.sd_g;
    split2(lj.sd_sig2, lj.dw_sd_sig2);
    split2(q.sigma, lj.dw_sd_sig);
    split2(lj.sd_k, lj.dw_sd_k);
    split2(lj.sd_g, lj.dw_sd_g);
    split2(0.5 * lj.sd_k, lj.dw_sd_hk);
}

// Process-wide autotuner cache: (precision, log2 atoms per replica, batched)
// -> (threads per atom, list type, cell split).
struct Tuning {
    int tpa, lt, split;
};
std::map<std::string, Tuning> &tune_cache()
{
    static std::map<std::string, Tuning> m;
    return m;
}

std::mutex &tune_mutex()
{
    static std::mutex m;
    return m;
}

// Lanes per atom of the full-list force kernels from the atom count: the
// choices md_autotune measured on GB300 for FCC liquids (mixed: 8 at 4k
// atoms, 4 at ~16k, 2 at ~55k, 1 from 131k; double word: 8 at 4k, 4 at ~16k,
// 2 from ~55k to ~442k (64 against 72 us per step at 131k), 1 at 1M; FP64,
// bound by its FP64 pipe: 8 at 4k, 4 up to ~256k, 2 up to ~2M, 1 at 4M).
int default_lanes(int64_t n, int32_t precision)
{
    if (precision == MD_MIXED) return n <= 8192 ? 8 : (n <= 32768 ? 4 : (n <= 98304 ? 2 : 1));
    if (precision == MD_DW) return n <= 8192 ? 8 : (n <= 32768 ? 4 : (n <= 600000 ? 2 : 1));
    return n <= 8192 ? 8 : (n <= 393216 ? 4 : (n <= 3000000 ? 2 : 1));
}

// Cell arrays large enough for the binning keys of `split` (8 per cell id
// when split; keys 8 c + octant must stay below 2^31).  Synchronises.
int ensure_key_arrays(md_ctx *c, int split)
{
    const int64_t want = split ? c->nids * 8 : c->nids;
    if (split && want >= ((int64_t)1 << 31)) return fail(c, MD_ERR_INVAL, "too many cells to split");
    if (want <= c->key_cap) return MD_OK;
    CK(cudaStreamSynchronize(c->st));
    int32_t *cnt = nullptr, *start = nullptr, *tmp = nullptr;
    const int64_t tlen = scan_tmp_elems(want);
    int rc;
    if ((rc = dalloc(c, &cnt, (size_t)want)) || (rc = dalloc(c, &start, (size_t)want + 1)) ||
        (rc = dalloc(c, &tmp, (size_t)tlen))) {
        cudaFree(cnt); cudaFree(start); cudaFree(tmp);
        return rc;
    }
    CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)want, c->st));
    cudaFree(c->cell_count); cudaFree(c->cell_start); cudaFree(c->scan_tmp);
    c->cell_count = cnt;
    c->cell_start = start;
    c->scan_tmp = tmp;
    c->scan_len = tlen;
    c->key_cap = want;
    // captured graphs hold the old arrays
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
    c->graphs.clear();
    return MD_OK;
}

// Switches lanes-per-atom / list type / cell split; a list-type or split
// change rebins and rebuilds the list.
int apply_tuning(md_ctx *c, int tpa, int lt, int split)
{
    const bool relist = lt != c->p.list_type || split != c->split;
    if (split != c->split) {
        const int rc = ensure_key_arrays(c, split);
        if (rc) return rc;
    }
    c->split = split;
    c->tpa = tpa;
    c->p.threads_per_atom = tpa;
    c->p.list_type = lt;
    if ((lt == MD_LIST_GROUP2 || lt == MD_LIST_GROUP4) && (c->gsz != lt || !c->gnb)) {
        const int rc = alloc_group(c, lt, group_cap0(c, lt));
        if (rc) return rc;
    }
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
    c->graphs.clear();
    if (relist) {
        c->list_valid = false;
        c->forces_valid = false;
        return ensure_forces(c);
    }
    return MD_OK;
}

}  // namespace

// Error text for calls without a context (read by md_last_error(NULL)).
namespace mdk {
void set_global_error(const std::string &msg) { g_create_error = msg; }
}  // namespace mdk

// ---------------------------------------------------------------------------
// Public ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *md_last_error(const md_ctx *c)
{
    return c ? c->err.c_str() : g_create_error.c_str();
}

static int create_impl(int32_t nrep, const md_box *boxes, const md_params *p,
                       const int64_t *counts, const double *pos, const double *vel, void *stream,
                       md_ctx **out, bool on_device)
{
    if (!out) return fail(nullptr, MD_ERR_INVAL, "out is NULL");
    *out = nullptr;
    md_ctx *c = new (std::nothrow) md_ctx();
    if (!c) return fail(nullptr, MD_ERR_NOMEM, "host allocation failed");
    int rc = make_context(c, boxes, p, counts, nrep, pos, vel, stream, on_device);
    if (rc) {
        g_create_error = c->err;
        free_all(c);
        delete c;
        return rc;
    }
    *out = c;
    return MD_OK;
}

int md_create_batch(int32_t nrep, const md_box *boxes, const md_params *p, const int64_t *counts,
                    const double *pos, const double *vel, void *stream, md_ctx **out)
{
    return create_impl(nrep, boxes, p, counts, pos, vel, stream, out, false);
}

int md_create(const md_box *box, const md_params *p, int64_t n, const double *pos,
              const double *vel, void *stream, md_ctx **out)
{
    return create_impl(1, box, p, &n, pos, vel, stream, out, false);
}

int md_create_device(const md_box *box, const md_params *p, int64_t n, const double *pos,
                     const double *vel, void *stream, md_ctx **out)
{
    return create_impl(1, box, p, &n, pos, vel, stream, out, true);
}

void md_destroy(md_ctx *c)
{
    if (!c) return;
    if (c->st) cudaStreamSynchronize(c->st);
    free_all(c);
    delete c;
}

int md_set_state(md_ctx *c, const double *pos, const double *vel)
{
    if (!c || !pos || !vel) return fail(c, MD_ERR_INVAL, "null argument");
    return set_state(c, pos, vel, false);
}

int md_set_state_device(md_ctx *c, const double *pos, const double *vel)
{
    if (!c || !pos || !vel) return fail(c, MD_ERR_INVAL, "null argument");
    return set_state(c, pos, vel, true);
}

int md_bin_cells(md_ctx *c)
{
    if (!c) return fail(c, MD_ERR_INVAL, "null context");
    int nl = 0;
    int rc = enq_bin(c, &nl);
    c->launches += nl;
    if (rc) return rc;
    DevStatus s;
    if ((rc = read_status(c, &s))) return rc;
    return check_flags(c, s);
}

int md_build_neighbors(md_ctx *c)
{
    if (!c) return fail(c, MD_ERR_INVAL, "null context");
    return rebuild_now(c, c->moved_since_bin);
}

int md_compute_forces(md_ctx *c)
{
    if (!c) return fail(c, MD_ERR_INVAL, "null context");
    int rc = ensure_list(c);
    if (rc) return rc;
    int nl = 0;
    rc = enq_force(c, EPI_F, false, &nl);
    c->launches += nl;
    return rc;
}

int md_integrate(md_ctx *c, int32_t phase)
{
    if (!c) return fail(c, MD_ERR_INVAL, "null context");
    if (phase != 1 && phase != 2) return fail(c, MD_ERR_INVAL, "phase must be 1 or 2");
    int rc = ensure_forces(c);
    if (rc) return rc;
    int nl = 0;
    Dev d = view(c);
    if (launch_integrate(d, c->lj, c->p.precision, phase, batched(c), c->st, &nl))
        return fail(c, MD_ERR_CUDA, "integrate launch failed");
    c->launches += nl;
    c->v32_fresh = false;
    if (phase == 1) {
        c->moved_since_bin = true;
        c->forces_valid = false;
    } else {
        c->step++;
    }
    return MD_OK;
}

int md_energy(md_ctx *c, double *pe, double *ke, double *w)
{
    if (!c) return fail(c, MD_ERR_INVAL, "null context");
    int rc = ensure_list(c);
    if (rc) return rc;
    int nl = 0;
    if ((rc = enq_force(c, EPI_F, true, &nl))) return rc;
    if ((rc = enq_energy(c, true, c->eout_d, &nl))) return rc;
    c->launches += nl;
    std::vector<double> h(3 * (size_t)c->nrep);
    CK(cudaMemcpyAsync(h.data(), c->eout_d, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    for (int32_t r = 0; r < c->nrep; r++) {
        if (pe) pe[r] = h[3 * r + 0];
        if (ke) ke[r] = h[3 * r + 1];
        if (w) w[r] = h[3 * r + 2];
    }
    return MD_OK;
}

int md_thermo(md_ctx *c, const double *energies, int64_t nrec, md_thermo_rec *out)
{
    if (!c || !out || nrec < 1 || (!energies && nrec != 1))
        return fail(c, MD_ERR_INVAL, "bad argument");
    const size_t nin = 3 * (size_t)nrec * (size_t)c->nrep, nout = 6 * (size_t)nrec * (size_t)c->nrep;
    int rc = MD_OK, nl = 0;
    double *buf = nullptr;   // records in, thermo records out
    if ((rc = dalloc(c, &buf, nin + nout))) return rc;
    if (energies) {
        cudaError_t e = cudaMemcpyAsync(buf, energies, sizeof(double) * nin, cudaMemcpyHostToDevice, c->st);
        if (e != cudaSuccess) rc = fail(c, MD_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
    } else if (!(rc = ensure_list(c)) && !(rc = enq_force(c, EPI_F, true, &nl))) {
        rc = enq_energy(c, true, buf, &nl);
    }
    if (!rc && launch_thermo(c->reps_d, c->nrep, nrec, buf, buf + nin, c->st, &nl))
        rc = fail(c, MD_ERR_CUDA, "thermo launch failed");
    c->launches += nl;
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(out, buf + nin, sizeof(double) * nout, cudaMemcpyDeviceToHost, c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
        if (e != cudaSuccess) rc = fail(c, MD_ERR_CUDA, std::string("thermo copy: ") + cudaGetErrorString(e));
    }
    cudaFree(buf);
    return rc;
}

int md_run(md_ctx *c, int64_t nsteps, int32_t energy_every, double *energies)
{
    if (!c || nsteps < 0) return fail(c, MD_ERR_INVAL, "bad argument");
    if (nsteps == 0) return MD_OK;
    const bool log = energies && energy_every > 0;
    const int32_t ev = log ? energy_every : 0;
    int rc = ensure_forces(c);
    if (rc) return rc;
    const int64_t nlog = log ? nsteps / energy_every : 0;
    if (log) {
        if (nlog > c->elog_cap) {
            if (c->elog_d) cudaFree(c->elog_d);
            c->elog_d = nullptr;
            if ((rc = dalloc(c, &c->elog_d, (size_t)nlog * 3 * c->nrep))) return rc;
            c->elog_cap = nlog;
            for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
            c->graphs.clear();
        }
        CK(cudaMemsetAsync(&c->status->elog_cursor, 0, sizeof(int64_t), c->st));
    }
    const int64_t s0 = c->step;
    int64_t first = s0 + 1;
    const int64_t last = s0 + nsteps;
    bool kd = true;
    for (int attempt = 0; attempt < 8; attempt++) {
        std::vector<PlannedRebuild> planned;
        const int xp0 = c->xp, pb0 = c->pb;
        CK(cudaMemsetAsync(&c->status->rebuild_count, 0, sizeof(int64_t), c->st));
        CK(cudaMemsetAsync(&c->status->dev_step, 0, sizeof(int64_t), c->st));
        if ((rc = run_span(c, s0, first, last, kd, ev, &planned))) return rc;
        DevStatus s;
        if ((rc = read_status(c, &s))) return rc;
        if ((rc = check_flags(c, s))) return rc;
        if (c->disp) c->rebuilds += s.rebuild_count;
        if (c->disp && (s.flags & FLAG_NL_OVERFLOW)) {
            // The rebuild before the force of step n_fail overflowed and every
            // kernel after it returned at once: the state is x_n (drifted,
            // binned, copied back).  Parities at that step follow from the
            // fused steps done before it.  Grow the list, build, resume there.
            const int64_t n_fail = first + s.overflow_step - 1;
            if (s.overflow_step < 1 || n_fail > last)
                return fail(c, MD_ERR_NL_OVERFLOW, "list overflow at an unknown step");
            const int64_t done = n_fail - first;
            c->pb = pb0 ^ (int)(done & 1);
            c->xp = x_flips(c) ? (xp0 ^ (int)(done & 1)) : xp0;
            c->moved_since_bin = false;
            c->list_valid = false;
            c->forces_valid = false;
            CK(cudaMemsetAsync(&c->status->flags, 0, sizeof(int32_t), c->st));
            if ((rc = grow_list(c, s.max_count))) return rc;
            if ((rc = rebuild_now(c, false))) return rc;
            if (log) {
                int64_t before = 0;
                for (int64_t t = s0 + 1; t < n_fail; t++) before += ((t - s0) % ev) == 0;
                CK(cudaMemcpyAsync(&c->status->elog_cursor, &before, sizeof(int64_t),
                                   cudaMemcpyHostToDevice, c->st));
                CK(cudaStreamSynchronize(c->st));
            }
            first = n_fail;
            kd = false;
            continue;
        }
        if (!(s.flags & FLAG_NL_OVERFLOW)) {
            if (!planned.empty() || c->disp) c->last_max = s.max_count;
            c->step = last;
            if (log) {
                CK(cudaMemcpyAsync(energies, c->elog_d, sizeof(double) * 3 * c->nrep * nlog,
                                   cudaMemcpyDeviceToHost, c->st));
                CK(cudaStreamSynchronize(c->st));
            }
            return MD_OK;
        }
        // The k-th rebuild of this span overflowed and every kernel after it
        // returned at once: the device state is x_n (drifted, binned), v at
        // the half step.  Grow the list and resume at that rebuild.
        const int64_t k = s.overflow_at;
        if (k < 1 || k > (int64_t)planned.size())
            return fail(c, MD_ERR_NL_OVERFLOW, "list overflow at an unknown rebuild");
        const PlannedRebuild &pr = planned[(size_t)k - 1];
        c->xp = pr.xp_after_bin;
        c->vp = pr.vp_after_bin;
        c->pb = pr.pb;
        c->moved_since_bin = false;
        c->list_valid = false;
        c->forces_valid = false;
        c->v32_fresh = false;
        CK(cudaMemsetAsync(&c->status->flags, 0, sizeof(int32_t), c->st));
        if ((rc = grow_list(c, s.max_count))) return rc;
        if (log) {
            int64_t before = 0;
            for (int64_t t = s0 + 1; t < pr.step; t++) before += ((t - s0) % ev) == 0;
            CK(cudaMemcpyAsync(&c->status->elog_cursor, &before, sizeof(int64_t),
                               cudaMemcpyHostToDevice, c->st));
            CK(cudaStreamSynchronize(c->st));
        }
        first = pr.step;
        kd = false;
    }
    return fail(c, MD_ERR_NL_OVERFLOW, "neighbour list kept overflowing");
}

int md_get_positions(md_ctx *c, double *out)
{
    if (!c || !out) return fail(c, MD_ERR_INVAL, "null argument");
    int nl = 0;
    if (launch_gather_out(view(c), 0, c->io_d, c->st, &nl)) return fail(c, MD_ERR_CUDA, "gather failed");
    c->launches += nl;
    CK(cudaMemcpyAsync(out, c->io_d, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return MD_OK;
}

int md_get_velocities(md_ctx *c, double *out)
{
    if (!c || !out) return fail(c, MD_ERR_INVAL, "null argument");
    int nl = 0;
    if (launch_gather_out(view(c), 1, c->io_d, c->st, &nl)) return fail(c, MD_ERR_CUDA, "gather failed");
    c->launches += nl;
    CK(cudaMemcpyAsync(out, c->io_d, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return MD_OK;
}

int md_get_forces(md_ctx *c, double *out)
{
    if (!c || !out) return fail(c, MD_ERR_INVAL, "null argument");
    int rc = ensure_forces(c);
    if (rc) return rc;
    int nl = 0;
    if (launch_gather_out(view(c), is_mixed(c) ? 3 : 2, c->io_d, c->st, &nl))
        return fail(c, MD_ERR_CUDA, "gather failed");
    c->launches += nl;
    CK(cudaMemcpyAsync(out, c->io_d, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return MD_OK;
}

int md_get_positions_device(md_ctx *c, double *out)
{
    if (!c || !out) return fail(c, MD_ERR_INVAL, "null argument");
    if (!is_device_pointer(out)) return fail(c, MD_ERR_INVAL, "out is not a device pointer");
    return gather_to(c, 0, out);
}

int md_get_velocities_device(md_ctx *c, double *out)
{
    if (!c || !out) return fail(c, MD_ERR_INVAL, "null argument");
    if (!is_device_pointer(out)) return fail(c, MD_ERR_INVAL, "out is not a device pointer");
    return gather_to(c, 1, out);
}

int md_get_forces_device(md_ctx *c, double *out)
{
    if (!c || !out) return fail(c, MD_ERR_INVAL, "null argument");
    if (!is_device_pointer(out)) return fail(c, MD_ERR_INVAL, "out is not a device pointer");
    int rc = ensure_forces(c);
    if (rc) return rc;
    return gather_to(c, is_mixed(c) ? 3 : 2, out);
}

int md_get_cells(md_ctx *c, int32_t *cell_start, int32_t *cell_atoms)
{
    if (!c || !cell_start || !cell_atoms) return fail(c, MD_ERR_INVAL, "null argument");
    const int sh = 3 * c->split;
    std::vector<int32_t> cs(((size_t)c->nids << sh) + 1), ids((size_t)c->n);
    CK(cudaMemcpyAsync(cs.data(), c->cell_start, sizeof(int32_t) * cs.size(), cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(ids.data(), c->id[c->vp], sizeof(int32_t) * ids.size(), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    // device cells are numbered by tiles; report them in (cx, cy, cz) order,
    // each cell's atoms by caller id (split cells hold them by octant first)
    int64_t o = 0;
    for (int32_t r = 0; r < c->nrep; r++) {
        const Rep &R = c->reps_h[r];
        int64_t at = R.atom_off;
        for (int cx = 0; cx < R.nc[0]; cx++)
            for (int cy = 0; cy < R.nc[1]; cy++)
                for (int cz = 0; cz < R.nc[2]; cz++) {
                    const int64_t id = cell_id(R, cx, cy, cz);
                    cell_start[o++] = (int32_t)(at - R.atom_off);
                    const int64_t first = at;
                    for (int32_t a = cs[id << sh]; a < cs[(id + 1) << sh]; a++)
                        cell_atoms[at++] = (int32_t)(ids[a] - R.atom_off);
                    std::sort(cell_atoms + first, cell_atoms + at);
                }
        cell_start[o++] = (int32_t)(at - R.atom_off);
    }
    return MD_OK;
}

int md_get_neighbors(md_ctx *c, int32_t *counts, int32_t *rows, int32_t cap)
{
    if (!c || !counts || !rows || cap <= 0) return fail(c, MD_ERR_INVAL, "bad argument");
    int rc = ensure_list(c);
    if (rc) return rc;
    if (list_g(c)) {
        // exact rows filtered from the group rows on the device (FP64
        // criterion), then copied out with their lengths
        int32_t *buf = nullptr;
        if ((rc = dalloc(c, &buf, (size_t)c->n * ((size_t)cap + 1)))) return rc;
        int nl = 0;
        if (launch_decode_group(view(c), c->lj, list_g(c), buf, buf + c->n, cap, c->st, &nl)) {
            cudaFree(buf);
            return fail(c, MD_ERR_CUDA, "decode failed");
        }
        c->launches += nl;
        cudaError_t e = cudaMemcpyAsync(counts, buf, sizeof(int32_t) * c->n, cudaMemcpyDeviceToHost, c->st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(rows, buf + c->n, sizeof(int32_t) * c->n * cap, cudaMemcpyDeviceToHost, c->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
        cudaFree(buf);
        if (e != cudaSuccess) return fail(c, MD_ERR_CUDA, cudaGetErrorString(e));
        for (int64_t a = 0; a < c->n; a++)
            if (counts[a] > cap) return fail(c, MD_ERR_INVAL, "a row is longer than cap");
        return MD_OK;
    }
    std::vector<int32_t> cnt((size_t)c->n), ids((size_t)c->n);
    CK(cudaMemcpyAsync(cnt.data(), c->nb_count, sizeof(int32_t) * c->n, cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(ids.data(), c->id[c->vp], sizeof(int32_t) * c->n, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    for (int64_t a = 0; a < c->n; a++) {
        if (cnt[a] > cap) return fail(c, MD_ERR_INVAL, "a row is longer than cap");
        counts[ids[a]] = cnt[a];
    }
    int32_t *rows_d = nullptr;
    if ((rc = dalloc(c, &rows_d, (size_t)c->n * (size_t)cap))) return rc;
    int nl = 0;
    if (launch_decode_list(view(c), rows_d, cap, c->st, &nl)) {
        cudaFree(rows_d);
        return fail(c, MD_ERR_CUDA, "decode failed");
    }
    c->launches += nl;
    cudaError_t e = cudaMemcpyAsync(rows, rows_d, sizeof(int32_t) * c->n * cap, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    cudaFree(rows_d);
    if (e != cudaSuccess) return fail(c, MD_ERR_CUDA, cudaGetErrorString(e));
    return MD_OK;
}

int md_get_info(md_ctx *c, md_info *info)
{
    if (!c || !info) return fail(c, MD_ERR_INVAL, "null argument");
    info->n = c->n;
    info->nrep = c->nrep;
    info->precision = c->p.precision;
    info->list_type = c->p.list_type;
    info->threads_per_atom = c->tpa;
    info->list_capacity = active_cap(c);
    info->max_neighbors = c->last_max;
    info->ncells = c->ncells;
    info->step = c->step;
    info->kernel_launches = c->launches;
    info->rebuilds = c->rebuilds;
    info->cell_split = c->split;
    return MD_OK;
}

int md_set_cell_split(md_ctx *c, int32_t split)
{
    if (!c || (split != 0 && split != 1)) return fail(c, MD_ERR_INVAL, "split must be 0 or 1");
    if (split == c->split) return MD_OK;
    CK(cudaStreamSynchronize(c->st));
    int rc = ensure_key_arrays(c, split);
    if (rc) return rc;
    c->split = split;
    // new binning keys: rebin and rebuild (the rows hold the same pairs; the
    // order of a cell's entries, and so the force sums' rounding, changes)
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
    c->graphs.clear();
    c->list_valid = false;
    c->forces_valid = false;
    return ensure_forces(c);
}

int md_set_step(md_ctx *c, int64_t step)
{
    if (!c || step < 0) return fail(c, MD_ERR_INVAL, "bad argument");
    c->step = step;
    return MD_OK;
}

int md_set_capacity(md_ctx *c, int32_t cap)
{
    if (!c || cap < 4) return fail(c, MD_ERR_INVAL, "bad argument");
    CK(cudaStreamSynchronize(c->st));
    int rc = realloc_active(c, cap);
    if (rc) return rc;
    c->list_valid = false;
    c->forces_valid = false;
    return rebuild_now(c, c->moved_since_bin);
}

int md_profile(md_ctx *c, int64_t nsteps, md_phase_times *out)
{
    if (!c || !out || nsteps < 1) return fail(c, MD_ERR_INVAL, "bad argument");
    int rc = ensure_forces(c);
    if (rc) return rc;
    std::memset(out, 0, sizeof(*out));
    const int64_t s0 = c->step, every = c->p.rebuild_every;
    // per op: an outer event pair around all of its launches and, for force
    // ops, an inner pair around the force kernel alone.  Ops are enqueued one
    // by one; with the displacement trigger the rebuild decision of each step
    // is read back from the device first (profiling only).
    std::vector<Op> ops;
    std::vector<cudaEvent_t> ev;
    std::vector<int> nls;
    CK(cudaMemsetAsync(&c->status->rebuild_count, 0, sizeof(int64_t), c->st));
    auto enqueue = [&](const Op &op) -> int {
        cudaEvent_t e[4];
        for (auto &x : e) CK(cudaEventCreate(&x));
        for (auto &x : e) ev.push_back(x);
        int nl = 0, r;
        CK(cudaEventRecord(e[0], c->st));
        if (op.kind == Op::FORCE) r = enq_force(c, op.last ? EPI_FK : EPI_FKKD, op.energy, &nl, &e[2]);
        else r = enq_op(c, op, &nl);
        if (r) return r;
        CK(cudaEventRecord(e[1], c->st));
        ops.push_back(op);
        nls.push_back(nl);
        c->launches += nl;
        if (op.kind == Op::REBUILD) c->rebuilds++;
        return MD_OK;
    };
    rc = enqueue({Op::KD, s0 + 1, false, false});
    for (int64_t n = s0 + 1; !rc && n <= s0 + nsteps; n++) {
        bool rebuild = false;
        if (c->disp) {
            int32_t need = 0;
            CK(cudaMemcpyAsync(&need, &c->status->need_rebuild, sizeof(int32_t), cudaMemcpyDeviceToHost, c->st));
            CK(cudaStreamSynchronize(c->st));
            if (need) CK(cudaMemsetAsync(&c->status->need_rebuild, 0, sizeof(int32_t), c->st));
            rebuild = need != 0;
        } else {
            rebuild = n % every == 0;
        }
        if (rebuild && (rc = enqueue({Op::REBUILD, n, false, false}))) break;
        rc = enqueue({Op::FORCE, n, n == s0 + nsteps, false});
    }
    if (!rc) {
        DevStatus s;
        if (!(rc = read_status(c, &s))) rc = check_flags(c, s);
        if (!rc && (s.flags & FLAG_NL_OVERFLOW)) rc = fail(c, MD_ERR_NL_OVERFLOW, "list overflow while profiling");
        if (!rc) c->last_max = s.max_count;
    }
    for (size_t k = 0; !rc && k < ops.size(); k++) {
        float all = 0, kern = 0;
        CK(cudaEventElapsedTime(&all, ev[4 * k], ev[4 * k + 1]));
        if (ops[k].kind == Op::FORCE) {
            CK(cudaEventElapsedTime(&kern, ev[4 * k + 2], ev[4 * k + 3]));
            out->force_ms += kern;
            out->force_launches += 1;
            out->other_ms += all - kern;
            out->other_launches += nls[k] - 1;
        } else if (ops[k].kind == Op::REBUILD) {
            out->neigh_ms += all;
            out->neigh_launches += nls[k];
        } else {
            out->other_ms += all;
            out->other_launches += nls[k];
        }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (rc) return rc;
    c->step = s0 + nsteps;
    out->steps = nsteps;
    // list entries per atom: row lengths (of the groups, for group lists)
    // summed over the rows and divided by the atom count
    int64_t nrows = c->n;
    const int32_t *lens = c->nb_count;
    if (list_g(c)) {
        int32_t ng = 0;
        CK(cudaMemcpy(&ng, c->gcell_start + c->nids, sizeof(int32_t), cudaMemcpyDeviceToHost));
        nrows = ng;
        lens = c->gnb_count;
    }
    std::vector<int32_t> cnt((size_t)nrows);
    CK(cudaMemcpy(cnt.data(), lens, sizeof(int32_t) * nrows, cudaMemcpyDeviceToHost));
    double sum = 0;
    for (int32_t q : cnt) sum += q;
    out->mean_neighbors = sum / (double)c->n;
    out->rows = nrows;
    return MD_OK;
}

int md_set_lj(md_ctx *c, double epsilon, double sigma)
{
    if (!c || !(epsilon > 0) || !(sigma > 0) || !std::isfinite(epsilon) || !std::isfinite(sigma))
        return fail(c, MD_ERR_INVAL, "bad argument");
    CK(cudaStreamSynchronize(c->st));
    c->p.epsilon = epsilon;
    c->p.sigma = sigma;
    c->lj.pot = 0;
    set_lj_constants(c);
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
    c->graphs.clear();
    c->forces_valid = false;
    return MD_OK;
}

int md_set_spring_dashpot(md_ctx *c, double k_spring, double gamma)
{
    if (!c || !(k_spring >= 0) || !(gamma >= 0) || !std::isfinite(k_spring) || !std::isfinite(gamma))
        return fail(c, MD_ERR_INVAL, "bad argument");
    if (!(c->p.cutoff >= c->p.sigma))
        return fail(c, MD_ERR_INVAL, "cutoff must be >= sigma (the sphere diameter) so lists hold every contact");
    CK(cudaStreamSynchronize(c->st));
    int rc = MD_OK;
    for (int b = 0; b < 2; b++) {
        if (!c->v32[b]) {
            if ((rc = dalloc(c, &c->v32[b], (size_t)c->n + 1))) return rc;
            // slot n (the sentinel) stays zero: the fused step writes slots < n
            CK(cudaMemsetAsync(c->v32[b], 0, sizeof(float4) * ((size_t)c->n + 1), c->st));
        }
        if (is_dw(c) && !c->vlo[b]) {
            if ((rc = dalloc(c, &c->vlo[b], (size_t)c->n + 1))) return rc;
            CK(cudaMemsetAsync(c->vlo[b], 0, sizeof(float4) * ((size_t)c->n + 1), c->st));
        }
    }
    c->v32_fresh = false;
    // contacts use full per-atom lists
    if (c->p.list_type != MD_LIST_FULL && (rc = apply_tuning(c, 1, MD_LIST_FULL, c->split))) return rc;
    c->lj.pot = 1;
    c->lj.sd_k = k_spring;
    c->lj.sd_g = gamma;
    set_lj_constants(c);
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
    c->graphs.clear();
    c->forces_valid = false;
    return MD_OK;
}

static int adjoint_impl(md_ctx *c, int64_t nsteps, int64_t window, int32_t ckpt, double *loss,
                        double *g_eps, double *g_sigma, double *g_x0, double *g_v0, bool on_device)
{
    if (!c || !loss || nsteps < 1 || window < 1 || window > nsteps || ckpt < 1)
        return fail(c, MD_ERR_INVAL, "bad argument");
    if (on_device && ((g_x0 && !is_device_pointer(g_x0)) || (g_v0 && !is_device_pointer(g_v0))))
        return fail(c, MD_ERR_INVAL, "g_x0 / g_v0 are not device pointers of the current device");
    if (c->nrep != 1) return fail(c, MD_ERR_INVAL, "md_adjoint takes a single system");
    if (c->disp)
        return fail(c, MD_ERR_INVAL, "md_adjoint needs the fixed rebuild schedule (rebuild_every > 0)");
    if (is_sd(c)) return fail(c, MD_ERR_INVAL, "md_adjoint differentiates the Lennard-Jones force only");
    const int64_t every = c->p.rebuild_every;
    if (every % ckpt != 0 || nsteps % ckpt != 0)
        return fail(c, MD_ERR_INVAL, "ckpt_every must divide rebuild_every and nsteps");
    const int64_t n = c->n, nck = nsteps / ckpt + 1;
    // precision of the reverse sweep's pair terms (the forward run always
    // uses the context's precision): by default the context's own
    const int pp = c->adj_prec < 0 ? c->p.precision : c->adj_prec;
    const bool mixed = pp == MD_MIXED;
    const bool dw = is_dw(c);
    const bool dwp = pp == MD_DW;
    if (dwp && !dw) return fail(c, MD_ERR_INVAL, "double-word pair terms need an MD_DW context");
    const int lt0 = c->p.list_type, tpa0 = c->tpa;
    int rc = MD_OK;
    // the adjoint walks full per-atom lists (with the default lanes per atom
    // for the atom count when the context runs another list type, whose
    // tuned lanes belong to that type: the group lists run one per atom)
    if (lt0 != MD_LIST_FULL &&
        (rc = apply_tuning(c, default_lanes(c->n, c->p.precision), MD_LIST_FULL, c->split)))
        return rc;

    // workspace: reused between calls, grown when a call needs more
    auto &W = c->adj;
    auto drop = [](auto *&p) { if (p) cudaFree(p); p = nullptr; };
    if (nck > W.nck) { drop(W.ck_x); drop(W.ck_v); drop(W.ck_id); drop(W.ck_p); drop(W.ck_plo); W.nck = 0; }
    if (ckpt > W.ckpt) { drop(W.blk_x); drop(W.blk_p); drop(W.blk_plo); W.ckpt = 0; }
    if ((!W.ck_x && ((rc = dalloc(c, &W.ck_x, (size_t)(nck * n))) || (rc = dalloc(c, &W.ck_v, (size_t)(nck * n))) ||
                     (rc = dalloc(c, &W.ck_id, (size_t)(nck * n))) || (rc = dalloc(c, &W.ck_p, (size_t)(nck * n))))) ||
        (!W.blk_x && ((rc = dalloc(c, &W.blk_x, (size_t)(ckpt * n))) || (rc = dalloc(c, &W.blk_p, (size_t)(ckpt * n))))) ||
        (!W.xbar && ((rc = dalloc(c, &W.xbar, (size_t)n)) || (rc = dalloc(c, &W.wbar, (size_t)n)) ||
                     (rc = dalloc(c, &W.ge, (size_t)n)) || (rc = dalloc(c, &W.gs, (size_t)n)) ||
                     (rc = dalloc(c, &W.g2, 2)))) ||
        ((mixed || dwp) && !W.wbar32 && (rc = dalloc(c, &W.wbar32, (size_t)n))) ||
        (dwp && !W.wbar_lo && (rc = dalloc(c, &W.wbar_lo, (size_t)n))) ||
        (dwp && !W.blk_plo && (rc = dalloc(c, &W.blk_plo, (size_t)(W.ckpt ? W.ckpt * n : ckpt * n)))) ||
        (dw && !W.ck_plo && (rc = dalloc(c, &W.ck_plo, (size_t)(W.nck ? W.nck * n : nck * n))))) {
        // release the whole workspace: a later call starts from scratch
        drop(W.ck_x); drop(W.ck_v); drop(W.ck_id); drop(W.ck_p); drop(W.ck_plo); drop(W.blk_x); drop(W.blk_p);
        drop(W.blk_plo); drop(W.wbar_lo);
        drop(W.xbar); drop(W.wbar); drop(W.wbar32); drop(W.ge); drop(W.gs); drop(W.g2);
        W.nck = W.ckpt = 0;
        return rc;
    }
    W.nck = std::max<int64_t>(W.nck, nck);
    W.ckpt = std::max<int64_t>(W.ckpt, ckpt);
    dvec4 *ck_x = W.ck_x, *ck_v = W.ck_v, *blk_x = W.blk_x, *xbar = W.xbar, *wbar = W.wbar;
    float4 *blk_p = W.blk_p, *ck_p = W.ck_p, *wbar32 = (mixed || dwp) ? W.wbar32 : nullptr;
    float4 *ck_plo = dw ? W.ck_plo : nullptr;
    float4 *blk_plo = dwp ? W.blk_plo : nullptr, *wbar_lo = dwp ? W.wbar_lo : nullptr;
    int32_t *ck_id = W.ck_id;
    double *ge = W.ge, *gs = W.gs, *g2 = W.g2;
    if (window > c->elog_cap) {
        if (c->elog_d) cudaFree(c->elog_d);
        c->elog_d = nullptr;
        if ((rc = dalloc(c, &c->elog_d, (size_t)window * 3))) return rc;
        c->elog_cap = window;
        for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second.exec);
        c->graphs.clear();
    }
    int nl = 0;
    auto save_ck = [&](int64_t k) {
        cudaMemcpyAsync(ck_x + k * n, c->x[c->xp], sizeof(dvec4) * n, cudaMemcpyDeviceToDevice, c->st);
        cudaMemcpyAsync(ck_v + k * n, c->v[c->vp], sizeof(dvec4) * n, cudaMemcpyDeviceToDevice, c->st);
        cudaMemcpyAsync(ck_id + k * n, c->id[c->vp], sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, c->st);
        cudaMemcpyAsync(ck_p + k * n, c->p32[c->pb], sizeof(float4) * n, cudaMemcpyDeviceToDevice, c->st);
        if (ck_plo)
            cudaMemcpyAsync(ck_plo + k * n, c->plo[c->pb], sizeof(float4) * n, cudaMemcpyDeviceToDevice, c->st);
    };
    auto load_ck = [&](int64_t k, bool with_id) {
        cudaMemcpyAsync(c->x[c->xp], ck_x + k * n, sizeof(dvec4) * n, cudaMemcpyDeviceToDevice, c->st);
        cudaMemcpyAsync(c->v[c->vp], ck_v + k * n, sizeof(dvec4) * n, cudaMemcpyDeviceToDevice, c->st);
        if (with_id)
            cudaMemcpyAsync(c->id[c->vp], ck_id + k * n, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, c->st);
        else {  // mid-epoch: the FP32 cell-relative copy of the same step
            cudaMemcpyAsync(c->p32[c->pb], ck_p + k * n, sizeof(float4) * n, cudaMemcpyDeviceToDevice, c->st);
            if (ck_plo)   // and on the double-word path its low parts
                cudaMemcpyAsync(c->plo[c->pb], ck_plo + k * n, sizeof(float4) * n, cudaMemcpyDeviceToDevice, c->st);
        }
    };
    // state at force point cb: the list of its epoch (built from the epoch's
    // start positions, which re-binning reproduces bit for bit), then x, v.
    // check: the rebuild reads the device status back (overflow repair);
    // else it is only enqueued (the forward sweep already built every list of
    // the run with this capacity, so the same positions cannot overflow it;
    // the status is read once after the reverse sweep).
    // list_epoch: the epoch whose list (and slot order) the context holds, or
    // -1.  A block of an epoch whose list is built only loads its checkpoint
    // (saved in that slot order): x, v and the FP32 positions.
    int64_t list_epoch = -1;
    auto restore = [&](int64_t cb, bool check) -> int {
        const int64_t e = cb - cb % every;
        if (!check && e == list_epoch) {
            load_ck(cb / ckpt, false);
            c->forces_valid = false;
            return MD_OK;
        }
        load_ck(e / ckpt, true);
        c->moved_since_bin = true;
        int r;
        if (check) {
            r = rebuild_now(c, true);
        } else if (!(r = enq_bin(c, &nl)) && !(r = enq_build(c, &nl))) {
            c->rebuilds++;
        }
        if (r) return r;
        list_epoch = check ? -1 : e;
        if (e != cb) load_ck(cb / ckpt, false);
        return MD_OK;
    };
    auto kick_drift = [&]() -> int {
        Dev d = view(c);
        if (launch_integrate(d, c->lj, c->p.precision, 1, false, c->st, &nl))
            return fail(c, MD_ERR_CUDA, "integrate launch failed");
        return MD_OK;
    };

    // ---- forward, with checkpoints ---------------------------------------
    // md_run's path: spans of fused steps replayed from the context's cached
    // graphs (the same trajectory bit for bit as separate kick-drift and
    // force launches), a span ending at every checkpoint and where the loss
    // window starts (energies logged on every step inside it).  The status is
    // read once at the end: a rebuild that overflowed stops every later
    // kernel, and the forward then reruns from step 0 with a larger list.
    std::vector<double> elog((size_t)window * 3);
    const int64_t w0 = nsteps - window;      // steps after w0 are in the loss window
    for (int attempt = 0;; attempt++) {
        if (attempt == 8) return fail(c, MD_ERR_NL_OVERFLOW, "neighbour list kept overflowing");
        if ((rc = attempt == 0 ? rebuild_now(c, true) : restore(0, true))) return rc;
        if ((rc = enq_force(c, EPI_F, false, &nl))) return rc;
        save_ck(0);
        CK(cudaMemsetAsync(&c->status->elog_cursor, 0, sizeof(int64_t), c->st));
        std::vector<PlannedRebuild> planned;
        for (int64_t s = 0; s < nsteps;) {
            int64_t last = std::min<int64_t>((s / ckpt + 1) * ckpt, nsteps);
            if (s < w0 && last > w0) last = w0;
            if ((rc = run_span(c, s, s + 1, last, true, s >= w0 ? 1 : 0, &planned))) return rc;
            s = last;
            if (s % ckpt == 0) save_ck(s / ckpt);
        }
        CK(cudaMemcpyAsync(elog.data(), c->elog_d, sizeof(double) * elog.size(), cudaMemcpyDeviceToHost, c->st));
        DevStatus st;
        if ((rc = read_status(c, &st)) || (rc = check_flags(c, st))) return rc;
        c->last_max = st.max_count;
        if (!(st.flags & FLAG_NL_OVERFLOW)) break;
        CK(cudaMemsetAsync(&c->status->flags, 0, sizeof(int32_t), c->st));
        if ((rc = grow_list(c, st.max_count))) return rc;
    }
    double acc = 0;
    for (int64_t k = 0; k < window; k++) acc += elog[3 * k];
    *loss = acc / (double)window;

    // ---- reverse sweep ------------------------------------------------------
    // the forward ended on the list of its last epoch, in that slot order
    list_epoch = nsteps - nsteps % every;
    CK(cudaMemsetAsync(xbar, 0, sizeof(dvec4) * n, c->st));
    CK(cudaMemsetAsync(wbar, 0, sizeof(dvec4) * n, c->st));
    if (wbar32) CK(cudaMemsetAsync(wbar32, 0, sizeof(float4) * n, c->st));
    if (wbar_lo) CK(cudaMemsetAsync(wbar_lo, 0, sizeof(float4) * n, c->st));
    CK(cudaMemsetAsync(ge, 0, sizeof(double) * n, c->st));
    CK(cudaMemsetAsync(gs, 0, sizeof(double) * n, c->st));
    const double cdt = c->lj.half_dt_m;
    for (int64_t b = nck - 1; b >= 0 && !rc; b--) {
        const int64_t cb = b * ckpt;
        const int64_t npts = (b == nck - 1) ? 1 : ckpt;
        if ((rc = restore(cb, false))) break;
        if ((rc = enq_force(c, EPI_F, false, &nl))) break;
        for (int64_t m = 0; m < npts && !rc; m++) {
            // the state at point cb + m, by the forward's own launches: a
            // kick-drift with the forces of cb for the first step of the block,
            // then one fused step per point (force at the previous point, both
            // half kicks, drift), so the recompute is the forward bit for bit
            if (m == 1) rc = kick_drift();
            else if (m > 1) rc = enq_force(c, EPI_FKKD, false, &nl);
            if (rc) break;
            // the snapshot the pair terms read: FP32 cell-relative positions
            // (mixed pair terms) or FP64 positions (FP64 pair terms, which
            // take only the cell coordinates from p32: fixed for the epoch)
            // (double-word pair terms: the high and low parts of the split positions)
            if (mixed || dwp)
                cudaMemcpyAsync(blk_p + m * n, c->p32[c->pb], sizeof(float4) * n, cudaMemcpyDeviceToDevice, c->st);
            else
                cudaMemcpyAsync(blk_x + m * n, c->x[c->xp], sizeof(dvec4) * n, cudaMemcpyDeviceToDevice, c->st);
            if (dwp)
                cudaMemcpyAsync(blk_plo + m * n, c->plo[c->pb], sizeof(float4) * n, cudaMemcpyDeviceToDevice, c->st);
        }
        for (int64_t m = npts - 1; m >= 0 && !rc; m--) {
            const int64_t pt = cb + m;
            if (pt < nsteps &&
                launch_adjoint_axpy(n, c->lj.dt, xbar, wbar, wbar32, wbar_lo, c->id[c->vp], c->st, &nl)) {
                rc = fail(c, MD_ERR_CUDA, "adjoint launch failed");
                break;
            }
            const double k = pt == nsteps ? 0.0 : (pt == 0 ? cdt : 2.0 * cdt);
            const double lw = pt > nsteps - window ? 1.0 / (double)window : 0.0;
            // the pair terms read the recomputed snapshot of force point pt
            // in place (same atom order and list as the whole block)
            Dev dv = view(c);
            if (mixed || dwp) dv.p32 = blk_p + m * n;
            else dv.x = blk_x + m * n;
            if (dwp) dv.plo = blk_plo + m * n;
            if (dwp ? launch_adjoint_pairs_dw(dv, c->lj, c->tpa, wbar32, wbar_lo, xbar, ge, gs, k, lw, c->st, &nl)
                    : launch_adjoint_pairs(dv, c->lj, mixed, c->tpa, wbar, wbar32, xbar, ge, gs, k, lw, c->st, &nl)) {
                rc = fail(c, MD_ERR_CUDA, "adjoint launch failed");
                break;
            }
        }
    }
    if (!rc && launch_sum2(n, ge, gs, g2, c->st, &nl)) rc = fail(c, MD_ERR_CUDA, "sum launch failed");
    if (!rc) {
        // the reverse sweep's rebuilds and kernels, checked once
        DevStatus st;
        if (!(rc = read_status(c, &st)) && !(rc = check_flags(c, st)) && (st.flags & FLAG_NL_OVERFLOW))
            rc = fail(c, MD_ERR_NL_OVERFLOW, "a recomputed list overflowed");
    }
    if (!rc && on_device) {
        // gradients straight into the caller's device buffers (n x 3)
        if ((g_x0 && launch_unpad3(n, xbar, g_x0, c->st, &nl)) ||
            (g_v0 && launch_unpad3(n, wbar, g_v0, c->st, &nl)))
            rc = fail(c, MD_ERR_CUDA, "gradient copy launch failed");
    }
    if (!rc) {
        double g[2];
        CK(cudaMemcpyAsync(g, g2, sizeof(g), cudaMemcpyDeviceToHost, c->st));
        std::vector<dvec4> hx, hw;
        if (!on_device) {
            hx.resize((size_t)n);
            hw.resize((size_t)n);
            CK(cudaMemcpyAsync(hx.data(), xbar, sizeof(dvec4) * n, cudaMemcpyDeviceToHost, c->st));
            CK(cudaMemcpyAsync(hw.data(), wbar, sizeof(dvec4) * n, cudaMemcpyDeviceToHost, c->st));
        }
        CK(cudaStreamSynchronize(c->st));
        if (g_eps) *g_eps = g[0];
        if (g_sigma) *g_sigma = g[1];
        for (int64_t a = 0; !on_device && a < n; a++) {
            if (g_x0) { g_x0[3 * a] = hx[a].x; g_x0[3 * a + 1] = hx[a].y; g_x0[3 * a + 2] = hx[a].z; }
            if (g_v0) { g_v0[3 * a] = hw[a].x; g_v0[3 * a + 1] = hw[a].y; g_v0[3 * a + 2] = hw[a].z; }
        }
        rc = restore(0, true);      // leave the context at the initial state
    }
    c->launches += nl;
    c->forces_valid = false;
    if (!rc && lt0 != MD_LIST_FULL) rc = apply_tuning(c, tpa0, lt0, c->split);
    return rc;
}

int md_adjoint(md_ctx *c, int64_t nsteps, int64_t window, int32_t ckpt, double *loss,
               double *g_eps, double *g_sigma, double *g_x0, double *g_v0)
{
    return adjoint_impl(c, nsteps, window, ckpt, loss, g_eps, g_sigma, g_x0, g_v0, false);
}

int md_adjoint_device(md_ctx *c, int64_t nsteps, int64_t window, int32_t ckpt, double *loss,
                      double *g_eps, double *g_sigma, double *g_x0, double *g_v0)
{
    return adjoint_impl(c, nsteps, window, ckpt, loss, g_eps, g_sigma, g_x0, g_v0, true);
}

int md_study_force_variant(md_ctx *c, int32_t variant, int32_t reps, double *us, double *forces)
{
    if (!c || !us || reps < 1 || variant < 0 || variant > 6) return fail(c, MD_ERR_INVAL, "bad argument");
    if (!is_mixed(c) || c->p.list_type != MD_LIST_FULL || is_sd(c) || c->nrep != 1)
        return fail(c, MD_ERR_STATE, "force studies take a single-system mixed LJ context with full lists");
    if ((variant == 3 || variant == 4) && kTile != 2)
        return fail(c, MD_ERR_STATE, "the shared-memory study stages 2x2x2-cell tiles (a build with MD_CELL_TILE = 2)");
    int rc = ensure_list(c);
    if (rc) return rc;
    float4 *fout = nullptr;
    float *lay = nullptr;
    if ((rc = dalloc(c, &fout, (size_t)c->n)) || (rc = dalloc(c, &lay, (size_t)study_layout_floats(c->n)))) {
        cudaFree(fout);
        return rc;
    }
    Dev d = view(c);
    d.f32 = fout;                                    // the library's kernel writes here too
    const int64_t ntiles = (int64_t)c->reps_h[0].nt[0] * c->reps_h[0].nt[1] * c->reps_h[0].nt[2];
    // variants 5 and 6: a texture object over the current FP32 positions
    cudaTextureObject_t tex = 0;
    if (variant >= 5) {
        int maxw = 0;
        cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxTexture1DLinearWidth, c->device);
        if ((int64_t)c->n + 1 > (int64_t)maxw) {
            cudaFree(fout);
            cudaFree(lay);
            return fail(c, MD_ERR_STATE, "more atoms than a linear texture holds");
        }
        cudaResourceDesc rd{};
        rd.resType = cudaResourceTypeLinear;
        rd.res.linear.devPtr = d.p32;
        rd.res.linear.desc = cudaCreateChannelDesc<float4>();
        rd.res.linear.sizeInBytes = sizeof(float4) * ((size_t)c->n + 1);
        cudaTextureDesc td{};
        td.addressMode[0] = cudaAddressModeClamp;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        if (cudaCreateTextureObject(&tex, &rd, &td, nullptr) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(fout);
            cudaFree(lay);
            return fail(c, MD_ERR_CUDA, "cudaCreateTextureObject failed");
        }
    }
    int nl = 0;
    auto launch = [&]() -> int {
        if (variant == 0) return launch_force(d, c->lj, MD_MIXED, false, 1, EPI_F, false, false, c->st, &nl);
        if (variant == 3 || variant == 4)
            return launch_study_tiles(d, c->lj, ntiles, variant == 4, fout, c->st, &nl);
        return launch_study_force(d, c->lj, variant, lay, tex, fout, c->st, &nl);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess && launch() != 0) e = cudaErrorLaunchFailure;   // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, c->st);
    for (int32_t r = 0; e == cudaSuccess && r < reps; r++)
        if (launch() != 0) e = cudaErrorLaunchFailure;
    if (e == cudaSuccess) e = cudaEventRecord(e1, c->st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    c->launches += nl;
    if (e == cudaSuccess) {
        *us = 1e3 * (double)ms / reps;
        DevStatus st;
        if (!(rc = read_status(c, &st)) && (st.flags & (FLAG_NL_OVERFLOW | FLAG_TIMEOUT))) {
            CK(cudaMemsetAsync(&c->status->flags, 0, sizeof(int32_t), c->st));
            rc = (st.flags & FLAG_TIMEOUT)
                     ? fail(c, MD_ERR_TIMEOUT, "a bulk copy into shared memory did not complete in time")
                     : fail(c, MD_ERR_STATE, "a tile neighbourhood holds more atoms than the staging array");
        }
        if (!rc && forces) {
            nl = 0;
            if (launch_gather_out(d, 3, c->io_d, c->st, &nl) != 0) rc = fail(c, MD_ERR_CUDA, "gather failed");
            c->launches += nl;
            if (!rc) {
                e = cudaMemcpyAsync(forces, c->io_d, sizeof(double) * 3 * c->n, cudaMemcpyDeviceToHost, c->st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (tex) cudaDestroyTextureObject(tex);
    cudaFree(fout);
    cudaFree(lay);
    if (e != cudaSuccess && !rc) rc = fail(c, MD_ERR_CUDA, std::string("study: ") + cudaGetErrorString(e));
    return rc;
}

int md_set_adjoint_precision(md_ctx *c, int32_t precision)
{
    if (!c || (precision != MD_FP64 && precision != MD_MIXED && precision != MD_DW))
        return fail(c, MD_ERR_INVAL, "precision must be MD_FP64, MD_MIXED or MD_DW");
    if (precision == MD_DW && !is_dw(c))
        return fail(c, MD_ERR_INVAL, "double-word pair terms need an MD_DW context");
    c->adj_prec = precision;
    return MD_OK;
}

int md_autotune(md_ctx *c, int32_t steps, md_params *chosen)
{
    if (!c || steps < 1) return fail(c, MD_ERR_INVAL, "bad argument");
    if (is_sd(c)) {   // one contact kernel: nothing to choose
        if (chosen) { *chosen = c->p; chosen->threads_per_atom = c->tpa; }
        return MD_OK;
    }
    const int64_t per_rep = c->n / c->nrep;
    int bucket = 0;
    while (((int64_t)1 << (bucket + 1)) <= per_rep) bucket++;
    const std::string key = std::to_string(c->p.precision) + ":" + std::to_string(bucket) + ":" +
                            std::to_string(c->nrep > 1);
    {
        std::lock_guard<std::mutex> g(tune_mutex());
        auto it = tune_cache().find(key);
        if (it != tune_cache().end()) {
            int rc = apply_tuning(c, it->second.tpa, it->second.lt, it->second.split);
            if (rc) return rc;
            if (chosen) { *chosen = c->p; chosen->threads_per_atom = c->tpa; }
            return MD_OK;
        }
    }
    int rc = ensure_forces(c);
    if (rc) return rc;
    // device backup of the current (cell-ordered) state
    dvec4 *xb = nullptr, *vb = nullptr;
    int32_t *ib = nullptr;
    if ((rc = dalloc(c, &xb, (size_t)c->n)) || (rc = dalloc(c, &vb, (size_t)c->n)) ||
        (rc = dalloc(c, &ib, (size_t)c->n))) {
        cudaFree(xb); cudaFree(vb); cudaFree(ib);
        return rc;
    }
    const int64_t step0 = c->step;
    auto save = [&]() {
        cudaMemcpyAsync(xb, c->x[c->xp], sizeof(dvec4) * c->n, cudaMemcpyDeviceToDevice, c->st);
        cudaMemcpyAsync(vb, c->v[c->vp], sizeof(dvec4) * c->n, cudaMemcpyDeviceToDevice, c->st);
        cudaMemcpyAsync(ib, c->id[c->vp], sizeof(int32_t) * c->n, cudaMemcpyDeviceToDevice, c->st);
    };
    auto restore = [&]() -> int {
        cudaMemcpyAsync(c->x[c->xp], xb, sizeof(dvec4) * c->n, cudaMemcpyDeviceToDevice, c->st);
        cudaMemcpyAsync(c->v[c->vp], vb, sizeof(dvec4) * c->n, cudaMemcpyDeviceToDevice, c->st);
        cudaMemcpyAsync(c->id[c->vp], ib, sizeof(int32_t) * c->n, cudaMemcpyDeviceToDevice, c->st);
        c->step = step0;
        c->moved_since_bin = true;
        c->list_valid = false;
        c->forces_valid = false;
        int r = ensure_forces(c);
        return r;
    };
    save();
    // (lanes per atom, list type); lists shared by groups are mixed-path only
    const int cands[7][2] = {{1, MD_LIST_FULL},   {2, MD_LIST_FULL}, {4, MD_LIST_FULL},
                             {8, MD_LIST_FULL},   {1, MD_LIST_HALF}, {1, MD_LIST_GROUP4},
                             {1, MD_LIST_GROUP2}};
    float best = 1e30f;
    int best_k = 0, best_split = c->split;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // times `steps` steps of one configuration from the saved state
    auto time_one = [&](int k, int split, float *ms) -> int {
        int r;
        if ((r = apply_tuning(c, cands[k][0], cands[k][1], split))) return r;
        if ((r = md_run(c, steps, 0, nullptr))) return r;  // warm-up (graph capture)
        if ((r = restore())) return r;
        CK(cudaEventRecord(e0, c->st));
        if ((r = md_run(c, steps, 0, nullptr))) return r;
        CK(cudaEventRecord(e1, c->st));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(ms, e0, e1));
        return restore();
    };
    // lanes per atom and list type at the current cell split, then the
    // winner with the other split (the cell size of the list build)
    // (the double-word path runs full lists only)
    const int ncand = is_mixed(c) ? 7 : (is_dw(c) ? 4 : 5);
    const int split0 = c->split;
    for (int k = 0; k < ncand && !rc; k++) {
        float ms = 0;
        if ((rc = time_one(k, split0, &ms))) break;
        if (ms < best) { best = ms; best_k = k; }
    }
    // (split cells need their binning keys 8 c + octant below 2^31)
    if (!rc && (split0 == 1 || c->nids * 8 < ((int64_t)1 << 31))) {
        float ms = 0;
        if (!(rc = time_one(best_k, 1 - split0, &ms)) && ms < best) {
            best = ms;
            best_split = 1 - split0;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(xb); cudaFree(vb); cudaFree(ib);
    if (rc) return rc;
    if ((rc = apply_tuning(c, cands[best_k][0], cands[best_k][1], best_split))) return rc;
    {
        std::lock_guard<std::mutex> g(tune_mutex());
        tune_cache()[key] = {cands[best_k][0], cands[best_k][1], best_split};
    }
    if (chosen) { *chosen = c->p; chosen->threads_per_atom = c->tpa; }
    return MD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Context construction
// ---------------------------------------------------------------------------
namespace {

// True if p is memory the current device can read (device or managed).
bool is_device_pointer(const void *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int make_context(md_ctx *c, const md_box *boxes, const md_params *p, const int64_t *counts,
                 int32_t nrep, const double *pos, const double *vel, void *stream, bool on_device)
{
    if (!boxes || !p || !counts || !pos || !vel || nrep <= 0)
        return fail(c, MD_ERR_INVAL, "null argument or nrep <= 0");
    const md_params &q = *p;
    if (!(q.epsilon > 0) || !(q.sigma > 0) || !(q.mass > 0) || !(q.cutoff > 0) || !(q.skin >= 0) ||
        !(q.dt > 0) || q.rebuild_every < 0 ||
        (q.precision != MD_FP64 && q.precision != MD_MIXED && q.precision != MD_DW) ||
        (q.list_type != MD_LIST_FULL && q.list_type != MD_LIST_HALF &&
         q.list_type != MD_LIST_GROUP2 && q.list_type != MD_LIST_GROUP4) ||
        !(q.threads_per_atom == 0 || q.threads_per_atom == 1 || q.threads_per_atom == 2 ||
          q.threads_per_atom == 4 || q.threads_per_atom == 8))
        return fail(c, MD_ERR_INVAL, "invalid md_params");
    if ((q.list_type == MD_LIST_GROUP2 || q.list_type == MD_LIST_GROUP4) && q.precision != MD_MIXED)
        return fail(c, MD_ERR_INVAL, "lists shared by groups of atoms need the mixed path");
    if (q.precision == MD_DW && q.list_type != MD_LIST_FULL)
        return fail(c, MD_ERR_INVAL, "the double-word path runs full per-atom lists");
    c->p = q;
    c->nrep = nrep;
    c->disp = q.rebuild_every == 0;
    {
        // trigger distance just below skin/2 (FP32 displacements are good to ~1e-7)
        const double h = std::max(0.0, 0.5 * q.skin - 1e-5);
        c->disp2_thr = std::nextafter((float)(h * h), 0.0f);
        if (!(c->disp2_thr > 0.f)) c->disp2_thr = 0.f;
    }
    c->tpa = q.threads_per_atom ? q.threads_per_atom : 1;
    const double rs = q.cutoff + q.skin;
    int64_t n = 0, cells = 0, ids = 0;   // cells, and cell ids with tile padding
    double maxrho = 0;
    int64_t maxn = 0;
    c->reps_h.resize(nrep);
    c->counts_h.assign(counts, counts + nrep);
    std::vector<int64_t> chunk_rep, chunk_first;
    for (int32_t r = 0; r < nrep; r++) {
        if (counts[r] <= 0) return fail(c, MD_ERR_INVAL, "a replica has no atoms");
        const double L[3] = {boxes[r].lx, boxes[r].ly, boxes[r].lz};
        Rep R{};
        double vol = 1;
        for (int d = 0; d < 3; d++) {
            if (!std::isfinite(L[d]) || !(L[d] > 0)) return fail(c, MD_ERR_INVAL, "invalid box");
            if (!(L[d] >= 2.0 * rs)) return fail(c, MD_ERR_BOX_TOO_SMALL, "box smaller than 2 (rc + skin)");
            R.L[d] = L[d];
            R.halfL[d] = 0.5 * L[d];
            R.nc[d] = (int32_t)std::floor(L[d] / rs);
            if (R.nc[d] > kMaxNc) return fail(c, MD_ERR_INVAL, "more than 1023 cells along a box edge");
            R.s[d] = L[d] / (double)R.nc[d];
            R.nsf[d] = -(float)R.s[d];
            R.invsf[d] = 1.0f / (float)R.s[d];
            // the split build's threshold s - rs - 1e-3 s, rounded down
            const double t = R.s[d] - rs - 1e-3 * R.s[d];
            R.splitf[d] = (float)t;
            if ((double)R.splitf[d] > t) R.splitf[d] = std::nextafter(R.splitf[d], -INFINITY);
            vol *= L[d];
        }
        for (int d = 0; d < 3; d++) R.nt[d] = (R.nc[d] + kTile - 1) / kTile;
        {
            // double-word positions: grid step g = 2^k, the least with
            // 2^24 g >= 2.5 max(s); s = s_h + s_l with s_h a multiple of g
            const double smax = std::max(R.s[0], std::max(R.s[1], R.s[2]));
            double g = std::ldexp(1.0, (int)std::floor(std::log2(2.5 * smax)) - 26);
            while (std::ldexp(g, 24) < 2.5 * smax) g *= 2.0;
            R.dw_magic = 1.5 * std::ldexp(g, 52);
            for (int d = 0; d < 3; d++) {
                const double sh = std::nearbyint(R.s[d] / g) * g;
                R.dw_sh[d] = (float)sh;
                R.dw_sl[d] = (float)(R.s[d] - sh);
            }
            // |p_h| + s_h <= 2^24 g keeps p_h +- s_h exact (one step g of margin)
            const double lim = std::ldexp(g, 24) - smax - g;
            R.dw_lim = (float)lim;
            if ((double)R.dw_lim > lim) R.dw_lim = std::nextafter(R.dw_lim, 0.0f);
        }
        R.cell_off = ids;
        R.ctr_off = 0;   // set below
        R.atom_off = n;
        R.natoms = counts[r];
        cells += (int64_t)R.nc[0] * R.nc[1] * R.nc[2];
        ids += (int64_t)R.nt[0] * R.nt[1] * R.nt[2] * kTile3;
        chunk_first.push_back((int64_t)chunk_rep.size() / 2);
        for (int64_t k = 0; k < energy_chunks_of(counts[r]); k++) {
            chunk_rep.push_back(r);
            chunk_rep.push_back(k);
        }
        n += counts[r];
        maxrho = std::max(maxrho, counts[r] / vol);
        maxn = std::max(maxn, counts[r]);
        c->reps_h[r] = R;
    }
    chunk_first.push_back((int64_t)chunk_rep.size() / 2);
    if (n > (int64_t)kJMask) return fail(c, MD_ERR_INVAL, "more than 67,108,863 atoms (26-bit list indices)");
    if (ids >= (int64_t)1 << 31) return fail(c, MD_ERR_INVAL, "too many cells");
    if (on_device) {
        if (!is_device_pointer(pos) || !is_device_pointer(vel))
            return fail(c, MD_ERR_INVAL, "pos/vel are not device pointers of the current device");
    } else {
        for (int64_t t = 0; t < 3 * n; t++)
            if (!std::isfinite(pos[t]) || !std::isfinite(vel[t]))
                return fail(c, MD_ERR_NONFINITE, "non-finite input");
    }
    c->n = n;
    if (q.threads_per_atom == 0) c->tpa = default_lanes(n, q.precision);
    c->ncells = cells;
    // whole cells: the split build (half-size cells) measured slower on the
    // LJ liquids (its lanes' octant runs diverge); md_set_cell_split and
    // md_autotune change it
    c->split = 0;
    c->nids = ids;
    c->nchunks = (int64_t)chunk_rep.size() / 2;

    set_lj_constants(c);

    CK(cudaGetDevice(&c->device));
    if (stream) {
        c->st = (cudaStream_t)stream;
    } else {
        CK(cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking));
        c->own_stream = true;
    }

    int rc;
    const size_t N = (size_t)n;
    if ((rc = dalloc(c, &c->reps_d, nrep))) return rc;
    if ((rc = dalloc(c, &c->rep_of_d, N))) return rc;
    // x, v and p32 carry one extra slot n: the sentinel atom that list
    // padding points at, parked far outside every cutoff
    const dvec4 far64 = mk_dvec4(1.0e6, 1.0e6, 1.0e6, 0.0), zero64 = mk_dvec4(0.0, 0.0, 0.0, 0.0);
    const float4 far32 = make_float4(1.0e4f, 1.0e4f, 1.0e4f, 0.0f);
    for (int b = 0; b < 2; b++) {
        if ((rc = dalloc(c, &c->x[b], N + 1))) return rc;
        if ((rc = dalloc(c, &c->v[b], N + 1))) return rc;
        if ((rc = dalloc(c, &c->id[b], N))) return rc;
        if ((rc = dalloc(c, &c->p32[b], N + 1))) return rc;
        CK(cudaMemcpy(c->x[b] + N, &far64, sizeof(dvec4), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->v[b] + N, &zero64, sizeof(dvec4), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->p32[b] + N, &far32, sizeof(float4), cudaMemcpyHostToDevice));
    }
    if ((rc = dalloc(c, &c->f32, N))) return rc;
    if (q.precision == MD_DW) {
        // low parts of the split positions; slot n (the sentinel) stays zero
        for (int b = 0; b < 2; b++) {
            if ((rc = dalloc(c, &c->plo[b], N + 1))) return rc;
            CK(cudaMemsetAsync(c->plo[b], 0, sizeof(float4) * (N + 1), c->st));
        }
    }
    if (c->disp) {
        if ((rc = dalloc(c, &c->p32_ref, N))) return rc;
        CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    }
    if ((rc = dalloc(c, &c->f64, N))) return rc;
    if ((rc = dalloc(c, &c->cell_key, N))) return rc;
    // binning keys: one per cell id (whole cells); md_set_cell_split grows
    // the arrays to 8 per cell id when cells are split
    if ((rc = dalloc(c, &c->cell_count, (size_t)ids))) return rc;
    if ((rc = dalloc(c, &c->cell_start, (size_t)ids + 1))) return rc;
    if ((rc = dalloc(c, &c->perm, N))) return rc;
    c->scan_len = scan_tmp_elems(ids);
    if ((rc = dalloc(c, &c->scan_tmp, (size_t)c->scan_len))) return rc;
    c->key_cap = ids;
    if ((rc = dalloc(c, &c->nb_count, N))) return rc;
    if ((rc = dalloc(c, &c->pe_atom, N))) return rc;
    if ((rc = dalloc(c, &c->w_atom, N))) return rc;
    if ((rc = dalloc(c, &c->pe64, N))) return rc;
    if ((rc = dalloc(c, &c->w64, N))) return rc;
    if ((rc = dalloc(c, &c->ke64, N))) return rc;
    if ((rc = dalloc(c, &c->status, 1))) return rc;
    if ((rc = dalloc(c, &c->chunk_rep_d, chunk_rep.size()))) return rc;
    if ((rc = dalloc(c, &c->chunk_first_d, chunk_first.size()))) return rc;
    if ((rc = dalloc(c, &c->partials_d, 3 * (size_t)c->nchunks))) return rc;
    if ((rc = dalloc(c, &c->eout_d, 3 * (size_t)nrep))) return rc;
    if ((rc = dalloc(c, &c->io_d, 6 * N))) return rc;

    // cell-centre table: (c + 0.5) s per replica and dimension, the same
    // expression the kernels would evaluate
    std::vector<double> ctr;
    for (int32_t r = 0; r < nrep; r++) {
        Rep &R = c->reps_h[r];
        R.ctr_off = (int64_t)ctr.size();
        for (int dd = 0; dd < 3; dd++)
            for (int32_t k = 0; k < R.nc[dd]; k++) ctr.push_back(((double)k + 0.5) * R.s[dd]);
    }
    if ((rc = dalloc(c, &c->ctr_d, ctr.size()))) return rc;
    // per replica: o s for each 6-bit cell-offset code of a list entry (codes
    // with a field of 3 do not occur and map to 0)
    std::vector<float4> offt(64 * (size_t)nrep);
    for (int32_t r = 0; r < nrep; r++)
        for (uint32_t code = 0; code < 64; code++) {
            float o[3];
            for (int dd = 0; dd < 3; dd++) {
                const uint32_t f = (code >> (2 * dd)) & 3u;
                o[dd] = f == 3u ? 0.0f : (float)((int)f - 1) * -c->reps_h[r].nsf[dd];
            }
            offt[64 * (size_t)r + code] = make_float4(o[0], o[1], o[2], 0.0f);
        }
    if ((rc = dalloc(c, &c->offtab_d, offt.size()))) return rc;
    CK(cudaMemcpyAsync(c->offtab_d, offt.data(), sizeof(float4) * offt.size(), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->ctr_d, ctr.data(), sizeof(double) * ctr.size(), cudaMemcpyHostToDevice, c->st));
    std::vector<int32_t> rep_of(N);
    for (int32_t r = 0; r < nrep; r++)
        for (int64_t a = 0; a < counts[r]; a++) rep_of[(size_t)(c->reps_h[r].atom_off + a)] = r;
    CK(cudaMemcpyAsync(c->reps_d, c->reps_h.data(), sizeof(Rep) * nrep, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->rep_of_d, rep_of.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->chunk_rep_d, chunk_rep.data(), sizeof(int64_t) * chunk_rep.size(), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->chunk_first_d, chunk_first.data(), sizeof(int64_t) * chunk_first.size(), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemsetAsync(c->cell_count, 0, sizeof(int32_t) * (size_t)ids, c->st));
    CK(cudaMemsetAsync(c->status, 0, sizeof(DevStatus), c->st));
    CK(cudaMemsetAsync(c->f32, 0, sizeof(float4) * N, c->st));
    CK(cudaMemsetAsync(c->f64, 0, sizeof(dvec4) * N, c->st));
    CK(cudaStreamSynchronize(c->st));

    // Initial capacity: expected full-list count at the densest replica with
    // margin, never more than the replica's size allows.
    c->expect_row = maxrho * 4.0 / 3.0 * M_PI * rs * rs * rs;
    const double expect = c->expect_row * (q.list_type == MD_LIST_HALF ? 0.5 : 1.0);
    int64_t cap0 = (int64_t)(1.3 * expect) + 16;
    cap0 = std::min<int64_t>(cap0, maxn + 3);
    if ((rc = alloc_list(c, (int32_t)std::max<int64_t>(cap0, 4)))) return rc;
    if (list_g(c) &&
        (rc = alloc_group(c, list_g(c), (int32_t)std::min<int64_t>(group_cap0(c, list_g(c)), maxn + 16))))
        return rc;
    return set_state(c, pos, vel, on_device);
}

// Replaces the state from host or device arrays (n x 3, caller order).
// Inputs are checked for non-finite values by the upload kernel
// (FLAG_NONFINITE, reported by the rebuild that follows).
int set_state(md_ctx *c, const double *pos, const double *vel, bool on_device)
{
    const double *src_x = pos, *src_v = vel;
    if (on_device) {
        if (!is_device_pointer(pos) || !is_device_pointer(vel))
            return fail(c, MD_ERR_INVAL, "pos/vel are not device pointers of the current device");
    } else {
        // no host-side scan: the upload kernel checks every value
        const size_t bytes = sizeof(double) * 3 * (size_t)c->n;
        CK(cudaMemcpyAsync(c->io_d, pos, bytes, cudaMemcpyHostToDevice, c->st));
        CK(cudaMemcpyAsync(c->io_d + 3 * c->n, vel, bytes, cudaMemcpyHostToDevice, c->st));
        src_x = c->io_d;
        src_v = c->io_d + 3 * c->n;
    }
    c->xp = 0;
    c->vp = 0;
    c->pb = 0;
    CK(cudaMemsetAsync(c->status, 0, sizeof(DevStatus), c->st));
    int nl = 0;
    Dev d = view(c);
    if (launch_scatter_in(d, src_x, src_v, c->st, &nl))
        return fail(c, MD_ERR_CUDA, "upload launch failed");
    c->launches += nl;
    c->moved_since_bin = true;
    c->list_valid = false;
    c->forces_valid = false;
    c->v32_fresh = false;
    int rc = rebuild_now(c, true);
    if (rc) return rc;
    return ensure_forces(c);
}

// Writes quantity `what` (launch_gather_out codes) in caller order to dst
// (device, n x 3 doubles) on the context's stream.
int gather_to(md_ctx *c, int what, double *dst)
{
    int nl = 0;
    if (launch_gather_out(view(c), what, dst, c->st, &nl)) return fail(c, MD_ERR_CUDA, "gather failed");
    c->launches += nl;
    return MD_OK;
}

}  // namespace
