// Internal declarations shared by the kernels and the host runtime of the
// GB300 LJ MD library.  Nothing here is part of the public ABI (include/md.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace mdk {

// FP64 3-vectors are stored padded to 32 bytes (one DRAM sector per atom).
typedef double4_32a dvec4;
__host__ __device__ __forceinline__ dvec4 mk_dvec4(double x, double y, double z, double w)
{
    return make_double4_32a(x, y, z, w);
}
#ifdef __CUDACC__
// Read-only (L1-cached) load of a padded FP64 3-vector.
__device__ __forceinline__ dvec4 ldg_dvec4(const dvec4 *p)
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    return mk_dvec4(a.x, a.y, b.x, b.y);
}
// Streaming (evict-first) load and store of a padded FP64 3-vector: per-atom
// state that a kernel touches once, kept from evicting gathered lines.
__device__ __forceinline__ dvec4 ld_cs_dvec4(const dvec4 *p)
{
    const double2 a = __ldcs(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldcs(reinterpret_cast<const double2 *>(p) + 1);
    return mk_dvec4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st_cs_dvec4(dvec4 *p, const dvec4 &v)
{
    __stcs(reinterpret_cast<double2 *>(p), make_double2(v.x, v.y));
    __stcs(reinterpret_cast<double2 *>(p) + 1, make_double2(v.z, v.w));
}
#endif

// A list entry packs the neighbour's slot index (low 26 bits) and the cell
// offset o in {-1,0,1}^3 of the neighbour's periodic image relative to the
// owner's cell, as o+1 in 2 bits per dimension: bits 26-27 x, 28-29 y, 30-31
// z.  Rows are padded to a multiple of 4 with entries that point at the
// sentinel slot n, an atom parked far outside every cutoff.
constexpr int kJBits = 26;
constexpr uint32_t kJMask = (1u << kJBits) - 1u;
constexpr uint32_t kZeroOffset = 0x15u;   // o = (0, 0, 0)
__host__ __device__ __forceinline__ uint32_t offset_code(int ox, int oy, int oz)
{
    return (uint32_t)(ox + 1) | ((uint32_t)(oy + 1) << 2) | ((uint32_t)(oz + 1) << 4);
}
constexpr int kMaxNc = 1023;        // cell coordinates are packed in 10 bits each

// Bits of the device error word.  Every kernel returns immediately while it
// is non-zero, so the state freezes at the first failure.
enum : int32_t {
    FLAG_NL_OVERFLOW = 1, FLAG_NONFINITE = 2, FLAG_BADPOS = 4, FLAG_BOUNDS = 8,
    FLAG_TIMEOUT = 16,  // a bounded device wait gave up
    FLAG_DWRANGE = 32   // double-word path: an atom left the range its split
                        // position keeps exact (see dw_split)
};

// Bounds checks of the debug build (MD_DEBUG_CHECKS=1): MD_CHECK(d, cond) is
// true when cond holds; otherwise it raises FLAG_BOUNDS and is false, and
// the caller skips the access.  In the normal build it is the constant true.
#ifndef MD_DEBUG_CHECKS
#define MD_DEBUG_CHECKS 0
#endif
#if MD_DEBUG_CHECKS
#define MD_CHECK(d, cond) ((cond) ? true : (atomicOr(&(d).status->flags, FLAG_BOUNDS), false))
#else
#define MD_CHECK(d, cond) true
#endif

// Device error word and step bookkeeping (one per context, in device memory).
struct DevStatus {
    int32_t flags;
    int32_t max_count;        // largest list row of the last build (counted even past cap)
    int64_t rebuild_count;    // binnings run since the host last cleared it
    int64_t overflow_at;      // rebuild_count when a build overflowed
    int64_t elog_cursor;      // next record of the on-device energy log
    // displacement-triggered rebuilds (md_params.rebuild_every == 0)
    int64_t dev_step;         // rebuild checks run since the host last cleared it
    int64_t overflow_step;    // dev_step when a build overflowed
    int32_t need_rebuild;     // set by any atom that moved more than the trigger distance
    int32_t pad_;
};

// One periodic replica.
struct Rep {
    double L[3];
    double halfL[3];
    double s[3];              // cell side L / nc (FP64)
    float nsf[3];             // -s in FP32 (stencil offsets of the mixed path)
    float invsf[3];           // fl32(1 / fl32(s)) (binning's quotient estimate)
    float splitf[3];          // split cells: s - rs - 1e-3 s in FP32, rounded down (the
                              // build skips the far half of a neighbour cell for atoms
                              // at least this far on the near side of their own centre)
    int32_t nc[3];
    int32_t nt[3];            // cell tiles per dimension, ceil(nc / MD_CELL_TILE)
    // double-word positions (precision MD_DW): grid step g = 2^k of the high
    // parts (the least power of two with 2^24 g >= 2.5 max(s)), the constant
    // 1.5 * 2^52 * g that rounds an FP64 number to a multiple of g, the cell
    // side split into s_h (a multiple of g) and s_l = fl32(s - s_h), and the
    // largest |high part| for which p_h +- s_h stays exact (2^24 g - max s)
    double dw_magic;
    float dw_sh[3], dw_sl[3];
    float dw_lim;
    int32_t dw_pad_;
    int64_t ctr_off;          // first entry of this replica in Dev::ctr
    int64_t cell_off;         // first global cell id of this replica
    int64_t atom_off;         // first atom slot of this replica
    int64_t natoms;
};

// Linear cell ids.  Cells are numbered tile by tile: T x T x T-cell tiles
// (T = MD_CELL_TILE, 2 unless a build sets it) in (tx, ty, tz) order with tz
// fastest, the cells of a tile in (x, y, z) order with z fastest.  Atoms are
// sorted by this id, so the 256 consecutive atoms of a thread block form a
// compact brick of cells instead of a pencil along z (T = 1 is the plain
// z-fastest order), whose neighbourhood (the cells its gathers touch) is
// about a third smaller.  When T does not divide nc the last tile of a row
// sticks out of the box; its missing cells get ids but never atoms.
#ifndef MD_CELL_TILE
#define MD_CELL_TILE 2
#endif
constexpr int kTile = MD_CELL_TILE;
static_assert(kTile == 1 || kTile == 2 || kTile == 4, "cell tiles of 1, 2 or 4 cells per edge");
constexpr int kTile3 = kTile * kTile * kTile;
__host__ __device__ __forceinline__ int64_t cell_id(const Rep &R, int cx, int cy, int cz)
{
    const int64_t tile = ((int64_t)(cx / kTile) * R.nt[1] + (cy / kTile)) * R.nt[2] + (cz / kTile);
    return R.cell_off + tile * kTile3 + ((cx % kTile) * kTile + (cy % kTile)) * kTile + (cz % kTile);
}
// Id of cell (cx, cy, cz) from the id `col` of (cx, cy, 0) (cell ids are
// below 2^31).
__host__ __device__ __forceinline__ int32_t cell_id_z(int32_t col, int cz)
{
    return col + (cz / kTile) * kTile3 + (cz % kTile);
}
__host__ __device__ __forceinline__ void cell_coords(const Rep &R, int64_t id, int &cx, int &cy,
                                                     int &cz)
{
    const int64_t local = id - R.cell_off;
    const int64_t tile = local / kTile3;
    const int l = (int)(local % kTile3);
    const int tz = (int)(tile % R.nt[2]);
    const int ty = (int)((tile / R.nt[2]) % R.nt[1]);
    const int tx = (int)(tile / ((int64_t)R.nt[2] * R.nt[1]));
    cx = kTile * tx + l / (kTile * kTile);
    cy = kTile * ty + (l / kTile) % kTile;
    cz = kTile * tz + l % kTile;
}

// LJ constants in both precisions.
struct LJ {
    double rc2, rs2, sigma6, c48e, c24e, c4e, eps, sigma;
    float rc2f, sigma6f, c48ef, c24ef, c4ef;
    double half_dt_m;         // dt / (2 m)
    double dt;
    double mass;
    float rs2f_lo, rs2f_hi;   // FP32 prefilter band around rs^2 (exact FP64 test inside)
    // double-word constants (precision MD_DW) as {fl32(c), fl32(c - fl32(c))}:
    // rc^2, 48 eps sigma^12, 24 eps sigma^6, 4 eps sigma^12, 4 eps sigma^6
    float dw_rc2[2], dw_a12[2], dw_a6[2], dw_b12[2], dw_b6[2];
    // adjoint pair terms in double word (s = sigma): 192 eps s^6, 672 eps s^12
    // (2 f'), 48 s^12, 24 s^6 (f / eps), 576 eps s^11, 144 eps s^5 (df/dsigma),
    // 2 s^12, 2 s^6 (dV/deps / 2), 24 eps s^11, 12 eps s^5 (dV/dsigma / 2)
    float dw_adj[10][2];
    // contact model in double word: sigma^2, sigma, K, gamma, K / 2
    float dw_sd_sig2[2], dw_sd_sig[2], dw_sd_k[2], dw_sd_g[2], dw_sd_hk[2];
    // spring-dashpot contact (Eq. 3; pot == 1): K, gamma, sigma^2 (sigma = diameter)
    int32_t pot;
    double sd_k, sd_g, sd_sig2;
    float sd_kf, sd_gf, sd_sig2f, sigmaf;
};

// Device pointers of one context (passed by value to kernels).
struct Dev {
    int64_t n;
    int64_t ncells;           // cell ids over all replicas, tile padding included
    int32_t split;            // 1: each cell's atoms are ordered by octant (the
                              // half-size cells of Sec. 3.2), cell_start holds 8
                              // entries per cell; 0: one entry per cell
    int32_t split_pad_;
    int32_t nrep;
    int32_t cap;              // list capacity (multiple of 4)
    const Rep *reps;
    const int32_t *rep_of;    // replica of each atom slot (static)
    dvec4 *x;               // current positions (FP64, .w unused)
    dvec4 *v;               // current velocities
    dvec4 *x_alt, *v_alt;   // reorder targets
    dvec4 *x_nxt;             // next positions of the fused FP64 step (other atoms
                              // still gather this step's x)
    int32_t *id, *id_alt;     // caller id of each slot
    float4 *p32, *p32_nxt;    // cell-relative FP32 positions; .w = packed cell coords
    float4 *p32_ref;          // p32 at the last binning (displacement trigger only, else null)
    float4 *plo, *plo_nxt;    // precision MD_DW: low parts of the split positions (p32
                              // then holds the high parts); null on the other paths
    float disp2_thr;          // squared trigger distance (FP32, below (skin/2)^2)
    float4 *f32;              // mixed-path forces
    dvec4 *f64;             // FP64-path forces
    // Binning keys: the global cell id, times 8 plus the octant when split
    // (octant = 4 hx + 2 hy + hz, h = 1 for the upper half of the cell along
    // that axis), so a cell's atoms are cell_start[key(c)] .. cell_start[key(c + 1)]
    int32_t *cell_key;        // binning key of each slot (binning scratch)
    int32_t *cell_count;      // per key (returns to zero after scatter)
    int32_t *cell_start;      // per key + 1
    int32_t *perm;            // scatter target: slot -> old slot
    int32_t *nb;              // list: int4 chunks, chunk q of atom i at ((q*n)+i)*4
    int32_t *nb_count;
    float *pe_atom, *w_atom;  // per-atom energy / virial (mixed)
    double *pe_atom64, *w_atom64, *ke_atom64;
    DevStatus *status;
    const double *ctr;        // cell-centre coordinates (c + 0.5) s: per replica
                              // nc_x, then nc_y, then nc_z values
    float4 *v32, *v32_nxt;    // contact model, mixed path: FP32 velocity copies
                              // (n + 1 each, slot n zero; flip with p32), else null;
                              // double-word path: the high parts of the copies
    float4 *vlo, *vlo_nxt;    // contact model, double-word path: their low parts
    // Lists shared by groups of G atoms of one cell (list types 2 and 4):
    // group table, per-cell group counts and their prefix sums (the number of
    // groups at gcell_start[ncells]), rows and row lengths.  Entry k of group
    // g is at int index ((k / 16) * ngmax + g) * 16 + k % 16: lane l of the
    // group's G lanes reads the int4 chunks l, l + 4, ... of each 16-entry
    // block.  Null when no group list was set up.
    int32_t *grp, *gcnt, *gcell_start, *gnb, *gnb_count;
    // which members each entry belongs to (bit k: member k's exact row holds
    // it; one byte per entry, laid out like the entries), and per group the
    // member pairs inside the list radius (bit a * G + b, both orders)
    uint8_t *gmask;
    uint16_t *gpair;
    int64_t ngmax;            // group slots allocated: ceil(n / G) + cells
    int32_t gcap;             // entries per group row (multiple of 16)
    const float4 *offtab;     // per replica 64 codes: (ox s_x, oy s_y, oz s_z) of a
                              // list entry's 6-bit cell-offset code
};

// Binning keys of cell c: its first key, and its atom range.
__host__ __device__ __forceinline__ int64_t key_of(const Dev &d, int64_t c)
{
    return c << (3 * d.split);
}
__host__ __device__ __forceinline__ int64_t nkeys(const Dev &d)
{
    return d.ncells << (3 * d.split);
}

#ifdef __CUDACC__
// Bit casts on host and device (the host side serves the conversion tests).
__host__ __device__ __forceinline__ long long bits_of(double a)
{
#ifdef __CUDA_ARCH__
    return __double_as_longlong(a);
#else
    long long b;
    memcpy(&b, &a, sizeof b);
    return b;
#endif
}
__host__ __device__ __forceinline__ double double_of(long long b)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double(b);
#else
    double a;
    memcpy(&a, &b, sizeof a);
    return a;
#endif
}
__host__ __device__ __forceinline__ unsigned int bits_of(float f)
{
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    unsigned int b;
    memcpy(&b, &f, sizeof b);
    return b;
#endif
}
__host__ __device__ __forceinline__ float float_of(unsigned int b)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float f;
    memcpy(&f, &b, sizeof f);
    return f;
#endif
}

// Conversions and compares of positive doubles done on their IEEE bit
// patterns with integer operations: on GB300 the FP64 pipe, which executes
// FP64 compares and FP64<->FP32 conversions, is a small fraction of the
// integer and FP32 rates.  Valid for finite a > 0 within FP32's normal range
// (f32_of_pos) and any finite float > 0 (f64_of_pos).
constexpr long long kF64F32Rebias = (long long)(1023 - 127) << 23;
// fl32(a), rounded to nearest with ties away from zero (add half of the 29
// dropped mantissa bits; a carry moves into the exponent as it should)
__host__ __device__ __forceinline__ float f32_of_pos(double a)
{
    const long long b = bits_of(a);
    return float_of((unsigned int)(((b + (1LL << 28)) >> 29) - kF64F32Rebias));
}
// (double)f, exact
__host__ __device__ __forceinline__ double f64_of_pos(float f)
{
    return double_of(((long long)bits_of(f) + kF64F32Rebias) << 29);
}
// a < b for a >= +0 and b > 0 (non-negative doubles order like their
// patterns; a NaN a compares false, as in FP64)
__host__ __device__ __forceinline__ bool lt_nonneg(double a, double b)
{
    return bits_of(a) < bits_of(b);
}

// Signed conversions with IEEE results on the bit patterns (checked bit for
// bit against the hardware conversions on every float and on random and
// edge-case doubles, ties included, by tests/bitconv_check.cu); the FP64
// pipe runs only for the rare operands outside FP32's normal range.  Zero
// takes the integer path of f64_of_f32.
// (double)f, exact
__host__ __device__ __forceinline__ double f64_of_f32(float f)
{
    const unsigned int u = bits_of(f);
    const unsigned int mag = u & 0x7fffffffu;
    const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
    if (mag - 0x00800000u < 0x7f000000u)               // normal
        return double_of((long long)(sign | (((unsigned long long)mag + kF64F32Rebias) << 29)));
    if (mag == 0) return double_of((long long)sign);
    return (double)f;                                   // subnormal, inf, NaN
}
// (float)a, rounded to nearest even
__host__ __device__ __forceinline__ float f32_of_f64(double a)
{
    const unsigned long long b = (unsigned long long)bits_of(a);
    const unsigned long long mag = b & 0x7fffffffffffffffULL;
    // |a| in [2^-126, 2^128): a normal FP32 result (or an overflow to inf,
    // which the rounding carry produces)
    if (mag - 0x3810000000000000ULL < 0x0fe0000000000000ULL) {
        const unsigned long long r = (mag + 0x0fffffffULL + ((mag >> 29) & 1ULL)) >> 29;
        return float_of((unsigned int)((b >> 32) & 0x80000000ULL) |
                        (unsigned int)(r - (unsigned long long)kF64F32Rebias));
    }
    return (float)a;
}

// Displacement trigger: flags a rebuild when atom i's new cell-relative
// position p lies farther than the trigger distance from its position at the
// last binning (same cell frame, FP32; error ~1e-7 against a trigger distance
// set 1e-5 below skin/2).
__device__ __forceinline__ void check_displacement(const Dev &d, int64_t i, const float4 &p)
{
    if (!d.p32_ref) return;
    const float4 r = d.p32_ref[i];
    const float dx = p.x - r.x, dy = p.y - r.y, dz = p.z - r.z;
    if (fmaf(dz, dz, fmaf(dy, dy, dx * dx)) > d.disp2_thr) d.status->need_rebuild = 1;
}

// Double-word positions (precision MD_DW): the cell-relative FP64 position p
// as h + l, h = p rounded to a multiple of the replica's grid step g (two
// FP64 additions of 1.5 * 2^52 * g), l = fl32(p - h) (p - h is exact).  h has
// at most 24 significant bits while |p| < 2^24 g, so it is an FP32 number,
// and sums and differences of such numbers below 2^24 g are exact in FP32:
// the force kernel forms the high part of each displacement without
// rounding.  l carries p to 2^-25 g.  Returns false (the caller raises
// FLAG_DWRANGE) when |h| exceeds R.dw_lim, past which h +- s_h could round.
__host__ __device__ __forceinline__ bool dw_split(const Rep &R, double p, float &h, float &l)
{
#ifdef __CUDA_ARCH__
    const double hd = __dsub_rn(__dadd_rn(p, R.dw_magic), R.dw_magic);
    l = f32_of_f64(__dsub_rn(p, hd));
#else
    const double hd = (p + R.dw_magic) - R.dw_magic;   // (the CPU check of the split)
    l = f32_of_f64(p - hd);
#endif
    h = f32_of_f64(hd);
    return fabsf(h) <= R.dw_lim;
}

// Velocity copies of slot i for the contact kernels: fl32(v) into vh and,
// on the double-word path, fl32(v - fl32(v)) into vl.
__device__ __forceinline__ void store_vel_copy(float4 *vh, float4 *vl, int64_t i, const dvec4 &v)
{
    const float hx = f32_of_f64(v.x), hy = f32_of_f64(v.y), hz = f32_of_f64(v.z);
    vh[i] = make_float4(hx, hy, hz, 0.f);
    if (vl)
        vl[i] = make_float4(f32_of_f64(v.x - f64_of_f32(hx)), f32_of_f64(v.y - f64_of_f32(hy)),
                            f32_of_f64(v.z - f64_of_f32(hz)), 0.f);
}

// p32 / plo entries of slot i from the cell-relative FP64 position (px, py,
// pz): on the double-word path the split above, else p32 = fl32(p).
__device__ __forceinline__ void store_cell_pos(const Dev &d, const Rep &R, float4 *p32,
                                               float4 *plo, int64_t i, double px, double py,
                                               double pz, uint32_t pack)
{
    if (plo) {
        float hx, hy, hz, lx, ly, lz;
        const bool ok = dw_split(R, px, hx, lx) & dw_split(R, py, hy, ly) & dw_split(R, pz, hz, lz);
        if (!ok) atomicOr(&d.status->flags, FLAG_DWRANGE);
        p32[i] = make_float4(hx, hy, hz, __uint_as_float(pack));
        plo[i] = make_float4(lx, ly, lz, 0.f);
    } else {
        p32[i] = make_float4(f32_of_f64(px), f32_of_f64(py), f32_of_f64(pz), __uint_as_float(pack));
    }
}
#endif

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the k_*.cu files).
// ---------------------------------------------------------------------------
int launch_bin(const Dev &d, int32_t *scan_tmp, int64_t scan_tmp_len, cudaStream_t st,
               int *nlaunch);
int launch_build(const Dev &d, const LJ &lj, bool half, int64_t ncells, cudaStream_t st,
                 int *nlaunch);

enum Epi : int { EPI_F = 0, EPI_FK = 1, EPI_FKKD = 2 };
int launch_force(const Dev &d, const LJ &lj, int precision, bool half, int tpa, int epi,
                 bool energy, bool batched, cudaStream_t st, int *nlaunch);
int launch_integrate(const Dev &d, const LJ &lj, int precision, int phase, bool batched,
                     cudaStream_t st, int *nlaunch);
// Double-word path (precision MD_DW, k_force_dw.cu): full per-atom lists,
// 1/2/4/8 lanes per atom, epilogues as the other full-list kernels; forces
// in d.f64, per-atom PE / W in d.pe_atom64 / d.w_atom64.
int launch_force_dw(const Dev &d, const LJ &lj, int tpa, int epi, bool energy, bool batched,
                    cudaStream_t st, int *nlaunch);
// Spring-dashpot forces (full list).  Mixed path: one kernel with the
// epilogue epi (EPI_F / EPI_FK / EPI_FKKD, as the LJ kernels), gathering the
// neighbours' FP32 velocities from d.v32 and, for EPI_FKKD, writing the next
// p32 and v32 to d.p32_nxt / d.v32_nxt.  FP64 path: force store only (epi is
// ignored; the update runs in launch_integrate).
int launch_force_sd(const Dev &d, const LJ &lj, bool mixed, int epi, bool energy,
                    cudaStream_t st, int *nlaunch);
// The same in double word (k_force_dw.cu): one fused kernel with the
// epilogue epi, gathering the neighbours' velocities from d.v32 / d.vlo and,
// for EPI_FKKD, writing the next p32 / plo and v32 / vlo.
int launch_force_sd_dw(const Dev &d, const LJ &lj, int epi, bool energy, cudaStream_t st,
                       int *nlaunch);
// d.v32 / d.vlo <- the double-word split of d.v for i <= n.
int launch_velocity_dw(const Dev &d, cudaStream_t st, int *nlaunch);
// d.v32[i] = fl32(d.v[i]) for i <= n (slot n: the sentinel's zero velocity);
// with d.vlo also the low parts.
int launch_velocity_f32(const Dev &d, cudaStream_t st, int *nlaunch);
// out3 != NULL: write (PE, KE, W) per replica there; otherwise append one
// record to log_base at status->elog_cursor and advance the cursor.
int launch_energy(const Dev &d, const LJ &lj, int precision, bool ke_from_v,
                  const int64_t *chunk_rep, const int64_t *chunk_first, int64_t nchunks,
                  double *partials, double *out3, double *log_base, cudaStream_t st,
                  int *nlaunch);
int64_t energy_chunks_of(int64_t natoms);
// (PE, KE, W) records (device, nrec x nrep x 3) -> (pe, ke, etot, W, T, P)
// records (device, nrec x nrep x 6)
int launch_thermo(const Rep *reps, int32_t nrep, int64_t nrec, const double *rec, double *out,
                  cudaStream_t st, int *nlaunch);
// what: 0 positions, 1 velocities, 2 FP64 forces, 3 mixed-path forces
int launch_gather_out(const Dev &d, int what, double *out_dev, cudaStream_t st, int *nlaunch);
int launch_scatter_in(const Dev &d, const double *pos_dev, const double *vel_dev,
                      cudaStream_t st, int *nlaunch);
int launch_decode_list(const Dev &d, int32_t *rows_dev, int32_t cap, cudaStream_t st,
                       int *nlaunch);
// Displacement-triggered rebuilds: move the binned state from the alt
// buffers into the current ones and record p32 as the reference; and the
// per-step check that sets a graph conditional to 1 when a rebuild is due.
int launch_copy_back(const Dev &d, cudaStream_t st, int *nlaunch);
int launch_rebuild_check(const Dev &d, cudaGraphConditionalHandle h, cudaStream_t st,
                         int *nlaunch);

int64_t scan_tmp_elems(int64_t nkeys_total);

// Force-kernel studies (k_study.cu): variants 1 (SoA gathers), 2 (AoSoA
// gathers), 5 (gathers through the texture path) and 6 (half of them) into
// fout; variants 3 and 4 (neighbourhood staged in shared memory by plain
// loads / by TMA bulk copies, one block per 2x2x2-cell tile).  Single
// replica, mixed path, full lists.
int64_t study_layout_floats(int64_t n);
int launch_study_force(const Dev &d, const LJ &lj, int variant, float *layouts,
                       cudaTextureObject_t tex, float4 *fout, cudaStream_t st, int *nlaunch);
int launch_study_tiles(const Dev &d, const LJ &lj, int64_t ntiles, bool tma, float4 *fout,
                       cudaStream_t st, int *nlaunch);

// Lists shared by groups of G atoms (k_bin.cu, k_build.cu, k_force.cu, k_misc.cu)
int launch_group_table(const Dev &d, int G, int64_t ncells, int32_t *tmp, int64_t tmp_len,
                       cudaStream_t st, int *nlaunch);
int launch_build_group(const Dev &d, const LJ &lj, int G, cudaStream_t st, int *nlaunch);
int launch_force_group(const Dev &d, const LJ &lj, int G, int epi, bool energy, bool batched,
                       cudaStream_t st, int *nlaunch);
// exact per-atom rows (FP64 criterion) from a group list: counts (n, caller
// order) and rows (n x cap, caller order, replica-local ids)
int launch_decode_group(const Dev &d, const LJ &lj, int G, int32_t *counts_dev, int32_t *rows_dev,
                        int32_t cap, cudaStream_t st, int *nlaunch);

// Adjoint (k_adjoint.cu)
// mixed: FP32 pair terms reading wbar32 (an FP32 copy of wbar in slot order
// kept by the axpy kernel); FP64 path: wbar32 may be null.
// lanes: 1, 2, 4 or 8 lanes per atom (the context's lanes per atom: several
// lanes keep small systems from leaving SMs idle)
int launch_adjoint_pairs(const Dev &d, const LJ &lj, bool mixed, int lanes, const dvec4 *wbar,
                         const float4 *wbar32, dvec4 *xbar, double *g_eps, double *g_sig,
                         double k, double lw, cudaStream_t st, int *nlaunch);
// wbar += dt xbar (caller order); wbar32 (may be null) <- its FP32 copy in
// the slot order of id (slot -> caller id)
// wbar_lo (may be null): the low parts fl32(w - fl32(w)) beside wbar32 (the
// double-word pair terms read both)
int launch_adjoint_axpy(int64_t n, double dt, const dvec4 *xbar, dvec4 *wbar, float4 *wbar32,
                        float4 *wbar_lo, const int32_t *id, cudaStream_t st, int *nlaunch);
// Adjoint pair terms in double word (k_force_dw.cu): d.p32 / d.plo the high
// and low parts of the snapshot's positions, wh / wl those of the adjoint w
// in slot order; full lists, single replica.
int launch_adjoint_pairs_dw(const Dev &d, const LJ &lj, int lanes, const float4 *wh,
                            const float4 *wl, dvec4 *xbar, double *g_eps, double *g_sig, double k,
                            double lw, cudaStream_t st, int *nlaunch);
int launch_sum2(int64_t n, const double *a, const double *b, double *out, cudaStream_t st,
                int *nlaunch);
int launch_unpad3(int64_t n, const dvec4 *a, double *out, cudaStream_t st, int *nlaunch);

}  // namespace mdk
