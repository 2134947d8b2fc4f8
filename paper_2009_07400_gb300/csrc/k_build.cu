// Verlet-list build (tinyMD Sec. 3.2, Fig. 1: scan the neighbour cells, keep
// every j within r = rc + skin; half lists store each pair once; Sec. 4.2:
// neighbour-major layout on GPUs).
//
// Half-list ownership: pair (i, j) is stored in row i iff j's image lies in
// i's upper half-space: del = x_i - x_j (FP64, as the list criterion) has
// del.z < 0, ties broken by del.y < 0, del.x < 0, then id_j > id_i.  del is
// exactly antisymmetric, so each pair is stored once and rows are balanced.
// Cell coordinates are monotone in z, so a lower neighbour cell that is not a
// periodic image holds no owned atom (skipped), an upper one holds only owned
// atoms, and only the same z-layer and image cells need the sign test (FP32,
// or FP64 when the FP32 value is within 1e-4 of zero).
//
// The list criterion is exact FP64: r^2 = ((dx*dx + dy*dy) + dz*dz) with dx
// the minimum-image difference, each operation rounded, compared strictly
// with (rc+skin)^2.  GB300's FP64 rate is a small fraction of its FP32 rate,
// so every candidate is first classified in FP32 from the cell-relative
// positions p = fl32(x - C_cell):
//     d = (p_i - p_j) + o * (-s)        (o = stencil offset of j's image)
// d is formed as (p_i + o(-s)) - p_j.  The FP32 r^2 of a candidate differs
// from the FP64 one by far less than 2.5e-4 rs^2 (a few FP32 ulps of
// |p| <= s/2 and |o s| <= s propagated through the three squares), so only
// candidates inside that band are decided by the FP64 test: about 3 % of the
// atoms meet one.  The FP64 test
// applies the image shift the way the minimum-image branch does,
// (x_i - x_j) -/+ L, with __dmul_rn/__dadd_rn so nothing is contracted.
//
// Each periodic image of each neighbour cell is visited once (all 27
// offsets, each with its own image shift), so boxes with fewer than three
// cells per dimension need no de-duplication: at most one image of an atom
// lies within rs < L/2.
//
// Split cells (optional, md_set_cell_split): the binning orders each cell's
// atoms by octant, and a neighbour cell is scanned as the runs of its
// octants that can hold a pair (the half-size cells of Sec. 3.2's footnote
// with their wider stencil); the rows hold the same pairs as with whole
// cells.
//
// Layout: entries of atom i are int4 chunks, chunk q at int4 index q*n + i;
// the last chunk of a row is padded with entries pointing at the far-away
// sentinel slot n.  Rows longer than the capacity are counted but not stored
// (overflow flag).
#include "md_internal.cuh"

#include <type_traits>

namespace mdk {

namespace {

__device__ __forceinline__ bool stopped(const DevStatus *st)
{
    return *((volatile const int32_t *)&st->flags) != 0;
}

__device__ __forceinline__ double image_diff(double xi, double xj, int k, double L)
{
    double t = __dsub_rn(xi, xj);
    if (k > 0) t = __dsub_rn(t, L);
    else if (k < 0) t = __dadd_rn(t, L);
    return t;
}


// Half-list ownership of candidate j (FP32 d = p_i + o(-s) - p_j first; the
// exact FP64 del when the FP32 z-component is within 1e-4 of zero).
__device__ __forceinline__ bool owns(const Dev &d, const LJ &lj, int64_t i, int32_t j, int32_t idi,
                                     float dx, float dy, float dz, int kx, int ky, int kz,
                                     const Rep &R, dvec4 &xi, bool &have_xi)
{
    (void)lj; (void)dx; (void)dy;
    if (fabsf(dz) > 1e-4f) return dz < 0.f;
    if (!have_xi) { xi = d.x[i]; have_xi = true; }
    const dvec4 xj = d.x[j];
    const double ez = image_diff(xi.z, xj.z, kz, R.L[2]);
    if (ez != 0.0) return ez < 0.0;
    const double ey = image_diff(xi.y, xj.y, ky, R.L[1]);
    if (ey != 0.0) return ey < 0.0;
    const double ex = image_diff(xi.x, xj.x, kx, R.L[0]);
    if (ex != 0.0) return ex < 0.0;
    return d.id[j] > idi;
}

// Builds row i; returns its length (rows longer than the capacity are
// counted in full but stored only up to the capacity).  SPLIT: the binning
// ordered each cell's atoms by octant (the context's cell split).  OFF32:
// every stored entry's offset from the row fits in 32 bits (cap n < 2^32),
// so the write position is a 32-bit offset (two instructions fewer per
// candidate than a 64-bit pointer: 36.3 against 38.3 us per step of
// neighbour work at 1M atoms); offsets of entries past the capacity may wrap,
// but those are never stored.
template <bool BATCHED, bool HALF, bool SPLIT, bool OFF32>
__device__ __forceinline__ int32_t build_row(const Dev &d, const LJ &lj, int64_t i)
{
    const Rep &R = d.reps[BATCHED ? d.rep_of[i] : 0];
    const float4 pi = d.p32[i];
    const uint32_t pack = __float_as_uint(pi.w);
    const int ci[3] = {(int)(pack & 1023u), (int)((pack >> 10) & 1023u), (int)((pack >> 20) & 1023u)};
    const int32_t idi = HALF ? d.id[i] : 0;
    const int64_t n = d.n;
    const int32_t cap = d.cap;
    int32_t *row = d.nb + 4 * i;          // entry k of row i: row[(k>>2)*4n + (k&3)]
    const float4 *p32 = d.p32;
    const float lo = lj.rs2f_lo, hi = lj.rs2f_hi;

    int32_t cnt = 0;
    // write position of entry cnt: OFF32 its offset from row (ints), else
    // its address; a step from entry 4q+3 to entry 4q+4 is 4n - 3 ints
    uint32_t wo = 0;
    int32_t *wp = row;
    const uint32_t wstep32 = (uint32_t)(4 * n - 3);
    const int64_t wstep = 4 * n - 3;
    auto put = [&](int32_t v) {
        if (OFF32) row[wo] = v;
        else *wp = v;
    };
    // next entry (step4: cnt % 4 == 3), if `yes`
    auto advance = [&](bool yes, bool step4) {
        if (OFF32) wo += yes ? (step4 ? wstep32 : 1u) : 0u;
        else wp += yes ? (step4 ? wstep : 1) : 0;
    };
    bool have_xi = false;
    dvec4 xi = mk_dvec4(0, 0, 0, 0);
    // Split cells: the octants of neighbour cell o that can hold a neighbour
    // (octant bits 4 hx + 2 hy + hz).  Along an axis with o = +1 the upper
    // half lies at least s (1 - 2e-4) - p beyond the atom (binned halves are
    // exact to 2e-4 cell units), so it is skipped when p <= s - rs - 1e-3 s;
    // likewise the lower half of the o = -1 cell when p >= -(s - rs - 1e-3 s).
    // far: bit 2a set = skip the upper half of the o = +1 cell along axis a,
    // bit 2a + 1 = skip the lower half of the o = -1 cell.
    uint32_t far = 0;
    {
        const float pc[3] = {pi.x, pi.y, pi.z};
#pragma unroll
        for (int a = 0; a < 3; a++)
            far |= ((uint32_t)(pc[a] <= R.splitf[a]) << (2 * a)) |
                   ((uint32_t)(pc[a] >= -R.splitf[a]) << (2 * a + 1));
    }
    // octants kept along axis a (lower-half octants `lo`) in neighbour cell o
    auto keep = [&](int a, int o, uint32_t lo) -> uint32_t {
        const uint32_t up = 0xFFu & ~lo;
        if (o > 0) return lo | (((far >> (2 * a)) & 1u) ? 0u : up);
        if (o < 0) return up | (((far >> (2 * a + 1)) & 1u) ? 0u : lo);
        return 0xFFu;
    };

    for (int ox = -1; ox <= 1; ox++) {
        int ux = ci[0] + ox, kx = 0;
        if (ux < 0) { ux += R.nc[0]; kx = -1; } else if (ux >= R.nc[0]) { ux -= R.nc[0]; kx = 1; }
        const float qx = pi.x + (float)ox * R.nsf[0];
        const uint32_t kx8 = keep(0, ox, 0x0Fu);
        for (int oy = -1; oy <= 1; oy++) {
            int uy = ci[1] + oy, ky = 0;
            if (uy < 0) { uy += R.nc[1]; ky = -1; } else if (uy >= R.nc[1]) { uy -= R.nc[1]; ky = 1; }
            const float qy = pi.y + (float)oy * R.nsf[1];
            const int32_t col = (int32_t)cell_id(R, ux, uy, 0);
            const uint32_t kxy8 = kx8 & keep(1, oy, 0x33u);
            for (int oz = -1; oz <= 1; oz++) {
                int uz = ci[2] + oz, kz = 0;
                if (uz < 0) { uz += R.nc[2]; kz = -1; } else if (uz >= R.nc[2]) { uz -= R.nc[2]; kz = 1; }
                const float qz = pi.z + (float)oz * R.nsf[2];
                const int32_t cid = cell_id_z(col, uz);
                if (!MD_CHECK(d, cid >= 0 && cid < d.ncells)) continue;
                if (HALF && oz < 0 && kz == 0) continue;        // entirely below
                const bool test_sign = HALF && (oz == 0 || kz != 0);
                const uint32_t tag = offset_code(ox, oy, oz) << kJBits;
                // full test of candidate j (self, ownership, FP64 in the band)
                auto accept = [&](int32_t j, float dx, float dy, float dz, float r2f) {
                    if (j == i) return;
                    if (test_sign && !owns(d, lj, i, j, idi, dx, dy, dz, kx, ky, kz, R, xi, have_xi))
                        return;
                    if (!(r2f < lo)) {                         // inside the band: decide in FP64
                        if (!have_xi) { xi = d.x[i]; have_xi = true; }
                        const dvec4 xj = d.x[j];
                        const double tx = image_diff(xi.x, xj.x, kx, R.L[0]);
                        const double ty = image_diff(xi.y, xj.y, ky, R.L[1]);
                        const double tz = image_diff(xi.z, xj.z, kz, R.L[2]);
                        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(tx, tx), __dmul_rn(ty, ty)),
                                                    __dmul_rn(tz, tz));
                        if (!(r2 < lj.rs2)) return;
                    }
                    if (cnt < cap) put((int32_t)((uint32_t)j | tag));
                    advance(true, (cnt & 3) == 3);
                    cnt++;
                };
                // candidates j0 .. j1 - 1 of this cell
                auto range = [&](int32_t j0, int32_t j1) {
                    if (!MD_CHECK(d, j0 >= 0 && j0 <= j1 && j1 <= d.n)) return;
                    // hot loop, 32 candidates at a time: a candidate clearly
                    // inside (FP32 r^2 below the band) is appended at once by a
                    // predicated store, so the lanes of a warp stay converged;
                    // the few in the band (and, in half lists, those whose
                    // ownership the FP32 sign cannot decide) are marked and go
                    // through accept() after the chunk
                    for (int32_t jb = j0; jb < j1; jb += 32) {
                        const int m = min(32, (int)(j1 - jb));
                        uint32_t slow = 0;
                        // CAP: the row may reach its capacity within this chunk
                        // (the per-candidate test costs ~7 % of the build, so it
                        // is compiled in only where it can matter)
                        auto scan = [&](auto CAP) {
#pragma unroll 4
                            for (int t = 0; t < m; t++) {
                                const int32_t j = jb + t;
                                const float4 pj = __ldg(p32 + j);
                                const float dx = qx - pj.x, dy = qy - pj.y, dz = qz - pj.z;
                                const float r2f = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                                bool in = (r2f < lo) & (j != (int32_t)i);
                                bool sl = (r2f >= lo) & (r2f < hi);
                                if (HALF && test_sign) {
                                    const bool amb = fabsf(dz) <= 1e-4f;
                                    sl |= amb & (r2f < lo);
                                    in &= !amb & (dz < 0.f);
                                }
                                if (CAP.value ? (in & (cnt < cap)) : in) put((int32_t)((uint32_t)j | tag));
                                advance(in, (cnt & 3) == 3);
                                cnt += in;
                                slow |= (uint32_t)sl << t;
                            }
                        };
                        if (cnt + m <= cap) scan(std::false_type{});
                        else scan(std::true_type{});
                        while (slow) {
                            const int t = __ffs(slow) - 1;
                            slow &= slow - 1;
                            const int32_t j = jb + t;
                            const float4 pj = __ldg(p32 + j);
                            const float dx = qx - pj.x, dy = qy - pj.y, dz = qz - pj.z;
                            accept(j, dx, dy, dz, fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
                        }
                    }
                };
                if (SPLIT) {
                    // the kept octants of this cell as runs of consecutive keys
                    const int64_t kb = key_of(d, cid);
                    uint32_t runs = kxy8 & keep(2, oz, 0x55u);
                    while (runs) {
                        const int q0 = __ffs(runs) - 1;
                        const int len = __ffs(~(runs >> q0)) - 1;
                        runs &= ~(((1u << len) - 1u) << q0);
                        range(d.cell_start[kb + q0], d.cell_start[kb + q0 + len]);
                    }
                } else {
                    range(d.cell_start[cid], d.cell_start[cid + 1]);
                }
            }
        }
    }
    if (cnt < cap) {   // pad the last chunk with entries for the sentinel slot n
        const int32_t pad = (int32_t)((uint32_t)n | (kZeroOffset << kJBits));
        for (int32_t k = cnt; (k & 3) != 0; k++) row[(int64_t)(k >> 2) * 4 * n + (k & 3)] = pad;
    }
    d.nb_count[i] = cnt;
    return cnt;
}

// The explicit minimum of one block per SM matters: with the bare block size
// ptxas capped the full-list instance at 56 registers and spilled; with it
// the kernel takes 72 registers (7 blocks of 4 warps per SM) and no spills.
template <bool BATCHED, bool HALF, bool SPLIT, bool OFF32>
__global__ void __launch_bounds__(128, 1) k_build(Dev d, LJ lj)
{
    if (stopped(d.status)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t cnt = i < d.n ? build_row<BATCHED, HALF, SPLIT, OFF32>(d, lj, i) : 0;
    // every lane of the warp reaches this point: reduce the row lengths
    const int32_t wmax = __reduce_max_sync(0xffffffffu, cnt);
    if ((threadIdx.x & 31) == 0) atomicMax(&d.status->max_count, wmax);
    if (cnt > d.cap) {
        atomicOr(&d.status->flags, FLAG_NL_OVERFLOW);
        d.status->overflow_at = d.status->rebuild_count;
        d.status->overflow_step = d.status->dev_step;
    }
}

// ---------------------------------------------------------------------------
// Lists shared by groups of G atoms of one cell.  A group's row holds every
// atom j outside the group that lies in the exact row of some member (the
// FP64 criterion above: FP32 classification, FP64 inside the band), with a
// byte of member bits per entry (bit k: j is in member k's row), so the force
// kernel applies exactly each member's Verlet row.  The pairs of members are
// decided the same way into a per-group mask.  Lanes: the G lanes of a group
// take the candidates of a stencil cell G * U at a time, each candidate
// against all members (their positions in registers), and append accepted
// ones in candidate order with a ballot (rank = accepted lanes of the group
// below the lane).  Every loop runs the warp's largest trip count (groups of
// a warp can sit in different cells) so lanes stay converged and every
// ballot has the whole warp.  Rows are padded with sentinel entries (mask 0)
// to a multiple of 16.
// ---------------------------------------------------------------------------

// FP64 decision of the band members `band` (bits) of candidate j with image
// flags k[3]: returns the bits of the members whose exact r^2 < rs^2.
template <int G>
__device__ __forceinline__ uint32_t exact_bits(const Dev &d, const LJ &lj, const Rep &R,
                                               int32_t a0, int32_t j, uint32_t band, int kx,
                                               int ky, int kz)
{
    uint32_t in = 0;
    const dvec4 xj = d.x[j];
#pragma unroll
    for (int k = 0; k < G; k++) {
        if (!((band >> k) & 1u)) continue;
        const dvec4 xi = d.x[a0 + k];
        const double tx = image_diff(xi.x, xj.x, kx, R.L[0]);
        const double ty = image_diff(xi.y, xj.y, ky, R.L[1]);
        const double tz = image_diff(xi.z, xj.z, kz, R.L[2]);
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(tx, tx), __dmul_rn(ty, ty)), __dmul_rn(tz, tz));
        if (r2 < lj.rs2) in |= 1u << k;
    }
    return in;
}

template <int G, bool BATCHED>
__global__ void __launch_bounds__(128, 4) k_build_group(Dev d, LJ lj)
{
    if (stopped(d.status)) return;
    constexpr int U = 2;                                    // candidates per lane per round
    constexpr unsigned gbits = (1u << G) - 1u;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gi = t / G;
    const int l = (int)(t % G);
    const int lane = threadIdx.x & 31;
    const int gbase = lane & ~(G - 1);
    const int32_t ng = d.gcell_start[d.ncells];
    // groups past the last one run the loops with empty ranges (no early
    // return: trip counts and ballots stay uniform over the warp)
    int32_t a0 = 0;
    int m = 0;
    if (gi < ng && MD_CHECK(d, gi < d.ngmax)) {
        const uint32_t gw = (uint32_t)d.grp[gi];
        a0 = (int32_t)(gw & kJMask);
        m = (int)(gw >> kJBits) + 1;
        if (!MD_CHECK(d, a0 + m <= d.n)) m = 0;
    }
    const Rep &R = d.reps[BATCHED && m > 0 ? d.rep_of[a0] : 0];
    float px[G], py[G], pz[G];
    uint32_t pack = 0;
#pragma unroll
    for (int k = 0; k < G; k++) {
        // absent members sit far away (and away from the sentinel slot)
        const float4 q = k < m ? d.p32[a0 + k] : make_float4(-1.0e4f, -1.0e4f, -1.0e4f, 0.f);
        px[k] = q.x; py[k] = q.y; pz[k] = q.z;
        if (k == 0 && m > 0) pack = __float_as_uint(q.w);
    }
    const int ci[3] = {(int)(pack & 1023u), (int)((pack >> 10) & 1023u), (int)((pack >> 20) & 1023u)};
    const int64_t ngmax = d.ngmax;
    const int32_t cap = d.gcap;
    const float4 *p32 = d.p32;
    const float lo = lj.rs2f_lo, hi = lj.rs2f_hi;
    int32_t *rows = d.gnb;
    uint8_t *masks = d.gmask;
    int32_t cnt = 0;

    for (int ox = -1; ox <= 1; ox++) {
        int ux = ci[0] + ox, kx = 0;
        if (ux < 0) { ux += R.nc[0]; kx = -1; } else if (ux >= R.nc[0]) { ux -= R.nc[0]; kx = 1; }
        const float offx = (float)ox * -R.nsf[0];
        for (int oy = -1; oy <= 1; oy++) {
            int uy = ci[1] + oy, ky = 0;
            if (uy < 0) { uy += R.nc[1]; ky = -1; } else if (uy >= R.nc[1]) { uy -= R.nc[1]; ky = 1; }
            const float offy = (float)oy * -R.nsf[1];
            const int32_t col = (int32_t)cell_id(R, ux, uy, 0);
            for (int oz = -1; oz <= 1; oz++) {
                int uz = ci[2] + oz, kz = 0;
                if (uz < 0) { uz += R.nc[2]; kz = -1; } else if (uz >= R.nc[2]) { uz -= R.nc[2]; kz = 1; }
                const float offz = (float)oz * -R.nsf[2];
                const int32_t cid = cell_id_z(col, uz);
                int32_t j0 = 0, j1 = 0;
                if (m > 0 && MD_CHECK(d, cid >= 0 && cid < d.ncells)) {
                    j0 = d.cell_start[key_of(d, cid)];
                    j1 = d.cell_start[key_of(d, cid + 1)];
                    if (!MD_CHECK(d, j0 >= 0 && j0 <= j1 && j1 <= d.n)) j1 = j0;
                }
                const uint32_t tag = offset_code(ox, oy, oz) << kJBits;
                const int nr = (j1 - j0 + G * U - 1) / (G * U);
                const int rmax = __reduce_max_sync(0xffffffffu, nr);
                for (int r = 0; r < rmax; r++) {
                    uint32_t mk[U];
                    int32_t jj[U];
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        const int32_t j = j0 + (r * U + u) * G + l;
                        const bool valid = j < j1 && (uint32_t)(j - a0) >= (uint32_t)m;
                        const float4 pj = __ldg(p32 + (j < j1 ? j : d.n));
                        const float qx = pj.x + offx, qy = pj.y + offy, qz = pj.z + offz;
                        uint32_t in = 0, band = 0;
#pragma unroll
                        for (int k = 0; k < G; k++) {
                            const float dx = px[k] - qx, dy = py[k] - qy, dz = pz[k] - qz;
                            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                            in |= (uint32_t)(r2 < lo) << k;
                            band |= (uint32_t)((r2 >= lo) & (r2 < hi)) << k;
                        }
                        if (!valid) in = band = 0;
                        if (band) in |= exact_bits<G>(d, lj, R, a0, j, band, kx, ky, kz);
                        mk[u] = in;
                        jj[u] = j;
                    }
#pragma unroll
                    for (int u = 0; u < U; u++) {
                        const bool acc = mk[u] != 0u;
                        const unsigned bal = (__ballot_sync(0xffffffffu, acc) >> gbase) & gbits;
                        if (acc) {
                            const int32_t k = cnt + __popc(bal & ((1u << l) - 1u));
                            if (k < cap) {
                                const int64_t at = ((int64_t)(k >> 4) * ngmax + gi) * 16 + (k & 15);
                                rows[at] = (int32_t)((uint32_t)jj[u] | tag);
                                masks[at] = (uint8_t)mk[u];
                            }
                        }
                        cnt += __popc(bal);
                    }
                }
            }
        }
    }
    if (m == 0) return;
    // pad the last 16-entry block with entries for the sentinel slot n
    const int32_t pad = (int32_t)((uint32_t)d.n | (kZeroOffset << kJBits));
    const int32_t end = min((cnt + 15) & ~15, cap);
    for (int32_t k = cnt + l; k < end; k += G) {
        const int64_t at = ((int64_t)(k >> 4) * ngmax + gi) * 16 + (k & 15);
        rows[at] = pad;
        masks[at] = 0;
    }
    if (l == 0) {
        // member pairs inside the list radius (same cell: the direct image)
        uint32_t pairs = 0;
        for (int a = 0; a < m; a++)
            for (int b = a + 1; b < m; b++) {
                const float dx = px[a] - px[b], dy = py[a] - py[b], dz = pz[a] - pz[b];
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                bool in = r2 < lo;
                if (!in && r2 < hi) {
                    const dvec4 xa = d.x[a0 + a], xb = d.x[a0 + b];
                    const double tx = image_diff(xa.x, xb.x, 0, R.L[0]);
                    const double ty = image_diff(xa.y, xb.y, 0, R.L[1]);
                    const double tz = image_diff(xa.z, xb.z, 0, R.L[2]);
                    in = __dadd_rn(__dadd_rn(__dmul_rn(tx, tx), __dmul_rn(ty, ty)), __dmul_rn(tz, tz)) < lj.rs2;
                }
                if (in) pairs |= (1u << (a * G + b)) | (1u << (b * G + a));
            }
        d.gpair[gi] = (uint16_t)pairs;
        d.gnb_count[gi] = cnt;
        atomicMax(&d.status->max_count, cnt);
        if (cnt > cap) {
            atomicOr(&d.status->flags, FLAG_NL_OVERFLOW);
            d.status->overflow_at = d.status->rebuild_count;
            d.status->overflow_step = d.status->dev_step;
        }
    }
}

// Per-atom rows of a group list: member k of group g holds the entries of
// the group's row with bit k set and the members paired with it; counts and
// rows in caller order (rows: replica-local ids, at most cap per row; counts
// are complete).
template <int G, bool BATCHED>
__global__ void __launch_bounds__(128) k_decode_group(Dev d, LJ lj, int32_t *counts,
                                                      int32_t *rows, int32_t cap)
{
    (void)lj;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gi = t / G;
    const int k = (int)(t % G);
    if (gi >= d.gcell_start[d.ncells] || !MD_CHECK(d, gi < d.ngmax)) return;
    const uint32_t gw = (uint32_t)d.grp[gi];
    const int32_t a0 = (int32_t)(gw & kJMask);
    const int m = (int)(gw >> kJBits) + 1;
    if (k >= m) return;
    const int32_t i = a0 + k;
    if (!MD_CHECK(d, i < d.n)) return;
    const Rep &R = d.reps[BATCHED ? d.rep_of[i] : 0];
    const int64_t o = d.id[i];
    int32_t cnt = 0;
    auto put = [&](int32_t j) {
        if (!MD_CHECK(d, j >= 0 && j < d.n)) return;
        if (cnt < cap) rows[o * cap + cnt] = (int32_t)(d.id[j] - R.atom_off);
        cnt++;
    };
    const uint32_t pairs = d.gpair[gi];
    for (int b = 0; b < m; b++)
        if ((pairs >> (k * G + b)) & 1u) put(a0 + b);
    const int32_t gc = MD_CHECK(d, d.gnb_count[gi] <= d.gcap) ? d.gnb_count[gi] : 0;
    for (int32_t e = 0; e < gc; e++) {
        const int64_t at = ((int64_t)(e >> 4) * d.ngmax + gi) * 16 + (e & 15);
        if ((d.gmask[at] >> k) & 1u) put((int32_t)((uint32_t)d.gnb[at] & kJMask));
    }
    counts[o] = cnt;
}

}  // namespace

int launch_decode_group(const Dev &d, const LJ &lj, int G, int32_t *counts, int32_t *rows,
                        int32_t cap, cudaStream_t st, int *nl)
{
    if (d.n <= 0) return 0;
    if ((G != 2 && G != 4) || !d.gnb || !d.grp || !d.gmask || !d.gpair) return -1;
    const bool b = d.nrep > 1;
    const unsigned g = (unsigned)((d.ngmax * G + 127) / 128);
    if (G == 4) {
        if (b) k_decode_group<4, true><<<g, 128, 0, st>>>(d, lj, counts, rows, cap);
        else k_decode_group<4, false><<<g, 128, 0, st>>>(d, lj, counts, rows, cap);
    } else {
        if (b) k_decode_group<2, true><<<g, 128, 0, st>>>(d, lj, counts, rows, cap);
        else k_decode_group<2, false><<<g, 128, 0, st>>>(d, lj, counts, rows, cap);
    }
    *nl += 1;
    return (int)cudaGetLastError();
}

int launch_build_group(const Dev &d, const LJ &lj, int G, cudaStream_t st, int *nl)
{
    if (d.n <= 0) return 0;
    if ((G != 2 && G != 4) || !d.gnb || !d.grp || !d.gmask || !d.gpair) return -1;
    const bool b = d.nrep > 1;
    const unsigned g = (unsigned)((d.ngmax * G + 127) / 128);
    if (G == 4) {
        if (b) k_build_group<4, true><<<g, 128, 0, st>>>(d, lj);
        else k_build_group<4, false><<<g, 128, 0, st>>>(d, lj);
    } else {
        if (b) k_build_group<2, true><<<g, 128, 0, st>>>(d, lj);
        else k_build_group<2, false><<<g, 128, 0, st>>>(d, lj);
    }
    *nl += 1;
    return (int)cudaGetLastError();
}

// A warp-per-cell build (lanes = the cell's atoms, broadcast candidate loads)
// executed ~40 % fewer instructions but measured slower on GB300 (1241 vs
// 1041 us at 1M atoms, latency-bound), so the build is one thread per atom.
// 32-bit write offsets when every stored entry's offset fits: the largest is
// (cap / 4 - 1) 4n + 3 < cap n + 4.
template <bool B, bool H, bool S>
void launch_build_as(const Dev &d, const LJ &lj, unsigned g, cudaStream_t st)
{
    if ((int64_t)d.cap * d.n + 4 < ((int64_t)1 << 32)) k_build<B, H, S, true><<<g, 128, 0, st>>>(d, lj);
    else k_build<B, H, S, false><<<g, 128, 0, st>>>(d, lj);
}

int launch_build(const Dev &d, const LJ &lj, bool half, int64_t ncells, cudaStream_t st, int *nl)
{
    (void)ncells;
    if (d.n <= 0) return 0;
    const bool b = d.nrep > 1;
    const unsigned g = (unsigned)((d.n + 127) / 128);
    if (d.split) {
        if (b && half) launch_build_as<true, true, true>(d, lj, g, st);
        else if (b) launch_build_as<true, false, true>(d, lj, g, st);
        else if (half) launch_build_as<false, true, true>(d, lj, g, st);
        else launch_build_as<false, false, true>(d, lj, g, st);
    } else {
        if (b && half) launch_build_as<true, true, false>(d, lj, g, st);
        else if (b) launch_build_as<true, false, false>(d, lj, g, st);
        else if (half) launch_build_as<false, true, false>(d, lj, g, st);
        else launch_build_as<false, false, false>(d, lj, g, st);
    }
    *nl += 1;
    return (int)cudaGetLastError();
}

}  // namespace mdk
