// Cell binning (tinyMD Sec. 3.2, Fig. 1: cells of side >= rc + skin; Sec. 6:
// "distribution over cells" every 20 steps).
//
// GPU design: a counting sort in four passes over HBM-resident SoA data.
//   1. k_bin_assign   one thread per atom: wrap x into the box (one
//                     conditional +/-L per component, written back only
//                     when it changed), cell = (int)(x/s) clamped to nc-1,
//                     and with split cells the octant of the atom in its
//                     cell (which half along each axis: the half-size cells
//                     of Sec. 3.2, which the list build scans); histogram of
//                     the keys (cell, or cell and octant) with one atomicAdd
//                     per distinct key of a warp.
//   2. scan           exclusive prefix sum of the histogram (three kernels,
//                     4096 cells per 1024-thread block, warp shuffles).
//   3. k_bin_scatter  one thread per atom: slot = start + count - 1 - rank,
//                     count taken down by one atomicSub per distinct cell of
//                     a warp (leaves the histogram at zero for the next
//                     binning).
//   4. k_sort_gather  a group of 32, 16, 8 or 4 lanes per key (from the
//                     mean occupancy): rank the key's members by caller
//                     id (so the order is the stable (cell, id) order, or
//                     (cell, octant, id) with split cells, independent of
//                     atomic arrival order) and gather x, v,
//                     id into the reordered buffers; also writes the
//                     cell-relative FP32 position p = fl32(x - C_cell) and
//                     the packed cell coordinates used by the mixed path.
#include <cfloat>

#include "md_internal.cuh"

namespace mdk {

namespace {

__device__ __forceinline__ bool stopped(const DevStatus *st)
{
    return *((volatile const int32_t *)&st->flags) != 0;
}

template <bool BATCHED>
__global__ void __launch_bounds__(256) k_bin_assign(Dev d)
{
    if (stopped(d.status)) return;
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a == 0) d.status->rebuild_count += 1;
    if (a >= d.n) return;
    const Rep &R = d.reps[BATCHED ? d.rep_of[a] : 0];
    const dvec4 x = d.x[a];
    double c[3] = {x.x, x.y, x.z};
    int32_t k[3];
    uint32_t oct = 0;
    int32_t bad = 0;
    bool moved = false;
    for (int q = 0; q < 3; q++) {
        double u = c[q];
        const double L = R.L[q];
        // The tests read the IEEE bit patterns as integers (GB300's FP64
        // pipe is narrow): all-ones exponent = inf or NaN; u < 0 iff the
        // sign is set and u is not -0.0; and for u >= 0, u >= L iff its
        // pattern is at least L's.  Only atoms outside [0, L) do FP64 work.
        const int64_t b = __double_as_longlong(u);
        if ((b & 0x7ff0000000000000LL) == 0x7ff0000000000000LL) {
            bad |= FLAG_NONFINITE;
            u = 0.0;
            moved = true;
        } else {
            const bool neg = b < 0 && b != (int64_t)0x8000000000000000LL;
            if (neg || b >= __double_as_longlong(L)) {
                u = neg ? u + L : u - L;
                if (u < 0.0 || u > L) { bad |= FLAG_BADPOS; u = 0.0; }
                moved = true;
            }
        }
        c[q] = u;
        // (int)(u / s) with the IEEE FP64 quotient.  GB300's FP64 divide is
        // slow, so the quotient is estimated in FP32 (error < 2e-4 for
        // u/s <= 1023) and the exact division runs only when the estimate
        // lies within 1e-3 of an integer, where the two could disagree.
        const float y = (float)u * R.invsf[q];
        int32_t kk = (int32_t)y;
        const float fr = y - (float)kk;
        if (fr < 1e-3f || fr > 1.0f - 1e-3f) kk = (int32_t)(u / R.s[q]);
        k[q] = kk >= R.nc[q] ? R.nc[q] - 1 : kk;
        // octant bit: the upper half of the cell along q.  y - k is the
        // position in the cell in cell units, within 2e-4 of u/s - k (the
        // list build allows 1e-3 for it); for the last cell it can reach 1
        oct = (oct << 1) | (uint32_t)(y - (float)k[q] >= 0.5f);
    }
    if (bad) atomicOr(&d.status->flags, bad);
    if (moved) d.x[a] = mk_dvec4(c[0], c[1], c[2], 0.0);
    int32_t key = (int32_t)key_of(d, cell_id(R, k[0], k[1], k[2]));
    if (d.split) key |= (int32_t)oct;
    if (!MD_CHECK(d, key >= 0 && key < nkeys(d))) return;
    d.cell_key[a] = key;
    // atoms arrive roughly in cell order, so lanes of a warp share keys:
    // one atomic per distinct key of the warp
    const unsigned same = __match_any_sync(__activemask(), key);
    if ((threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&d.cell_count[key], __popc(same));
}

// Block-wide exclusive scan of 4 values per thread (1024 threads).
__device__ __forceinline__ int32_t block_exclusive(int32_t v, int32_t *warp_tot, int32_t *total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        int32_t t = warp_tot[lane];
        int32_t s = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t u = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += u;
        }
        warp_tot[lane] = s - t;
        if (lane == 31) *total = s;
    }
    __syncthreads();
    return inc - v + warp_tot[w];
}

constexpr int kScanPer = 4096;  // elements per scan block (1024 threads x 4)

// Phase A: per-block exclusive scan of in[] into out[], block total to tot[b].
__global__ void __launch_bounds__(1024) k_scan_block(const int32_t *in, int32_t *out,
                                                      int64_t len, int32_t *tot)
{
    __shared__ int32_t wt[32];
    __shared__ int32_t total;
    int64_t base = (int64_t)blockIdx.x * kScanPer + threadIdx.x * 4;
    int32_t v[4];
#pragma unroll
    for (int q = 0; q < 4; q++) v[q] = (base + q < len) ? in[base + q] : 0;
    int32_t sum = v[0] + v[1] + v[2] + v[3];
    int32_t ex = block_exclusive(sum, wt, &total);
#pragma unroll
    for (int q = 0; q < 4; q++) {
        if (base + q < len) out[base + q] = ex;
        ex += v[q];
    }
    if (threadIdx.x == 0) tot[blockIdx.x] = total;
}

// Phase B: one block scans the block totals (any count, in chunks of 4096)
// and writes the grand total to out[len].
__global__ void __launch_bounds__(1024) k_scan_tops(int32_t *tot, int64_t nb, int32_t *out,
                                                     int64_t len)
{
    __shared__ int32_t wt[32];
    __shared__ int32_t total;
    int32_t carry = 0;
    for (int64_t c0 = 0; c0 < nb; c0 += kScanPer) {
        int64_t base = c0 + threadIdx.x * 4;
        int32_t v[4];
#pragma unroll
        for (int q = 0; q < 4; q++) v[q] = (base + q < nb) ? tot[base + q] : 0;
        int32_t ex = block_exclusive(v[0] + v[1] + v[2] + v[3], wt, &total);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (base + q < nb) tot[base + q] = carry + ex;
            ex += v[q];
        }
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[len] = carry;
}

// Phase C: add each block's offset.
__global__ void __launch_bounds__(1024) k_scan_add(int32_t *out, int64_t len, const int32_t *tot)
{
    int64_t base = (int64_t)blockIdx.x * kScanPer + threadIdx.x * 4;
    int32_t off = tot[blockIdx.x];
#pragma unroll
    for (int q = 0; q < 4; q++)
        if (base + q < len) out[base + q] += off;
}

__global__ void __launch_bounds__(256) k_bin_scatter(Dev d)
{
    if (stopped(d.status)) return;
    int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= d.n) return;
    int32_t key = d.cell_key[a];
    if (!MD_CHECK(d, key >= 0 && key < nkeys(d))) return;
    // one atomic per distinct key of the warp (atoms arrive roughly in cell
    // order); the slots of a key are re-ranked by id afterwards, so their
    // order here does not matter
    const unsigned same = __match_any_sync(__activemask(), key);
    const int leader = __ffs(same) - 1;
    int32_t top = 0;
    if ((int)(threadIdx.x & 31) == leader) top = atomicSub(&d.cell_count[key], __popc(same));
    top = __shfl_sync(same, top, leader);
    const int32_t below = __popc(same & ((1u << (threadIdx.x & 31)) - 1u));
    int32_t pos = d.cell_start[key] + top - 1 - below;
    if (!MD_CHECK(d, pos >= 0 && pos < d.n)) return;
    d.perm[pos] = (int32_t)a;
}

// G lanes per key (G = 32, 16, 8 or 4, chosen from the mean key
// occupancy, so that small cells do not leave most of a warp idle): rank
// each key's members by caller id with shuffles inside the group, gather
// into the new order.  All 32 lanes run the same number of loop trips (the
// warp's largest key), so every shuffle has the whole warp converged.
template <int G, bool BATCHED>
__global__ void __launch_bounds__(256) k_sort_gather(Dev d, int64_t nk)
{
    if (stopped(d.status)) return;
    const int gl = threadIdx.x % G;
    const int64_t key = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    int32_t start = 0, m = 0;
    if (key < nk) {
        start = d.cell_start[key];
        m = d.cell_start[key + 1] - start;
        if (!MD_CHECK(d, start >= 0 && m >= 0 && start + m <= d.n)) m = 0;
    }
    int32_t mmax = m;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mmax = max(mmax, __shfl_xor_sync(0xffffffffu, mmax, o));
    for (int32_t base = 0; base < mmax; base += G) {
        const int32_t mine = base + gl;
        const bool have = mine < m;
        const int32_t old = have ? d.perm[start + mine] : 0;
        const int32_t my_id = have ? d.id[old] : INT32_MAX;
        int32_t rank = 0;
        for (int32_t c0 = 0; c0 < mmax; c0 += G) {
            const int32_t other = (c0 + gl < m) ? d.id[d.perm[start + c0 + gl]] : INT32_MAX;
#pragma unroll
            for (int t = 0; t < G; t++) rank += (__shfl_sync(0xffffffffu, other, t, G) < my_id);
        }
        if (!have) continue;
        const int32_t ns = start + rank;
        const dvec4 x = d.x[old];
        const dvec4 v = d.v[old];
        d.x_alt[ns] = x;
        d.v_alt[ns] = v;
        d.id_alt[ns] = my_id;
        // contact model: the velocity copies in the new order
        if (d.v32) store_vel_copy(d.v32, d.vlo, ns, v);
        const Rep &R = d.reps[BATCHED ? d.rep_of[ns] : 0];
        int cx, cy, cz;
        cell_coords(R, key >> (3 * d.split), cx, cy, cz);
        // centres (c + 0.5) s from the table the force epilogue uses, so
        // both compute p = fl32(x - C) from the same C
        const double *ct = d.ctr + R.ctr_off;
        const double px = x.x - __ldg(ct + cx);
        const double py = x.y - __ldg(ct + R.nc[0] + cy);
        const double pz = x.z - __ldg(ct + R.nc[0] + R.nc[1] + cz);
        const uint32_t pack = (uint32_t)cx | ((uint32_t)cy << 10) | ((uint32_t)cz << 20);
        store_cell_pos(d, R, d.p32, d.plo, ns, px, py, pz, pack);
    }
}

// Groups of up to G consecutive atoms of one cell (the rows of a list shared
// by a group): per cell the number of groups, ceil(count / G) ...
__global__ void __launch_bounds__(256) k_group_count(Dev d, int64_t ncells, int G)
{
    if (stopped(d.status)) return;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    const int32_t m = d.cell_start[key_of(d, c + 1)] - d.cell_start[key_of(d, c)];
    d.gcnt[c] = (m + G - 1) / G;
}

// ... and, after the scan of those counts into gcell_start, the group table:
// group gcell_start[c] + k of cell c holds atoms start + kG .. start + kG +
// size - 1, packed as the first atom's slot (low kJBits bits) and size - 1.
__global__ void __launch_bounds__(256) k_group_fill(Dev d, int64_t ncells, int G)
{
    if (stopped(d.status)) return;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    const int32_t start = d.cell_start[key_of(d, c)];
    const int32_t m = d.cell_start[key_of(d, c + 1)] - start;
    const int32_t g0 = d.gcell_start[c];
    for (int32_t k = 0; k * G < m; k++) {
        const int32_t size = min(G, m - k * G);
        if (!MD_CHECK(d, g0 + k < d.ngmax && start + k * G < d.n)) return;
        d.grp[g0 + k] = (int32_t)((uint32_t)(start + k * G) | ((uint32_t)(size - 1) << kJBits));
    }
}

template <int G>
void launch_sort_gather(const Dev &d, int64_t nk, cudaStream_t st)
{
    const unsigned gs = (unsigned)((nk * G + 255) / 256);
    if (d.nrep > 1) k_sort_gather<G, true><<<gs, 256, 0, st>>>(d, nk);
    else k_sort_gather<G, false><<<gs, 256, 0, st>>>(d, nk);
}

inline unsigned blocks_for(int64_t n, int per) { return (unsigned)((n + per - 1) / per); }

}  // namespace

int64_t scan_tmp_elems(int64_t nkeys_total)
{
    return (nkeys_total + kScanPer - 1) / kScanPer + 1;
}

// Bins the atoms of d (all replicas).  On return the reordered state is in
// d.x_alt / d.v_alt / d.id_alt and d.p32 (the caller swaps the pointers).
int launch_bin(const Dev &d, int32_t *tmp, int64_t tmp_len, cudaStream_t st, int *nl)
{
    if (d.n <= 0) return 0;
    const bool batched = d.nrep > 1;
    const int64_t nk = nkeys(d);
    unsigned gb = blocks_for(d.n, 256);
    if (batched) k_bin_assign<true><<<gb, 256, 0, st>>>(d);
    else k_bin_assign<false><<<gb, 256, 0, st>>>(d);
    int64_t nb = (nk + kScanPer - 1) / kScanPer;
    if (nb + 1 > tmp_len) return -1;
    k_scan_block<<<(unsigned)nb, 1024, 0, st>>>(d.cell_count, d.cell_start, nk, tmp);
    k_scan_tops<<<1, 1024, 0, st>>>(tmp, nb, d.cell_start, nk);
    k_scan_add<<<(unsigned)nb, 1024, 0, st>>>(d.cell_start, nk, tmp);
    k_bin_scatter<<<gb, 256, 0, st>>>(d);
    // lanes per key from the mean occupancy (about 19 atoms per cell at the
    // LJ benchmark's density, 2.4 per octant; about 3 per cell for dense
    // granular packings)
    const int64_t mean = d.n / (nk > 0 ? nk : 1);
    if (mean >= 12) launch_sort_gather<32>(d, nk, st);
    else if (mean >= 6) launch_sort_gather<16>(d, nk, st);
    else if (mean >= 3) launch_sort_gather<8>(d, nk, st);
    else launch_sort_gather<4>(d, nk, st);
    *nl += 6;
    return (int)cudaGetLastError();
}

// Group table of the current binning for groups of G atoms (G = 2 or 4):
// d.gcnt <- groups per cell, d.gcell_start <- their exclusive prefix sums
// (the total, the number of groups, at d.gcell_start[ncells]), d.grp <- the
// groups.  tmp: the binning's scan scratch.
int launch_group_table(const Dev &d, int G, int64_t ncells, int32_t *tmp, int64_t tmp_len,
                       cudaStream_t st, int *nl)
{
    if (d.n <= 0) return 0;
    const int64_t nb = (ncells + kScanPer - 1) / kScanPer;
    if (nb + 1 > tmp_len || !d.gcnt || !d.gcell_start || !d.grp) return -1;
    const unsigned gc = blocks_for(ncells, 256);
    k_group_count<<<gc, 256, 0, st>>>(d, ncells, G);
    k_scan_block<<<(unsigned)nb, 1024, 0, st>>>(d.gcnt, d.gcell_start, ncells, tmp);
    k_scan_tops<<<1, 1024, 0, st>>>(tmp, nb, d.gcell_start, ncells);
    k_scan_add<<<(unsigned)nb, 1024, 0, st>>>(d.gcell_start, ncells, tmp);
    k_group_fill<<<gc, 256, 0, st>>>(d, ncells, G);
    *nl += 5;
    return (int)cudaGetLastError();
}

}  // namespace mdk
