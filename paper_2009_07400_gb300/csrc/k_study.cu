// Variants of the mixed full-list force pass that the library measured and
// did not adopt, kept runnable so the measurements can be repeated
// (md_study_force_variant).  Each computes the forces of the current state
// over the current per-atom list (one lane per atom, forces only, no
// integration) into a scratch array.
//
//   1  SoA gathers: the neighbour's FP32 cell-relative position from three
//      float arrays (three 4-byte gathers per pair instead of one 16-byte one).
//   2  AoSoA gathers: blocks of four atoms stored x0..x3, y0..y3, z0..z3
//      (the clustered layout of the paper's Sec. 4.2), three 4-byte gathers
//      from one 48-byte block.
//   3  Neighbourhood in shared memory: one block per 2x2x2-cell tile stages
//      the positions of the tile's 4x4x4-cell neighbourhood in the tile's
//      frame, and every pair reads its neighbour from there (the entry's
//      cell offset picks the staged cell; no per-pair offset select).
//   4  The same with the staging done by the TMA: each staged cell is a
//      contiguous, 16-byte aligned range of the position array, copied by
//      one bulk copy (cp.async.bulk) that completes on a shared-memory
//      mbarrier; the block then shifts the staged positions into the tile
//      frame in place.  Its forces are bitwise those of variant 3.
//   5  The library's AoS float4 gathers through the texture path
//      (tex1Dfetch on a texture object over the position array) instead of
//      the load/store unit's global loads.
//   6  Half of the gathers through each path: the pairs of a list chunk
//      alternate between a global load and a texture fetch.
//
// Variants 1, 2, 5 and 6 evaluate every pair with the library kernel's
// arithmetic in the same order, so their forces are bitwise those of the
// library.
// Variant 3 forms displacements in the tile frame (coordinates up to two
// cells from its centre), so its FP32 rounding differs.
#include "md_internal.cuh"

namespace mdk {

namespace {

__device__ __forceinline__ float rcp_fast(float a)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

__device__ __forceinline__ void kahan(float &s, float &c, float term)
{
    const float y = term - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// SoA (3 arrays of n + 1) and AoSoA (blocks of 4: 12 floats) copies of p32,
// slot n the far-away sentinel like p32's.
__global__ void __launch_bounds__(256) k_study_layouts(const float4 *p32, int64_t n1, float *soa,
                                                        float *aosoa)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n1) return;
    const float4 p = p32[j];
    soa[j] = p.x;
    soa[n1 + j] = p.y;
    soa[2 * n1 + j] = p.z;
    float *b = aosoa + (j >> 2) * 12 + (j & 3);
    b[0] = p.x;
    b[4] = p.y;
    b[8] = p.z;
}

// Variants 1, 2, 5 and 6: the library's pair loop (one lane per atom, int4
// list chunks, offsets selected in registers, four pairs per Kahan step) with
// the gather replaced.
template <int LAYOUT>
__global__ void __launch_bounds__(256) k_study_gather(Dev d, LJ lj, const float *soa,
                                                      const float *aosoa, int64_t n1,
                                                      cudaTextureObject_t tex, float4 *fout)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const int64_t n = d.n;
    const Rep &R = d.reps[0];
    const float nsx = R.nsf[0], nsy = R.nsf[1], nsz = R.nsf[2];
    const float4 pi = d.p32[i];
    const int cnt = d.nb_count[i];
    const int nq = (cnt + 3) >> 2;
    const int4 *nb4 = reinterpret_cast<const int4 *>(d.nb);
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    const float qx0 = pi.x - nsx, qx2 = pi.x + nsx;
    const float qy0 = pi.y - nsy, qy2 = pi.y + nsy;
    const float qz0 = pi.z - nsz, qz2 = pi.z + nsz;
    auto pair = [&](uint32_t e, bool via_tex, float &px, float &py, float &pz) {
        const uint32_t j = e & kJMask;
        float jx, jy, jz;
        if (LAYOUT == 5 || LAYOUT == 6) {
            const float4 p = via_tex ? tex1Dfetch<float4>(tex, (int)j) : __ldg(d.p32 + j);
            jx = p.x;
            jy = p.y;
            jz = p.z;
        } else if (LAYOUT == 1) {
            jx = __ldg(soa + j);
            jy = __ldg(soa + n1 + j);
            jz = __ldg(soa + 2 * n1 + j);
        } else {
            const float *b = aosoa + (j >> 2) * 12 + (j & 3);
            jx = __ldg(b);
            jy = __ldg(b + 4);
            jz = __ldg(b + 8);
        }
        const uint32_t c = e >> kJBits;
        const float dx = ((c & 2u) ? qx2 : ((c & 1u) ? pi.x : qx0)) - jx;
        const float dy = ((c & 8u) ? qy2 : ((c & 4u) ? pi.y : qy0)) - jy;
        const float dz = ((c & 32u) ? qz2 : ((c & 16u) ? pi.z : qz0)) - jz;
        const float rsq = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float sr2 = rcp_fast(rsq);
        const float t = sr2 * sr2 * sr2 * lj.sigma6f;
        float f = sr2 * t * fmaf(lj.c48ef, t, -lj.c24ef);
        f = rsq < lj.rc2f ? f : 0.f;
        px = fmaf(f, dx, px);
        py = fmaf(f, dy, py);
        pz = fmaf(f, dz, pz);
    };
    int4 nxt = nq > 0 ? __ldcs(nb4 + i) : make_int4(0, 0, 0, 0);
    for (int q = 0; q < nq; q++) {
        const int4 e = nxt;
        if (q + 1 < nq) nxt = __ldcs(nb4 + (int64_t)(q + 1) * n + i);
        float px = 0.f, py = 0.f, pz = 0.f;
        pair((uint32_t)e.x, LAYOUT == 5, px, py, pz);
        pair((uint32_t)e.y, LAYOUT >= 5, px, py, pz);
        pair((uint32_t)e.z, LAYOUT == 5, px, py, pz);
        pair((uint32_t)e.w, LAYOUT >= 5, px, py, pz);
        kahan(sx, cx, px);
        kahan(sy, cy, py);
        kahan(sz, cz, pz);
    }
    fout[i] = make_float4(sx - cx, sy - cy, sz - cz, 0.f);
}

constexpr int kTileSlots = 3008;   // staged atoms per block (47 KiB of float4; static shared
                                   // memory stays below 48 KiB with the tables)
constexpr long long kWaitCycles = 20000000;   // bulk-copy wait limit (~10 ms at 2 GHz)

// Variants 3 and 4: block b = 2x2x2-cell tile b of the (single) replica.
// Staged cell L = (lx, ly, lz) in [0, 4)^3 is the cell at (2 t + l - 1) per
// dimension (periodic), its atoms shifted into the tile frame (origin at the
// tile's centre): p + (l - 1.5) s.  A pair's staged slot is off[L] + j with
// L = (the atom's local cell) + (the entry's cell offset).  Returns with the
// overflow flag raised if a neighbourhood holds more than kTileSlots atoms,
// and (TMA) with the timeout flag if the bulk copies do not complete within
// kWaitCycles (the block then waits once more, bounded, before it leaves).
template <bool TMA>
__global__ void __launch_bounds__(256) k_study_tiles(Dev d, LJ lj, float4 *fout)
{
    __shared__ __align__(128) float4 pos[kTileSlots];
    __shared__ int32_t off[64];
    __shared__ int32_t base[65];
    __shared__ __align__(8) uint64_t bar;
    const Rep &R = d.reps[0];
    const int64_t tile = blockIdx.x;
    const int tz = (int)(tile % R.nt[2]);
    const int ty = (int)((tile / R.nt[2]) % R.nt[1]);
    const int tx = (int)(tile / ((int64_t)R.nt[2] * R.nt[1]));
    const float s[3] = {-R.nsf[0], -R.nsf[1], -R.nsf[2]};
    // cell ranges of the 64 staged cells and their slot bases
    if (threadIdx.x < 64) {
        const int l[3] = {(int)threadIdx.x >> 4, ((int)threadIdx.x >> 2) & 3, (int)threadIdx.x & 3};
        const int t3[3] = {tx, ty, tz};
        int g[3];
        for (int q = 0; q < 3; q++) {
            g[q] = 2 * t3[q] + l[q] - 1;
            if (g[q] < 0) g[q] += R.nc[q];
            else if (g[q] >= R.nc[q]) g[q] -= R.nc[q];
        }
        int32_t j0 = 0, j1 = 0;
        if (g[0] < R.nc[0] && g[1] < R.nc[1] && g[2] < R.nc[2]) {   // (nc < 2 never occurs)
            const int64_t cid = cell_id(R, g[0], g[1], g[2]);
            j0 = d.cell_start[key_of(d, cid)];
            j1 = d.cell_start[key_of(d, cid + 1)];
        }
        base[threadIdx.x] = j1 - j0;        // counts, summed below
        off[threadIdx.x] = j0;              // first atom, for now
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t acc = 0;
        for (int L = 0; L < 64; L++) {
            const int32_t c = base[L];
            base[L] = acc;
            acc += c;
        }
        base[64] = acc;
    }
    __syncthreads();
    const int32_t total = base[64];
    if (total > kTileSlots) {
        if (threadIdx.x == 0) atomicOr(&d.status->flags, FLAG_NL_OVERFLOW);
        return;
    }
    if (TMA) {
        // one bulk copy per non-empty cell (16-byte aligned source and
        // destination, 16 bytes per atom), completing on the mbarrier; the
        // expected byte count is registered before any copy is issued
        const uint32_t bar_a = (uint32_t)__cvta_generic_to_shared(&bar);
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a),
                         "r"((uint32_t)total * 16u) : "memory");
        }
        __syncthreads();
        if (threadIdx.x < 64) {
            const int32_t cnt = base[threadIdx.x + 1] - base[threadIdx.x];
            if (cnt > 0) {
                const uint32_t dst = (uint32_t)__cvta_generic_to_shared(pos + base[threadIdx.x]);
                const float4 *src = d.p32 + off[threadIdx.x];
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                    "l"(src), "r"((uint32_t)cnt * 16u), "r"(bar_a) : "memory");
            }
        }
        auto wait = [&]() {
            const long long t0 = clock64();
            uint32_t ok = 0;
            while (!ok && clock64() - t0 < kWaitCycles)
                asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                             : "=r"(ok) : "r"(bar_a) : "memory");
            return ok != 0;
        };
        // every thread waits; the block leaves together if any gave up
        if (__syncthreads_or(!wait())) {
            if (threadIdx.x == 0) atomicOr(&d.status->flags, FLAG_TIMEOUT);
            __syncthreads_or(!wait());      // the copies of this block, once more
            return;
        }
        for (int32_t k = threadIdx.x; k < total; k += blockDim.x) {
            int L = 0;
            while (base[L + 1] <= k) L++;
            const float4 p = pos[k];
            pos[k] = make_float4(p.x + ((float)(L >> 4) - 1.5f) * s[0], p.y + ((float)((L >> 2) & 3) - 1.5f) * s[1],
                                 p.z + ((float)(L & 3) - 1.5f) * s[2], 0.f);
        }
    } else {
        // stage: every staged slot from its cell, shifted into the tile frame
        for (int32_t k = threadIdx.x; k < total; k += blockDim.x) {
            int L = 0;
            while (base[L + 1] <= k) L++;
            const int32_t j = off[L] + (k - base[L]);
            const float4 p = d.p32[j];
            pos[k] = make_float4(p.x + ((float)(L >> 4) - 1.5f) * s[0], p.y + ((float)((L >> 2) & 3) - 1.5f) * s[1],
                                 p.z + ((float)(L & 3) - 1.5f) * s[2], 0.f);
        }
    }
    __syncthreads();
    if (threadIdx.x < 64) off[threadIdx.x] = base[threadIdx.x] - off[threadIdx.x];   // slot = off[L] + j
    __syncthreads();
    // the tile's own atoms: cells 8 tile .. 8 tile + 7 are consecutive
    const int32_t a0 = d.cell_start[key_of(d, R.cell_off + tile * 8)],
                  a1 = d.cell_start[key_of(d, R.cell_off + tile * 8 + 8)];
    const int4 *nb4 = reinterpret_cast<const int4 *>(d.nb);
    const int64_t n = d.n;
    for (int32_t i = a0 + (int32_t)threadIdx.x; i < a1; i += blockDim.x) {
        const float4 p = d.p32[i];
        const uint32_t pack = __float_as_uint(p.w);
        const int li[3] = {(int)(pack & 1023u) - (2 * tx - 1), (int)((pack >> 10) & 1023u) - (2 * ty - 1),
                           (int)((pack >> 20) & 1023u) - (2 * tz - 1)};
        const float pix = p.x + ((float)li[0] - 1.5f) * s[0];
        const float piy = p.y + ((float)li[1] - 1.5f) * s[1];
        const float piz = p.z + ((float)li[2] - 1.5f) * s[2];
        // local cell of an entry with cell code c (o + 1 per dimension):
        // (li + o) per dimension, i.e. lc0 + x-field * 16 + y-field * 4 + z-field
        const int lc0 = (li[0] - 1) * 16 + (li[1] - 1) * 4 + (li[2] - 1);
        const int cnt = d.nb_count[i];
        const int nq = (cnt + 3) >> 2;
        float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
        auto pair = [&](uint32_t e, float &px, float &py, float &pz) {
            const uint32_t j = e & kJMask;
            const uint32_t c = e >> kJBits;
            float4 pj = make_float4(1.0e4f, 1.0e4f, 1.0e4f, 0.f);       // padding: far away
            if (j < (uint32_t)n) {
                const int L = lc0 + (int)(c & 3u) * 16 + (int)((c >> 2) & 3u) * 4 + (int)(c >> 4);
                pj = pos[off[L] + (int32_t)j];
            }
            const float dx = pix - pj.x, dy = piy - pj.y, dz = piz - pj.z;
            const float rsq = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float sr2 = rcp_fast(rsq);
            const float t = sr2 * sr2 * sr2 * lj.sigma6f;
            float f = sr2 * t * fmaf(lj.c48ef, t, -lj.c24ef);
            f = rsq < lj.rc2f ? f : 0.f;
            px = fmaf(f, dx, px);
            py = fmaf(f, dy, py);
            pz = fmaf(f, dz, pz);
        };
        for (int q = 0; q < nq; q++) {
            const int4 e = __ldcs(nb4 + (int64_t)q * n + i);
            float px = 0.f, py = 0.f, pz = 0.f;
            pair((uint32_t)e.x, px, py, pz);
            pair((uint32_t)e.y, px, py, pz);
            pair((uint32_t)e.z, px, py, pz);
            pair((uint32_t)e.w, px, py, pz);
            kahan(sx, cx, px);
            kahan(sy, cy, py);
            kahan(sz, cz, pz);
        }
        fout[i] = make_float4(sx - cx, sy - cy, sz - cz, 0.f);
    }
}

}  // namespace

int64_t study_layout_floats(int64_t n) { return 3 * (n + 1) + 12 * ((n + 1 + 3) / 4); }

// Variants 1, 2, 5 and 6 into fout (n float4, cell order).  layouts: device
// scratch of study_layout_floats(n) floats (variants 1 and 2 fill it on every
// call); tex: a texture object over d.p32 (n + 1 float4; variants 5 and 6).
int launch_study_force(const Dev &d, const LJ &lj, int variant, float *layouts,
                       cudaTextureObject_t tex, float4 *fout, cudaStream_t st, int *nl)
{
    if (d.n <= 0 || d.nrep != 1) return -1;
    const int64_t n1 = d.n + 1;
    const unsigned g = (unsigned)((d.n + 255) / 256);
    float *soa = layouts, *aosoa = layouts + 3 * n1;
    if (variant == 1 || variant == 2) {
        k_study_layouts<<<(unsigned)((n1 + 255) / 256), 256, 0, st>>>(d.p32, n1, soa, aosoa);
        if (variant == 1) k_study_gather<1><<<g, 256, 0, st>>>(d, lj, soa, aosoa, n1, tex, fout);
        else k_study_gather<2><<<g, 256, 0, st>>>(d, lj, soa, aosoa, n1, tex, fout);
        *nl += 2;
    } else if (variant == 5 || variant == 6) {
        if (variant == 5) k_study_gather<5><<<g, 256, 0, st>>>(d, lj, soa, aosoa, n1, tex, fout);
        else k_study_gather<6><<<g, 256, 0, st>>>(d, lj, soa, aosoa, n1, tex, fout);
        *nl += 1;
    } else {
        return -1;   // variants 3 and 4: launch_study_tiles
    }
    return (int)cudaGetLastError();
}

int launch_study_tiles(const Dev &d, const LJ &lj, int64_t ntiles, bool tma, float4 *fout,
                       cudaStream_t st, int *nl)
{
    if (d.n <= 0 || d.nrep != 1 || ntiles <= 0) return -1;
    if (tma) k_study_tiles<true><<<(unsigned)ntiles, 256, 0, st>>>(d, lj, fout);
    else k_study_tiles<false><<<(unsigned)ntiles, 256, 0, st>>>(d, lj, fout);
    *nl += 1;
    return (int)cudaGetLastError();
}

}  // namespace mdk
