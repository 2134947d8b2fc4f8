// LJ 12-6 forces over the Verlet list (tinyMD Sec. 3.2, Eq. 2) in the
// operation order of the potential kernel of Sec. 4.2:
//     sr2 = 1/rsq; sr6 = sr2*sr2*sr2*sigma^6; f = 48 eps sr6 (sr6 - 1/2) sr2
//     F_i += f * del,  del = x_i - x_j,  only if rsq < rc^2.
//
// GPU mapping (Sec. 3.1/4.1: one thread per particle; here TPA = 1, 2, 4 or 8
// lanes per atom, the larger counts for systems too small to fill the GPU): the neighbour-major list is streamed from HBM as int4
// chunks (ld.global.cs: evict-first, it is read once per step), neighbour
// positions are gathered through the read-only L1 path (16 B float4 in the
// mixed path, so the whole position array stays L2-resident), and the
// per-atom sum stays in registers.  No tensor cores: the pair gather is not a
// dense contraction.
//
// Pair arithmetic as executed: t = sr2^3 sigma^6 (the paper's sr6) and
// f = sr2 t (48 eps t - 24 eps), the same product regrouped so that the two
// constant factors fold into one FMA.
//
// Mixed path: positions are FP32 offsets from the centre of the atom's cell
// at the last binning; a neighbour's displacement is
//     d = (p_i - o s) - p_j
// with o its stencil offset (2 bits per dimension in the list entry), so
// |d|'s FP32 rounding error is that of numbers of size ~s rather than of the
// box length.  Per-atom sums are Kahan
// compensated: the four pairs of a list chunk are summed in a plain FP32
// partial and each partial enters a Kahan sum (the compensation then covers
// the long per-atom sum, where the rounding error accumulates).  The
// reciprocal is the hardware approximation (rcp.approx, relative error
// below 2^-22), which keeps the force error far inside the 1e-5 budget.
// Positions and velocities are integrated in FP64.
//
// Epilogues (velocity Verlet, Sec. 3.2 Eq. 1, kick-drift-kick, c = dt/(2m)):
//   EPI_F    store F
//   EPI_FK   store F; v += c F                          (last step of a run)
//   EPI_FKKD v += c F (full step n); v += c F; x += dt v; write the FP32
//            position of step n+1 into the other p32 buffer (other atoms are
//            still gathering this step's positions), and in the FP64 path
//            the FP64 position into the other x buffer for the same reason.
#include "md_internal.cuh"

namespace mdk {

namespace {

__device__ __forceinline__ bool stopped(const DevStatus *st)
{
    return *((volatile const int32_t *)&st->flags) != 0;
}

__device__ __forceinline__ int4 ld_stream(const int4 *p) { return __ldcs(p); }


// Kahan (compensated) accumulation: s + c tracks the exact running sum.
__device__ __forceinline__ void kahan_add(float &s, float &c, float term)
{
    const float y = term - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// FP64 reciprocal: a correctly rounded FP32 reciprocal of fl32(a) as the
// seed (relative error <= 2^-23), refined by one Newton-Raphson step
// r <- r + r (1 - a r), which squares it to <= 2^-46 (~1.4e-14), far inside
// the FP64 path's 1e-10 force tolerance.  The seed's two conversions run as
// integer operations on the bit patterns: GB300's FP64 pipe bounds this path,
// and this keeps it to the two FMAs of the Newton step.
__device__ __forceinline__ double rcp_nr(double a)
{
    const double r = f64_of_pos(__frcp_rn(f32_of_pos(a)));
    return fma(r, fma(-a, r, 1.0), r);
}

// FP32 reciprocal on the special-function unit (one instruction).
__device__ __forceinline__ float rcp_approx(float a)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}



// FP64 epilogue shared by both precisions.  fx..fz: force on atom i.
template <int EPI, bool ENERGY>
__device__ __forceinline__ void epilogue(const Dev &d, const LJ &lj, const Rep &R, int64_t i,
                                         double fx, double fy, double fz, uint32_t pack,
                                         bool mixed)
{
    if (EPI == EPI_F || EPI == EPI_FK) {
        if (mixed) d.f32[i] = make_float4((float)fx, (float)fy, (float)fz, 0.f);
        else d.f64[i] = mk_dvec4(fx, fy, fz, 0.0);
    }
    if (EPI == EPI_F) return;
    // the per-atom FP64 state is read and written once per step: streaming
    // (evict-first) accesses keep it from evicting the L1 lines of the
    // neighbour gathers (-2 % kernel time at 1M atoms)
    dvec4 v = ld_cs_dvec4(d.v + i);
    v.x = fma(lj.half_dt_m, fx, v.x);
    v.y = fma(lj.half_dt_m, fy, v.y);
    v.z = fma(lj.half_dt_m, fz, v.z);
    if (ENERGY) d.ke_atom64[i] = 0.5 * lj.mass * fma(v.x, v.x, fma(v.y, v.y, v.z * v.z));
    if (EPI == EPI_FKKD) {
        v.x = fma(lj.half_dt_m, fx, v.x);
        v.y = fma(lj.half_dt_m, fy, v.y);
        v.z = fma(lj.half_dt_m, fz, v.z);
        dvec4 x = mixed ? ld_cs_dvec4(d.x + i) : d.x[i];   // the FP64 path gathers x
        x.x = fma(lj.dt, v.x, x.x);
        x.y = fma(lj.dt, v.y, x.y);
        x.z = fma(lj.dt, v.z, x.z);
        // the FP64 path gathers neighbours from x itself: write the next
        // positions to the other buffer; the mixed path gathers p32 only
        if (mixed) st_cs_dvec4(d.x + i, x);
        else d.x_nxt[i] = x;
        // cell centres (c + 0.5) s from the per-replica table: the same values
        // as computing them, without integer conversions and FP64 products
        // on GB300's narrow FP64 pipe
        const double *ct = d.ctr + R.ctr_off;
        const double cx = __ldg(ct + (pack & 1023u));
        const double cy = __ldg(ct + R.nc[0] + ((pack >> 10) & 1023u));
        const double cz = __ldg(ct + R.nc[0] + R.nc[1] + ((pack >> 20) & 1023u));
        const float4 pn = make_float4((float)(x.x - cx), (float)(x.y - cy), (float)(x.z - cz),
                                      __uint_as_float(pack));
        d.p32_nxt[i] = pn;
        check_displacement(d, i, pn);
    }
    st_cs_dvec4(d.v + i, v);
}

// ---------------------------------------------------------------------------
// Mixed precision, full list.
// ---------------------------------------------------------------------------

// One tile of atoms of the mixed full-list kernel (tile = gt / blockDim).
template <int TPA, bool BATCHED, int EPI, bool ENERGY>
__device__ __forceinline__ void mixed_full_tile(const Dev &d, const LJ &lj, int64_t gt)
{
    const int64_t i0 = gt / TPA;
    const int sub = (int)(gt % TPA);
    const bool valid = i0 < d.n;
    if (TPA == 1 && !valid) return;
    const int64_t i = valid ? i0 : d.n - 1;
    const int64_t n = d.n;
    const Rep &R = d.reps[BATCHED ? d.rep_of[i] : 0];
    const float nsx = R.nsf[0], nsy = R.nsf[1], nsz = R.nsf[2];
    const float4 pi = d.p32[i];
    const int cnt = valid && MD_CHECK(d, d.nb_count[i] <= d.cap) ? d.nb_count[i] : 0;
    const int nq = (cnt + 3) >> 2;
    const int4 *nb4 = reinterpret_cast<const int4 *>(d.nb);

    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    float pe = 0.f, w = 0.f, cpe = 0.f, cw = 0.f;
    const float4 *p32 = d.p32;
    // p_i - o s for o = -1, 0, +1; ns = -s
    const float qx0 = pi.x - nsx, qx2 = pi.x + nsx;
    const float qy0 = pi.y - nsy, qy2 = pi.y + nsy;
    const float qz0 = pi.z - nsz, qz2 = pi.z + nsz;

    // one pair: adds f*d to (px, py, pz) and, with ENERGY, V and f r^2
    auto pair = [&](uint32_t e, float &px, float &py, float &pz, float &pv, float &pw) {
        if (!MD_CHECK(d, (e & kJMask) <= (uint32_t)d.n)) return;
        const float4 pj = __ldg(p32 + (e & kJMask));
        const uint32_t c = e >> kJBits;
        // the stencil offset selects p_i + s, p_i or p_i - s in registers
        // (measured faster than offset tables in shared memory, whose reads
        // compete with the gathers for the L1 data pipe)
        const float dx = ((c & 2u) ? qx2 : ((c & 1u) ? pi.x : qx0)) - pj.x;
        const float dy = ((c & 8u) ? qy2 : ((c & 4u) ? pi.y : qy0)) - pj.y;
        const float dz = ((c & 32u) ? qz2 : ((c & 16u) ? pi.z : qz0)) - pj.z;
        const float rsq = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float sr2 = rcp_approx(rsq);
        const float t = sr2 * sr2 * sr2 * lj.sigma6f;
        float f = sr2 * t * fmaf(lj.c48ef, t, -lj.c24ef);
        const bool in = rsq < lj.rc2f;
        f = in ? f : 0.f;
        px = fmaf(f, dx, px);
        py = fmaf(f, dy, py);
        pz = fmaf(f, dz, pz);
        if (ENERGY) {
            pv += in ? lj.c4ef * t * (t - 1.f) : 0.f;
            pw = fmaf(f, rsq, pw);
        }
    };

    auto chunk = [&](const int4 &e) {
        float px = 0.f, py = 0.f, pz = 0.f, pv = 0.f, pw = 0.f;
        pair((uint32_t)e.x, px, py, pz, pv, pw);
        pair((uint32_t)e.y, px, py, pz, pv, pw);
        pair((uint32_t)e.z, px, py, pz, pv, pw);
        pair((uint32_t)e.w, px, py, pz, pv, pw);
        kahan_add(sx, cx, px);
        kahan_add(sy, cy, py);
        kahan_add(sz, cz, pz);
        if (ENERGY) {
            kahan_add(pe, cpe, pv);
            kahan_add(w, cw, pw);
        }
    };
    // the next list chunk is loaded one round ahead (deeper prefetch and
    // two chunks per round measured slower: more registers, less occupancy)
    int q = sub;
    int4 nxt = q < nq ? ld_stream(nb4 + (int64_t)q * n + i) : make_int4(0, 0, 0, 0);
    for (; q < nq; q += TPA) {
        const int4 e = nxt;
        if (q + TPA < nq) nxt = ld_stream(nb4 + (int64_t)(q + TPA) * n + i);
        chunk(e);
    }
    float fx = sx - cx, fy = sy - cy, fz = sz - cz;
    if (ENERGY) {
        pe -= cpe;
        w -= cw;
    }
    if (TPA > 1) {
#pragma unroll
        for (int o = TPA / 2; o > 0; o >>= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            fy += __shfl_xor_sync(0xffffffffu, fy, o);
            fz += __shfl_xor_sync(0xffffffffu, fz, o);
            if (ENERGY) {
                pe += __shfl_xor_sync(0xffffffffu, pe, o);
                w += __shfl_xor_sync(0xffffffffu, w, o);
            }
        }
        if (sub != 0 || !valid) return;
    }
    if (ENERGY) {
        d.pe_atom[i] = 0.5f * pe;
        d.w_atom[i] = 0.5f * w;
    }
    epilogue<EPI, ENERGY>(d, lj, R, i, (double)fx, (double)fy, (double)fz,
                          __float_as_uint(pi.w), true);
}

// ---------------------------------------------------------------------------
// Mixed precision, list shared by a group of G atoms of one cell.  The G
// lanes of a group split the group's row (lane l takes the int4 chunks l,
// l + G, ... of each 16-entry block); each lane gathers its entries'
// positions once and evaluates each of them against the members, whose
// positions it holds in registers, so a gathered position serves up to G
// pairs and nothing is exchanged between lanes inside the loop.  Each entry
// carries a byte of member bits from the build (bit k: the entry is in member
// k's exact Verlet row), so every member sums exactly the pairs of its own
// row, as with per-atom lists.  The entry's cell offset (shared by the
// members: one cell) is applied to the neighbour,
//     d_k = p_k - (p_j + o s),
// from a 64-entry table of o s per replica.  Each lane keeps a Kahan sum per
// member over its chunks (four pairs per chunk and member in a plain
// partial); the G lanes' sums are combined by a fixed butterfly (every lane
// ends with the same totals), and lane k runs the epilogue of member k.
// Pairs inside the group: lane l takes member l against the members its
// pair mask names.
// ---------------------------------------------------------------------------
template <int G, bool BATCHED, int EPI, bool ENERGY>
__global__ void __launch_bounds__(256) k_force_mixed_group(Dev d, LJ lj)
{
    if (stopped(d.status)) return;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gi = t / G;
    const int l = (int)(t % G);
    const int lane = threadIdx.x & 31;
    const unsigned gmask = ((1u << G) - 1u) << (lane & ~(G - 1));
    if (gi >= d.gcell_start[d.ncells]) return;             // whole groups leave together
    if (!MD_CHECK(d, gi < d.ngmax)) return;
    const uint32_t gw = (uint32_t)d.grp[gi];
    const int64_t a0 = gw & kJMask;
    const int m = (int)(gw >> kJBits) + 1;
    if (!MD_CHECK(d, a0 + m <= d.n)) return;
    const int32_t rep = BATCHED ? d.rep_of[a0] : 0;
    const Rep &R = d.reps[rep];
    const float4 *offt = d.offtab + 64 * rep;
    const float4 *p32 = d.p32;
    float qx[G], qy[G], qz[G];
    uint32_t pack = 0;
#pragma unroll
    for (int k = 0; k < G; k++) {
        // absent members sit far away (and away from the sentinel slot)
        const float4 q = k < m ? p32[a0 + k] : make_float4(-1.0e4f, -1.0e4f, -1.0e4f, 0.f);
        qx[k] = q.x; qy[k] = q.y; qz[k] = q.z;
        if (k == 0) pack = __float_as_uint(q.w);
    }
    float sx[G], sy[G], sz[G], cx[G], cy[G], cz[G], pe[G], w[G], cpe[G], cw[G];
#pragma unroll
    for (int k = 0; k < G; k++) {
        sx[k] = sy[k] = sz[k] = cx[k] = cy[k] = cz[k] = 0.f;
        pe[k] = w[k] = cpe[k] = cw[k] = 0.f;
    }
    // one pair: member position (x, y, z) against the neighbour image
    // (jx, jy, jz); adds f d to (fx, fy, fz) and, with ENERGY, V and f r^2
    auto pair = [&](float x, float y, float z, float jx, float jy, float jz, bool live, float &fx,
                    float &fy, float &fz, float &pv, float &pw) {
        const float dx = x - jx, dy = y - jy, dz = z - jz;
        const float rsq = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const float sr2 = rcp_approx(rsq);
        const float tt = sr2 * sr2 * sr2 * lj.sigma6f;
        float f = sr2 * tt * fmaf(lj.c48ef, tt, -lj.c24ef);
        const bool in = live & (rsq < lj.rc2f);
        f = in ? f : 0.f;
        fx = fmaf(f, dx, fx);
        fy = fmaf(f, dy, fy);
        fz = fmaf(f, dz, fz);
        if (ENERGY) {
            pv += in ? lj.c4ef * tt * (tt - 1.f) : 0.f;
            pw = fmaf(f, rsq, pw);
        }
    };
    auto add_partials = [&](const float (&px)[G], const float (&py)[G], const float (&pz)[G],
                            const float (&pv)[G], const float (&pw)[G]) {
#pragma unroll
        for (int k = 0; k < G; k++) {
            kahan_add(sx[k], cx[k], px[k]);
            kahan_add(sy[k], cy[k], py[k]);
            kahan_add(sz[k], cz[k], pz[k]);
            if (ENERGY) {
                kahan_add(pe[k], cpe[k], pv[k]);
                kahan_add(w[k], cw[k], pw[k]);
            }
        }
    };
    {   // pairs inside the group: member l against the members paired with it
        float px[G], py[G], pz[G], pv[G], pw[G];
#pragma unroll
        for (int k = 0; k < G; k++) px[k] = py[k] = pz[k] = pv[k] = pw[k] = 0.f;
        float jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
        for (int k = 0; k < G; k++)
            if (k == l) { jx = qx[k]; jy = qy[k]; jz = qz[k]; }
        const uint32_t pairs = (uint32_t)d.gpair[gi] >> (l * G);
#pragma unroll
        for (int k = 0; k < G; k++) {
            // k == l would be the self pair (d = 0): moved out of range (its
            // pair bit is never set)
            const float ox = k == l ? 1.0e4f : 0.f;
            pair(qx[k] + ox, qy[k], qz[k], jx, jy, jz, (pairs >> k) & 1u, px[k], py[k], pz[k], pv[k], pw[k]);
        }
        add_partials(px, py, pz, pv, pw);
    }
    const int cnt = MD_CHECK(d, d.gnb_count[gi] <= d.gcap) ? d.gnb_count[gi] : 0;
    // the lane's int4 chunks: l, l + G, ... of every 16-entry block (4 chunks
    // per block: one per lane for G = 4, two for G = 2)
    constexpr int kPer = 4 / G;
    const int nq = ((cnt + 15) >> 4) * kPer;
    // chunk c of the rows as int4 index c; its four member-bit bytes as the
    // uint32 of the same index
    const int64_t c0 = gi * 4 + l;
    const int64_t bstride = d.ngmax * 4;                   // chunks between 16-entry blocks
    const int4 *nb4 = reinterpret_cast<const int4 *>(d.gnb);
    const uint32_t *mb4 = reinterpret_cast<const uint32_t *>(d.gmask);
    auto chunk_at = [&](int q) { return c0 + (int64_t)(q / kPer) * bstride + (q % kPer) * G; };
    int4 nxt = nq > 0 ? ld_stream(nb4 + chunk_at(0)) : make_int4(0, 0, 0, 0);
    uint32_t mnxt = nq > 0 ? __ldcs(mb4 + chunk_at(0)) : 0u;
    for (int q = 0; q < nq; q++) {
        const int4 e4 = nxt;
        const uint32_t mw = mnxt;
        if (q + 1 < nq) {
            nxt = ld_stream(nb4 + chunk_at(q + 1));
            mnxt = __ldcs(mb4 + chunk_at(q + 1));
        }
        const uint32_t es[4] = {(uint32_t)e4.x, (uint32_t)e4.y, (uint32_t)e4.z, (uint32_t)e4.w};
        float4 pj[4], of[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const uint32_t j = es[u] & kJMask;
            if (!MD_CHECK(d, j <= (uint32_t)d.n)) { pj[u] = make_float4(1.0e4f, 1.0e4f, 1.0e4f, 0.f); of[u] = make_float4(0.f, 0.f, 0.f, 0.f); continue; }
            pj[u] = __ldg(p32 + j);
            of[u] = __ldg(offt + (es[u] >> kJBits));
        }
        float px[G], py[G], pz[G], pv[G], pw[G];
#pragma unroll
        for (int k = 0; k < G; k++) px[k] = py[k] = pz[k] = pv[k] = pw[k] = 0.f;
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const float jx = pj[u].x + of[u].x, jy = pj[u].y + of[u].y, jz = pj[u].z + of[u].z;
#pragma unroll
            for (int k = 0; k < G; k++)
                pair(qx[k], qy[k], qz[k], jx, jy, jz, (mw >> (8 * u + k)) & 1u, px[k], py[k], pz[k],
                     pv[k], pw[k]);
        }
        add_partials(px, py, pz, pv, pw);
    }
    // combine the lanes' sums (fixed butterfly: every lane gets the same bits)
    float fx[G], fy[G], fz[G], ev[G], ew[G];
#pragma unroll
    for (int k = 0; k < G; k++) {
        fx[k] = sx[k] - cx[k];
        fy[k] = sy[k] - cy[k];
        fz[k] = sz[k] - cz[k];
        ev[k] = pe[k] - cpe[k];
        ew[k] = w[k] - cw[k];
    }
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
#pragma unroll
        for (int k = 0; k < G; k++) {
            fx[k] += __shfl_xor_sync(gmask, fx[k], o);
            fy[k] += __shfl_xor_sync(gmask, fy[k], o);
            fz[k] += __shfl_xor_sync(gmask, fz[k], o);
            if (ENERGY) {
                ev[k] += __shfl_xor_sync(gmask, ev[k], o);
                ew[k] += __shfl_xor_sync(gmask, ew[k], o);
            }
        }
    }
    if (l >= m) return;
    float gx = 0.f, gy = 0.f, gz = 0.f, gv = 0.f, gww = 0.f;
#pragma unroll
    for (int k = 0; k < G; k++)
        if (k == l) { gx = fx[k]; gy = fy[k]; gz = fz[k]; gv = ev[k]; gww = ew[k]; }
    const int64_t i = a0 + l;
    if (ENERGY) {
        d.pe_atom[i] = 0.5f * gv;
        d.w_atom[i] = 0.5f * gww;
    }
    epilogue<EPI, ENERGY>(d, lj, R, i, (double)gx, (double)gy, (double)gz, pack, true);
}

// o + 1 -> o, a 3-entry table per block for the half-list kernel.
__device__ __forceinline__ void fill_offsets(float (&ot)[3])
{
    if (threadIdx.x < 3) ot[threadIdx.x] = (float)((int)threadIdx.x - 1);
    __syncthreads();
}

template <int TPA, bool BATCHED, int EPI, bool ENERGY>
__global__ void __launch_bounds__(256) k_force_mixed_full(Dev d, LJ lj)
{
    if (stopped(d.status)) return;
    mixed_full_tile<TPA, BATCHED, EPI, ENERGY>(d, lj, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// Mixed precision, half list: i-side Kahan sum in registers, j-side through
// vector FP32 atomics (red.global.add.v4.f32); f32 must be zero on entry.
// ---------------------------------------------------------------------------
template <bool BATCHED, bool ENERGY>
__global__ void __launch_bounds__(256) k_force_mixed_half(Dev d, LJ lj)
{
    __shared__ float ot[3];
    fill_offsets(ot);
    if (stopped(d.status)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const int64_t n = d.n;
    const Rep &R = d.reps[BATCHED ? d.rep_of[i] : 0];
    const float nsx = R.nsf[0], nsy = R.nsf[1], nsz = R.nsf[2];
    const float4 pi = d.p32[i];
    const int cnt = MD_CHECK(d, d.nb_count[i] <= d.cap) ? d.nb_count[i] : 0;
    const int nq = (cnt + 3) >> 2;
    const int4 *nb4 = reinterpret_cast<const int4 *>(d.nb);
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    float pe = 0.f, w = 0.f, cpe = 0.f, cw = 0.f;

    auto pair = [&](int32_t e) {
        const uint32_t c = (uint32_t)e >> kJBits;
        const int32_t j = (int32_t)((uint32_t)e & kJMask);
        if (j == n) return;                                 // padding
        if (!MD_CHECK(d, j < n)) return;
        const float4 pj = __ldg(&d.p32[j]);
        const float dx = fmaf(ot[c & 3u], nsx, pi.x - pj.x);
        const float dy = fmaf(ot[(c >> 2) & 3u], nsy, pi.y - pj.y);
        const float dz = fmaf(ot[c >> 4], nsz, pi.z - pj.z);
        const float rsq = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        if (!(rsq < lj.rc2f)) return;
        const float sr2 = rcp_approx(rsq);
        const float sr6 = sr2 * sr2 * sr2 * lj.sigma6f;
        const float f = sr2 * sr6 * fmaf(lj.c48ef, sr6, -lj.c24ef);
        const float tx = f * dx, ty = f * dy, tz = f * dz;
        kahan_add(sx, cx, tx);
        kahan_add(sy, cy, ty);
        kahan_add(sz, cz, tz);
        atomicAdd(&d.f32[j], make_float4(-tx, -ty, -tz, 0.f));
        if (ENERGY) {
            kahan_add(pe, cpe, lj.c4ef * sr6 * (sr6 - 1.f));
            kahan_add(w, cw, f * rsq);
        }
    };
    for (int q = 0; q < nq; q++) {
        const int4 e = ld_stream(nb4 + (int64_t)q * n + i);
        pair(e.x);
        pair(e.y);
        pair(e.z);
        pair(e.w);
    }
    atomicAdd(&d.f32[i], make_float4(sx - cx, sy - cy, sz - cz, 0.f));
    if (ENERGY) {
        d.pe_atom[i] = pe - cpe;
        d.w_atom[i] = w - cw;
    }
}

// ---------------------------------------------------------------------------
// FP64, full list.  The image shift of a neighbour is added to (x_i - x_j)
// exactly as the minimum-image branch would; atoms in interior cells never
// need one, so the per-pair shift is only applied in warps that have an atom
// on a box face.
// ---------------------------------------------------------------------------
struct Shift {
    double lo[3], hi[3];  // added for o = -1 / o = +1 (0 unless on a face)
};

template <bool EDGE>
__device__ __forceinline__ void f64_pair(const Dev &d, const LJ &lj, const dvec4 &xi,
                                         const Shift &sh, int32_t e, double &fx, double &fy,
                                         double &fz, double &pe, double &w, bool energy)
{
    const uint32_t c = (uint32_t)e >> kJBits;
    const int32_t j = (int32_t)((uint32_t)e & kJMask);
    if (!MD_CHECK(d, j <= d.n)) return;
    const dvec4 xj = ldg_dvec4(&d.x[j]);
    double dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
    if (EDGE) {
        const int ox = (int)(c & 3u) - 1, oy = (int)((c >> 2) & 3u) - 1, oz = (int)(c >> 4) - 1;
        if (ox) dx = dx + (ox < 0 ? sh.lo[0] : sh.hi[0]);
        if (oy) dy = dy + (oy < 0 ? sh.lo[1] : sh.hi[1]);
        if (oz) dz = dz + (oz < 0 ? sh.lo[2] : sh.hi[2]);
    }
    const double rsq = fma(dz, dz, fma(dy, dy, dx * dx));
    // rsq < rc^2 on the bit patterns (an integer compare instead of an FP64
    // one); padding points at the far-away sentinel
    const bool in = lt_nonneg(rsq, lj.rc2);
    const double sr2 = rcp_nr(rsq);
    const double t = sr2 * sr2 * sr2 * lj.sigma6;
    double f = sr2 * t * fma(lj.c48e, t, -lj.c24e);
    f = in ? f : 0.0;
    fx = fma(f, dx, fx);
    fy = fma(f, dy, fy);
    fz = fma(f, dz, fz);
    if (energy) {
        pe += in ? lj.c4e * t * (t - 1.0) : 0.0;
        w = fma(f, rsq, w);
    }
}

__device__ __forceinline__ Shift make_shift(const Rep &R, uint32_t pack, bool &edge)
{
    const int c[3] = {(int)(pack & 1023u), (int)((pack >> 10) & 1023u), (int)((pack >> 20) & 1023u)};
    Shift sh;
    edge = false;
#pragma unroll
    for (int q = 0; q < 3; q++) {
        sh.lo[q] = c[q] == 0 ? R.L[q] : 0.0;            // image of cell -1 sits at x - L
        sh.hi[q] = c[q] == R.nc[q] - 1 ? -R.L[q] : 0.0;  // image of cell nc sits at x + L
        edge |= (c[q] == 0) || (c[q] == R.nc[q] - 1);
    }
    return sh;
}

template <int TPA, bool BATCHED, int EPI, bool ENERGY>
__global__ void __launch_bounds__(256) k_force_f64_full(Dev d, LJ lj)
{
    if (stopped(d.status)) return;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i0 = gt / TPA;
    const int sub = (int)(gt % TPA);
    const bool valid = i0 < d.n;
    if (TPA == 1 && !valid) return;
    const int64_t i = valid ? i0 : d.n - 1;
    const int64_t n = d.n;
    const Rep &R = d.reps[BATCHED ? d.rep_of[i] : 0];
    const dvec4 xi = d.x[i];
    const uint32_t pack = __float_as_uint(d.p32[i].w);
    bool edge;
    const Shift sh = make_shift(R, pack, edge);
    const int cnt = valid && MD_CHECK(d, d.nb_count[i] <= d.cap) ? d.nb_count[i] : 0;
    const int nq = (cnt + 3) >> 2;
    const int4 *nb4 = reinterpret_cast<const int4 *>(d.nb);
    double fx = 0, fy = 0, fz = 0, pe = 0, w = 0;
    const bool any_edge = __any_sync(__activemask(), edge);
    for (int q = sub; q < nq; q += TPA) {
        const int4 e = ld_stream(nb4 + (int64_t)q * n + i);
        if (any_edge) {
            f64_pair<true>(d, lj, xi, sh, e.x, fx, fy, fz, pe, w, ENERGY);
            f64_pair<true>(d, lj, xi, sh, e.y, fx, fy, fz, pe, w, ENERGY);
            f64_pair<true>(d, lj, xi, sh, e.z, fx, fy, fz, pe, w, ENERGY);
            f64_pair<true>(d, lj, xi, sh, e.w, fx, fy, fz, pe, w, ENERGY);
        } else {
            f64_pair<false>(d, lj, xi, sh, e.x, fx, fy, fz, pe, w, ENERGY);
            f64_pair<false>(d, lj, xi, sh, e.y, fx, fy, fz, pe, w, ENERGY);
            f64_pair<false>(d, lj, xi, sh, e.z, fx, fy, fz, pe, w, ENERGY);
            f64_pair<false>(d, lj, xi, sh, e.w, fx, fy, fz, pe, w, ENERGY);
        }
    }
    if (TPA > 1) {
#pragma unroll
        for (int o = TPA / 2; o > 0; o >>= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            fy += __shfl_xor_sync(0xffffffffu, fy, o);
            fz += __shfl_xor_sync(0xffffffffu, fz, o);
            if (ENERGY) {
                pe += __shfl_xor_sync(0xffffffffu, pe, o);
                w += __shfl_xor_sync(0xffffffffu, w, o);
            }
        }
        if (sub != 0 || !valid) return;
    }
    if (ENERGY) {
        d.pe_atom64[i] = 0.5 * pe;
        d.w_atom64[i] = 0.5 * w;
    }
    epilogue<EPI, ENERGY>(d, lj, R, i, fx, fy, fz, pack, false);
}

// FP64, half list: j-side through FP64 atomics; f64 must be zero on entry.
template <bool BATCHED, bool ENERGY>
__global__ void __launch_bounds__(256) k_force_f64_half(Dev d, LJ lj)
{
    if (stopped(d.status)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const int64_t n = d.n;
    const Rep &R = d.reps[BATCHED ? d.rep_of[i] : 0];
    const dvec4 xi = d.x[i];
    const uint32_t pack = __float_as_uint(d.p32[i].w);
    bool edge;
    const Shift sh = make_shift(R, pack, edge);
    const int cnt = MD_CHECK(d, d.nb_count[i] <= d.cap) ? d.nb_count[i] : 0;
    const int nq = (cnt + 3) >> 2;
    const int4 *nb4 = reinterpret_cast<const int4 *>(d.nb);
    double fx = 0, fy = 0, fz = 0, pe = 0, w = 0;
    for (int q = 0; q < nq; q++) {
        const int4 e4 = ld_stream(nb4 + (int64_t)q * n + i);
        const int32_t es[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
        for (int t = 0; t < 4; t++) {
            double gx = 0, gy = 0, gz = 0, pp = 0, ww = 0;
            f64_pair<true>(d, lj, xi, sh, es[t], gx, gy, gz, pp, ww, ENERGY);
            if (gx != 0.0 || gy != 0.0 || gz != 0.0) {
                const int32_t j = (int32_t)((uint32_t)es[t] & kJMask);
                atomicAdd(&d.f64[j].x, -gx);
                atomicAdd(&d.f64[j].y, -gy);
                atomicAdd(&d.f64[j].z, -gz);
            }
            fx += gx; fy += gy; fz += gz; pe += pp; w += ww;
        }
    }
    atomicAdd(&d.f64[i].x, fx);
    atomicAdd(&d.f64[i].y, fy);
    atomicAdd(&d.f64[i].z, fz);
    if (ENERGY) {
        d.pe_atom64[i] = pe;
        d.w_atom64[i] = w;
    }
}

template <int TPA, bool B>
int launch_full(const Dev &d, const LJ &lj, bool mixed, int epi, bool energy, cudaStream_t st)
{
    const int64_t threads = d.n * TPA;
    const unsigned g = (unsigned)((threads + 255) / 256);
#define MD_FULL(EP, EN)                                                                    \
    do {                                                                                   \
        if (mixed) k_force_mixed_full<TPA, B, EP, EN><<<g, 256, 0, st>>>(d, lj);           \
        else k_force_f64_full<TPA, B, EP, EN><<<g, 256, 0, st>>>(d, lj);                   \
    } while (0)
    if (epi == EPI_F) { if (energy) MD_FULL(EPI_F, true); else MD_FULL(EPI_F, false); }
    else if (epi == EPI_FK) { if (energy) MD_FULL(EPI_FK, true); else MD_FULL(EPI_FK, false); }
    else { if (energy) MD_FULL(EPI_FKKD, true); else MD_FULL(EPI_FKKD, false); }
#undef MD_FULL
    return 0;
}

template <int G, bool B>
void launch_group_g(const Dev &d, const LJ &lj, int epi, bool energy, cudaStream_t st)
{
    const unsigned g = (unsigned)((d.ngmax * G + 255) / 256);
#define MD_GRP(EP, EN) k_force_mixed_group<G, B, EP, EN><<<g, 256, 0, st>>>(d, lj)
    if (epi == EPI_F) { if (energy) MD_GRP(EPI_F, true); else MD_GRP(EPI_F, false); }
    else if (epi == EPI_FK) { if (energy) MD_GRP(EPI_FK, true); else MD_GRP(EPI_FK, false); }
    else { if (energy) MD_GRP(EPI_FKKD, true); else MD_GRP(EPI_FKKD, false); }
#undef MD_GRP
}

}  // namespace

// Mixed path over a list shared by groups of G = 2 or 4 atoms; epilogues as
// the full-list kernels.
int launch_force_group(const Dev &d, const LJ &lj, int G, int epi, bool energy, bool batched,
                       cudaStream_t st, int *nl)
{
    if (d.n <= 0) return 0;
    if ((G != 2 && G != 4) || !d.gnb || !d.grp || !d.offtab || !d.gmask || !d.gpair) return -1;
    if (G == 4) {
        if (batched) launch_group_g<4, true>(d, lj, epi, energy, st);
        else launch_group_g<4, false>(d, lj, epi, energy, st);
    } else {
        if (batched) launch_group_g<2, true>(d, lj, epi, energy, st);
        else launch_group_g<2, false>(d, lj, epi, energy, st);
    }
    *nl += 1;
    return (int)cudaGetLastError();
}

// Half lists only support EPI_F (the caller zeroes the force array first and
// integrates in a separate kernel).
int launch_force(const Dev &d, const LJ &lj, int precision, bool half, int tpa, int epi,
                 bool energy, bool batched, cudaStream_t st, int *nl)
{
    if (d.n <= 0) return 0;
    const bool mixed = precision == 1;
    if (half) {
        if (epi != EPI_F) return -1;
        const unsigned g = (unsigned)((d.n + 255) / 256);
#define MD_HALF(B, EN)                                                   \
    do {                                                                 \
        if (mixed) k_force_mixed_half<B, EN><<<g, 256, 0, st>>>(d, lj);  \
        else k_force_f64_half<B, EN><<<g, 256, 0, st>>>(d, lj);          \
    } while (0)
        if (batched) { if (energy) MD_HALF(true, true); else MD_HALF(true, false); }
        else { if (energy) MD_HALF(false, true); else MD_HALF(false, false); }
#undef MD_HALF
    } else if (batched) {
        if (tpa == 8) launch_full<8, true>(d, lj, mixed, epi, energy, st);
        else if (tpa == 4) launch_full<4, true>(d, lj, mixed, epi, energy, st);
        else if (tpa == 2) launch_full<2, true>(d, lj, mixed, epi, energy, st);
        else launch_full<1, true>(d, lj, mixed, epi, energy, st);
    } else {
        if (tpa == 8) launch_full<8, false>(d, lj, mixed, epi, energy, st);
        else if (tpa == 4) launch_full<4, false>(d, lj, mixed, epi, energy, st);
        else if (tpa == 2) launch_full<2, false>(d, lj, mixed, epi, energy, st);
        else launch_full<1, false>(d, lj, mixed, epi, energy, st);
    }
    *nl += 1;
    return (int)cudaGetLastError();
}

}  // namespace mdk
