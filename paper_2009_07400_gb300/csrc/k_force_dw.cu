// LJ 12-6 forces over the Verlet list (tinyMD Sec. 3.2, Eq. 2) in
// double-word arithmetic: every quantity of the pair kernel is an unevaluated
// sum h + l of two FP32 numbers, which carries about 48 significant bits, so
// the forces agree with an FP64 evaluation to ~1e-13 while every operation
// runs on the FP32 pipe.  GB300's FP64 pipe is about 1/64 of its FP32 rate
// and bounds the FP64 path (17 FP64 operations per pair); the double-word
// pair takes about 160 FP32-pipe instructions instead (ncu: 418 M warp
// instructions for 78.6 M listed pairs before the constant folding below).
// Precision MD_DW.
//
// Building blocks (dw_arith.cuh, with their CPU check of exactness and
// error bounds in the tests): TwoSum, Fast2Sum, the FMA exact product, the
// double-word product and sum, and the Newton-refined reciprocal and
// reciprocal square root.
// Intermediate results are not renormalised (their low parts stay within a
// few ulps of the high parts, which the multiplication tolerates); the
// per-atom sums are renormalised once per list chunk.  The cut-off test
// takes the sign of (r2_h - rc2_h) + (r2_l - rc2_l): the first difference is
// exact near rc^2 (Sterbenz), so the sign is that of r^2 - rc^2 unless they
// differ by less than ~2^-47 rc^2.  All arithmetic uses the _rn intrinsics
// so that nothing is contracted or reassociated.  (Renormalising r^2 first
// measured 13 % slower together with the unfolded constants below: 73
// instead of 64 registers.)
//
// Positions: p32 holds the high parts of the cell-relative positions, on a
// grid of step g = 2^k with 2^24 g >= 2.5 cell sides, plo the low parts
// (dw_split).  The displacement of a listed pair,
//     d = (p_i - o s) - p_j,
// then has an exact FP32 high part (p_ih -+ s_h - p_jh: multiples of g below
// 2^24 g) and a low part (p_il -+ s_l) - p_jl rounded once, so the
// cancellation of nearby positions loses nothing; d is good to ~2^-45.
//
// Reciprocal: 1/r^2 from the hardware approximation of 1/fl(r2_h + r2_l)
// refined by one FP32 Newton step (within ~1 ulp), then one Newton step in
// double word, y (1 + e) with e = 1 - r^2 y: relative error ~2^-46.
//
// Pair arithmetic as executed, with sigma and epsilon folded into double-word
// constants (A12 = 48 eps sigma^12, A6 = 24 eps sigma^6, B12 = 4 eps
// sigma^12, B6 = 4 eps sigma^6): sr6 = sr2^3,
//     f = sr2 sr6 (A12 sr6 - A6),   V = sr6 (B12 sr6 - B6),
// the paper's f = 48 eps sr6' (sr6' - 1/2) sr2 and 4 eps sr6' (sr6' - 1)
// with sr6' = sigma^6 sr6, regrouped.
//
// Epilogue: the FP64 velocity-Verlet update of the mixed path (x and v
// updated in place), with the force F = (double)h + (double)l; the next
// positions' split goes to the other p32 / plo buffers.
//
// The file also holds the double-word adjoint pair terms (md_adjoint on an
// MD_DW context) and the double-word spring-dashpot contact step (Eq. 3),
// which share these building blocks.
#include "md_internal.cuh"
#include "dw_arith.cuh"

namespace mdk {

namespace {

__device__ __forceinline__ bool stopped(const DevStatus *st)
{
    return *((volatile const int32_t *)&st->flags) != 0;
}

using namespace dwa;

__device__ __forceinline__ float rcp_approx(float a)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

__device__ __forceinline__ double to_f64(dw a)
{
    return f64_of_f32(a.h) + f64_of_f32(a.l);
}

__device__ __forceinline__ dw dw_const(const float c[2])
{
    return {c[0], c[1]};
}

// FP64 epilogue (velocity Verlet, Sec. 3.2 Eq. 1, as the mixed path: x and v
// in place with streaming accesses), the next split positions into
// p32_nxt / plo_nxt.
template <int EPI, bool ENERGY>
__device__ __forceinline__ void dw_epilogue(const Dev &d, const LJ &lj, const Rep &R, int64_t i,
                                            double fx, double fy, double fz, uint32_t pack)
{
    if (EPI == EPI_F || EPI == EPI_FK) d.f64[i] = mk_dvec4(fx, fy, fz, 0.0);
    if (EPI == EPI_F) return;
    dvec4 v = ld_cs_dvec4(d.v + i);
    v.x = fma(lj.half_dt_m, fx, v.x);
    v.y = fma(lj.half_dt_m, fy, v.y);
    v.z = fma(lj.half_dt_m, fz, v.z);
    if (ENERGY) d.ke_atom64[i] = 0.5 * lj.mass * fma(v.x, v.x, fma(v.y, v.y, v.z * v.z));
    if (EPI == EPI_FKKD) {
        v.x = fma(lj.half_dt_m, fx, v.x);
        v.y = fma(lj.half_dt_m, fy, v.y);
        v.z = fma(lj.half_dt_m, fz, v.z);
        dvec4 x = ld_cs_dvec4(d.x + i);
        x.x = fma(lj.dt, v.x, x.x);
        x.y = fma(lj.dt, v.y, x.y);
        x.z = fma(lj.dt, v.z, x.z);
        st_cs_dvec4(d.x + i, x);
        const double *ct = d.ctr + R.ctr_off;
        const double cx = __ldg(ct + (pack & 1023u));
        const double cy = __ldg(ct + R.nc[0] + ((pack >> 10) & 1023u));
        const double cz = __ldg(ct + R.nc[0] + R.nc[1] + ((pack >> 20) & 1023u));
        store_cell_pos(d, R, d.p32_nxt, d.plo_nxt, i, x.x - cx, x.y - cy, x.z - cz, pack);
        if (d.p32_ref) check_displacement(d, i, d.p32_nxt[i]);
    }
    st_cs_dvec4(d.v + i, v);
}

// One atom (TPA lanes) over its full list.
template <int TPA, bool BATCHED, int EPI, bool ENERGY>
__global__ void __launch_bounds__(256) k_force_dw_full(Dev d, LJ lj)
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
    const float4 hi = d.p32[i], li = d.plo[i];
    const int cnt = valid && MD_CHECK(d, d.nb_count[i] <= d.cap) ? d.nb_count[i] : 0;
    const int nq = (cnt + 3) >> 2;
    const int4 *nb4 = reinterpret_cast<const int4 *>(d.nb);
    const float4 *p32 = d.p32, *plo = d.plo;

    // p_i - o s for o = -1 (field 0) and o = +1 (field 2): high parts exact
    const float qhx0 = __fadd_rn(hi.x, R.dw_sh[0]), qhx2 = __fsub_rn(hi.x, R.dw_sh[0]);
    const float qhy0 = __fadd_rn(hi.y, R.dw_sh[1]), qhy2 = __fsub_rn(hi.y, R.dw_sh[1]);
    const float qhz0 = __fadd_rn(hi.z, R.dw_sh[2]), qhz2 = __fsub_rn(hi.z, R.dw_sh[2]);
    const float qlx0 = __fadd_rn(li.x, R.dw_sl[0]), qlx2 = __fsub_rn(li.x, R.dw_sl[0]);
    const float qly0 = __fadd_rn(li.y, R.dw_sl[1]), qly2 = __fsub_rn(li.y, R.dw_sl[1]);
    const float qlz0 = __fadd_rn(li.z, R.dw_sl[2]), qlz2 = __fsub_rn(li.z, R.dw_sl[2]);
    const dw rc2 = dw_const(lj.dw_rc2);
    const dw a12 = dw_const(lj.dw_a12), a6n = {-lj.dw_a6[0], -lj.dw_a6[1]};

    dw ax = {0.f, 0.f}, ay = {0.f, 0.f}, az = {0.f, 0.f}, ape = {0.f, 0.f}, aw = {0.f, 0.f};

    auto pair = [&](uint32_t e) {
        if (!MD_CHECK(d, (e & kJMask) <= (uint32_t)d.n)) return;
        const uint32_t j = e & kJMask;
        const float4 hj = __ldg(p32 + j);
        const float4 lj4 = __ldg(plo + j);
        const uint32_t c = e >> kJBits;
        const bool x2 = c & 2u, x1 = c & 1u, y2 = c & 8u, y1 = c & 4u, z2 = c & 32u, z1 = c & 16u;
        const float dxh = __fsub_rn(x2 ? qhx2 : (x1 ? hi.x : qhx0), hj.x);
        const float dyh = __fsub_rn(y2 ? qhy2 : (y1 ? hi.y : qhy0), hj.y);
        const float dzh = __fsub_rn(z2 ? qhz2 : (z1 ? hi.z : qhz0), hj.z);
        const float dxl = __fsub_rn(x2 ? qlx2 : (x1 ? li.x : qlx0), lj4.x);
        const float dyl = __fsub_rn(y2 ? qly2 : (y1 ? li.y : qly0), lj4.y);
        const float dzl = __fsub_rn(z2 ? qlz2 : (z1 ? li.z : qlz0), lj4.z);
        dw r2 = dw_add(dw_add(dw_sq_of(dxh, dxl), dw_sq_of(dyh, dyl)), dw_sq_of(dzh, dzl));
        const bool in = __fadd_rn(__fsub_rn(r2.h, rc2.h), __fsub_rn(r2.l, rc2.l)) < 0.f;
        // 1 / r^2
        const float rf = __fadd_rn(r2.h, r2.l);
        const dw sr2 = dw_recip(r2, rf, rcp_approx(rf));
        const dw sr6 = dw_mul(dw_mul(sr2, sr2), sr2);
        dw f = dw_mul(dw_mul(sr2, sr6), dw_add(dw_mul(a12, sr6), a6n));
        f.h = in ? f.h : 0.f;
        f.l = in ? f.l : 0.f;
        ax = dw_add(ax, dw_mul(f, dw{dxh, dxl}));
        ay = dw_add(ay, dw_mul(f, dw{dyh, dyl}));
        az = dw_add(az, dw_mul(f, dw{dzh, dzl}));
        if (ENERGY) {
            dw v = dw_mul(sr6, dw_add(dw_mul(dw_const(lj.dw_b12), sr6), dw{-lj.dw_b6[0], -lj.dw_b6[1]}));
            v.h = in ? v.h : 0.f;
            v.l = in ? v.l : 0.f;
            ape = dw_add(ape, v);
            aw = dw_add(aw, dw_mul(f, r2));
        }
    };

    int q = sub;
    int4 nxt = q < nq ? __ldcs(nb4 + (int64_t)q * n + i) : make_int4(0, 0, 0, 0);
    for (; q < nq; q += TPA) {
        const int4 e = nxt;
        if (q + TPA < nq) nxt = __ldcs(nb4 + (int64_t)(q + TPA) * n + i);
        pair((uint32_t)e.x);
        pair((uint32_t)e.y);
        pair((uint32_t)e.z);
        pair((uint32_t)e.w);
        // keep the low parts of the sums near an ulp of the high parts
        ax = fast_two_sum(ax.h, ax.l);
        ay = fast_two_sum(ay.h, ay.l);
        az = fast_two_sum(az.h, az.l);
        if (ENERGY) {
            ape = fast_two_sum(ape.h, ape.l);
            aw = fast_two_sum(aw.h, aw.l);
        }
    }
    if (TPA > 1) {
        // butterfly: two_sum is symmetric, so every lane ends with the same sums
#pragma unroll
        for (int o = TPA / 2; o > 0; o >>= 1) {
            ax = dw_add(ax, dw{__shfl_xor_sync(0xffffffffu, ax.h, o), __shfl_xor_sync(0xffffffffu, ax.l, o)});
            ay = dw_add(ay, dw{__shfl_xor_sync(0xffffffffu, ay.h, o), __shfl_xor_sync(0xffffffffu, ay.l, o)});
            az = dw_add(az, dw{__shfl_xor_sync(0xffffffffu, az.h, o), __shfl_xor_sync(0xffffffffu, az.l, o)});
            if (ENERGY) {
                ape = dw_add(ape, dw{__shfl_xor_sync(0xffffffffu, ape.h, o),
                                     __shfl_xor_sync(0xffffffffu, ape.l, o)});
                aw = dw_add(aw, dw{__shfl_xor_sync(0xffffffffu, aw.h, o),
                                   __shfl_xor_sync(0xffffffffu, aw.l, o)});
            }
        }
        if (sub != 0 || !valid) return;
    }
    if (ENERGY) {
        d.pe_atom64[i] = 0.5 * to_f64(ape);
        d.w_atom64[i] = 0.5 * to_f64(aw);
    }
    dw_epilogue<EPI, ENERGY>(d, lj, R, i, to_f64(ax), to_f64(ay), to_f64(az), __float_as_uint(hi.w));
}

template <int TPA, bool B>
void launch_dw(const Dev &d, const LJ &lj, int epi, bool energy, cudaStream_t st)
{
    const unsigned g = (unsigned)((d.n * TPA + 255) / 256);
#define MD_DW_K(EP, EN) k_force_dw_full<TPA, B, EP, EN><<<g, 256, 0, st>>>(d, lj)
    if (epi == EPI_F) { if (energy) MD_DW_K(EPI_F, true); else MD_DW_K(EPI_F, false); }
    else if (epi == EPI_FK) { if (energy) MD_DW_K(EPI_FK, true); else MD_DW_K(EPI_FK, false); }
    else { if (energy) MD_DW_K(EPI_FKKD, true); else MD_DW_K(EPI_FKKD, false); }
#undef MD_DW_K
}


// ---------------------------------------------------------------------------
// Adjoint pair terms in double word (md_adjoint on an MD_DW context, pair
// precision MD_DW): the Jacobian-vector product J(x) w and the parameter
// derivatives of k_adjoint.cu's FP64 kernel, term for term, with sigma and
// epsilon folded into double-word constants (s = sigma, sr8 = sr2 sr6,
// sr10 = sr8 sr2):
//   f            = sr8 (A12 sr6 - A6)        A12 = 48 eps s^12, A6 = 24 eps s^6
//   2 f'         = sr10 (D6 - D12 sr6)       D6 = 192 eps s^6, D12 = 672 eps s^12
//   f / eps      = sr8 (E12 sr6 - E6)        E12 = 48 s^12, E6 = 24 s^6
//   df / dsigma  = sr8 (S12 sr6 - S6)        S12 = 576 eps s^11, S6 = 144 eps s^5
//   dV/deps / 2  = sr6 (P12 sr6 - P6)        P12 = 2 s^12, P6 = 2 s^6
//   dV/dsigma / 2 = sr6 (Q12 sr6 - Q6)       Q12 = 24 eps s^11, Q6 = 12 eps s^5
// (f' = df/d(r^2)).  Per pair, with u the adjoint w and du = u_i - u_j:
//   (J u)_i += f du + 2 f' d (d . du),  g_eps += (f / eps)(d . u_i),
//   g_sigma += (df / dsigma)(d . u_i), and inside the loss window F_i and the
//   PE derivatives.  Geometry from the high and low parts of the positions
// (snapshots in p32 / plo), the neighbour's u from double-word copies in slot
// order (wbar_h, wbar_l, written by the axpy kernel); per-atom sums in double
// word, added to the FP64 adjoint state (caller order) once per atom.
struct DwAdjArgs {
    const float4 *wh, *wl;   // u in slot order: high and low parts
    dvec4 *xbar;             // caller order, updated
    double *g_eps, *g_sig;   // caller order, updated
    double k, lw;
};

__device__ __forceinline__ dw dw_axb(dw a, dw x, dw b)   // a x - b
{
    return dw_add(dw_mul(a, x), dw{-b.h, -b.l});
}

template <bool WINDOW, int TPA>
__global__ void __launch_bounds__(128) k_adjoint_pairs_dw(Dev d, LJ lj, DwAdjArgs a)
{
    if (stopped(d.status)) return;
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i0 = gt / TPA;
    const int sub = (int)(gt % TPA);
    const bool valid = i0 < d.n;
    if (TPA == 1 && !valid) return;
    const int64_t i = valid ? i0 : d.n - 1;   // idle lanes still join the shuffles
    const Rep &R = d.reps[0];
    const int32_t idi = d.id[i];
    const float4 hi = d.p32[i], li = d.plo[i];
    const float4 uih = a.wh[i], uil = a.wl[i];
    const dw uix = {uih.x, uil.x}, uiy = {uih.y, uil.y}, uiz = {uih.z, uil.z};
    const int cnt = valid && MD_CHECK(d, d.nb_count[i] <= d.cap) ? d.nb_count[i] : 0;
    const int4 *nb4 = reinterpret_cast<const int4 *>(d.nb);
    const float qhx0 = __fadd_rn(hi.x, R.dw_sh[0]), qhx2 = __fsub_rn(hi.x, R.dw_sh[0]);
    const float qhy0 = __fadd_rn(hi.y, R.dw_sh[1]), qhy2 = __fsub_rn(hi.y, R.dw_sh[1]);
    const float qhz0 = __fadd_rn(hi.z, R.dw_sh[2]), qhz2 = __fsub_rn(hi.z, R.dw_sh[2]);
    const float qlx0 = __fadd_rn(li.x, R.dw_sl[0]), qlx2 = __fsub_rn(li.x, R.dw_sl[0]);
    const float qly0 = __fadd_rn(li.y, R.dw_sl[1]), qly2 = __fsub_rn(li.y, R.dw_sl[1]);
    const float qlz0 = __fadd_rn(li.z, R.dw_sl[2]), qlz2 = __fsub_rn(li.z, R.dw_sl[2]);
    const dw rc2 = dw_const(lj.dw_rc2);
    const dw zero = {0.f, 0.f};
    dw jx = zero, jy = zero, jz = zero, ge = zero, gs = zero;
    dw fx = zero, fy = zero, fz = zero, pe_e = zero, pe_s = zero;
    for (int q = sub; 4 * q < cnt; q += TPA) {
      const int4 e4 = __ldcs(nb4 + (int64_t)q * d.n + i);
      const uint32_t es[4] = {(uint32_t)e4.x, (uint32_t)e4.y, (uint32_t)e4.z, (uint32_t)e4.w};
#pragma unroll
      for (int t4 = 0; t4 < 4; t4++) {
        if (4 * q + t4 >= cnt) break;
        const uint32_t e = es[t4];
        const uint32_t j = e & kJMask;
        if (!MD_CHECK(d, j < (uint32_t)d.n)) continue;
        const float4 hj = __ldg(d.p32 + j), lj4 = __ldg(d.plo + j);
        const uint32_t c = e >> kJBits;
        const bool x2 = c & 2u, x1 = c & 1u, y2 = c & 8u, y1 = c & 4u, z2 = c & 32u, z1 = c & 16u;
        const float dxh = __fsub_rn(x2 ? qhx2 : (x1 ? hi.x : qhx0), hj.x);
        const float dyh = __fsub_rn(y2 ? qhy2 : (y1 ? hi.y : qhy0), hj.y);
        const float dzh = __fsub_rn(z2 ? qhz2 : (z1 ? hi.z : qhz0), hj.z);
        const float dxl = __fsub_rn(x2 ? qlx2 : (x1 ? li.x : qlx0), lj4.x);
        const float dyl = __fsub_rn(y2 ? qly2 : (y1 ? li.y : qly0), lj4.y);
        const float dzl = __fsub_rn(z2 ? qlz2 : (z1 ? li.z : qlz0), lj4.z);
        const dw r2 = dw_add(dw_add(dw_sq_of(dxh, dxl), dw_sq_of(dyh, dyl)), dw_sq_of(dzh, dzl));
        if (!(__fadd_rn(__fsub_rn(r2.h, rc2.h), __fsub_rn(r2.l, rc2.l)) < 0.f)) continue;
        const float rf = __fadd_rn(r2.h, r2.l);
        const dw sr2 = dw_recip(r2, rf, rcp_approx(rf));
        const dw sr6 = dw_mul(dw_mul(sr2, sr2), sr2);
        const dw sr8 = dw_mul(sr2, sr6);
        const dw f = dw_mul(sr8, dw_axb(dw_const(lj.dw_a12), sr6, dw_const(lj.dw_a6)));
        // 2 f' = sr10 (D6 - D12 sr6)
        const dw fp2 = dw_mul(dw_mul(sr8, sr2), dw_add(dw_const(lj.dw_adj[0]),
                                                       dw_mul(dw{-lj.dw_adj[1][0], -lj.dw_adj[1][1]}, sr6)));
        const dw dx = {dxh, dxl}, dy = {dyh, dyl}, dz = {dzh, dzl};
        const float4 ujh = __ldg(a.wh + j), ujl = __ldg(a.wl + j);
        const dw dux = dw_add(uix, dw{-ujh.x, -ujl.x});
        const dw duy = dw_add(uiy, dw{-ujh.y, -ujl.y});
        const dw duz = dw_add(uiz, dw{-ujh.z, -ujl.z});
        const dw g = dw_mul(fp2, dw_add(dw_add(dw_mul(dx, dux), dw_mul(dy, duy)), dw_mul(dz, duz)));
        jx = dw_add(jx, dw_add(dw_mul(f, dux), dw_mul(g, dx)));
        jy = dw_add(jy, dw_add(dw_mul(f, duy), dw_mul(g, dy)));
        jz = dw_add(jz, dw_add(dw_mul(f, duz), dw_mul(g, dz)));
        const dw dui = dw_add(dw_add(dw_mul(dx, uix), dw_mul(dy, uiy)), dw_mul(dz, uiz));
        ge = dw_add(ge, dw_mul(dw_mul(sr8, dw_axb(dw_const(lj.dw_adj[2]), sr6, dw_const(lj.dw_adj[3]))), dui));
        gs = dw_add(gs, dw_mul(dw_mul(sr8, dw_axb(dw_const(lj.dw_adj[4]), sr6, dw_const(lj.dw_adj[5]))), dui));
        if (WINDOW) {   // -F/W and dPE/dtheta: only inside the loss window
            fx = dw_add(fx, dw_mul(f, dx));
            fy = dw_add(fy, dw_mul(f, dy));
            fz = dw_add(fz, dw_mul(f, dz));
            pe_e = dw_add(pe_e, dw_mul(sr6, dw_axb(dw_const(lj.dw_adj[6]), sr6, dw_const(lj.dw_adj[7]))));
            pe_s = dw_add(pe_s, dw_mul(sr6, dw_axb(dw_const(lj.dw_adj[8]), sr6, dw_const(lj.dw_adj[9]))));
        }
      }
      jx = fast_two_sum(jx.h, jx.l);
      jy = fast_two_sum(jy.h, jy.l);
      jz = fast_two_sum(jz.h, jz.l);
      ge = fast_two_sum(ge.h, ge.l);
      gs = fast_two_sum(gs.h, gs.l);
    }
    if (TPA > 1) {
        auto red = [](dw &v, int o) {
            v = dw_add(v, dw{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)});
        };
#pragma unroll
        for (int o = TPA / 2; o > 0; o >>= 1) {
            red(jx, o); red(jy, o); red(jz, o); red(ge, o); red(gs, o);
            if (WINDOW) { red(fx, o); red(fy, o); red(fz, o); red(pe_e, o); red(pe_s, o); }
        }
        if (sub != 0 || !valid) return;
    }
    dvec4 xb = a.xbar[idi];
    xb.x += a.k * to_f64(jx) - a.lw * to_f64(fx);
    xb.y += a.k * to_f64(jy) - a.lw * to_f64(fy);
    xb.z += a.k * to_f64(jz) - a.lw * to_f64(fz);
    a.xbar[idi] = xb;
    a.g_eps[idi] += a.k * to_f64(ge) + a.lw * to_f64(pe_e);
    a.g_sig[idi] += a.k * to_f64(gs) + a.lw * to_f64(pe_s);
}


// ---------------------------------------------------------------------------
// Spring-dashpot contact forces (Sec. 3.2, Eq. 3) in double word: the mixed
// contact kernel's mapping (one thread per sphere over its full row, the
// velocity-Verlet update fused into the epilogue) with every pair quantity a
// double word.  Spheres touch when r^2 < sigma^2 (strict; the sign test of
// the LJ kernel); then
//     F_i += x_ij [K (sigma - r) - gamma (x_ij . v_ij) / r] / r.
// 1/r: the hardware reciprocal square root of fl(r2_h + r2_l), one FP32
// Newton step y (3 - a y^2) / 2, then one double-word step y (1 + e / 2) with
// e = 1 - r^2 y^2 (y^2 exact by two_prod): relative error ~2^-47; r = r^2 / r.
// sigma - r cancels for touching spheres; its high parts are subtracted
// exactly (two_sum).  The neighbours' velocities come from double-word
// copies (v32: high parts, vlo: low parts) that the binning, the velocity
// copy kernel and this epilogue keep, like the positions.
__device__ __forceinline__ float rsqrt_approx(float a)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

template <int EPI, bool ENERGY>
__device__ __forceinline__ void dw_sd_epilogue(const Dev &d, const LJ &lj, const Rep &R, int64_t i,
                                               double fx, double fy, double fz, uint32_t pack)
{
    if (EPI == EPI_F || EPI == EPI_FK) d.f64[i] = mk_dvec4(fx, fy, fz, 0.0);
    if (EPI == EPI_F) return;
    dvec4 v = ld_cs_dvec4(d.v + i);
    v.x = fma(lj.half_dt_m, fx, v.x);
    v.y = fma(lj.half_dt_m, fy, v.y);
    v.z = fma(lj.half_dt_m, fz, v.z);
    if (ENERGY) d.ke_atom64[i] = 0.5 * lj.mass * fma(v.x, v.x, fma(v.y, v.y, v.z * v.z));
    if (EPI == EPI_FKKD) {
        v.x = fma(lj.half_dt_m, fx, v.x);
        v.y = fma(lj.half_dt_m, fy, v.y);
        v.z = fma(lj.half_dt_m, fz, v.z);
        dvec4 x = ld_cs_dvec4(d.x + i);
        x.x = fma(lj.dt, v.x, x.x);
        x.y = fma(lj.dt, v.y, x.y);
        x.z = fma(lj.dt, v.z, x.z);
        st_cs_dvec4(d.x + i, x);
        const double *ct = d.ctr + R.ctr_off;
        const double cx = __ldg(ct + (pack & 1023u));
        const double cy = __ldg(ct + R.nc[0] + ((pack >> 10) & 1023u));
        const double cz = __ldg(ct + R.nc[0] + R.nc[1] + ((pack >> 20) & 1023u));
        store_cell_pos(d, R, d.p32_nxt, d.plo_nxt, i, x.x - cx, x.y - cy, x.z - cz, pack);
        if (d.p32_ref) check_displacement(d, i, d.p32_nxt[i]);
        store_vel_copy(d.v32_nxt, d.vlo_nxt, i, v);
    }
    st_cs_dvec4(d.v + i, v);
}

// At most 64 registers (4 blocks of 256 per SM instead of 3 at 77): the
// kernel waits on its gathers, and the extra warps hide more of that than
// the 8-16 bytes of spills cost (153 against 163 us per step at 1M spheres,
// the same results).
template <bool BATCHED, bool ENERGY, int EPI>
__global__ void __launch_bounds__(256, 4) k_force_sd_dw(Dev d, LJ lj)
{
    if (stopped(d.status)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const int64_t n = d.n;
    const Rep &R = d.reps[BATCHED ? d.rep_of[i] : 0];
    const float4 hi = d.p32[i], li = d.plo[i];
    const float4 vih = d.v32[i], vil = d.vlo[i];
    const float qhx0 = __fadd_rn(hi.x, R.dw_sh[0]), qhx2 = __fsub_rn(hi.x, R.dw_sh[0]);
    const float qhy0 = __fadd_rn(hi.y, R.dw_sh[1]), qhy2 = __fsub_rn(hi.y, R.dw_sh[1]);
    const float qhz0 = __fadd_rn(hi.z, R.dw_sh[2]), qhz2 = __fsub_rn(hi.z, R.dw_sh[2]);
    const float qlx0 = __fadd_rn(li.x, R.dw_sl[0]), qlx2 = __fsub_rn(li.x, R.dw_sl[0]);
    const float qly0 = __fadd_rn(li.y, R.dw_sl[1]), qly2 = __fsub_rn(li.y, R.dw_sl[1]);
    const float qlz0 = __fadd_rn(li.z, R.dw_sl[2]), qlz2 = __fsub_rn(li.z, R.dw_sl[2]);
    const dw sig2 = dw_const(lj.dw_sd_sig2), sig = dw_const(lj.dw_sd_sig);
    const dw kk = dw_const(lj.dw_sd_k), gn = {-lj.dw_sd_g[0], -lj.dw_sd_g[1]};
    const int cnt = MD_CHECK(d, d.nb_count[i] <= d.cap) ? d.nb_count[i] : 0;
    const int nq = (cnt + 3) >> 2;
    const int4 *nb4 = reinterpret_cast<const int4 *>(d.nb);
    const dw zero = {0.f, 0.f};
    dw ax = zero, ay = zero, az = zero, ape = zero, aw = zero;
    for (int q = 0; q < nq; q++) {
        const int4 e4 = __ldcs(nb4 + (int64_t)q * n + i);
        const uint32_t es[4] = {(uint32_t)e4.x, (uint32_t)e4.y, (uint32_t)e4.z, (uint32_t)e4.w};
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const uint32_t e = es[t];
            const uint32_t j = MD_CHECK(d, (e & kJMask) <= (uint32_t)d.n) ? (e & kJMask) : (uint32_t)d.n;
            const float4 hj = __ldg(d.p32 + j), lj4 = __ldg(d.plo + j);
            const uint32_t c = e >> kJBits;
            const bool x2 = c & 2u, x1 = c & 1u, y2 = c & 8u, y1 = c & 4u, z2 = c & 32u, z1 = c & 16u;
            const float dxh = __fsub_rn(x2 ? qhx2 : (x1 ? hi.x : qhx0), hj.x);
            const float dyh = __fsub_rn(y2 ? qhy2 : (y1 ? hi.y : qhy0), hj.y);
            const float dzh = __fsub_rn(z2 ? qhz2 : (z1 ? hi.z : qhz0), hj.z);
            const float dxl = __fsub_rn(x2 ? qlx2 : (x1 ? li.x : qlx0), lj4.x);
            const float dyl = __fsub_rn(y2 ? qly2 : (y1 ? li.y : qly0), lj4.y);
            const float dzl = __fsub_rn(z2 ? qlz2 : (z1 ? li.z : qlz0), lj4.z);
            const dw r2 = dw_add(dw_add(dw_sq_of(dxh, dxl), dw_sq_of(dyh, dyl)), dw_sq_of(dzh, dzl));
            if (!(__fadd_rn(__fsub_rn(r2.h, sig2.h), __fsub_rn(r2.l, sig2.l)) < 0.f)) continue;
            const float4 vjh = __ldg(d.v32 + j), vjl = __ldg(d.vlo + j);
            // 1/r and r
            const float af = __fadd_rn(r2.h, r2.l);
            const dw ir = dw_rsqrt(r2, af, rsqrt_approx(af));
            const dw r = dw_mul(r2, ir);
            const dw dx = {dxh, dxl}, dy = {dyh, dyl}, dz = {dzh, dzl};
            const dw vx = dw_add(dw{vih.x, vil.x}, dw{-vjh.x, -vjl.x});
            const dw vy = dw_add(dw{vih.y, vil.y}, dw{-vjh.y, -vjl.y});
            const dw vz = dw_add(dw{vih.z, vil.z}, dw{-vjh.z, -vjl.z});
            const dw vn = dw_mul(dw_add(dw_add(dw_mul(dx, vx), dw_mul(dy, vy)), dw_mul(dz, vz)), ir);
            const dw ov = dw_add(sig, dw{-r.h, -r.l});
            const dw fo = dw_mul(dw_add(dw_mul(kk, ov), dw_mul(gn, vn)), ir);
            ax = dw_add(ax, dw_mul(fo, dx));
            ay = dw_add(ay, dw_mul(fo, dy));
            az = dw_add(az, dw_mul(fo, dz));
            if (ENERGY) {
                ape = dw_add(ape, dw_mul(dw_const(lj.dw_sd_hk), dw_mul(ov, ov)));
                aw = dw_add(aw, dw_mul(fo, r2));
            }
        }
        ax = fast_two_sum(ax.h, ax.l);
        ay = fast_two_sum(ay.h, ay.l);
        az = fast_two_sum(az.h, az.l);
    }
    if (ENERGY) {
        d.pe_atom64[i] = 0.5 * to_f64(ape);
        d.w_atom64[i] = 0.5 * to_f64(aw);
    }
    dw_sd_epilogue<EPI, ENERGY>(d, lj, R, i, to_f64(ax), to_f64(ay), to_f64(az), __float_as_uint(hi.w));
}

// Double-word velocity copies (v32: high parts, vlo: low parts) for the
// contact kernel, where something other than its fused step changed v.
__global__ void __launch_bounds__(256) k_velocity_dw(Dev d)
{
    if (stopped(d.status)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > d.n) return;                     // slot n: the sentinel (zero velocity)
    store_vel_copy(d.v32, d.vlo, i, d.v[i]);
}

template <bool B, bool EN>
void launch_sd_dw(const Dev &d, const LJ &lj, int epi, unsigned g, cudaStream_t st)
{
    if (epi == EPI_F) k_force_sd_dw<B, EN, EPI_F><<<g, 256, 0, st>>>(d, lj);
    else if (epi == EPI_FK) k_force_sd_dw<B, EN, EPI_FK><<<g, 256, 0, st>>>(d, lj);
    else k_force_sd_dw<B, EN, EPI_FKKD><<<g, 256, 0, st>>>(d, lj);
}

}  // namespace

int launch_force_dw(const Dev &d, const LJ &lj, int tpa, int epi, bool energy, bool batched,
                    cudaStream_t st, int *nl)
{
    if (d.n <= 0) return 0;
    if (!d.plo || !d.plo_nxt) return -1;
    if (batched) {
        if (tpa == 8) launch_dw<8, true>(d, lj, epi, energy, st);
        else if (tpa == 4) launch_dw<4, true>(d, lj, epi, energy, st);
        else if (tpa == 2) launch_dw<2, true>(d, lj, epi, energy, st);
        else launch_dw<1, true>(d, lj, epi, energy, st);
    } else {
        if (tpa == 8) launch_dw<8, false>(d, lj, epi, energy, st);
        else if (tpa == 4) launch_dw<4, false>(d, lj, epi, energy, st);
        else if (tpa == 2) launch_dw<2, false>(d, lj, epi, energy, st);
        else launch_dw<1, false>(d, lj, epi, energy, st);
    }
    *nl += 1;
    return (int)cudaGetLastError();
}

}  // namespace mdk

namespace mdk {

int launch_adjoint_pairs_dw(const Dev &d, const LJ &lj, int lanes, const float4 *wh,
                            const float4 *wl, dvec4 *xbar, double *g_eps, double *g_sig, double k,
                            double lw, cudaStream_t st, int *nl)
{
    if (lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8) return -1;
    if (!wh || !wl || !d.plo) return -1;
    if (d.n <= 0) return 0;
    DwAdjArgs a{wh, wl, xbar, g_eps, g_sig, k, lw};
    const unsigned g = (unsigned)((d.n * lanes + 127) / 128);
    const bool win = lw != 0.0;
#define MD_ADJDW(W)                                                                   \
    do {                                                                              \
        if (lanes == 8) k_adjoint_pairs_dw<W, 8><<<g, 128, 0, st>>>(d, lj, a);        \
        else if (lanes == 4) k_adjoint_pairs_dw<W, 4><<<g, 128, 0, st>>>(d, lj, a);   \
        else if (lanes == 2) k_adjoint_pairs_dw<W, 2><<<g, 128, 0, st>>>(d, lj, a);   \
        else k_adjoint_pairs_dw<W, 1><<<g, 128, 0, st>>>(d, lj, a);                   \
    } while (0)
    if (win) MD_ADJDW(true);
    else MD_ADJDW(false);
#undef MD_ADJDW
    *nl += 1;
    return (int)cudaGetLastError();
}

}  // namespace mdk

namespace mdk {

int launch_velocity_dw(const Dev &d, cudaStream_t st, int *nl)
{
    if (d.n <= 0) return 0;
    if (!d.v32 || !d.vlo) return -1;
    k_velocity_dw<<<(unsigned)((d.n + 256) / 256), 256, 0, st>>>(d);
    *nl += 1;
    return (int)cudaGetLastError();
}

int launch_force_sd_dw(const Dev &d, const LJ &lj, int epi, bool energy, cudaStream_t st, int *nl)
{
    if (d.n <= 0) return 0;
    if (!d.plo || !d.plo_nxt || !d.v32 || !d.v32_nxt || !d.vlo || !d.vlo_nxt) return -1;
    const unsigned g = (unsigned)((d.n + 255) / 256);
    const bool b = d.nrep > 1;
    if (b && energy) launch_sd_dw<true, true>(d, lj, epi, g, st);
    else if (b) launch_sd_dw<true, false>(d, lj, epi, g, st);
    else if (energy) launch_sd_dw<false, true>(d, lj, epi, g, st);
    else launch_sd_dw<false, false>(d, lj, epi, g, st);
    *nl += 1;
    return (int)cudaGetLastError();
}

}  // namespace mdk
