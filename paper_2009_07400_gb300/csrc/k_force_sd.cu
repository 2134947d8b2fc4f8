// Spring-dashpot contact forces (tinyMD Sec. 3.2, Eq. 3) over the same cell
// binning and Verlet list as the Lennard-Jones path.  Spheres of diameter
// sigma touch when r = |x_ij| < sigma (strict); then
//     F_i += K xi + gamma xi_dot,  xi = xhat (sigma - r),
//     xi_dot = -xhat (xhat . v_ij),  xhat = x_ij / r,
// i.e. F_i += x_ij [K (sigma - r) - gamma (x_ij . v_ij) / r] / r, with
// x_ij = x_i - x_j (minimum image) and v_ij = v_i - v_j.  The list radius
// is cutoff + skin with cutoff >= sigma.
//
// GPU mapping: one thread per atom over its full-list row (neighbour-major
// int4 chunks), like the LJ kernels.  The pair term reads the neighbours'
// velocities, those of the half step (the latest ones, as in the oracle).
// Mixed path: displacements from the cell-relative FP32 positions plus the
// stencil offset (as the LJ mixed kernel), velocities from FP32 copies, FP32
// pair arithmetic (r by a correctly rounded square root, since sigma - r
// cancels) with compensated per-atom sums; the velocity-Verlet update is
// fused into the kernel's epilogue like the LJ step, which writes the next
// FP32 positions and the next FP32 velocity copies into the other buffers
// of their pairs (the neighbours still gather this step's), so one launch
// makes a time step.  FP64 path: FP64 throughout, 1/r by a refined FP32
// estimate (below FP64 rounding after two steps); it gathers the FP64
// velocities themselves, so it stores the force and the update runs in its
// own kernel afterwards.
#include "md_internal.cuh"

namespace mdk {

namespace {

__device__ __forceinline__ bool stopped(const DevStatus *st)
{
    return *((volatile const int32_t *)&st->flags) != 0;
}

__device__ __forceinline__ void kahan(float &s, float &c, float term)
{
    const float y = term - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

__device__ __forceinline__ float rcp_approx(float a)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

// FP32 copies of the velocities for the mixed contact kernel (the neighbour
// gathers then read 16 B instead of 32 B and convert nothing on GB300's
// narrow FP64 pipe).  The fused step keeps them current; this pass runs only
// where something else changed the velocities (the first step of a run, a
// new state, a lone final kick).
__global__ void __launch_bounds__(256) k_velocity_f32(Dev d)
{
    if (stopped(d.status)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > d.n) return;                     // slot n: the sentinel (zero velocity)
    const dvec4 v = d.v[i];
    // conversions on the bit patterns (IEEE results, no FP64-pipe work)
    d.v32[i] = make_float4(f32_of_f64(v.x), f32_of_f64(v.y), f32_of_f64(v.z), 0.f);
}

// Velocity-Verlet epilogue of the mixed contact step, in the operation order
// of the standalone update (kick; with EPI_FKKD the second kick, the drift,
// the next p32 and the next v32).  f: the FP32 force on atom i.
template <int EPI, bool ENERGY>
__device__ __forceinline__ void sd_epilogue(const Dev &d, const LJ &lj, const Rep &R, int64_t i,
                                            float4 f, uint32_t pack)
{
    if (EPI == EPI_F || EPI == EPI_FK) d.f32[i] = f;
    if (EPI == EPI_F) return;
    const double fx = f64_of_f32(f.x), fy = f64_of_f32(f.y), fz = f64_of_f32(f.z);
    dvec4 v = ld_cs_dvec4(d.v + i);        // streaming: keeps the gathered lines in L1
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
        st_cs_dvec4(d.x + i, x);             // neighbours gather p32 and v32 only
        const double *ct = d.ctr + R.ctr_off;
        const double cx = __ldg(ct + (pack & 1023u));
        const double cy = __ldg(ct + R.nc[0] + ((pack >> 10) & 1023u));
        const double cz = __ldg(ct + R.nc[0] + R.nc[1] + ((pack >> 20) & 1023u));
        const float4 pn = make_float4(f32_of_f64(x.x - cx), f32_of_f64(x.y - cy),
                                      f32_of_f64(x.z - cz), __uint_as_float(pack));
        d.p32_nxt[i] = pn;
        check_displacement(d, i, pn);
        d.v32_nxt[i] = make_float4(f32_of_f64(v.x), f32_of_f64(v.y), f32_of_f64(v.z), 0.f);
    }
    st_cs_dvec4(d.v + i, v);
}

template <bool BATCHED, bool ENERGY, int EPI>
__global__ void __launch_bounds__(256) k_force_sd_mixed(Dev d, LJ lj)
{
    if (stopped(d.status)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const int64_t n = d.n;
    const Rep &R = d.reps[BATCHED ? d.rep_of[i] : 0];
    const float4 pi = d.p32[i];
    const float4 *v32 = d.v32;
    const float4 vi = v32[i];
    // p_i - o s for o = -1, 0, +1 (nsf = -s), selected per pair in registers
    const float qx0 = pi.x - R.nsf[0], qx2 = pi.x + R.nsf[0];
    const float qy0 = pi.y - R.nsf[1], qy2 = pi.y + R.nsf[1];
    const float qz0 = pi.z - R.nsf[2], qz2 = pi.z + R.nsf[2];
    const int cnt = MD_CHECK(d, d.nb_count[i] <= d.cap) ? d.nb_count[i] : 0;
    const int nq = (cnt + 3) >> 2;
    const int4 *nb4 = reinterpret_cast<const int4 *>(d.nb);
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    float pe = 0.f, w = 0.f, cpe = 0.f, cw = 0.f;
    for (int q = 0; q < nq; q++) {
        const int4 e4 = __ldcs(nb4 + (int64_t)q * n + i);
        const uint32_t es[4] = {(uint32_t)e4.x, (uint32_t)e4.y, (uint32_t)e4.z, (uint32_t)e4.w};
        // the chunk's position and velocity gathers are issued together, the
        // velocity before the contact test: in dense packings nearly every
        // listed pair touches, and the two dependent gather latencies per
        // pair were the kernel's limiter (74 -> 70 us at 1M spheres; a
        // dilute gas pays an extra L1 gather per non-touching pair instead)
        float4 pjs[4], vjs[4];
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const int32_t j = (int32_t)(es[t] & kJMask);
            const int32_t jl = MD_CHECK(d, j <= d.n) ? j : (int32_t)d.n;   // checked in debug builds
            pjs[t] = __ldg(d.p32 + jl);
            vjs[t] = __ldg(v32 + jl);
        }
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const uint32_t c = es[t] >> kJBits;   // (a bad j was replaced by the sentinel above)
            const float4 pj = pjs[t];
            // d = (p_i - o s) - p_j with o = code - 1 per dimension
            const float dx = ((c & 2u) ? qx2 : ((c & 1u) ? pi.x : qx0)) - pj.x;
            const float dy = ((c & 8u) ? qy2 : ((c & 4u) ? pi.y : qy0)) - pj.y;
            const float dz = ((c & 32u) ? qz2 : ((c & 16u) ? pi.z : qz0)) - pj.z;
            const float rsq = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (!(rsq < lj.sd_sig2f)) continue;            // padding is far away
            const float4 vj = vjs[t];
            const float vx = vi.x - vj.x, vy = vi.y - vj.y, vz = vi.z - vj.z;
            const float r = sqrtf(rsq);                     // correctly rounded: sigma - r cancels
            const float ir = rcp_approx(r);
            const float vn = fmaf(dz, vz, fmaf(dy, vy, dx * vx)) * ir;
            const float ov = lj.sigmaf - r;
            const float fo = (lj.sd_kf * ov - lj.sd_gf * vn) * ir;
            kahan(sx, cx, fo * dx);
            kahan(sy, cy, fo * dy);
            kahan(sz, cz, fo * dz);
            if (ENERGY) {
                kahan(pe, cpe, 0.5f * lj.sd_kf * ov * ov);
                kahan(w, cw, fo * rsq);
            }
        }
    }
    if (ENERGY) {
        d.pe_atom[i] = 0.5f * (pe - cpe);
        d.w_atom[i] = 0.5f * (w - cw);
    }
    sd_epilogue<EPI, ENERGY>(d, lj, R, i, make_float4(sx - cx, sy - cy, sz - cz, 0.f),
                             __float_as_uint(pi.w));
}

template <bool BATCHED, bool ENERGY>
__global__ void __launch_bounds__(256) k_force_sd_f64(Dev d, LJ lj)
{
    if (stopped(d.status)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const int64_t n = d.n;
    const Rep &R = d.reps[BATCHED ? d.rep_of[i] : 0];
    const dvec4 xi = d.x[i];
    const dvec4 vi = d.v[i];
    const uint32_t pack = __float_as_uint(d.p32[i].w);
    const int ci[3] = {(int)(pack & 1023u), (int)((pack >> 10) & 1023u), (int)((pack >> 20) & 1023u)};
    const int cnt = MD_CHECK(d, d.nb_count[i] <= d.cap) ? d.nb_count[i] : 0;
    const int nq = (cnt + 3) >> 2;
    const int4 *nb4 = reinterpret_cast<const int4 *>(d.nb);
    double fx = 0, fy = 0, fz = 0, pe = 0, w = 0;
    for (int q = 0; q < nq; q++) {
        const int4 e4 = __ldcs(nb4 + (int64_t)q * n + i);
        const uint32_t es[4] = {(uint32_t)e4.x, (uint32_t)e4.y, (uint32_t)e4.z, (uint32_t)e4.w};
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const uint32_t e = es[t];
            const int32_t j = (int32_t)(e & kJMask);
            const uint32_t c = e >> kJBits;
            if (!MD_CHECK(d, j <= d.n)) continue;
            const dvec4 xj = ldg_dvec4(d.x + j);
            double dd[3] = {xi.x - xj.x, xi.y - xj.y, xi.z - xj.z};
            // periodic image: a neighbour cell across the box face sits one
            // box length away (same rule as the list criterion)
            const int o[3] = {(int)(c & 3u) - 1, (int)((c >> 2) & 3u) - 1, (int)(c >> 4) - 1};
#pragma unroll
            for (int k = 0; k < 3; k++) {
                if (o[k] < 0 && ci[k] == 0) dd[k] += R.L[k];
                else if (o[k] > 0 && ci[k] == R.nc[k] - 1) dd[k] -= R.L[k];
            }
            const double rsq = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
            if (!lt_nonneg(rsq, lj.sd_sig2)) continue;
            const dvec4 vj = ldg_dvec4(d.v + j);
            // 1/r: FP32 reciprocal square root refined by two Newton steps
            // y <- y (3 - rsq y^2) / 2 (relative error 2^-22 -> ~2^-44 ->
            // below FP64 rounding), then r = rsq / r; cheaper on GB300's FP64
            // pipe than an FP64 square root and two divisions (the seed's
            // conversions are integer operations on the bit patterns)
            double ir = f64_of_pos(rsqrtf(f32_of_pos(rsq)));
            ir = ir * fma(-0.5 * rsq, ir * ir, 1.5);
            ir = ir * fma(-0.5 * rsq, ir * ir, 1.5);
            const double r = rsq * ir;
            const double vn = (dd[0] * (vi.x - vj.x) + dd[1] * (vi.y - vj.y) + dd[2] * (vi.z - vj.z)) * ir;
            const double ov = lj.sigma - r;
            const double fo = (lj.sd_k * ov - lj.sd_g * vn) * ir;
            fx = fma(fo, dd[0], fx);
            fy = fma(fo, dd[1], fy);
            fz = fma(fo, dd[2], fz);
            if (ENERGY) {
                pe += 0.5 * lj.sd_k * ov * ov;
                w = fma(fo, rsq, w);
            }
        }
    }
    d.f64[i] = mk_dvec4(fx, fy, fz, 0.0);
    if (ENERGY) {
        d.pe_atom64[i] = 0.5 * pe;
        d.w_atom64[i] = 0.5 * w;
    }
}

template <bool B, bool EN>
void launch_sd_mixed(const Dev &d, const LJ &lj, int epi, unsigned g, cudaStream_t st)
{
    if (epi == EPI_F) k_force_sd_mixed<B, EN, EPI_F><<<g, 256, 0, st>>>(d, lj);
    else if (epi == EPI_FK) k_force_sd_mixed<B, EN, EPI_FK><<<g, 256, 0, st>>>(d, lj);
    else k_force_sd_mixed<B, EN, EPI_FKKD><<<g, 256, 0, st>>>(d, lj);
}

}  // namespace

int launch_velocity_f32(const Dev &d, cudaStream_t st, int *nl)
{
    if (d.n <= 0) return 0;
    if (!d.v32) return -1;
    k_velocity_f32<<<(unsigned)((d.n + 256) / 256), 256, 0, st>>>(d);
    *nl += 1;
    return (int)cudaGetLastError();
}

int launch_force_sd(const Dev &d, const LJ &lj, bool mixed, int epi, bool energy,
                    cudaStream_t st, int *nl)
{
    if (d.n <= 0) return 0;
    const unsigned g = (unsigned)((d.n + 255) / 256);
    const bool b = d.nrep > 1;
    if (mixed) {
        if (!d.v32 || !d.v32_nxt) return -1;
        if (b && energy) launch_sd_mixed<true, true>(d, lj, epi, g, st);
        else if (b) launch_sd_mixed<true, false>(d, lj, epi, g, st);
        else if (energy) launch_sd_mixed<false, true>(d, lj, epi, g, st);
        else launch_sd_mixed<false, false>(d, lj, epi, g, st);
    } else {
        if (b && energy) k_force_sd_f64<true, true><<<g, 256, 0, st>>>(d, lj);
        else if (b) k_force_sd_f64<true, false><<<g, 256, 0, st>>>(d, lj);
        else if (energy) k_force_sd_f64<false, true><<<g, 256, 0, st>>>(d, lj);
        else k_force_sd_f64<false, false><<<g, 256, 0, st>>>(d, lj);
    }
    *nl += 1;
    return (int)cudaGetLastError();
}

}  // namespace mdk
