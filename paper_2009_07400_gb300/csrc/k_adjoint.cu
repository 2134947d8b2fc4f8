// Reverse-mode derivative of a velocity-Verlet LJ rollout (not in the paper;
// the forward map is tinyMD's Sec. 3.2 Eq. 1 with the Eq. 2 force).
//
// Leapfrog form of the forward map (c = dt/(2m), w_n = v_{n+1/2}):
//     w_0 = v_0 + c F(x_0);  w_n = w_{n-1} + 2c F(x_n)  (1 <= n < S)
//     x_{n+1} = x_n + dt w_n
//     loss = (1/W) sum_{n = S-W+1 .. S} PE(x_n)
// Reverse sweep over force points n = S .. 0 with X = dloss/dx_{n+1}-carry,
// Wb = dloss/dw_n:
//     Wb += dt X
//     X  += k_n J(x_n) Wb,      theta_bar += k_n dF/dtheta(x_n) . Wb
//     X  += -F(x_n)/W,          theta_bar += dPE/dtheta(x_n)/W   (window)
// with k_n = 2c (n >= 1), c (n = 0), 0 (n = S: v_S does not enter the loss).
// J = dF/dx is symmetric; for one pair, with f the scalar of F_i = f d:
//     (J u)_i = sum_j [ f (u_i - u_j) + 2 f' d (d . (u_i - u_j)) ],
//     f' = df/d(r^2) = 48 eps sr2^2 t (2 - 7 t),   t = sigma^6 sr2^3,
//     df/deps = f/eps,  df/dsigma = 144 eps sr2 t (4t - 1) / sigma,
//     V = 4 eps t (t - 1),  dV/dsigma = 24 eps t (2t - 1) / sigma.
// rc is held fixed; pairs crossing it are a measure-zero set whose jump the
// derivative ignores.  The FP64 path evaluates the pair terms in FP64; the
// mixed path in FP32 (its forward forces are FP32 too), with per-atom sums
// added to the FP64 adjoint state.  Adjoint vectors live in caller order (the atom order
// changes at every rebuild); one thread per atom of the cell-ordered state
// owns the caller-order entry of its atom, so no atomics are needed.
#include "md_internal.cuh"

namespace mdk {

namespace {

__device__ __forceinline__ bool stopped(const DevStatus *st)
{
    return *((volatile const int32_t *)&st->flags) != 0;
}

// FP64 reciprocal: correctly rounded FP32 seed, two Newton steps (relative
// error below FP64 rounding); avoids an FP64 division per pair on GB300's
// narrow FP64 pipe (the seed's conversions are integer operations on the
// bit patterns).
__device__ __forceinline__ double rcp64(double a)
{
    double r = f64_of_pos(__frcp_rn(f32_of_pos(a)));
    r = fma(r, fma(-a, r, 1.0), r);
    return fma(r, fma(-a, r, 1.0), r);
}

// FP32 reciprocal on the special-function unit (relative error below 2^-22,
// as in the mixed force kernel).
__device__ __forceinline__ float rcp_approx(float a)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

struct AdjArgs {
    const float4 *wbar32; // FP32 copy of wbar in slot order (mixed path)
    const dvec4 *wbar;   // dloss/dw (caller order)
    dvec4 *xbar;         // dloss/dx carry (caller order), updated
    double *g_eps;       // per-atom accumulators (caller order)
    double *g_sig;
    double k;            // k_n
    double lw;           // 1/W inside the loss window, else 0
};

// FP64 path: FP64 pair geometry (the image shift of the neighbour's stencil
// slot is added to (x_i - x_j) as the minimum-image branch would) and FP64
// arithmetic.
template <bool WINDOW, int TPA>
__global__ void __launch_bounds__(128) k_adjoint_pairs(Dev d, LJ lj, AdjArgs a)
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
    const dvec4 xi = d.x[i];
    const float4 pi = d.p32[i];
    const uint32_t pack = __float_as_uint(pi.w);
    const int c[3] = {(int)(pack & 1023u), (int)((pack >> 10) & 1023u), (int)((pack >> 20) & 1023u)};
    double lo[3], hi[3];
    for (int q = 0; q < 3; q++) {
        lo[q] = c[q] == 0 ? R.L[q] : 0.0;
        hi[q] = c[q] == R.nc[q] - 1 ? -R.L[q] : 0.0;
    }
    const dvec4 ui = a.wbar[idi];
    const int cnt = valid && MD_CHECK(d, d.nb_count[i] <= d.cap) ? d.nb_count[i] : 0;
    const int4 *nb4 = reinterpret_cast<const int4 *>(d.nb);
    const double eps = lj.eps, sigma6 = lj.sigma6, sigma = lj.sigma;
    const double inv_eps = 1.0 / eps, inv_sigma = 1.0 / sigma;   // once per atom
    double jx = 0, jy = 0, jz = 0, fx = 0, fy = 0, fz = 0, ge = 0, gs = 0, pe_e = 0, pe_s = 0;
    // the TPA lanes of an atom take the row's int4 chunks in turn; each
    // chunk is loaded once
    for (int q = sub; 4 * q < cnt; q += TPA) {
      const int4 e4 = nb4[(int64_t)q * d.n + i];
      const int32_t es[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
      for (int t4 = 0; t4 < 4; t4++) {
        if (4 * q + t4 >= cnt) break;
        const int32_t e = es[t4];
        const uint32_t code = (uint32_t)e >> kJBits;
        const int ox = (int)(code & 3u) - 1, oy = (int)((code >> 2) & 3u) - 1, oz = (int)(code >> 4) - 1;
        const int32_t j = (int32_t)((uint32_t)e & kJMask);
        if (!MD_CHECK(d, j <= d.n)) continue;
        const dvec4 xj = d.x[j];
        double dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
        if (ox) dx = dx + (ox < 0 ? lo[0] : hi[0]);
        if (oy) dy = dy + (oy < 0 ? lo[1] : hi[1]);
        if (oz) dz = dz + (oz < 0 ? lo[2] : hi[2]);
        const double rsq = dx * dx + dy * dy + dz * dz;
        if (!lt_nonneg(rsq, lj.rc2)) continue;
        const double sr2 = rcp64(rsq);
        const double t = sr2 * sr2 * sr2 * sigma6;
        const double f = 48.0 * eps * t * (t - 0.5) * sr2;
        const double fp = 48.0 * eps * sr2 * sr2 * t * (2.0 - 7.0 * t);
        const dvec4 uj = a.wbar[d.id[j]];
        const double dux = ui.x - uj.x, duy = ui.y - uj.y, duz = ui.z - uj.z;
        const double ddu = dx * dux + dy * duy + dz * duz;
        jx += f * dux + 2.0 * fp * dx * ddu;
        jy += f * duy + 2.0 * fp * dy * ddu;
        jz += f * duz + 2.0 * fp * dz * ddu;
        const double dui = dx * ui.x + dy * ui.y + dz * ui.z;
        ge += (f * inv_eps) * dui;
        gs += (144.0 * eps * sr2 * t * (4.0 * t - 1.0) * inv_sigma) * dui;
        if (WINDOW) {   // -F/W and dPE/dtheta: only inside the loss window
            fx += f * dx;
            fy += f * dy;
            fz += f * dz;
            pe_e += 0.5 * 4.0 * t * (t - 1.0);
            pe_s += 0.5 * 24.0 * eps * t * (2.0 * t - 1.0) * inv_sigma;
        }
      }
    }
    if (TPA > 1) {
#pragma unroll
        for (int o = TPA / 2; o > 0; o >>= 1) {
            jx += __shfl_xor_sync(0xffffffffu, jx, o);
            jy += __shfl_xor_sync(0xffffffffu, jy, o);
            jz += __shfl_xor_sync(0xffffffffu, jz, o);
            ge += __shfl_xor_sync(0xffffffffu, ge, o);
            gs += __shfl_xor_sync(0xffffffffu, gs, o);
            if (WINDOW) {
                fx += __shfl_xor_sync(0xffffffffu, fx, o);
                fy += __shfl_xor_sync(0xffffffffu, fy, o);
                fz += __shfl_xor_sync(0xffffffffu, fz, o);
                pe_e += __shfl_xor_sync(0xffffffffu, pe_e, o);
                pe_s += __shfl_xor_sync(0xffffffffu, pe_s, o);
            }
        }
        if (sub != 0 || !valid) return;
    }
    dvec4 xb = a.xbar[idi];
    xb.x += a.k * jx - a.lw * fx;
    xb.y += a.k * jy - a.lw * fy;
    xb.z += a.k * jz - a.lw * fz;
    a.xbar[idi] = xb;
    a.g_eps[idi] += a.k * ge + a.lw * pe_e;
    a.g_sig[idi] += a.k * gs + a.lw * pe_s;
}

// Mixed path: the same pair terms in FP32 (geometry from the cell-relative
// FP32 positions, the neighbour's adjoint from an FP32 copy that the axpy
// kernel writes in slot order, so it is gathered like the positions: one
// local 16-byte load per pair instead of the caller id and a scattered
// load), summed per atom in FP32 and added to the FP64 adjoint state once
// per atom.  The FP64 pipe then only sees the per-atom updates.
template <bool WINDOW, int TPA>
__global__ void __launch_bounds__(128) k_adjoint_pairs_f32(Dev d, LJ lj, AdjArgs a)
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
    const float4 pi = d.p32[i];
    const float4 ui = a.wbar32[i];
    const int cnt = valid && MD_CHECK(d, d.nb_count[i] <= d.cap) ? d.nb_count[i] : 0;
    const int4 *nb4 = reinterpret_cast<const int4 *>(d.nb);
    const float eps = (float)lj.eps, sig6 = lj.sigma6f;
    const float inv_eps = (float)(1.0 / lj.eps), inv_sig = (float)(1.0 / lj.sigma);
    const float qx0 = pi.x - R.nsf[0], qx2 = pi.x + R.nsf[0];
    const float qy0 = pi.y - R.nsf[1], qy2 = pi.y + R.nsf[1];
    const float qz0 = pi.z - R.nsf[2], qz2 = pi.z + R.nsf[2];
    float jx = 0, jy = 0, jz = 0, fx = 0, fy = 0, fz = 0, ge = 0, gs = 0, pe_e = 0, pe_s = 0;
    for (int q = sub; 4 * q < cnt; q += TPA) {
      const int4 e4 = nb4[(int64_t)q * d.n + i];
      const int32_t es[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
      for (int t4 = 0; t4 < 4; t4++) {
        if (4 * q + t4 >= cnt) break;
        const uint32_t e = (uint32_t)es[t4];
        const uint32_t c = e >> kJBits;
        const int32_t j = (int32_t)(e & kJMask);
        if (!MD_CHECK(d, j < d.n)) continue;
        const float4 pj = d.p32[j];
        const float dx = ((c & 2u) ? qx2 : ((c & 1u) ? pi.x : qx0)) - pj.x;
        const float dy = ((c & 8u) ? qy2 : ((c & 4u) ? pi.y : qy0)) - pj.y;
        const float dz = ((c & 32u) ? qz2 : ((c & 16u) ? pi.z : qz0)) - pj.z;
        const float rsq = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        if (!(rsq < lj.rc2f)) continue;
        const float sr2 = rcp_approx(rsq);
        const float t = sr2 * sr2 * sr2 * sig6;
        const float f = 48.0f * eps * t * (t - 0.5f) * sr2;
        const float fp = 48.0f * eps * sr2 * sr2 * t * (2.0f - 7.0f * t);
        const float4 uj = a.wbar32[j];
        const float dux = ui.x - uj.x, duy = ui.y - uj.y, duz = ui.z - uj.z;
        const float ddu = fmaf(dz, duz, fmaf(dy, duy, dx * dux));
        jx += f * dux + 2.0f * fp * dx * ddu;
        jy += f * duy + 2.0f * fp * dy * ddu;
        jz += f * duz + 2.0f * fp * dz * ddu;
        const float dui = fmaf(dz, ui.z, fmaf(dy, ui.y, dx * ui.x));
        ge += (f * inv_eps) * dui;
        gs += (144.0f * eps * sr2 * t * (4.0f * t - 1.0f) * inv_sig) * dui;
        if (WINDOW) {
            fx += f * dx;
            fy += f * dy;
            fz += f * dz;
            pe_e += 2.0f * t * (t - 1.0f);
            pe_s += 12.0f * eps * t * (2.0f * t - 1.0f) * inv_sig;
        }
      }
    }
    if (TPA > 1) {
#pragma unroll
        for (int o = TPA / 2; o > 0; o >>= 1) {
            jx += __shfl_xor_sync(0xffffffffu, jx, o);
            jy += __shfl_xor_sync(0xffffffffu, jy, o);
            jz += __shfl_xor_sync(0xffffffffu, jz, o);
            ge += __shfl_xor_sync(0xffffffffu, ge, o);
            gs += __shfl_xor_sync(0xffffffffu, gs, o);
            if (WINDOW) {
                fx += __shfl_xor_sync(0xffffffffu, fx, o);
                fy += __shfl_xor_sync(0xffffffffu, fy, o);
                fz += __shfl_xor_sync(0xffffffffu, fz, o);
                pe_e += __shfl_xor_sync(0xffffffffu, pe_e, o);
                pe_s += __shfl_xor_sync(0xffffffffu, pe_s, o);
            }
        }
        if (sub != 0 || !valid) return;
    }
    dvec4 xb = a.xbar[idi];
    xb.x += a.k * (double)jx - a.lw * (double)fx;
    xb.y += a.k * (double)jy - a.lw * (double)fy;
    xb.z += a.k * (double)jz - a.lw * (double)fz;
    a.xbar[idi] = xb;
    a.g_eps[idi] += a.k * (double)ge + a.lw * (double)pe_e;
    a.g_sig[idi] += a.k * (double)gs + a.lw * (double)pe_s;
}

// wbar += dt xbar (caller order) for the atom in slot s, and the FP32 copy
// of the result into slot s (the current slot order, id: slot -> caller id);
// with wbar_lo also the low parts fl32(w - fl32(w)) (a double-word copy).
__global__ void __launch_bounds__(256) k_adjoint_axpy(int64_t n, double dt, const dvec4 *xbar,
                                                      dvec4 *wbar, float4 *wbar32,
                                                      float4 *wbar_lo, const int32_t *id)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t a = id[s];
    dvec4 w = wbar[a];
    const dvec4 x = xbar[a];
    w.x = fma(dt, x.x, w.x);
    w.y = fma(dt, x.y, w.y);
    w.z = fma(dt, x.z, w.z);
    wbar[a] = w;
    if (wbar32) {
        const float hx = (float)w.x, hy = (float)w.y, hz = (float)w.z;
        wbar32[s] = make_float4(hx, hy, hz, 0.f);
        if (wbar_lo)
            wbar_lo[s] = make_float4((float)(w.x - (double)hx), (float)(w.y - (double)hy),
                                     (float)(w.z - (double)hz), 0.f);
    }
}

// out (n x 3 doubles) <- a (padded FP64 3-vectors), same atom order.
__global__ void __launch_bounds__(256) k_unpad3(int64_t n, const dvec4 *a, double *out)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const dvec4 v = a[t];
    out[3 * t] = v.x;
    out[3 * t + 1] = v.y;
    out[3 * t + 2] = v.z;
}

// Deterministic sum of two per-atom arrays (one block, fixed order).
__global__ void __launch_bounds__(1024) k_sum2(int64_t n, const double *a, const double *b,
                                               double *out)
{
    __shared__ double sa[32], sb[32];
    double x = 0, y = 0;
    for (int64_t t = threadIdx.x; t < n; t += blockDim.x) {
        x += a[t];
        y += b[t];
    }
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sa[w] = x; sb[w] = y; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double p = 0, q = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) { p += sa[k]; q += sb[k]; }
        out[0] = p;
        out[1] = q;
    }
}

}  // namespace

int launch_adjoint_pairs(const Dev &d, const LJ &lj, bool mixed, int lanes, const dvec4 *wbar,
                         const float4 *wbar32, dvec4 *xbar, double *g_eps, double *g_sig,
                         double k, double lw, cudaStream_t st, int *nl)
{
    AdjArgs a{wbar32, wbar, xbar, g_eps, g_sig, k, lw};
    if (lanes != 1 && lanes != 2 && lanes != 4 && lanes != 8) return -1;
    if (mixed && !wbar32) return -1;
    const unsigned g = (unsigned)((d.n * lanes + 127) / 128);
    const bool win = lw != 0.0;
#define MD_ADJ(K, W)                                                             \
    do {                                                                         \
        if (lanes == 8) K<W, 8><<<g, 128, 0, st>>>(d, lj, a);                    \
        else if (lanes == 4) K<W, 4><<<g, 128, 0, st>>>(d, lj, a);               \
        else if (lanes == 2) K<W, 2><<<g, 128, 0, st>>>(d, lj, a);               \
        else K<W, 1><<<g, 128, 0, st>>>(d, lj, a);                               \
    } while (0)
    if (mixed) { if (win) MD_ADJ(k_adjoint_pairs_f32, true); else MD_ADJ(k_adjoint_pairs_f32, false); }
    else { if (win) MD_ADJ(k_adjoint_pairs, true); else MD_ADJ(k_adjoint_pairs, false); }
#undef MD_ADJ
    *nl += 1;
    return (int)cudaGetLastError();
}

int launch_adjoint_axpy(int64_t n, double dt, const dvec4 *xbar, dvec4 *wbar, float4 *wbar32,
                        float4 *wbar_lo, const int32_t *id, cudaStream_t st, int *nl)
{
    if (wbar_lo && !wbar32) return -1;
    k_adjoint_axpy<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, dt, xbar, wbar, wbar32, wbar_lo, id);
    *nl += 1;
    return (int)cudaGetLastError();
}

int launch_unpad3(int64_t n, const dvec4 *a, double *out, cudaStream_t st, int *nl)
{
    if (n <= 0) return 0;
    k_unpad3<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, a, out);
    *nl += 1;
    return (int)cudaGetLastError();
}

int launch_sum2(int64_t n, const double *a, const double *b, double *out, cudaStream_t st, int *nl)
{
    k_sum2<<<1, 1024, 0, st>>>(n, a, b, out);
    *nl += 1;
    return (int)cudaGetLastError();
}

}  // namespace mdk
