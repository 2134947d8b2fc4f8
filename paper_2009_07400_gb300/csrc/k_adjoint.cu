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
// derivative ignores.  Adjoint vectors live in caller order (the atom order
// changes at every rebuild); one thread per atom of the cell-ordered state
// owns the caller-order entry of its atom, so no atomics are needed.
#include "md_internal.cuh"

namespace mdk {

namespace {

__device__ __forceinline__ bool stopped(const DevStatus *st)
{
    return *((volatile const int32_t *)&st->flags) != 0;
}

struct AdjArgs {
    const dvec4 *wbar;   // dloss/dw (caller order)
    dvec4 *xbar;         // dloss/dx carry (caller order), updated
    double *g_eps;       // per-atom accumulators (caller order)
    double *g_sig;
    double k;            // k_n
    double lw;           // 1/W inside the loss window, else 0
};

// FP64 pair geometry: the image shift of the neighbour's stencil slot is added
// to (x_i - x_j) as the minimum-image branch would.
template <bool MIXED>
__global__ void __launch_bounds__(128) k_adjoint_pairs(Dev d, LJ lj, AdjArgs a)
{
    if (stopped(d.status)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
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
    const int cnt = MD_CHECK(d, d.nb_count[i] <= d.cap) ? d.nb_count[i] : 0;
    const int4 *nb4 = reinterpret_cast<const int4 *>(d.nb);
    const double eps = lj.eps, sigma6 = lj.sigma6, sigma = lj.sigma;
    double jx = 0, jy = 0, jz = 0, fx = 0, fy = 0, fz = 0, ge = 0, gs = 0, pe_e = 0, pe_s = 0;
    for (int k = 0; k < cnt; k++) {
        const int4 e4 = nb4[(int64_t)(k >> 2) * d.n + i];
        const int32_t e = (k & 3) == 0 ? e4.x : (k & 3) == 1 ? e4.y : (k & 3) == 2 ? e4.z : e4.w;
        const uint32_t code = (uint32_t)e >> kJBits;
        const int ox = (int)(code & 3u) - 1, oy = (int)((code >> 2) & 3u) - 1, oz = (int)(code >> 4) - 1;
        const int32_t j = (int32_t)((uint32_t)e & kJMask);
        if (!MD_CHECK(d, j <= d.n)) continue;
        double dx, dy, dz;
        if (MIXED) {
            // cell-relative FP32 geometry, as in the mixed force kernel
            const float4 pj = d.p32[j];
            dx = (double)fmaf((float)ox, R.nsf[0], pi.x - pj.x);
            dy = (double)fmaf((float)oy, R.nsf[1], pi.y - pj.y);
            dz = (double)fmaf((float)oz, R.nsf[2], pi.z - pj.z);
        } else {
            const dvec4 xj = d.x[j];
            dx = xi.x - xj.x;
            dy = xi.y - xj.y;
            dz = xi.z - xj.z;
            if (ox) dx = dx + (ox < 0 ? lo[0] : hi[0]);
            if (oy) dy = dy + (oy < 0 ? lo[1] : hi[1]);
            if (oz) dz = dz + (oz < 0 ? lo[2] : hi[2]);
        }
        const double rsq = dx * dx + dy * dy + dz * dz;
        if (!(rsq < lj.rc2)) continue;
        const double sr2 = 1.0 / rsq;
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
        ge += (f / eps) * dui;
        gs += (144.0 * eps * sr2 * t * (4.0 * t - 1.0) / sigma) * dui;
        fx += f * dx;
        fy += f * dy;
        fz += f * dz;
        pe_e += 0.5 * 4.0 * t * (t - 1.0);
        pe_s += 0.5 * 24.0 * eps * t * (2.0 * t - 1.0) / sigma;
    }
    dvec4 xb = a.xbar[idi];
    xb.x += a.k * jx - a.lw * fx;
    xb.y += a.k * jy - a.lw * fy;
    xb.z += a.k * jz - a.lw * fz;
    a.xbar[idi] = xb;
    a.g_eps[idi] += a.k * ge + a.lw * pe_e;
    a.g_sig[idi] += a.k * gs + a.lw * pe_s;
}

__global__ void __launch_bounds__(256) k_adjoint_axpy(int64_t n, double dt, const dvec4 *xbar,
                                                      dvec4 *wbar)
{
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    dvec4 w = wbar[a];
    const dvec4 x = xbar[a];
    w.x = fma(dt, x.x, w.x);
    w.y = fma(dt, x.y, w.y);
    w.z = fma(dt, x.z, w.z);
    wbar[a] = w;
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

int launch_adjoint_pairs(const Dev &d, const LJ &lj, bool mixed, const dvec4 *wbar, dvec4 *xbar,
                         double *g_eps, double *g_sig, double k, double lw, cudaStream_t st,
                         int *nl)
{
    AdjArgs a{wbar, xbar, g_eps, g_sig, k, lw};
    const unsigned g = (unsigned)((d.n + 127) / 128);
    if (mixed) k_adjoint_pairs<true><<<g, 128, 0, st>>>(d, lj, a);
    else k_adjoint_pairs<false><<<g, 128, 0, st>>>(d, lj, a);
    *nl += 1;
    return (int)cudaGetLastError();
}

int launch_adjoint_axpy(int64_t n, double dt, const dvec4 *xbar, dvec4 *wbar, cudaStream_t st,
                        int *nl)
{
    k_adjoint_axpy<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, dt, xbar, wbar);
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
