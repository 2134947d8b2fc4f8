// Velocity-Verlet half steps (tinyMD Sec. 3.2, Eq. 1), the FP64 energy /
// virial reductions, and the gathers that map the cell-ordered state back to
// the caller's atom order.
#include "md_internal.cuh"

namespace mdk {

namespace {

__device__ __forceinline__ bool stopped(const DevStatus *st)
{
    return *((volatile const int32_t *)&st->flags) != 0;
}

// phase 1: v += c F; x += dt v            (c = dt / (2m))
// phase 2: v += c F
// phase 3: v += c F (full step; KE when asked); v += c F; x += dt v
// Positions change in place, so the FP32 cell-relative copy (on the
// double-word path its high and low parts) is refreshed in place too (no
// other kernel reads it concurrently).
template <bool BATCHED, bool MIXED>
__global__ void __launch_bounds__(256) k_integrate(Dev d, LJ lj, int phase, int want_ke)
{
    if (stopped(d.status)) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    double fx, fy, fz;
    if (MIXED) {
        // conversions on the bit patterns: this kernel is bound by GB300's
        // narrow FP64 pipe, which would otherwise run them
        const float4 f = d.f32[i];
        fx = f64_of_f32(f.x); fy = f64_of_f32(f.y); fz = f64_of_f32(f.z);
    } else {
        const dvec4 f = d.f64[i];
        fx = f.x; fy = f.y; fz = f.z;
    }
    dvec4 v = d.v[i];
    v.x = fma(lj.half_dt_m, fx, v.x);
    v.y = fma(lj.half_dt_m, fy, v.y);
    v.z = fma(lj.half_dt_m, fz, v.z);
    if (phase == 3) {
        if (want_ke) d.ke_atom64[i] = 0.5 * lj.mass * fma(v.x, v.x, fma(v.y, v.y, v.z * v.z));
        v.x = fma(lj.half_dt_m, fx, v.x);
        v.y = fma(lj.half_dt_m, fy, v.y);
        v.z = fma(lj.half_dt_m, fz, v.z);
    }
    d.v[i] = v;
    if (phase == 2) return;
    dvec4 x = d.x[i];
    x.x = fma(lj.dt, v.x, x.x);
    x.y = fma(lj.dt, v.y, x.y);
    x.z = fma(lj.dt, v.z, x.z);
    d.x[i] = x;
    const Rep &R = d.reps[BATCHED ? d.rep_of[i] : 0];
    const float4 p = d.p32[i];
    const uint32_t pack = __float_as_uint(p.w);
    // cell centres (c + 0.5) s from the per-replica table (no FP64 arithmetic)
    const double *ct = d.ctr + R.ctr_off;
    const double cx = __ldg(ct + (pack & 1023u));
    const double cy = __ldg(ct + R.nc[0] + ((pack >> 10) & 1023u));
    const double cz = __ldg(ct + R.nc[0] + R.nc[1] + ((pack >> 20) & 1023u));
    store_cell_pos(d, R, d.p32, d.plo, i, x.x - cx, x.y - cy, x.z - cz, pack);
    check_displacement(d, i, d.p32[i]);
}

// After a binning with the displacement trigger: the reordered state goes
// back into the current buffers (so the buffer roles of the captured step
// graph do not depend on whether the rebuild ran) and p32 becomes the
// reference of the next displacement checks.
__global__ void __launch_bounds__(256) k_copy_back(Dev d)
{
    if (stopped(d.status)) return;
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= d.n) return;
    d.x[a] = d.x_alt[a];
    d.v[a] = d.v_alt[a];
    d.id[a] = d.id_alt[a];
    d.p32_ref[a] = d.p32[a];
}

// One thread: decides whether the step's conditional rebuild runs (an atom
// moved past the trigger distance and no error is pending) and prepares the
// status word for it.
__global__ void k_rebuild_check(DevStatus *st, cudaGraphConditionalHandle h)
{
    const bool go = st->need_rebuild != 0 && *((volatile const int32_t *)&st->flags) == 0;
    st->dev_step += 1;
    if (go) {
        st->need_rebuild = 0;
        st->max_count = 0;
    }
    cudaGraphSetConditional(h, go ? 1u : 0u);
}

constexpr int kChunk = 1024;   // atoms per reduction chunk (1024: a 16k-atom system still fills 16 blocks)

// Per-chunk FP64 partial sums of (PE, KE, W).  Chunks never straddle
// replicas: chunk c of replica r covers atoms [off_r + c*kChunk, ...).
template <bool MIXED>
__global__ void __launch_bounds__(256) k_energy_chunks(Dev d, LJ lj, const int64_t *chunk_rep,
                                                       int ke_from_v, double *partials)
{
    if (stopped(d.status)) return;
    const int64_t c = blockIdx.x;
    const int64_t r = chunk_rep[2 * c], k = chunk_rep[2 * c + 1];
    const Rep &R = d.reps[r];
    const int64_t a0 = R.atom_off + k * kChunk;
    const int64_t a1 = min(R.atom_off + R.natoms, a0 + kChunk);
    double pe = 0, ke = 0, w = 0;
    for (int64_t a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
        if (MIXED) { pe += (double)d.pe_atom[a]; w += (double)d.w_atom[a]; }
        else { pe += d.pe_atom64[a]; w += d.w_atom64[a]; }
        if (ke_from_v) {
            const dvec4 v = d.v[a];
            ke += 0.5 * lj.mass * fma(v.x, v.x, fma(v.y, v.y, v.z * v.z));
        } else {
            ke += d.ke_atom64[a];
        }
    }
    __shared__ double sh[3][8];
    for (int o = 16; o > 0; o >>= 1) {
        pe += __shfl_xor_sync(0xffffffffu, pe, o);
        ke += __shfl_xor_sync(0xffffffffu, ke, o);
        w += __shfl_xor_sync(0xffffffffu, w, o);
    }
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sh[0][wid] = pe; sh[1][wid] = ke; sh[2][wid] = w; }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0;
        for (int q = 0; q < 8; q++) s += sh[threadIdx.x][q];
        partials[3 * c + threadIdx.x] = s;
    }
}

// One block; warp w sums (replica, quantity) pairs t = w, w + 32, ...: lane l
// adds chunks l, l+32, ... in order, then a fixed shuffle tree combines the
// lanes, so the result does not depend on scheduling.  With log_base the
// record goes to the on-device energy log at the cursor, which the block then
// advances.
__global__ void __launch_bounds__(1024) k_energy_final(const int64_t *chunk_first, int32_t nrep,
                                                       const double *partials, double *out,
                                                       double *log_base, DevStatus *st)
{
    if (stopped(st)) return;
    double *dst = out ? out : log_base + st->elog_cursor * 3 * (int64_t)nrep;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t t = w; t < 3 * (int64_t)nrep; t += 32) {
        const int64_t r = t / 3, q = t % 3;
        double s = 0;
        for (int64_t c = chunk_first[r] + lane; c < chunk_first[r + 1]; c += 32) s += partials[3 * c + q];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) dst[t] = s;
    }
    __syncthreads();
    if (!out && threadIdx.x == 0) st->elog_cursor += 1;
}

// Thermodynamic outputs of (PE, KE, W) records, one thread per (record,
// replica): total energy, T = 2 KE / (3 N - 3) (the momentum-free degrees of
// freedom) and P = (N T + W / 3) / V.  rec: nrec x nrep x 3; out: nrec x
// nrep x 6 (pe, ke, etot, w, T, P).  N = 1 has no free degree: T and P are
// reported as 0.
__global__ void __launch_bounds__(256) k_thermo(const Rep *reps, int32_t nrep, int64_t nrec,
                                                const double *rec, double *out)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nrec * nrep) return;
    const Rep &R = reps[t % nrep];
    const double pe = rec[3 * t], ke = rec[3 * t + 1], w = rec[3 * t + 2];
    const double nat = (double)R.natoms;
    const double vol = R.L[0] * R.L[1] * R.L[2];
    const double temp = R.natoms > 1 ? 2.0 * ke / (3.0 * nat - 3.0) : 0.0;
    double *o = out + 6 * t;
    o[0] = pe;
    o[1] = ke;
    o[2] = pe + ke;
    o[3] = w;
    o[4] = temp;
    o[5] = R.natoms > 1 ? (nat * temp + w / 3.0) / vol : 0.0;
}

// out (n x 3, caller order) <- x / v / F of the cell-ordered state.
__global__ void __launch_bounds__(256) k_gather_out(Dev d, int what, int mixed, double *out)
{
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= d.n) return;
    double3 q;
    if (what == 0) { const dvec4 t = d.x[a]; q = make_double3(t.x, t.y, t.z); }
    else if (what == 1) { const dvec4 t = d.v[a]; q = make_double3(t.x, t.y, t.z); }
    else if (mixed) { const float4 t = d.f32[a]; q = make_double3(t.x, t.y, t.z); }
    else { const dvec4 t = d.f64[a]; q = make_double3(t.x, t.y, t.z); }
    const int64_t o = d.id[a];
    out[3 * o + 0] = q.x;
    out[3 * o + 1] = q.y;
    out[3 * o + 2] = q.z;
}

// Caller-order input (n x 3) -> state in caller order (id = identity).
__global__ void __launch_bounds__(256) k_scatter_in(Dev d, const double *pos, const double *vel)
{
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= d.n) return;
    const double x0 = pos[3 * a], x1 = pos[3 * a + 1], x2 = pos[3 * a + 2];
    const double v0 = vel[3 * a], v1 = vel[3 * a + 1], v2 = vel[3 * a + 2];
    // inputs from device memory are checked here (host inputs were already)
    if (!(isfinite(x0) && isfinite(x1) && isfinite(x2) && isfinite(v0) && isfinite(v1) && isfinite(v2)))
        atomicOr(&d.status->flags, FLAG_NONFINITE);
    d.x[a] = mk_dvec4(x0, x1, x2, 0.0);
    d.v[a] = mk_dvec4(v0, v1, v2, 0.0);
    d.id[a] = (int32_t)a;
}

// rows (n x cap, caller order, replica-local ids) <- decoded list.
template <bool BATCHED>
__global__ void __launch_bounds__(256) k_decode_list(Dev d, int32_t *rows, int32_t cap)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.n) return;
    const Rep &R = d.reps[BATCHED ? d.rep_of[i] : 0];
    const int32_t cnt = MD_CHECK(d, d.nb_count[i] <= d.cap) ? d.nb_count[i] : 0;
    const int64_t o = d.id[i];
    const int4 *nb4 = reinterpret_cast<const int4 *>(d.nb);
    for (int32_t k = 0; k < cnt && k < cap; k++) {
        const int4 e4 = nb4[(int64_t)(k >> 2) * d.n + i];
        const int32_t e = (k & 3) == 0 ? e4.x : (k & 3) == 1 ? e4.y : (k & 3) == 2 ? e4.z : e4.w;
        const int32_t j = (int32_t)((uint32_t)e & kJMask);
        if (!MD_CHECK(d, j < d.n)) continue;
        rows[o * cap + k] = (int32_t)(d.id[j] - R.atom_off);
    }
}

}  // namespace

int launch_integrate(const Dev &d, const LJ &lj, int precision, int phase, bool batched,
                     cudaStream_t st, int *nl)
{
    if (d.n <= 0) return 0;
    const unsigned g = (unsigned)((d.n + 255) / 256);
    const int want_ke = phase >= 4 ? 1 : 0;
    const int ph = phase >= 4 ? 3 : phase;
    const bool m = precision == 1;
    if (batched && m) k_integrate<true, true><<<g, 256, 0, st>>>(d, lj, ph, want_ke);
    else if (batched) k_integrate<true, false><<<g, 256, 0, st>>>(d, lj, ph, want_ke);
    else if (m) k_integrate<false, true><<<g, 256, 0, st>>>(d, lj, ph, want_ke);
    else k_integrate<false, false><<<g, 256, 0, st>>>(d, lj, ph, want_ke);
    *nl += 1;
    return (int)cudaGetLastError();
}

// chunk_rep: device, (replica, chunk index) per chunk; chunk_first: device,
// nrep+1 first-chunk offsets.  out3: device, nrep x 3 (PE, KE, W).
int launch_energy(const Dev &d, const LJ &lj, int precision, bool ke_from_v,
                  const int64_t *chunk_rep, const int64_t *chunk_first, int64_t nchunks,
                  double *partials, double *out3, double *log_base, cudaStream_t st, int *nl)
{
    if (precision == 1)
        k_energy_chunks<true><<<(unsigned)nchunks, 256, 0, st>>>(d, lj, chunk_rep, ke_from_v ? 1 : 0, partials);
    else
        k_energy_chunks<false><<<(unsigned)nchunks, 256, 0, st>>>(d, lj, chunk_rep, ke_from_v ? 1 : 0, partials);
    k_energy_final<<<1, 1024, 0, st>>>(chunk_first, d.nrep, partials, out3, log_base, d.status);
    *nl += 2;
    return (int)cudaGetLastError();
}

int64_t energy_chunks_of(int64_t natoms) { return (natoms + kChunk - 1) / kChunk; }

int launch_thermo(const Rep *reps, int32_t nrep, int64_t nrec, const double *rec, double *out,
                  cudaStream_t st, int *nl)
{
    const int64_t t = nrec * nrep;
    if (t <= 0) return 0;
    k_thermo<<<(unsigned)((t + 255) / 256), 256, 0, st>>>(reps, nrep, nrec, rec, out);
    *nl += 1;
    return (int)cudaGetLastError();
}

int launch_gather_out(const Dev &d, int what, double *out, cudaStream_t st, int *nl)
{
    if (d.n <= 0) return 0;
    const unsigned g = (unsigned)((d.n + 255) / 256);
    const int mixed = (what == 3) ? 1 : 0;
    k_gather_out<<<g, 256, 0, st>>>(d, what >= 2 ? 2 : what, mixed, out);
    *nl += 1;
    return (int)cudaGetLastError();
}

int launch_scatter_in(const Dev &d, const double *pos, const double *vel, cudaStream_t st, int *nl)
{
    if (d.n <= 0) return 0;
    const unsigned g = (unsigned)((d.n + 255) / 256);
    k_scatter_in<<<g, 256, 0, st>>>(d, pos, vel);
    *nl += 1;
    return (int)cudaGetLastError();
}

int launch_copy_back(const Dev &d, cudaStream_t st, int *nl)
{
    if (d.n <= 0 || !d.p32_ref) return d.p32_ref ? 0 : -1;
    k_copy_back<<<(unsigned)((d.n + 255) / 256), 256, 0, st>>>(d);
    *nl += 1;
    return (int)cudaGetLastError();
}

int launch_rebuild_check(const Dev &d, cudaGraphConditionalHandle h, cudaStream_t st, int *nl)
{
    k_rebuild_check<<<1, 1, 0, st>>>(d.status, h);
    *nl += 1;
    return (int)cudaGetLastError();
}

int launch_decode_list(const Dev &d, int32_t *rows, int32_t cap, cudaStream_t st, int *nl)
{
    if (d.n <= 0) return 0;
    const unsigned g = (unsigned)((d.n + 255) / 256);
    if (d.nrep > 1) k_decode_list<true><<<g, 256, 0, st>>>(d, rows, cap);
    else k_decode_list<false><<<g, 256, 0, st>>>(d, rows, cap);
    *nl += 1;
    return (int)cudaGetLastError();
}

}  // namespace mdk
