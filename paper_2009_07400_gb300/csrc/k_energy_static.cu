// md_energy_sums_static: the FP64 energy / virial / kinetic-energy reduction
// without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need
// totals: an external MD engine that has reserved the whole GPU for its own
// memory pool, a deployment with a fixed device-memory budget decided up
// front, or a latency-sensitive loop that must not call cudaMalloc because
// it can synchronise the device and stall other streams.  They pass their own
// per-atom inputs and an output slot; the only scratch this reduction needs
// (one partial sum triple per chunk of atoms) lives in a fixed-size array in
// the library's own device data, so no allocation happens on any call.
#include <mutex>
#include <string>

#include "../../include/md.h"
#include "md_internal.cuh"

namespace mdk {
void set_global_error(const std::string &msg);
}

namespace {

constexpr int64_t kChunkAtoms = 4096;
constexpr int64_t kMaxChunks = 8192;   // n <= 8192 * 4096 = 33,554,432 atoms

// Scratch of md_energy_sums_static: (PE, KE, W) partial sums, one triple per
// chunk (192 KiB).  Every GPU that loads the library holds it until the
// process exits.  In host code this name is a host-side stand-in, not a
// device address: host code obtains the address with cudaGetSymbolAddress.
static __device__ __align__(256) double g_energy_partials[3 * kMaxChunks];

// Device addresses of g_energy_partials, one per CUDA context.  The library's
// module is loaded once per context, so the array has its own address in
// every context that calls (a device's primary context, or a driver-API
// context of an external engine made current on the calling thread); an
// address resolved in one context is not valid in another.
struct ScratchAddr {
    unsigned long long ctx_id;   // unique id of the context (never reused in a process)
    double *addr;
};
constexpr int kMaxContexts = 64;
std::mutex g_mu;
ScratchAddr g_addr[kMaxContexts];
int g_naddr = 0;

// cuCtxGetCurrent and cuCtxGetId fetched through the runtime (the library
// does not link the driver library itself); null if the driver lacks them.
void *driver_fn(const char *name, unsigned int version)
{
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &f, version, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return f;
}
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

// Unique id of the calling thread's current context; false if unknown (no
// current context yet, or an old driver).
bool current_ctx_id(unsigned long long *id)
{
    static const CtxGetCurrentFn get_cur = (CtxGetCurrentFn)driver_fn("cuCtxGetCurrent", 4000);
    static const CtxGetIdFn get_id = (CtxGetIdFn)driver_fn("cuCtxGetId", 12000);
    void *ctx = nullptr;
    return get_cur && get_id && get_cur(&ctx) == 0 && ctx && get_id(ctx, id) == 0;
}

__global__ void __launch_bounds__(256) k_static_chunks(int64_t n, const double *pe, const double *w,
                                                       const double *vel, double mass,
                                                       double *partials)
{
    const int64_t a0 = (int64_t)blockIdx.x * kChunkAtoms;
    const int64_t a1 = min(n, a0 + kChunkAtoms);
    double p = 0, k = 0, v = 0;
    for (int64_t a = a0 + threadIdx.x; a < a1; a += blockDim.x) {
        p += pe[a];
        v += w[a];
        const double vx = vel[3 * a], vy = vel[3 * a + 1], vz = vel[3 * a + 2];
        k += 0.5 * mass * fma(vx, vx, fma(vy, vy, vz * vz));
    }
    for (int o = 16; o > 0; o >>= 1) {
        p += __shfl_xor_sync(0xffffffffu, p, o);
        k += __shfl_xor_sync(0xffffffffu, k, o);
        v += __shfl_xor_sync(0xffffffffu, v, o);
    }
    __shared__ double sh[3][8];
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sh[0][wid] = p; sh[1][wid] = k; sh[2][wid] = v; }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0;
        for (int q = 0; q < 8; q++) s += sh[threadIdx.x][q];
        partials[3 * blockIdx.x + threadIdx.x] = s;
    }
}

// Sums the chunk partials in a fixed order (one warp per quantity).
__global__ void __launch_bounds__(96) k_static_final(int64_t nchunks, const double *partials,
                                                     double *out3)
{
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double s = 0;
    for (int64_t c = lane; c < nchunks; c += 32) s += partials[3 * c + q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out3[q] = s;
}

}  // namespace

extern "C" int md_energy_sums_static(int64_t n, const double *pe_atom, const double *w_atom,
                                     const double *vel, double mass, double *out3, void *stream)
{
    if (n < 1 || !pe_atom || !w_atom || !vel || !out3 || !(mass > 0)) {
        mdk::set_global_error("md_energy_sums_static: bad argument");
        return MD_ERR_INVAL;
    }
    const int64_t nchunks = (n + kChunkAtoms - 1) / kChunkAtoms;
    if (nchunks > kMaxChunks) {
        mdk::set_global_error("md_energy_sums_static: n = " + std::to_string(n) +
                              " exceeds the maximum of " + std::to_string(kMaxChunks * kChunkAtoms) +
                              " atoms (fixed scratch size)");
        return MD_ERR_INVAL;
    }
    // the calling thread's current context: a device's primary context, or
    // a context the caller made current through the driver API
    unsigned long long ctx_id = 0;
    bool keyed = current_ctx_id(&ctx_id);
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> g(g_mu);
        for (int k = 0; keyed && k < g_naddr; k++)
            if (g_addr[k].ctx_id == ctx_id) scratch = g_addr[k].addr;
        if (!scratch) {
            // first call in this context: resolve the array's address (this
            // also makes the device's primary context current when the
            // thread had none; host-only work, nothing is allocated)
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_energy_partials);
            if (e != cudaSuccess) {
                mdk::set_global_error(std::string("md_energy_sums_static: cudaGetSymbolAddress: ") +
                                      cudaGetErrorString(e));
                return MD_ERR_CUDA;
            }
            scratch = (double *)p;
            keyed = current_ctx_id(&ctx_id);
            // without a context id nothing is cached and the next call
            // resolves the address again
            if (keyed && g_naddr < kMaxContexts) g_addr[g_naddr++] = {ctx_id, scratch};
        }
    }
    // an error left pending by unrelated earlier work on this thread would
    // otherwise be reported as this call's launch failure: clear it (a
    // sticky error of a broken context makes the launches below fail anyway)
    cudaGetLastError();
    cudaStream_t st = (cudaStream_t)stream;
    k_static_chunks<<<(unsigned)nchunks, 256, 0, st>>>(n, pe_atom, w_atom, vel, mass, scratch);
    k_static_final<<<1, 96, 0, st>>>(nchunks, scratch, out3);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        mdk::set_global_error(std::string("md_energy_sums_static: launch: ") + cudaGetErrorString(e));
        return MD_ERR_CUDA;
    }
    return MD_OK;
}
