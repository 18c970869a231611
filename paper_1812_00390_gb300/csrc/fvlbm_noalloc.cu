// Total mass without any allocation by the call.
//
// fvlbm_mass keeps its block partial sums in the solver's workspace.  This
// variant keeps them in a fixed array in the library's own device memory
// instead, so a call needs no device (or host) allocation at all.  It exists
// for callers that may not allocate while they run: processes whose device
// memory is reserved up front by another allocator (a framework's caching pool
// or a fixed serving budget), and real-time loops or plugins that are not
// allowed to touch the device heap.  The paper has no counterpart.
//
// The array belongs to this file's device module.  With CUDA's default lazy
// module loading the module, and so the array, is loaded into a device's
// memory the first time the process uses it there: the first call's
// cudaGetSymbolAddress.  That first call per device can therefore allocate;
// callers make it once before the region in which they may not allocate (and
// before any stream capture).  Later calls allocate nothing.
#include <mutex>

#include <cuda_runtime.h>

#include "fvlbm_device.cuh"
#include "fvlbm_internal.h"

namespace fvlbm {

namespace {

constexpr int NA_THREADS = 256;
constexpr int64_t NA_MAX_CHUNKS = 8192;   // chunks of 4096 cells: up to 33.5 M cells
constexpr int64_t NA_MAX_INST = 4096;     // instances per solver
constexpr int NA_MAX_DEVICES = 64;

// Partial sums [NA_MAX_CHUNKS], then per-instance results [NA_MAX_INST].
// Every GPU on which the module is loaded (first call there) holds these 96 KB
// until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[NA_MAX_CHUNKS + NA_MAX_INST];

std::mutex g_setup_mutex;
double* g_scratch_ptr[NA_MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, not a device address).
int scratch_address(int device, double** out) {
    if (device < 0 || device >= NA_MAX_DEVICES) return fail(FVLBM_ERR_ARG, "device %d out of range", device);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return fail(FVLBM_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        g_scratch_ptr[device] = (double*)p;
    }
    *out = g_scratch_ptr[device];
    return FVLBM_OK;
}

// sum of A_i rho_i over each chunk of one instance, rho from the stored state
// in FP64, in the same order as the workspace reduction of fvlbm_mass
template <typename S, bool DEV>
__global__ void mass_chunks_static_kernel(DevView v, double* part) {
    __shared__ double sh[NA_THREADS];
    const int64_t ch = blockIdx.x;
    const int64_t b = v.chunk[3 * ch], e = v.chunk[3 * ch + 1];
    double s0 = 0;
    for (int64_t i = b + threadIdx.x; i < e; i += NA_THREADS) {
        double r, jx, jy;
        CellIO<S>::moments64(v.fa, i, v.inst[v.grp[i]], r, jx, jy);
        const double rho = DEV ? 1.0 + r : r;
        s0 += v.area[i] * rho;
    }
    sh[threadIdx.x] = s0;
    __syncthreads();
    for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[ch] = sh[0];
}

__global__ void mass_final_static_kernel(DevView v, const double* part, double* out) {
    const int inst = blockIdx.x * blockDim.x + threadIdx.x;
    if (inst >= v.n_inst) return;
    double s = 0;  // every call starts from zero; nothing from an earlier call is reused
    for (int64_t ch = 0; ch < v.n_chunk; ch++)
        if (v.chunk[3 * ch + 2] == inst) s += part[ch];
    out[inst] = s;
}

template <typename S, bool DEV>
void launch(const DevView& v, cudaStream_t st, double* part, double* res) {
    if (v.n_chunk > 0) mass_chunks_static_kernel<S, DEV><<<(unsigned)v.n_chunk, NA_THREADS, 0, st>>>(v, part);
    mass_final_static_kernel<<<(unsigned)((v.n_inst + 127) / 128), 128, 0, st>>>(v, part, res);
}

}  // namespace
}  // namespace fvlbm

using namespace fvlbm;

extern "C" int fvlbm_mass_noalloc(fvlbm_solver* s, double* mass) {
    clear_error();
    SolverRef r;
    if (!mass) return fail(FVLBM_ERR_ARG, "fvlbm_mass_noalloc: mass is null");
    int rc = solver_ref(s, &r);
    if (rc) return rc;
    const DevView& v = *r.view;
    if (v.n_chunk > NA_MAX_CHUNKS || v.n_inst > NA_MAX_INST)
        return fail(FVLBM_ERR_ARG,
                    "fvlbm_mass_noalloc: solver too large for the fixed scratch (%lld chunks of 4096 cells, "
                    "%d instances; limits %lld chunks = %lld cells, %lld instances)",
                    (long long)v.n_chunk, v.n_inst, (long long)NA_MAX_CHUNKS, (long long)(NA_MAX_CHUNKS * 4096),
                    (long long)NA_MAX_INST);
    DeviceGuard dg(r.device);
    if (!dg.ok) return fail(FVLBM_ERR_CUDA, "fvlbm_mass_noalloc: cannot select device %d", r.device);
    double* scratch = nullptr;
    rc = scratch_address(r.device, &scratch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)r.stream;
    double* part = scratch;
    double* res = scratch + NA_MAX_CHUNKS;
    switch (r.prec) {
        case FVLBM_FP64: launch<double, false>(v, st, part, res); break;
        case FVLBM_FP32_DEV: launch<float, true>(v, st, part, res); break;
        case FVLBM_FP16_DEV: launch<__half, true>(v, st, part, res); break;
        case FVLBM_BF16_DEV: launch<__nv_bfloat16, true>(v, st, part, res); break;
        default: return fail(FVLBM_ERR_ARG, "fvlbm_mass_noalloc: unknown precision %d", r.prec);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(mass, res, sizeof(double) * v.n_inst, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return fail(FVLBM_ERR_CUDA, "fvlbm_mass_noalloc: %s", cudaGetErrorString(e));
    return solver_sync_check(s);
}
