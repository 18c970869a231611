// CUDA kernels of one FVLBM stage (sm_103a).
//
// One stage evaluates RHS(f) of Eq. (rhs) and applies one update of the time
// scheme (Sec. 2.3).  It runs as two deterministic per-cell gathers (no
// atomics):
//
//  face_values   Steps 1-3.  Per cell: rho, u (Sec. 2.1), boundary ghost /
//                wall values (Sec. 2.4.1, Eq. wallbc), the weighted
//                least-squares gradient of f_1..f_8 (Eq. leastsquare, with
//                precomputed coefficients), then the face value of every
//                (face, direction) for which this cell is the upwind side
//                (Eq. lslrflux), and every direction of its boundary faces
//                (Sec. 2.4.2).  Each (face, direction) has exactly one writer.
//  update        Steps 4-5.  Per cell: flux sum -sum_m (e.n dl / A) f_m
//                over its faces, BGK collision -(f - f^eq)/tau with f^eq of
//                the same stage state, and out = base + beta dt RHS (or the
//                AB2 combination).
//
// Precision modes: FP64 keeps f; the deviation modes keep g = f - w and do all
// arithmetic in FP32 (the flux of the constant w vanishes because the face
// vectors of a closed cell sum to zero).  FP32 stores g itself; the 16-bit
// modes store the split format of fvlbm_device.cuh: rho - 1 and rho u in FP32
// and the non-equilibrium parts of directions 3..8 in FP16 or BF16, times a
// power-of-two scale per (instance, direction).
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "fvlbm_internal.h"
#include "fvlbm_device.cuh"
#include "fvlbm_stage.cuh"

namespace fvlbm {

// Step 0: f = f^eq(rho0, u0) of the cell's instance.
template <typename T, typename S, bool DEV>
__global__ void init_eq_kernel(DevView v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.n_cell) return;
    const InstParam& P = v.inst[v.grp[i]];
    T f[FVLBM_Q];
    for (int a = 0; a < FVLBM_Q; a++) f[a] = feqs<T, DEV>(a, rarg<T, DEV>(P.rho0), T(P.u0x), T(P.u0y));
    CellIO<S>::template store<T, DEV>(v.fa, i, P, f);
}

// rho, u in FP64 from the stored state (Step 6).
template <typename T, typename S, bool DEV>
__global__ void macros_kernel(DevView v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.n_cell) return;
    double r, mx, my;
    CellIO<S>::moments64(v.fa, i, v.inst[v.grp[i]], r, mx, my);
    double rho = DEV ? 1.0 + r : r;
    v.rho[i] = rho;
    v.ux[i] = mx / rho;
    v.uy[i] = my / rho;
}

// f and rho, u in the caller's cell order, [n_cell][9] (get / set) or
// [n_cell] and [n_cell][2] (macros), in a buffer the device reaches: for set
// the caller's host buffer itself when the GPU reads pageable host memory,
// otherwise (and for get and macros) the device staging buffer v.conv that one
// copy fills or empties.  One thread per caller cell c.  get / set pass a
// block's ORDERED_CELLS x 9 doubles through shared memory, so that every warp
// access to the caller's buffer covers 32 consecutive doubles (a per-thread
// row of 9 would touch each host line once per direction).
constexpr int ORDERED_CELLS = 256;

template <typename T, typename S, bool DEV>
__global__ void __launch_bounds__(ORDERED_CELLS) get_f_ordered_kernel(DevView v, double* __restrict__ out) {
    __shared__ double buf[ORDERED_CELLS * FVLBM_Q];
    const int64_t c0 = (int64_t)blockIdx.x * ORDERED_CELLS;
    const int64_t c = c0 + threadIdx.x;
    if (c < v.n_cell) {
        const int64_t i = v.iperm[c];
        T f[FVLBM_Q];
        CellIO<S>::template load<T, DEV>(v.fa, i, v.inst[v.grp[i]], f);
        for (int a = 0; a < FVLBM_Q; a++)
            buf[threadIdx.x * FVLBM_Q + a] = DEV ? (double)f[a] + wgt<double>(a) : (double)f[a];
    }
    __syncthreads();
    const int nw = (int)(v.n_cell - c0 < ORDERED_CELLS ? v.n_cell - c0 : ORDERED_CELLS) * FVLBM_Q;
    for (int w = threadIdx.x; w < nw; w += ORDERED_CELLS) out[c0 * FVLBM_Q + w] = buf[w];
}

template <typename T, typename S, bool DEV>
__global__ void __launch_bounds__(ORDERED_CELLS) set_f_ordered_kernel(DevView v, const double* __restrict__ in) {
    __shared__ double buf[ORDERED_CELLS * FVLBM_Q];
    const int64_t c0 = (int64_t)blockIdx.x * ORDERED_CELLS;
    const int nw = (int)(v.n_cell - c0 < ORDERED_CELLS ? v.n_cell - c0 : ORDERED_CELLS) * FVLBM_Q;
    for (int w = threadIdx.x; w < nw; w += ORDERED_CELLS) buf[w] = in[c0 * FVLBM_Q + w];
    __syncthreads();
    const int64_t c = c0 + threadIdx.x;
    if (c >= v.n_cell) return;
    const int64_t i = v.iperm[c];
    T f[FVLBM_Q];
    for (int a = 0; a < FVLBM_Q; a++) {
        const double x = buf[threadIdx.x * FVLBM_Q + a];
        f[a] = (T)(DEV ? x - wgt<double>(a) : x);
    }
    CellIO<S>::template store<T, DEV>(v.fa, i, v.inst[v.grp[i]], f);
}

template <typename T, typename S, bool DEV>
__global__ void macros_ordered_kernel(DevView v, double* __restrict__ rho_out, double* __restrict__ u_out) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= v.n_cell) return;
    const int64_t i = v.iperm[c];
    double r, mx, my;
    CellIO<S>::moments64(v.fa, i, v.inst[v.grp[i]], r, mx, my);
    const double rho = DEV ? 1.0 + r : r;
    if (rho_out) rho_out[c] = rho;
    if (u_out) {
        u_out[2 * c] = mx / rho;
        u_out[2 * c + 1] = my / rho;
    }
}

// Deterministic FP64 reductions: one block per chunk of one instance, fixed
// tree order; then one thread per instance sums its chunks in order.
constexpr int RED_THREADS = 256;

__global__ void reduce_chunks_kernel(DevView v, int what) {
    __shared__ double sh[3][RED_THREADS];
    const int64_t ch = blockIdx.x;
    const int64_t b = v.chunk[3 * ch], e = v.chunk[3 * ch + 1];
    double s0 = 0, s1 = 0, s2 = 0;
    for (int64_t i = b + threadIdx.x; i < e; i += RED_THREADS) {
        if (what == RED_MASS) {
            s0 += v.area[i] * v.rho[i];
        } else {
            double ox = v.uold[i], oy = v.uold[v.np + i];
            double dx = v.ux[i] - ox, dy = v.uy[i] - oy;
            s0 += dx * dx + dy * dy;
            s1 += ox * ox + oy * oy;
            v.uold[i] = v.ux[i];
            v.uold[v.np + i] = v.uy[i];
        }
    }
    sh[0][threadIdx.x] = s0;
    sh[1][threadIdx.x] = s1;
    sh[2][threadIdx.x] = s2;
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int q = 0; q < 3; q++) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; q++) v.part[3 * ch + q] = sh[q][0];
}

__global__ void reduce_final_kernel(DevView v) {
    const int inst = blockIdx.x * blockDim.x + threadIdx.x;
    if (inst >= v.n_inst) return;
    double s[3] = {0, 0, 0};
    for (int64_t ch = 0; ch < v.n_chunk; ch++)
        if (v.chunk[3 * ch + 2] == inst)
            for (int q = 0; q < 3; q++) s[q] += v.part[3 * ch + q];
    for (int q = 0; q < 3; q++) v.red[3 * inst + q] = s[q];
}

// ------------------------------------------------------------------ launchers
#define DISPATCH_PREC(prec, ...)                                            \
    switch (prec) {                                                          \
        case FVLBM_FP64: { typedef double T; typedef double S; const bool DEV = false; __VA_ARGS__; } \
        case FVLBM_FP32_DEV: { typedef float T; typedef float S; const bool DEV = true; __VA_ARGS__; } \
        case FVLBM_FP16_DEV: { typedef float T; typedef __half S; const bool DEV = true; __VA_ARGS__; } \
        case FVLBM_BF16_DEV: { typedef float T; typedef __nv_bfloat16 S; const bool DEV = true; __VA_ARGS__; } \
        default: return fail(FVLBM_ERR_ARG, "unknown precision %d", prec); \
    }

int launch_stage(const DevView& v, int prec, void* stream, const void* fin, const void* fbase, void* fout,
                 double beta, int mode, void* const* ev) {
    switch (prec) {
        case FVLBM_FP64: return stage_fp64(v, stream, fin, fbase, fout, beta, mode, ev);
        case FVLBM_FP32_DEV: return stage_fp32(v, stream, fin, fbase, fout, beta, mode, ev);
        case FVLBM_FP16_DEV: return stage_fp16(v, stream, fin, fbase, fout, beta, mode, ev);
        case FVLBM_BF16_DEV: return stage_bf16(v, stream, fin, fbase, fout, beta, mode, ev);
    }
    return fail(FVLBM_ERR_ARG, "unknown precision %d", prec);
}

int launch_init_eq(const DevView& v, int prec, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    DISPATCH_PREC(prec, init_eq_kernel<T, S, DEV><<<grid_of(v.n_cell, 256), 256, 0, st>>>(v);
                  return check_launch("init kernel"));
}

int launch_macros(const DevView& v, int prec, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    DISPATCH_PREC(prec, macros_kernel<T, S, DEV><<<grid_of(v.n_cell, 256), 256, 0, st>>>(v);
                  return check_launch("macros kernel"));
}

int launch_reduce(const DevView& v, void* stream, int what) {
    cudaStream_t st = (cudaStream_t)stream;
    if (v.n_chunk > 0) reduce_chunks_kernel<<<(unsigned)v.n_chunk, RED_THREADS, 0, st>>>(v, what);
    reduce_final_kernel<<<grid_of(v.n_inst, 128), 128, 0, st>>>(v);
    return check_launch("reduction kernels");
}

}  // namespace fvlbm

// ------------------------------------------------------------------ FMA peak
// Dependent FMA chains, 8 per thread, enough warps to fill every SM: the
// sustained FMA rate of the device in FP64 or FP32 (2 flop per FMA).
namespace fvlbm {
template <typename T>
__global__ void fma_peak_kernel(T* out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = (T)(threadIdx.x + k);
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = x[k] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) s += x[k];
    if (s == (T)-1) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}
}  // namespace fvlbm

extern "C" int fvlbm_fma_peak(int32_t device, int32_t fp64, double* tflops) {
    using namespace fvlbm;
    clear_error();
    if (!tflops) return fail(FVLBM_ERR_ARG, "fvlbm_fma_peak: null output");
    int prev = -1;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return fail(FVLBM_ERR_UNSUPPORTED, "no CUDA device %d", device);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int threads = 256, blocks = sms * 8, iters = fp64 ? 2048 : 16384;
    void* out = nullptr;
    cudaEvent_t e0, e1;
    int rc = FVLBM_OK;
    if (cudaMalloc(&out, sizeof(double) * threads * blocks) != cudaSuccess) rc = fail(FVLBM_ERR_OOM, "fma peak buffer");
    if (!rc) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        for (int rep = 0; rep < 4; rep++) {
            cudaEventRecord(e0);
            if (fp64) fma_peak_kernel<double><<<blocks, threads>>>((double*)out, iters, 0.999999, 1e-7);
            else fma_peak_kernel<float><<<blocks, threads>>>((float*)out, iters, 0.999999f, 1e-7f);
            cudaEventRecord(e1);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = fail(FVLBM_ERR_CUDA, "fma peak: %s", cudaGetErrorString(e));
        else *tflops = 2.0 * 8.0 * iters * (double)threads * blocks / (best * 1e-3) / 1e12;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(out);
    }
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
}

namespace fvlbm {
int launch_get_f_ordered(const DevView& v, int prec, void* stream, double* f) {
    cudaStream_t st = (cudaStream_t)stream;
    DISPATCH_PREC(prec, get_f_ordered_kernel<T, S, DEV><<<grid_of(v.n_cell, ORDERED_CELLS), ORDERED_CELLS, 0, st>>>(v, f);
                  return check_launch("get_f kernel"));
}

int launch_set_f_ordered(const DevView& v, int prec, void* stream, const double* f) {
    cudaStream_t st = (cudaStream_t)stream;
    DISPATCH_PREC(prec, set_f_ordered_kernel<T, S, DEV><<<grid_of(v.n_cell, ORDERED_CELLS), ORDERED_CELLS, 0, st>>>(v, f);
                  return check_launch("set_f kernel"));
}

int launch_macros_ordered(const DevView& v, int prec, void* stream, double* rho, double* u) {
    cudaStream_t st = (cudaStream_t)stream;
    DISPATCH_PREC(prec, macros_ordered_kernel<T, S, DEV><<<grid_of(v.n_cell, 256), 256, 0, st>>>(v, rho, u);
                  return check_launch("macros kernel"));
}
}  // namespace fvlbm
