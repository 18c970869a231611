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
// vectors of a closed cell sum to zero), storing g in FP32, FP16 (times a
// power-of-two scale per instance and direction) or BF16.
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "fvlbm_internal.h"
#include "fvlbm_device.cuh"

namespace fvlbm {

template <typename T> __device__ __forceinline__ T inst_dt(const InstParam& p);
template <> __device__ __forceinline__ double inst_dt<double>(const InstParam& p) { return p.dt; }
template <> __device__ __forceinline__ float inst_dt<float>(const InstParam& p) { return p.dt_f; }
template <typename T> __device__ __forceinline__ T inst_inv_tau(const InstParam& p);
template <> __device__ __forceinline__ double inst_inv_tau<double>(const InstParam& p) { return p.inv_tau; }
template <> __device__ __forceinline__ float inst_inv_tau<float>(const InstParam& p) { return p.inv_tau_f; }

// ------------------------------------------------------------------ physics
// Density and velocity (Sec. 2.1).  FP64 mode: r = rho = sum f.  Deviation
// mode: r = rho - 1 = sum g, kept unrounded by the 1 so that the density
// deviation keeps FP32 relative precision.
template <typename T, bool DEV>
__device__ __forceinline__ void moments(const T* f, T& r, T& ux, T& uy) {
    T s = 0, mx = 0, my = 0;
#pragma unroll
    for (int a = 0; a < FVLBM_Q; a++) {
        s += f[a];
        mx += T(EXA(a)) * f[a];
        my += T(EYA(a)) * f[a];
    }
    r = s;
    const T rho = DEV ? T(1) + s : s;
    ux = mx / rho;
    uy = my / rho;
}

// Eq. (feq).  FP64 mode: r = rho, returns f^eq.  Deviation mode: r = rho - 1,
// returns f^eq - w = w [(rho - 1) + rho (3 e.u + 4.5 (e.u)^2 - 1.5 u^2)].
template <typename T, bool DEV>
__device__ __forceinline__ T feqs(int a, T r, T ux, T uy) {
    T eu = T(EXA(a)) * ux + T(EYA(a)) * uy;
    T uu = ux * ux + uy * uy;
    T poly = T(3) * eu + T(4.5) * eu * eu - T(1.5) * uu;
    if (DEV) return wgt<T>(a) * (r + (T(1) + r) * poly);
    return r * wgt<T>(a) * (T(1) + poly);
}

// Density argument of feqs for a given density.
template <typename T, bool DEV>
__device__ __forceinline__ T rarg(double rho) { return DEV ? T(rho - 1.0) : T(rho); }

// Stencil value minus the cell value for a boundary slot (Sec. 2.4.1):
//   wall      f^eq(rho, u_w) - f^eq(rho, u)                        Eq. (wallbc)
//   inlet     f^eq(rho*, u_inf) - f^eq(rho, u), rho* = rho_inf or rho
//   outlet    0 (external) or f^eq(rho_inf, u) - f^eq(rho, u) (internal)
//   symmetry  f^eq(rho, u*) - f, u* = u mirrored in the face line
template <typename T, bool DEV>
__device__ __forceinline__ T bc_delta(uint32_t kind, const BcParam& b, int a, T fa, T rho, T ux, T uy, T fe,
                                      T nhx, T nhy) {
    switch (kind) {
        case SK_WALL: return feqs<T, DEV>(a, rho, T(b.uwx), T(b.uwy)) - fe;
        case SK_INLET: return feqs<T, DEV>(a, b.external ? rarg<T, DEV>(b.rho_inf) : rho, T(b.uix), T(b.uiy)) - fe;
        case SK_OUTLET: return b.external ? T(0) : feqs<T, DEV>(a, rarg<T, DEV>(b.rho_inf), ux, uy) - fe;
        default: {  // symmetry
            T un = ux * nhx + uy * nhy;
            return feqs<T, DEV>(a, rho, ux - T(2) * un * nhx, uy - T(2) * un * nhy) - fa;
        }
    }
}

template <typename T>
__device__ __forceinline__ bool finite_val(T x) { return isfinite(x); }

// ------------------------------------------------------------------ kernels
template <typename T, typename S, int MAXF, bool DEV>
__global__ void __launch_bounds__(256) face_values_kernel(DevView v, const S* __restrict__ fin) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.n_cell) return;
    const int64_t np = v.np;
    const InstParam& P = v.inst[v.grp[i]];
    const T* cg = (const T*)v.cg;
    const T* rv = (const T*)v.rv;
    const T* nv = (const T*)v.nv;
    T* fv = (T*)v.fv;

    T f[FVLBM_Q];
#pragma unroll
    for (int a = 0; a < FVLBM_Q; a++) f[a] = Store<S>::ld(fin, a * np + i, P.inv_scale[a], P.off[a]);
    T rho, ux, uy;
    moments<T, DEV>(f, rho, ux, uy);

    // Step 2: gradient of f_1..f_8
    T gx[FVLBM_Q - 1], gy[FVLBM_Q - 1];
#pragma unroll
    for (int a = 0; a < FVLBM_Q - 1; a++) gx[a] = gy[a] = T(0);
#pragma unroll
    for (int k = 0; k < MAXF; k++) {
        const uint32_t meta = v.meta[k * np + i];
        const uint32_t kind = meta & 0xFF;
        if (kind == SK_NONE) continue;
        const T cx = cg[(0 * MAXF + k) * np + i], cy = cg[(1 * MAXF + k) * np + i];
        if (kind == SK_INTERIOR) {
            const int64_t j = v.nbr[k * np + i];
#pragma unroll
            for (int a = 1; a < FVLBM_Q; a++) {
                T d = Store<S>::ld(fin, a * np + j, P.inv_scale[a], P.off[a]) - f[a];
                gx[a - 1] += cx * d;
                gy[a - 1] += cy * d;
            }
        } else {
            const BcParam& b = v.bc[meta >> 16];
            T nx = nv[(0 * MAXF + k) * np + i], ny = nv[(1 * MAXF + k) * np + i];
            T inv = T(1) / sqrt(nx * nx + ny * ny);
#pragma unroll
            for (int a = 1; a < FVLBM_Q; a++) {
                T d = bc_delta<T, DEV>(kind, b, a, f[a], rho, ux, uy, feqs<T, DEV>(a, rho, ux, uy), nx * inv, ny * inv);
                gx[a - 1] += cx * d;
                gy[a - 1] += cy * d;
            }
        }
    }

    // Steps 1, 3: face values written by their upwind cell; boundary faces in full
#pragma unroll
    for (int k = 0; k < MAXF; k++) {
        const uint32_t meta = v.meta[k * np + i];
        const uint32_t kind = meta & 0xFF;
        if (kind == SK_NONE) continue;
        const uint32_t mask = (meta >> 8) & 0xFF;
        const int64_t fid = v.fid[k * np + i];
        const T rx = rv[(0 * MAXF + k) * np + i], ry = rv[(1 * MAXF + k) * np + i];
        if (kind == SK_INTERIOR) {
#pragma unroll
            for (int a = 1; a < FVLBM_Q; a++)
                if (mask & (1u << (a - 1))) fv[(a - 1) * v.n_face + fid] = f[a] + gx[a - 1] * rx + gy[a - 1] * ry;
        } else {
            const BcParam& b = v.bc[meta >> 16];
            T nx = nv[(0 * MAXF + k) * np + i], ny = nv[(1 * MAXF + k) * np + i];
            T inv = T(1) / sqrt(nx * nx + ny * ny);
#pragma unroll
            for (int a = 1; a < FVLBM_Q; a++) {
                const bool out = (mask >> (a - 1)) & 1u;
                T val;
                if (kind == SK_OUTLET && b.external) {
                    val = f[a];
                } else if ((kind == SK_INLET || kind == SK_OUTLET) && out) {
                    val = f[a] + gx[a - 1] * rx + gy[a - 1] * ry;
                } else {
                    T d = bc_delta<T, DEV>(kind, b, a, f[a], rho, ux, uy, feqs<T, DEV>(a, rho, ux, uy), nx * inv, ny * inv);
                    val = kind == SK_SYMMETRY ? f[a] + T(0.5) * d : f[a] + d;
                }
                fv[(a - 1) * v.n_face + fid] = val;
            }
        }
    }
}

template <typename T, typename S, int MAXF, bool DEV>
__global__ void __launch_bounds__(256) update_kernel(DevView v, const S* __restrict__ fin, const S* fbase, S* fout,
                                                     T beta, int mode) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.n_cell) return;
    const int64_t np = v.np;
    const InstParam& P = v.inst[v.grp[i]];
    const T* nv = (const T*)v.nv;
    const T* fv = (const T*)v.fv;

    T f[FVLBM_Q];
#pragma unroll
    for (int a = 0; a < FVLBM_Q; a++) f[a] = Store<S>::ld(fin, a * np + i, P.inv_scale[a], P.off[a]);
    T rho, ux, uy;
    moments<T, DEV>(f, rho, ux, uy);

    T flux[FVLBM_Q];
#pragma unroll
    for (int a = 0; a < FVLBM_Q; a++) flux[a] = T(0);
#pragma unroll
    for (int k = 0; k < MAXF; k++) {
        const uint32_t kind = v.meta[k * np + i] & 0xFF;
        if (kind == SK_NONE) continue;
        const int64_t fid = v.fid[k * np + i];
        const T nx = nv[(0 * MAXF + k) * np + i], ny = nv[(1 * MAXF + k) * np + i];
#pragma unroll
        for (int a = 1; a < FVLBM_Q; a++) {
            const T en = T(EXA(a)) * nx + T(EYA(a)) * ny;
            // deviation mode: the face vectors of a closed cell sum to zero, so
            // subtracting the cell value leaves the flux unchanged in exact
            // arithmetic and removes the rounding of the FP32 face vectors
            // from the constant part of g
            const T face = fv[(a - 1) * v.n_face + fid];
            flux[a] += en * (DEV ? face - f[a] : face);
        }
    }
    const T inv_tau = inst_inv_tau<T>(P);
    const T dt = inst_dt<T>(P);
    bool bad = false;
    T* rp = (T*)v.rprev;
#pragma unroll
    for (int a = 0; a < FVLBM_Q; a++) {
        const T rhs = -flux[a] - (f[a] - feqs<T, DEV>(a, rho, ux, uy)) * inv_tau;
        T out;
        if (mode == MODE_RK) {
            const T base = (fbase == fin) ? f[a] : Store<S>::ld(fbase, a * np + i, P.inv_scale[a], P.off[a]);
            out = base + beta * dt * rhs;
        } else if (mode == MODE_AB2_FIRST) {
            out = f[a] + dt * rhs;
            rp[a * np + i] = rhs;
        } else {
            out = f[a] + dt * (T(1.5) * rhs - T(0.5) * rp[a * np + i]);
            rp[a * np + i] = rhs;
        }
        bad |= !finite_val(out);
        Store<S>::st(fout, a * np + i, out, P.scale[a], P.off[a]);
    }
    if (bad) *v.flag = 1;
}

// Step 0: f = f^eq(rho0, u0) of the cell's instance.
template <typename T, typename S, bool DEV>
__global__ void init_eq_kernel(DevView v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.n_cell) return;
    const InstParam& P = v.inst[v.grp[i]];
    S* f = (S*)v.fa;
    for (int a = 0; a < FVLBM_Q; a++)
        Store<S>::st(f, a * v.np + i, feqs<T, DEV>(a, rarg<T, DEV>(P.rho0), T(P.u0x), T(P.u0y)), P.scale[a], P.off[a]);
}

// rho, u in FP64 from the stored state (Step 6).
template <typename T, typename S, bool DEV>
__global__ void macros_kernel(DevView v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.n_cell) return;
    const InstParam& P = v.inst[v.grp[i]];
    const S* f = (const S*)v.fa;
    double r = 0, mx = 0, my = 0;
    for (int a = 0; a < FVLBM_Q; a++) {
        double x = (double)Store<S>::ld(f, a * v.np + i, P.inv_scale[a], P.off[a]);
        r += x;
        mx += EXA(a) * x;
        my += EYA(a) * x;
    }
    double rho = DEV ? 1.0 + r : r;
    v.rho[i] = rho;
    v.ux[i] = mx / rho;
    v.uy[i] = my / rho;
}

// FP64 [9][np] staging <-> state.
template <typename T, typename S, bool DEV>
__global__ void get_f_kernel(DevView v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.n_cell) return;
    const InstParam& P = v.inst[v.grp[i]];
    const S* f = (const S*)v.fa;
    for (int a = 0; a < FVLBM_Q; a++) {
        double x = (double)Store<S>::ld(f, a * v.np + i, P.inv_scale[a], P.off[a]);
        v.conv[a * v.np + i] = DEV ? x + wgt<double>(a) : x;
    }
}

template <typename T, typename S, bool DEV>
__global__ void set_f_kernel(DevView v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.n_cell) return;
    const InstParam& P = v.inst[v.grp[i]];
    S* f = (S*)v.fa;
    for (int a = 0; a < FVLBM_Q; a++) {
        double x = v.conv[a * v.np + i];
        Store<S>::st(f, a * v.np + i, (T)(DEV ? x - wgt<double>(a) : x), P.scale[a], P.off[a]);
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
static inline unsigned grid_of(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

static int check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(FVLBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return FVLBM_OK;
}

template <typename T, typename S, bool DEV>
static int stage_t(const DevView& v, cudaStream_t st, const void* fin, const void* fbase, void* fout,
                   double beta, int mode, void* const* ev) {
    const unsigned g = grid_of(v.n_cell, 256);
    if (ev) cudaEventRecord((cudaEvent_t)ev[0], st);
    if (v.maxf == 4) face_values_kernel<T, S, 4, DEV><<<g, 256, 0, st>>>(v, (const S*)fin);
    else face_values_kernel<T, S, 8, DEV><<<g, 256, 0, st>>>(v, (const S*)fin);
    if (ev) cudaEventRecord((cudaEvent_t)ev[1], st);
    if (v.maxf == 4)
        update_kernel<T, S, 4, DEV><<<g, 256, 0, st>>>(v, (const S*)fin, (const S*)fbase, (S*)fout, (T)beta, mode);
    else
        update_kernel<T, S, 8, DEV><<<g, 256, 0, st>>>(v, (const S*)fin, (const S*)fbase, (S*)fout, (T)beta, mode);
    if (ev) cudaEventRecord((cudaEvent_t)ev[2], st);
    return check_launch("stage kernels");
}

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
    cudaStream_t st = (cudaStream_t)stream;
    DISPATCH_PREC(prec, return (stage_t<T, S, DEV>(v, st, fin, fbase, fout, beta, mode, ev)));
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

int launch_get_f(const DevView& v, int prec, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    DISPATCH_PREC(prec, get_f_kernel<T, S, DEV><<<grid_of(v.n_cell, 256), 256, 0, st>>>(v);
                  return check_launch("get_f kernel"));
}

int launch_set_f(const DevView& v, int prec, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    DISPATCH_PREC(prec, set_f_kernel<T, S, DEV><<<grid_of(v.n_cell, 256), 256, 0, st>>>(v);
                  return check_launch("set_f kernel"));
}

int launch_reduce(const DevView& v, void* stream, int what) {
    cudaStream_t st = (cudaStream_t)stream;
    if (v.n_chunk > 0) reduce_chunks_kernel<<<(unsigned)v.n_chunk, RED_THREADS, 0, st>>>(v, what);
    reduce_final_kernel<<<grid_of(v.n_inst, 128), 128, 0, st>>>(v);
    return check_launch("reduction kernels");
}

}  // namespace fvlbm
