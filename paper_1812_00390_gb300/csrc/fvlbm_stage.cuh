// Templated CUDA kernels of one FVLBM stage (included by one translation unit
// per precision so that the build compiles them in parallel).
#pragma once

#include "fvlbm_device.cuh"
#include "fvlbm_internal.h"

namespace fvlbm {

template <typename T> __device__ __forceinline__ T inst_dt(const InstParam& p);
template <> __device__ __forceinline__ double inst_dt<double>(const InstParam& p) { return p.dt; }
template <> __device__ __forceinline__ float inst_dt<float>(const InstParam& p) { return p.dt_f; }
template <typename T> __device__ __forceinline__ T inst_inv_tau(const InstParam& p);
template <> __device__ __forceinline__ double inst_inv_tau<double>(const InstParam& p) { return p.inv_tau; }
template <> __device__ __forceinline__ float inst_inv_tau<float>(const InstParam& p) { return p.inv_tau_f; }

// ------------------------------------------------------------------ physics
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
    CellIO<S>::template load<T, DEV>(fin, i, np, P, f);
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
            T fj[FVLBM_Q];
            CellIO<S>::template load<T, DEV>(fin, j, np, v.inst[v.grp[j]], fj);
#pragma unroll
            for (int a = 1; a < FVLBM_Q; a++) {
                T d = fj[a] - f[a];
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
    CellIO<S>::template load<T, DEV>(fin, i, np, P, f);
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
    T fb[FVLBM_Q], out[FVLBM_Q];
    if (mode == MODE_RK && fbase != fin) CellIO<S>::template load<T, DEV>(fbase, i, np, P, fb);
#pragma unroll
    for (int a = 0; a < FVLBM_Q; a++) {
        const T rhs = -flux[a] - (f[a] - feqs<T, DEV>(a, rho, ux, uy)) * inv_tau;
        if (mode == MODE_RK) {
            out[a] = (fbase == fin ? f[a] : fb[a]) + beta * dt * rhs;
        } else if (mode == MODE_AB2_FIRST) {
            out[a] = f[a] + dt * rhs;
            rp[a * np + i] = rhs;
        } else {
            out[a] = f[a] + dt * (T(1.5) * rhs - T(0.5) * rp[a * np + i]);
            rp[a * np + i] = rhs;
        }
        bad |= !finite_val(out[a]);
    }
    CellIO<S>::template store<T, DEV>(fout, i, np, P, out);
    if (bad) *v.flag = 1;
}

// Fused stage: one CTA per tile of TILE consecutive cells (Hilbert order).
//   phase 1  f of the tile, its 1-ring and its 2-ring into shared memory
//   phase 2  gradients (Eq. leastsquare) of the tile and 1-ring cells, kept in
//            shared memory
//   phase 3  per tile cell: face values (Eq. lslrflux / Sec. 2.4.2) from the
//            upwind side -- its own gradient, or the neighbour's from shared
//            memory -- flux sum, collision and time update (Eq. rhs, Sec. 2.3)
// Each face value is evaluated by both cells of the face from the same data,
// so no face-value array goes through memory.
template <typename T, typename S, int MAXF, bool DEV, int TILE>
__global__ void __launch_bounds__(TILE) stage_tile_kernel(DevView v, const S* __restrict__ fin,
                                                          const S* fbase, S* fout, T beta, int mode) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lmax = v.lmax, gmax = v.gmax;
    T* fs = (T*)smem_raw;            // [9][lmax]
    T* gxs = fs + FVLBM_Q * lmax;    // [8][gmax]
    T* gys = gxs + (FVLBM_Q - 1) * gmax;
    const int64_t np = v.np;
    const int64_t t = blockIdx.x;
    const int64_t c0 = t * TILE;
    const int nt = (int)min((int64_t)TILE, v.n_cell - c0);
    const int64_t h0 = v.halo_ptr[t];
    const int nh = (int)(v.halo_ptr[t + 1] - h0);
    const int n1 = v.n_r1[t];
    const int nl = nt + nh;
    const T* cg = (const T*)v.cg;
    const T* rv = (const T*)v.rv;
    const T* rn = (const T*)v.rn;
    const T* nv = (const T*)v.nv;

    // phase 1
    for (int l = threadIdx.x; l < nl; l += TILE) {
        const int64_t gi = l < nt ? c0 + l : (int64_t)v.halo[h0 + l - nt];
        T f[FVLBM_Q];
        CellIO<S>::template load<T, DEV>(fin, gi, np, v.inst[v.grp[gi]], f);
#pragma unroll
        for (int a = 0; a < FVLBM_Q; a++) fs[a * lmax + l] = f[a];
    }
    __syncthreads();

    // phase 2
    for (int l = threadIdx.x; l < nt + n1; l += TILE) {
        const bool own = l < nt;
        const int64_t gi = own ? c0 + l : (int64_t)v.halo[h0 + l - nt];
        T f[FVLBM_Q];
#pragma unroll
        for (int a = 0; a < FVLBM_Q; a++) f[a] = fs[a * lmax + l];
        T rho, ux, uy;
        moments<T, DEV>(f, rho, ux, uy);
        T gx[FVLBM_Q - 1], gy[FVLBM_Q - 1];
#pragma unroll
        for (int a = 0; a < FVLBM_Q - 1; a++) gx[a] = gy[a] = T(0);
#pragma unroll
        for (int k = 0; k < MAXF; k++) {
            const uint32_t meta = v.meta[k * np + gi];
            const uint32_t kind = meta & 0xFF;
            if (kind == SK_NONE) continue;
            const T cx = cg[(0 * MAXF + k) * np + gi], cy = cg[(1 * MAXF + k) * np + gi];
            if (kind == SK_INTERIOR) {
                const int lj = own ? (int)v.lnbr[k * np + gi] : (int)v.r1nbr[(h0 + l - nt) * MAXF + k];
#pragma unroll
                for (int a = 1; a < FVLBM_Q; a++) {
                    const T d = fs[a * lmax + lj] - f[a];
                    gx[a - 1] += cx * d;
                    gy[a - 1] += cy * d;
                }
            } else {
                const BcParam& b = v.bc[meta >> 16];
                const T nx = nv[(0 * MAXF + k) * np + gi], ny = nv[(1 * MAXF + k) * np + gi];
                const T inv = T(1) / sqrt(nx * nx + ny * ny);
#pragma unroll
                for (int a = 1; a < FVLBM_Q; a++) {
                    const T d = bc_delta<T, DEV>(kind, b, a, f[a], rho, ux, uy, feqs<T, DEV>(a, rho, ux, uy),
                                                 nx * inv, ny * inv);
                    gx[a - 1] += cx * d;
                    gy[a - 1] += cy * d;
                }
            }
        }
#pragma unroll
        for (int a = 0; a < FVLBM_Q - 1; a++) {
            gxs[a * gmax + l] = gx[a];
            gys[a * gmax + l] = gy[a];
        }
    }
    __syncthreads();

    // phase 3
    const int l = threadIdx.x;
    if (l >= nt) return;
    const int64_t gi = c0 + l;
    const InstParam& P = v.inst[v.grp[gi]];
    T f[FVLBM_Q];
#pragma unroll
    for (int a = 0; a < FVLBM_Q; a++) f[a] = fs[a * lmax + l];
    T rho, ux, uy;
    moments<T, DEV>(f, rho, ux, uy);
    T flux[FVLBM_Q];
#pragma unroll
    for (int a = 0; a < FVLBM_Q; a++) flux[a] = T(0);
#pragma unroll
    for (int k = 0; k < MAXF; k++) {
        const uint32_t meta = v.meta[k * np + gi];
        const uint32_t kind = meta & 0xFF;
        if (kind == SK_NONE) continue;
        const uint32_t mask = (meta >> 8) & 0xFF;
        const T nx = nv[(0 * MAXF + k) * np + gi], ny = nv[(1 * MAXF + k) * np + gi];
        const T rx = rv[(0 * MAXF + k) * np + gi], ry = rv[(1 * MAXF + k) * np + gi];
        if (kind == SK_INTERIOR) {
            const int lj = (int)v.lnbr[k * np + gi];
            const T sx = rn[(0 * MAXF + k) * np + gi], sy = rn[(1 * MAXF + k) * np + gi];
#pragma unroll
            for (int a = 1; a < FVLBM_Q; a++) {
                const T en = T(EXA(a)) * nx + T(EYA(a)) * ny;
                T face;
                if (mask & (1u << (a - 1)))
                    face = f[a] + gxs[(a - 1) * gmax + l] * rx + gys[(a - 1) * gmax + l] * ry;
                else
                    face = fs[a * lmax + lj] + gxs[(a - 1) * gmax + lj] * sx + gys[(a - 1) * gmax + lj] * sy;
                flux[a] += en * (DEV ? face - f[a] : face);
            }
        } else {
            const BcParam& b = v.bc[meta >> 16];
            const T inv = T(1) / sqrt(nx * nx + ny * ny);
#pragma unroll
            for (int a = 1; a < FVLBM_Q; a++) {
                const bool out = (mask >> (a - 1)) & 1u;
                T face;
                if (kind == SK_OUTLET && b.external) {
                    face = f[a];
                } else if ((kind == SK_INLET || kind == SK_OUTLET) && out) {
                    face = f[a] + gxs[(a - 1) * gmax + l] * rx + gys[(a - 1) * gmax + l] * ry;
                } else {
                    const T d = bc_delta<T, DEV>(kind, b, a, f[a], rho, ux, uy, feqs<T, DEV>(a, rho, ux, uy),
                                                 nx * inv, ny * inv);
                    face = kind == SK_SYMMETRY ? f[a] + T(0.5) * d : f[a] + d;
                }
                const T en = T(EXA(a)) * nx + T(EYA(a)) * ny;
                flux[a] += en * (DEV ? face - f[a] : face);
            }
        }
    }
    const T inv_tau = inst_inv_tau<T>(P);
    const T dt = inst_dt<T>(P);
    bool bad = false;
    T* rp = (T*)v.rprev;
    T fb[FVLBM_Q], outv[FVLBM_Q];
    if (mode == MODE_RK && fbase != fin) CellIO<S>::template load<T, DEV>(fbase, gi, np, P, fb);
#pragma unroll
    for (int a = 0; a < FVLBM_Q; a++) {
        const T rhs = -flux[a] - (f[a] - feqs<T, DEV>(a, rho, ux, uy)) * inv_tau;
        if (mode == MODE_RK) {
            outv[a] = (fbase == fin ? f[a] : fb[a]) + beta * dt * rhs;
        } else if (mode == MODE_AB2_FIRST) {
            outv[a] = f[a] + dt * rhs;
            rp[a * np + gi] = rhs;
        } else {
            outv[a] = f[a] + dt * (T(1.5) * rhs - T(0.5) * rp[a * np + gi]);
            rp[a * np + gi] = rhs;
        }
        bad |= !finite_val(outv[a]);
    }
    CellIO<S>::template store<T, DEV>(fout, gi, np, P, outv);
    if (bad) *v.flag = 1;
}


static inline unsigned grid_of(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

static inline int check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(FVLBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return FVLBM_OK;
}

template <typename T, typename S, int MAXF, bool DEV, int TILE>
static int tile_launch(const DevView& v, cudaStream_t st, const void* fin, const void* fbase, void* fout,
                       double beta, int mode) {
    auto kern = stage_tile_kernel<T, S, MAXF, DEV, TILE>;
    const size_t smem = tile_smem_bytes(v, sizeof(T));
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return fail(FVLBM_ERR_CUDA, "fused stage: %zu B shared memory: %s", smem, cudaGetErrorString(e));
    }
    kern<<<(unsigned)v.n_tiles, TILE, smem, st>>>(v, (const S*)fin, (const S*)fbase, (S*)fout, (T)beta, mode);
    return FVLBM_OK;
}

template <typename T, typename S, int MAXF, bool DEV>
static int tile_dispatch(const DevView& v, cudaStream_t st, const void* fin, const void* fbase, void* fout,
                         double beta, int mode) {
    switch (v.tile) {
        case 128: return tile_launch<T, S, MAXF, DEV, 128>(v, st, fin, fbase, fout, beta, mode);
        case 256: return tile_launch<T, S, MAXF, DEV, 256>(v, st, fin, fbase, fout, beta, mode);
        case 512: return tile_launch<T, S, MAXF, DEV, 512>(v, st, fin, fbase, fout, beta, mode);
        case 1024: return tile_launch<T, S, MAXF, DEV, 1024>(v, st, fin, fbase, fout, beta, mode);
    }
    return fail(FVLBM_ERR_ARG, "unsupported tile size %d", v.tile);
}

template <typename T, typename S, bool DEV>
static int stage_t(const DevView& v, cudaStream_t st, const void* fin, const void* fbase, void* fout,
                   double beta, int mode, void* const* ev) {
    if (ev) cudaEventRecord((cudaEvent_t)ev[0], st);
    if (v.strategy == STRATEGY_TILE) {
        int rc = v.maxf == 4 ? tile_dispatch<T, S, 4, DEV>(v, st, fin, fbase, fout, beta, mode)
                             : tile_dispatch<T, S, 8, DEV>(v, st, fin, fbase, fout, beta, mode);
        if (rc) return rc;
        if (ev) {
            cudaEventRecord((cudaEvent_t)ev[1], st);
            cudaEventRecord((cudaEvent_t)ev[2], st);
        }
        return check_launch("fused stage kernel");
    }
    const int bs = v.block > 0 ? v.block : 256;   // smaller blocks spread small meshes over all SMs
    const unsigned g = grid_of(v.n_cell, bs);
    if (v.maxf == 4) face_values_kernel<T, S, 4, DEV><<<g, bs, 0, st>>>(v, (const S*)fin);
    else face_values_kernel<T, S, 8, DEV><<<g, bs, 0, st>>>(v, (const S*)fin);
    if (ev) cudaEventRecord((cudaEvent_t)ev[1], st);
    if (v.maxf == 4)
        update_kernel<T, S, 4, DEV><<<g, bs, 0, st>>>(v, (const S*)fin, (const S*)fbase, (S*)fout, (T)beta, mode);
    else
        update_kernel<T, S, 8, DEV><<<g, bs, 0, st>>>(v, (const S*)fin, (const S*)fbase, (S*)fout, (T)beta, mode);
    if (ev) cudaEventRecord((cudaEvent_t)ev[2], st);
    return check_launch("stage kernels");
}

}  // namespace fvlbm
