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
// Ghost state of a boundary slot (Sec. 2.4.1): the stencil value of direction
// a minus the cell value is
//   wall      f^eq(rho, u_w) - f^eq(rho, u)                        Eq. (wallbc)
//   inlet     f^eq(rho*, u_inf) - f^eq(rho, u), rho* = rho_inf (external) or rho
//   outlet    0 (external) or f^eq(rho_inf, u) - f^eq(rho, u) (internal)
//   symmetry  f^eq(rho, u*) - f_a, u* = u mirrored in the face line
// i.e. f^eq(r, u_g) minus f^eq(rho, u) (or f_a for symmetry), with the ghost
// density / velocity (r, u_g) found once per slot.
template <typename T> struct Ghost {
    T r, ux, uy;
    bool zero;    // external outlet: no difference
    bool sym;     // symmetry: subtract f_a
    bool io;      // inlet / internal outlet: faces the cell flows out through are reconstructed
};

// Boundary constants in the arithmetic type (FP32: rounded on the host).
template <typename T> struct BcVal;
template <> struct BcVal<double> {
    static __device__ __forceinline__ double uwx(const BcParam& b) { return b.uwx; }
    static __device__ __forceinline__ double uwy(const BcParam& b) { return b.uwy; }
    static __device__ __forceinline__ double uix(const BcParam& b) { return b.uix; }
    static __device__ __forceinline__ double uiy(const BcParam& b) { return b.uiy; }
    template <bool DEV> static __device__ __forceinline__ double rho(const BcParam& b) { return rarg<double, DEV>(b.rho_inf); }
};
template <> struct BcVal<float> {
    static __device__ __forceinline__ float uwx(const BcParam& b) { return b.uwx_f; }
    static __device__ __forceinline__ float uwy(const BcParam& b) { return b.uwy_f; }
    static __device__ __forceinline__ float uix(const BcParam& b) { return b.uix_f; }
    static __device__ __forceinline__ float uiy(const BcParam& b) { return b.uiy_f; }
    template <bool DEV> static __device__ __forceinline__ float rho(const BcParam& b) { return DEV ? b.rdev_f : b.rho_f; }
};

template <typename T, bool DEV, typename NormalFn>
__device__ __forceinline__ Ghost<T> ghost_state(uint32_t kind, const BcParam& b, T rho, T ux, T uy, NormalFn normal) {
    Ghost<T> g{rho, ux, uy, false, false, false};
    if (kind == SK_WALL) {
        g.ux = BcVal<T>::uwx(b);
        g.uy = BcVal<T>::uwy(b);
    } else if (kind == SK_INLET) {
        if (b.external) g.r = BcVal<T>::template rho<DEV>(b);
        g.ux = BcVal<T>::uix(b);
        g.uy = BcVal<T>::uiy(b);
        g.io = true;
    } else if (kind == SK_OUTLET) {
        if (b.external) {
            g.zero = true;
        } else {
            g.r = BcVal<T>::template rho<DEV>(b);
            g.io = true;
        }
    } else {   // symmetry: the face's unit normal is needed only here
        const typename Vec2<T>::type n = normal();
        const T inv = T(1) / sqrt(n.x * n.x + n.y * n.y);
        const T nhx = n.x * inv, nhy = n.y * inv;
        const T un = ux * nhx + uy * nhy;
        g.ux = ux - T(2) * un * nhx;
        g.uy = uy - T(2) * un * nhy;
        g.sym = true;
    }
    return g;
}

// Stencil value minus cell value of direction a (fe = f^eq_a(rho, u)).
template <typename T, bool DEV>
__device__ __forceinline__ T ghost_delta(const Ghost<T>& g, int a, T fa, T fe) {
    if (g.zero) return T(0);
    return feqs<T, DEV>(a, g.r, g.ux, g.uy) - (g.sym ? fa : fe);
}

template <typename T>
__device__ __forceinline__ bool finite_val(T x) { return isfinite(x); }

// rho, u of a cell for its boundary slots (ghost states); cells with interior
// slots only do not need them before the collision.
template <typename T, bool DEV, int MAXF>
__device__ __forceinline__ void boundary_moments(const uint2* d, const T* f, T& rho, T& ux, T& uy) {
    bool bc = false;
#pragma unroll
    for (int k = 0; k < MAXF; k++) bc |= (d[k].x & 0xFF) > SK_INTERIOR;
    rho = ux = uy = T(0);
    if (bc) moments<T, DEV>(f, rho, ux, uy);
}

// Least-squares gradient (Eq. leastsquare) of f_1..f_8 of one cell from the
// differences to its stencil values.  d: the cell's slot descriptors;
// fnb(k, fj) fills fj[1..8] with the neighbour values across interior slot k.
// On boundary slots it also writes the face values that are ghost values
// (Sec. 2.4.2: all directions of walls, symmetry planes and external outlets,
// inflow directions of inlets and internal outlets; half way to the ghost for
// symmetry) into face(k) (stride `stride`; null: not written).
template <typename T, bool DEV, int MAXF, typename Geo, typename Nb, typename Row>
__device__ __forceinline__ void lsq_gradient(const uint2* d, const Geo& G, const BcParam* bcs, const T* f,
                                             T rho, T ux, T uy, T* gx, T* gy, Nb fnb, int64_t stride, Row face) {
#pragma unroll
    for (int a = 0; a < FVLBM_Q - 1; a++) gx[a] = gy[a] = T(0);
#pragma unroll
    for (int k = 0; k < MAXF; k++) {
        const uint32_t kind = d[k].x & 0xFF;
        if (kind == SK_NONE) continue;
        const typename Vec2<T>::type c = G.cg(k);
        if (kind == SK_INTERIOR) {
            T fj[FVLBM_Q];
            fnb(k, fj);
#pragma unroll
            for (int a = 1; a < FVLBM_Q; a++) {
                const T dd = fj[a] - f[a];
                gx[a - 1] += c.x * dd;
                gy[a - 1] += c.y * dd;
            }
        } else {
            // the ghost difference enters the gradient and, for every direction
            // not reconstructed from the gradient, gives the face value at once
            const Ghost<T> g = ghost_state<T, DEV>(kind, bcs[d[k].x >> 16], rho, ux, uy, [&] { return G.nv(k); });
            const uint32_t mask = (d[k].x >> 8) & 0xFF;
            T* fo = face(k);
#pragma unroll
            for (int a = 1; a < FVLBM_Q; a++) {
                const T dd = ghost_delta<T, DEV>(g, a, f[a], feqs<T, DEV>(a, rho, ux, uy));
                gx[a - 1] += c.x * dd;
                gy[a - 1] += c.y * dd;
                if (fo && !(g.io && ((mask >> (a - 1)) & 1u)))
                    fo[(a - 1) * stride] = g.sym ? f[a] + T(0.5) * dd : f[a] + dd;
            }
        }
    }
}

// Values of one cell on its faces (Eq. lslrflux, Sec. 2.4.2) into a face
// table with direction stride `stride`: on interior faces the directions in
// the slot's writer mask; on inlet and internal-outlet faces the directions
// the cell flows out through (the reconstruction f_i + grad f_i . r; every
// other boundary face value is the ghost value, written by lsq_gradient).
// face(k) is the slot's row in the table, or null to skip the slot.
template <typename T, bool DEV, int MAXF, typename Geo, typename Row>
__device__ __forceinline__ void write_faces(const uint2* d, const Geo& G, const BcParam* bcs, const T* f,
                                            T rho, T ux, T uy, const T* gx, const T* gy, int64_t stride, Row face) {
#pragma unroll
    for (int k = 0; k < MAXF; k++) {
        const uint32_t kind = d[k].x & 0xFF;
        if (kind == SK_NONE) continue;
        T* fo = face(k);
        if (!fo) continue;
        const uint32_t mask = (d[k].x >> 8) & 0xFF;
        const typename Vec2<T>::type r = G.rv(k);
        if (kind == SK_INTERIOR) {
#pragma unroll
            for (int a = 1; a < FVLBM_Q; a++)
                if (mask & (1u << (a - 1))) fo[(a - 1) * stride] = f[a] + gx[a - 1] * r.x + gy[a - 1] * r.y;
        } else {
            // inlet / internal outlet: directions the cell flows out through
            // take the reconstruction (the others were written with the gradient)
            const BcParam& b = bcs[d[k].x >> 16];
            if (kind == SK_INLET || (kind == SK_OUTLET && !b.external)) {
#pragma unroll
                for (int a = 1; a < FVLBM_Q; a++)
                    if ((mask >> (a - 1)) & 1u) fo[(a - 1) * stride] = f[a] + gx[a - 1] * r.x + gy[a - 1] * r.y;
            }
        }
    }
}

// Flux sum of Eq. (rhs) from a face table: sum over the slots of
// (e_a . n dl / A) f_face (deviation mode: of f_face - f_a, the same in exact
// arithmetic because the face vectors of a closed cell sum to zero, without
// the rounding of the FP32 face vectors acting on the constant part of g).
// face(k, fa) fills fa[0..7] with the values of directions 1..8 on slot k.
template <typename T, bool DEV, int MAXF, typename Face>
__device__ __forceinline__ void flux_sum(const uint2* d, const typename Vec2<T>::type* n, const T* f, T* flux,
                                         Face face) {
#pragma unroll
    for (int a = 0; a < FVLBM_Q; a++) flux[a] = T(0);
#pragma unroll
    for (int k = 0; k < MAXF; k++) {
        if ((d[k].x & 0xFF) == SK_NONE) continue;
        T fa[FVLBM_Q - 1];
        face(k, fa);
#pragma unroll
        for (int a = 1; a < FVLBM_Q; a++) {
            const T en = T(EXA(a)) * n[k].x + T(EYA(a)) * n[k].y;
            flux[a] += en * (DEV ? fa[a - 1] - f[a] : fa[a - 1]);
        }
    }
}

// cp.async copy of one 4- or 8-byte element from global to shared memory.
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* dst, const T* src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
// Hint: bring a 16-byte aligned range (a multiple of 16 bytes) into L2.
__device__ __forceinline__ void prefetch_l2(const void* p, int64_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"((uint32_t)bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// Geometry of a fused-stage gradient cell: with up to 4 slots its
// least-squares vectors in registers (loaded before the staging barrier; 8
// slots would spill), else and for its reconstruction and face vectors from
// global memory (through L1, which the small shared-memory footprint leaves
// large).
template <typename T, int MAXF> struct RegGeo {
    typedef typename Vec2<T>::type T2;
    static constexpr bool REGS = MAXF <= 4;
    T2 c[REGS ? MAXF : 1];
    GeoRef<T, MAXF> G;
    __device__ __forceinline__ void load(const void* desc, const void* geo, uint32_t i) {
        G = GeoRef<T, MAXF>(desc, geo, i);
        if constexpr (REGS) {
#pragma unroll
            for (int k = 0; k < MAXF; k++) c[k] = G.cg(k);
        }
    }
    __device__ __forceinline__ T2 cg(int k) const {
        if constexpr (REGS) return c[k];
        else return G.cg(k);
    }
    __device__ __forceinline__ T2 rv(int k) const { return G.rv(k); }
    __device__ __forceinline__ T2 nv(int k) const { return G.nv(k); }
};

// Collision and time update of one cell (Eq. rhs, Sec. 2.3): rhs = -flux -
// (f - f^eq) / tau, then out = base + beta dt rhs (multistage; the base state
// is fb when use_fb, else f itself) or the AB2 combination.  Returns false
// when an output is not finite.
template <typename T, typename S, bool DEV, bool FMA_RK = false, typename I>
__device__ __forceinline__ bool update_cell(const DevView& v, const InstParam& P, I i, const T* f, T rho, T ux,
                                            T uy, const T* flux, const T* fb, bool use_fb, S* fout, T beta,
                                            int mode) {
    const T inv_tau = inst_inv_tau<T>(P);
    const T dt = inst_dt<T>(P);
    bool bad = false;
    T* rp = (T*)v.rprev;
    T out[FVLBM_Q];
    if constexpr (FMA_RK) {
        if (mode == MODE_RK) {
            // base + beta dt rhs = base - c1 flux + c2 (f^eq - f), c1 = beta dt,
            // c2 = beta dt / tau: fewer FP64 operations
            const T c1 = beta * dt, c2 = c1 * inv_tau;
#pragma unroll
            for (int a = 0; a < FVLBM_Q; a++) {
                out[a] = fma(c2, feqs<T, DEV>(a, rho, ux, uy) - f[a], fma(-c1, flux[a], use_fb ? fb[a] : f[a]));
                bad |= !finite_val(out[a]);
            }
            CellIO<S>::template store<T, DEV>(fout, i, P, out);
            return !bad;
        }
    }
    // Deviation modes: the collision term f^eq - f carries no mass or momentum
    // (f^eq has the cell's rho and rho u), so directions 0..2 follow from
    // directions 3..8 through those identities.  Evaluated directly in FP32,
    // its nine rounding errors (about eps |g| each, |g| >> |f^eq - f|) would
    // add a spurious mass and momentum source of about eps |g| / tau per unit
    // time, which dominated the velocity error at small tau.
    T col[FVLBM_Q];
    if constexpr (DEV) {
#pragma unroll
        for (int a = 3; a < FVLBM_Q; a++) col[a] = feqs<T, DEV>(a, rho, ux, uy) - f[a];
        col[1] = col[3] - col[5] + col[6] + col[7] - col[8];
        col[2] = col[4] - col[5] - col[6] + col[7] + col[8];
        col[0] = -(col[1] + col[2] + col[3] + col[4] + col[5] + col[6] + col[7] + col[8]);
    }
#pragma unroll
    for (int a = 0; a < FVLBM_Q; a++) {
        const T rhs = DEV ? -flux[a] + col[a] * inv_tau : -flux[a] - (f[a] - feqs<T, DEV>(a, rho, ux, uy)) * inv_tau;
        if (mode == MODE_RK) {
            out[a] = (use_fb ? fb[a] : f[a]) + beta * dt * rhs;
        } else if (mode == MODE_AB2_FIRST) {
            out[a] = f[a] + dt * rhs;
            rp[a * v.np + i] = rhs;
        } else {
            out[a] = f[a] + dt * (T(1.5) * rhs - T(0.5) * rp[a * v.np + i]);
            rp[a * v.np + i] = rhs;
        }
    }
    // one test: the sum of the outputs is not finite when any output is not
    T sum = out[0];
#pragma unroll
    for (int a = 1; a < FVLBM_Q; a++) sum += out[a];
    bad = !finite_val(sum);
    CellIO<S>::template store<T, DEV>(fout, i, P, out);
    return !bad;
}

// ------------------------------------------------------------------ kernels
// Two-kernel stage, kernel 1 (Steps 1-3): per cell the gradient, then the
// value of every (face, direction) it is the upwind side of, and every
// direction of its boundary faces, into the face table (one writer each).
template <typename T, typename S, int MAXF, bool DEV>
__global__ void __launch_bounds__(256) face_values_kernel(DevView v, const S* __restrict__ fin) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.n_grad) return;   // owned cells and, in a partition, the first ghost ring
    const GeoRef<T, MAXF> G(v.desc, v.geo, i);
    const int32_t* nb = v.nbr + blk_index(i, MAXF);
    uint2 d[MAXF];
#pragma unroll
    for (int k = 0; k < MAXF; k++) d[k] = G.desc(k);
    T f[FVLBM_Q];
    CellIO<S>::template load<T, DEV>(fin, i, v.inst[v.grp[i]], f);
    T rho, ux, uy;
    boundary_moments<T, DEV, MAXF>(d, f, rho, ux, uy);
    T gx[FVLBM_Q - 1], gy[FVLBM_Q - 1];
    T* fv = (T*)v.fv;
    auto row = [&](int k) { return fv + d[k].y; };
    lsq_gradient<T, DEV, MAXF>(d, G, v.bc, f, rho, ux, uy, gx, gy, [&](int k, T* fj) {
        const int64_t j = nb[k * BLK];
        CellIO<S>::template load<T, DEV>(fin, j, v.inst[v.grp[j]], fj);
    }, v.n_face, row);
    write_faces<T, DEV, MAXF>(d, G, v.bc, f, rho, ux, uy, gx, gy, v.n_face, row);
}

// Two-kernel stage, kernel 2 (Steps 4-5): flux sum over the cell's faces,
// collision and time update.
template <typename T, typename S, int MAXF, bool DEV>
__global__ void __launch_bounds__(256) update_kernel(DevView v, const S* __restrict__ fin, const S* fbase, S* fout,
                                                     T beta, int mode) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.n_cell) return;
    const InstParam& P = v.inst[v.grp[i]];
    const GeoRef<T, MAXF> G(v.desc, v.geo, i);
    uint2 d[MAXF];
    typename Vec2<T>::type n[MAXF];
#pragma unroll
    for (int k = 0; k < MAXF; k++) {
        d[k] = G.desc(k);
        n[k] = G.nv(k);
    }
    T f[FVLBM_Q];
    CellIO<S>::template load<T, DEV>(fin, i, P, f);
    T rho, ux, uy;
    moments<T, DEV>(f, rho, ux, uy);
    T flux[FVLBM_Q];
    const T* fv = (const T*)v.fv;
    flux_sum<T, DEV, MAXF>(d, n, f, flux, [&](int k, T* fa) {
        const T* p = fv + d[k].y;
#pragma unroll
        for (int a = 0; a < FVLBM_Q - 1; a++) fa[a] = p[a * v.n_face];
    });
    T fb[FVLBM_Q];
    const bool rk_base = mode == MODE_RK && fbase != fin;
    if (rk_base) CellIO<S>::template load<T, DEV>(fbase, i, P, fb);
    // the FP64 two-kernel stage is bound by the FP64 units: the shorter multistage form
    if (!update_cell<T, S, DEV, sizeof(T) == 8>(v, P, i, f, rho, ux, uy, flux, fb, rk_base, fout, beta, mode))
        *v.flag = 1;
}

// Slots (bit k) that some active thread of the warp uses: a polygon with
// fewer faces than MAXF leaves its last slots empty, and when every cell of a
// warp does (a warp of triangles in a 4-slot mesh), the warp skips them as a
// whole.  Slots 0..2 are always used.
template <int MAXF>
__device__ __forceinline__ uint32_t warp_slots(const uint2* d) {
    uint32_t u = 7u;
#pragma unroll
    for (int k = 3; k < MAXF; k++)
        if ((d[k].x & 0xFF) != SK_NONE) u |= 1u << k;
    return __reduce_or_sync(__activemask(), u);
}

// Fused stage, phase 2 for one local cell x (a tile cell, or a 1-ring entry),
// everything in shared memory: its least-squares gradient (Eq. leastsquare)
// and its values on the tile's faces.  The planner links every slot without
// a neighbour (boundary faces, unused slots) to the cell itself, and gives
// unused slots zero geometry and an empty mask, so the loops over the slots
// test no slot kind:
//   1. gradient over all slots from the neighbour differences (zero for the
//      self-linked slots);
//   2. only for cells with boundary slots (rare): the ghost differences of
//      Sec. 2.4.1 enter the gradient, and the boundary face values that are
//      ghost values are written (Sec. 2.4.2);
//   3. every slot writes the reconstruction f + grad f . (x_f - x_i)
//      (Eq. lslrflux) for the directions in its mask: the upwind ones on
//      interior faces, the outflow ones on inlet and internal-outlet faces,
//      none elsewhere; a 1-ring entry writes only the faces it shares with
//      the tile (the others carry no local face).
template <typename T, bool DEV, int MAXF, int LS, int FS, typename Geo>
__device__ __forceinline__ void tile_gradient_faces(const uint2* dx, const Geo& H, const BcParam* bcs, const T* fs,
                                                    T* fvs, int x, T* f) {
#pragma unroll
    for (int a = 0; a < FVLBM_Q; a++) f[a] = fs[a * LS + x];
    T gx[FVLBM_Q - 1], gy[FVLBM_Q - 1];
#pragma unroll
    for (int a = 0; a < FVLBM_Q - 1; a++) gx[a] = gy[a] = T(0);
    const uint32_t used = warp_slots<MAXF>(dx);
#pragma unroll
    for (int k = 0; k < MAXF; k++) {
        if (k >= 3 && !((used >> k) & 1u)) continue;
        const typename Vec2<T>::type c = H.cg(k);
        const T* p = fs + (dx[k].y & 0xFFFF);
#pragma unroll
        for (int a = 1; a < FVLBM_Q; a++) {
            const T dd = p[a * LS] - f[a];
            gx[a - 1] += c.x * dd;
            gy[a - 1] += c.y * dd;
        }
    }
    bool bc = false;
#pragma unroll
    for (int k = 0; k < MAXF; k++) bc |= (dx[k].x & 0xFF) > SK_INTERIOR;
    if (bc) {
        T rho, ux, uy;
        moments<T, DEV>(f, rho, ux, uy);
#pragma unroll
        for (int k = 0; k < MAXF; k++) {
            const uint32_t kind = dx[k].x & 0xFF;
            if (kind <= SK_INTERIOR) continue;
            const Ghost<T> g = ghost_state<T, DEV>(kind, bcs[dx[k].x >> 16], rho, ux, uy, [&] { return H.nv(k); });
            const typename Vec2<T>::type c = H.cg(k);
            const uint32_t mask = (dx[k].x >> 8) & 0xFF;
            const uint32_t lf = dx[k].y >> 16;
            T* fo = lf == LINK_NONE ? nullptr : fvs + lf;
#pragma unroll
            for (int a = 1; a < FVLBM_Q; a++) {
                const T dd = ghost_delta<T, DEV>(g, a, f[a], feqs<T, DEV>(a, rho, ux, uy));
                gx[a - 1] += c.x * dd;
                gy[a - 1] += c.y * dd;
                if (fo && !((mask >> (a - 1)) & 1u)) fo[(a - 1) * FS] = g.sym ? f[a] + T(0.5) * dd : f[a] + dd;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < MAXF; k++) {
        if (k >= 3 && !((used >> k) & 1u)) continue;
        const uint32_t lf = dx[k].y >> 16;
        const uint32_t mask = lf == LINK_NONE ? 0u : (dx[k].x >> 8) & 0xFF;
        T* fo = fvs + (lf == LINK_NONE ? 0u : lf);
        const typename Vec2<T>::type r = H.rv(k);
#pragma unroll
        for (int a = 1; a < FVLBM_Q; a++)
            if ((mask >> (a - 1)) & 1u) fo[(a - 1) * FS] = f[a] + gx[a - 1] * r.x + gy[a - 1] * r.y;
    }
}

// Fused stage: one CTA per tile of consecutive cells (Hilbert order; tile
// and 1-ring together at most TILE cells), everything between the state read
// and the state write in shared memory:
//   phase 1  cp.async of the state of the tile, its 1-ring and its 2-ring
//            (the 16-bit formats raw, each cell decoded by the thread that
//            staged it) and of the instance id of each tile cell; the slot
//            descriptors and the
//            least-squares vectors of each thread's gradient cell into
//            registers
//   phase 2  per tile and 1-ring cell (one per thread): the gradient
//            (Eq. leastsquare) and its values on the tile's faces
//            (Eq. lslrflux / Sec. 2.4.2): on interior faces the directions it
//            writes (upwind side), on boundary faces (tile cells) every
//            direction -- one writer per (face, direction), into a table of
//            the tile's faces; a tile cell's thread keeps its state
//   phase 3  per tile cell: flux sum from the face table, collision and the
//            time update (Eq. rhs, Sec. 2.3)
// The global loads of each phase are issued before the barrier that precedes
// it, so that their latency overlaps the wait, and each CTA prefetches into L2
// the data of a tile that starts somewhat under one CTA lifetime later (pf =
// 5/8 of the resident CTAs ahead).  The kernel is bound by shared-memory
// traffic more than by DRAM: what a thread can hold in registers (its own
// state, its least-squares vectors) or read through L1 (reconstruction and
// face vectors) stays out of shared memory, whose small footprint leaves L1
// large.  Shared-memory strides are compile-time constants (TileDims); the
// planner keeps every tile within them.
template <typename T, typename S, int MAXF, bool DEV, int TILE>
__global__ void __launch_bounds__(TILE, (sizeof(T) == 4 ? 1024 : 512) / TILE > 0 ? (sizeof(T) == 4 ? 1024 : 512) / TILE : 1)
    stage_tile_kernel(DevView v, const S* __restrict__ fin, const S* fbase, S* fout, T beta, int mode, int pf) {
    constexpr int LS = TileDims<TILE, MAXF, sizeof(T)>::LS;
    constexpr int FS = TileDims<TILE, MAXF, sizeof(T)>::FS;
    typedef typename Vec2<T>::type T2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* fs = (T*)smem_raw;            // [9][LS]  f of the local cells
    T* fvs = fs + FVLBM_Q * LS;      // [8][FS]  face values of directions 1..8
    int32_t* sgrp = (int32_t*)(fvs + (FVLBM_Q - 1) * FS);   // [TILE] instance of each tile cell
    // cell, halo and 1-ring indices in 32 bits: the set-up keeps every array
    // of a fused-stage solver below 2^32 elements
    const uint32_t t = blockIdx.x;
    const uint32_t c0 = (uint32_t)v.tile_begin[t];
    const int nt = (int)((uint32_t)v.tile_begin[t + 1] - c0);
    const uint32_t h0 = (uint32_t)v.halo_ptr[t];
    const int nh = (int)((uint32_t)v.halo_ptr[t + 1] - h0);
    const uint32_t q0 = (uint32_t)v.r1_ptr[t];
    const int n1 = (int)((uint32_t)v.r1_ptr[t + 1] - q0);
    const int l = threadIdx.x;
    const bool mine = l < nt;          // this thread owns tile cell l
    const uint32_t gi = c0 + l;

    // phase 1 (thread l's first local cell is local cell l).  The 16-bit split
    // formats are staged raw (moments, packed non-equilibrium words, instance)
    // in the face-table area, which is free until phase 2, and decoded by the
    // thread that staged them.
    constexpr bool PLAIN = sizeof(S) == sizeof(T);
    float* rawc = (float*)fvs;                     // [3][LS]
    uint32_t* raww = (uint32_t*)(rawc + 3 * LS);   // [3][LS]
    int32_t* rawg = (int32_t*)(raww + 3 * LS);     // [LS]
    static_assert(PLAIN || 7 * LS * 4 <= (FVLBM_Q - 1) * FS * (int)sizeof(T), "raw staging fits the face table");
    uint32_t gl = c0;
    for (int x = l; x < nt + nh; x += TILE) {
        const uint32_t gx = x < nt ? c0 + x : (uint32_t)v.halo[h0 + (x - nt)];
        if (x == l) gl = gx;
        if constexpr (PLAIN) {
            const S* p = fin + blk_index(gx, FVLBM_Q);
#pragma unroll
            for (int a = 0; a < FVLBM_Q; a++) cp_async_elem<T>(fs + a * LS + x, (const T*)p + a * BLK);
        } else {
            const float* pc = CellIO<S>::cptr(fin, gx);
            const uint32_t* pw = CellIO<S>::wptr(fin, gx);
#pragma unroll
            for (int q = 0; q < 3; q++) {
                cp_async_elem<float>(rawc + q * LS + x, pc + q * BLK);
                cp_async_elem<uint32_t>(raww + q * LS + x, pw + q * BLK);
            }
            cp_async_elem<int32_t>(rawg + x, v.grp + gx);
        }
    }
    // Phase 2 gives local cell x (tile cell, or 1-ring entry x - nt) to thread
    // x: with the planner's bound nt + n1 <= TILE every thread has at most one.
    // Its descriptors and local links are in flight during the wait.
    const int n2 = nt + n1;
    auto links = [&](int x, uint32_t g, uint2* d) {
        const GeoRef<T, MAXF> H(v.desc, v.geo, g);
        const uint32_t* rl = x < nt ? nullptr : v.r1link + blk_index(q0 + (uint32_t)(x - nt), MAXF);
#pragma unroll
        for (int k = 0; k < MAXF; k++) {
            d[k] = H.desc(k);
            if (x >= nt) d[k].y = rl[k * BLK];   // the 1-ring entry's local links
        }
    };
    if (l < nt) cp_async_elem<int32_t>(sgrp + l, v.grp + c0 + l);
    uint2 d[MAXF];
    RegGeo<T, MAXF> H;
    if (l < n2) {
        links(l, gl, d);
        H.load(v.desc, v.geo, gl);
    }
    // A CTA that starts somewhat before this one ends works on about tile
    // t + pf (pf = 5/8 of the CTAs resident on the GPU): bring that tile's
    // state and geometry into L2 now, so that its staging reads L2 rather than
    // HBM.  The last thread does it once its own copies are in flight, so that
    // the loads of the other tile's bounds overlap them.
    if (l == TILE - 1 && pf > 0 && t + pf < v.n_tiles) {
        const int64_t tp = t + pf;
        const int64_t b0 = v.tile_begin[tp] >> BLK_SHIFT;
        const int64_t nb = ((v.tile_begin[tp + 1] + BLK - 1) >> BLK_SHIFT) - b0;
        constexpr int64_t SB = CellIO<S>::BLOCK_BYTES;
        constexpr int64_t DB = (int64_t)MAXF * BLK * sizeof(uint2);
        constexpr int64_t GB = (int64_t)3 * MAXF * BLK * sizeof(T2);
        prefetch_l2((const unsigned char*)fin + b0 * SB, nb * SB);
        if (mode == MODE_RK && fbase != fin) prefetch_l2((const unsigned char*)fbase + b0 * SB, nb * SB);
        prefetch_l2((const unsigned char*)v.desc + b0 * DB, nb * DB);
        prefetch_l2((const unsigned char*)v.geo + b0 * GB, nb * GB);
        // its halo list and 1-ring links (16-byte aligned cover of each range)
        auto range = [&](const void* base, int64_t begin, int64_t end) {
            const int64_t a = begin & ~(int64_t)15, e = (end + 15) & ~(int64_t)15;
            if (e > a) prefetch_l2((const unsigned char*)base + a, e - a);
        };
        range(v.halo, 4 * v.halo_ptr[tp], 4 * v.halo_ptr[tp + 1]);
        range(v.grp, 4 * v.tile_begin[tp], 4 * v.tile_begin[tp + 1]);   // instance ids
        constexpr int64_t LB = (int64_t)MAXF * BLK * 4;   // bytes per block of 32 entries
        range(v.r1link, (v.r1_ptr[tp] >> BLK_SHIFT) * LB, ((v.r1_ptr[tp + 1] + BLK - 1) >> BLK_SHIFT) * LB);
    }
    cp_async_wait_all();
    // a 16-bit state is decoded by the thread that staged it (its own copies
    // are complete after the wait), so one barrier serves both
    if constexpr (PLAIN) __syncthreads();
    if constexpr (!PLAIN) {
        for (int x = l; x < nt + nh; x += TILE) {
            const uint32_t w[3] = {raww[x], raww[LS + x], raww[2 * LS + x]};
            T f[FVLBM_Q];
            CellIO<S>::template decode<T>(rawc[x], rawc[LS + x], rawc[2 * LS + x], w, v.inst[rawg[x]], f);
#pragma unroll
            for (int a = 0; a < FVLBM_Q; a++) fs[a * LS + x] = f[a];
        }
        __syncthreads();
    }

    // phase 2 (a tile cell's thread keeps its state for phase 3)
    T f[FVLBM_Q];
    if (l < n2) {
        tile_gradient_faces<T, DEV, MAXF, LS, FS>(d, H, v.bc, fs, fvs, l, f);
    }
    // phase 3 inputs, in flight during the wait
    T2 n[MAXF];
    T fb[FVLBM_Q];
    const bool rk_base = mode == MODE_RK && fbase != fin;
    if (mine) {
        const GeoRef<T, MAXF> G(v.desc, v.geo, gi);
#pragma unroll
        for (int k = 0; k < MAXF; k++) n[k] = G.nv(k);
        if (rk_base) CellIO<S>::template load<T, DEV>(fbase, gi, v.inst[v.grp[gi]], fb);
    }
    __syncthreads();

    // phase 3: flux of every slot from the face table, with no test of the
    // slot kind (unused slots read face row 0 with a zero face vector)
    if (!mine) return;
    const InstParam& P = v.inst[sgrp[l]];
    T rho, ux, uy;
    moments<T, DEV>(f, rho, ux, uy);
    T flux[FVLBM_Q];
#pragma unroll
    for (int a = 0; a < FVLBM_Q; a++) flux[a] = T(0);
    const uint32_t used = warp_slots<MAXF>(d);
#pragma unroll
    for (int k = 0; k < MAXF; k++) {
        if (k >= 3 && !((used >> k) & 1u)) continue;
        const T* p = fvs + (d[k].y >> 16);
#pragma unroll
        for (int a = 1; a < FVLBM_Q; a++) {
            const T en = T(EXA(a)) * n[k].x + T(EYA(a)) * n[k].y;
            flux[a] += en * (DEV ? p[(a - 1) * FS] - f[a] : p[(a - 1) * FS]);
        }
    }
    if (!update_cell<T, S, DEV>(v, P, gi, f, rho, ux, uy, flux, fb, rk_base, fout, beta, mode))
        *v.flag = 1;
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
    const size_t smem = TileDims<TILE, MAXF, sizeof(T)>::BYTES;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return fail(FVLBM_ERR_CUDA, "fused stage: %zu B shared memory: %s", smem, cudaGetErrorString(e));
    }
    // prefetch distance: 5/8 of the CTAs that fit on the GPU at once (queried
    // once per kernel; a function-local static is initialised once even when
    // several host threads launch at the same time).  Measured on GB300 over
    // 0.5 to 1.5 times the resident CTAs: 0.6 to 0.75 was best, longer
    // distances let the prefetched lines age out of L2 before their tile runs.
    static const int per_sm = [&] {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, TILE, smem) != cudaSuccess) {
            cudaGetLastError();
            n = 0;
        }
        return n;
    }();
    const int pf = per_sm * v.sms * 5 / 8;
    kern<<<(unsigned)v.n_tiles, TILE, smem, st>>>(v, (const S*)fin, (const S*)fbase, (S*)fout, (T)beta, mode, pf);
    return FVLBM_OK;
}

// Tile sizes whose shared memory exceeds a CTA's are not instantiated (the
// planner never selects them).
constexpr size_t TILE_SMEM_LIMIT = 227 * 1024;

template <typename T, typename S, int MAXF, bool DEV, int TILE>
static int tile_launch_if_fits(const DevView& v, cudaStream_t st, const void* fin, const void* fbase, void* fout,
                               double beta, int mode) {
    if constexpr (TileDims<TILE, MAXF, sizeof(T)>::BYTES <= TILE_SMEM_LIMIT)
        return tile_launch<T, S, MAXF, DEV, TILE>(v, st, fin, fbase, fout, beta, mode);
    return fail(FVLBM_ERR_UNSUPPORTED, "tile size %d does not fit in shared memory", TILE);
}

template <typename T, typename S, int MAXF, bool DEV>
static int tile_dispatch(const DevView& v, cudaStream_t st, const void* fin, const void* fbase, void* fout,
                         double beta, int mode) {
    switch (v.tile) {
        case 128: return tile_launch_if_fits<T, S, MAXF, DEV, 128>(v, st, fin, fbase, fout, beta, mode);
        case 256: return tile_launch_if_fits<T, S, MAXF, DEV, 256>(v, st, fin, fbase, fout, beta, mode);
        case 512: return tile_launch_if_fits<T, S, MAXF, DEV, 512>(v, st, fin, fbase, fout, beta, mode);
        case 1024: return tile_launch_if_fits<T, S, MAXF, DEV, 1024>(v, st, fin, fbase, fout, beta, mode);
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
    const unsigned g = grid_of(v.n_cell, bs), gg = grid_of(v.n_grad, bs);
    if (v.maxf == 4) face_values_kernel<T, S, 4, DEV><<<gg, bs, 0, st>>>(v, (const S*)fin);
    else face_values_kernel<T, S, 8, DEV><<<gg, bs, 0, st>>>(v, (const S*)fin);
    if (ev) cudaEventRecord((cudaEvent_t)ev[1], st);
    if (v.maxf == 4)
        update_kernel<T, S, 4, DEV><<<g, bs, 0, st>>>(v, (const S*)fin, (const S*)fbase, (S*)fout, (T)beta, mode);
    else
        update_kernel<T, S, 8, DEV><<<g, bs, 0, st>>>(v, (const S*)fin, (const S*)fbase, (S*)fout, (T)beta, mode);
    if (ev) cudaEventRecord((cudaEvent_t)ev[2], st);
    return check_launch("stage kernels");
}

}  // namespace fvlbm
