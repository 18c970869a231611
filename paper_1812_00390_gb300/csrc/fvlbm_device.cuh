// Device-side helpers shared by the library's CUDA translation units: the
// D2Q9 lattice of Sec. 2.1 and the storage formats of the state.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "fvlbm_internal.h"

namespace fvlbm {

#define EXA(a) ((a) == 1 || (a) == 5 || (a) == 8 ? 1 : ((a) == 3 || (a) == 6 || (a) == 7 ? -1 : 0))
#define EYA(a) ((a) == 2 || (a) == 5 || (a) == 6 ? 1 : ((a) == 4 || (a) == 7 || (a) == 8 ? -1 : 0))

template <typename T>
__device__ __forceinline__ T wgt(int a) {
    return a == 0 ? T(4.0 / 9.0) : (a < 5 ? T(1.0 / 9.0) : T(1.0 / 36.0));
}

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
    const T inv_rho = T(1) / (DEV ? T(1) + s : s);
    ux = mx * inv_rho;
    uy = my * inv_rho;
}

// Eq. (feq).  FP64 mode: r = rho, returns f^eq.  Deviation mode: r = rho - 1,
// returns f^eq - w = w [(rho - 1) + rho (3 e.u + 4.5 (e.u)^2 - 1.5 u^2)].
// The polynomial is evaluated as e.u (3 + 4.5 e.u) - 1.5 u^2 (two fused
// multiply-adds per direction once u^2 is known).
template <typename T, bool DEV>
__device__ __forceinline__ T feqs(int a, T r, T ux, T uy) {
    const T eu = T(EXA(a)) * ux + T(EYA(a)) * uy;
    const T uu15 = T(1.5) * (ux * ux + uy * uy);
    if (DEV) {
        const T poly = fma(eu, fma(T(4.5), eu, T(3)), -uu15);
        return wgt<T>(a) * fma(T(1) + r, poly, r);
    }
    return r * wgt<T>(a) * fma(eu, fma(T(4.5), eu, T(3)), T(1) - uu15);
}

// Density argument of feqs for a given density.
template <typename T, bool DEV>
__device__ __forceinline__ T rarg(double rho) { return DEV ? T(rho - 1.0) : T(rho); }

// ------------------------------------------------------------------ storage
// Per-cell arrays are stored in blocks of BLK = 32 consecutive cells (internal
// order): a block holds component 0 of its 32 cells, then component 1, ...  A
// cell's component c sits at (i / 32) * ncomp * 32 + c * 32 + i % 32, so a
// warp of consecutive cells reads whole 128-byte lines, and one address per
// cell serves every component (constant offsets c * 32).
__host__ __device__ __forceinline__ int64_t blk_index(int64_t i, int ncomp) {
    return (i >> BLK_SHIFT) * ((int64_t)ncomp << BLK_SHIFT) + (i & (BLK - 1));
}
// The same in 32-bit arithmetic, for the fused stage kernel, whose solvers
// keep every blocked array below 2^32 elements (checked at set-up).
__host__ __device__ __forceinline__ uint32_t blk_index(uint32_t i, int ncomp) {
    return (i >> BLK_SHIFT) * ((uint32_t)ncomp << BLK_SHIFT) + (i & (BLK - 1));
}

// Whole-cell access to the stored state (T: arithmetic type, DEV: deviation
// mode, the stored quantity is g = f - w).
//  double / float   9 components per cell: g_a (f_a in FP64 mode).
//  __half / bf16    split format: 3 FP32 components rho - 1, rho u_x, rho u_y,
//                   then the six 16-bit non-equilibrium parts
//                   n_a = g_a - g^eq_a(rho, u) of directions a = 3..8, times
//                   a power-of-two scale per (instance, direction), packed in
//                   pairs into three 32-bit components.
//                   n_0, n_1, n_2 follow from sum_a n_a = 0 and
//                   sum_a e_a n_a = 0 (the non-equilibrium part carries no mass
//                   or momentum), so rho and u never round through 16 bits;
//                   only the small non-equilibrium part does.
template <typename S> struct CellIO;

template <typename S> struct PlainIO {
    template <typename T, bool DEV, typename I>
    __device__ static void load(const void* base, I i, const InstParam&, T* f) {
        const S* p = (const S*)base + blk_index(i, FVLBM_Q);
#pragma unroll
        for (int a = 0; a < FVLBM_Q; a++) f[a] = (T)p[a * BLK];
    }
    template <typename T, bool DEV, typename I>
    __device__ static void store(void* base, I i, const InstParam&, const T* f) {
        S* p = (S*)base + blk_index(i, FVLBM_Q);
#pragma unroll
        for (int a = 0; a < FVLBM_Q; a++) p[a * BLK] = (S)f[a];
    }
    // FP64 moments of the stored state: r = sum f (FP64 mode) or sum g (deviation), j = sum e g
    __device__ static void moments64(const void* base, int64_t i, const InstParam&, double& r, double& jx, double& jy) {
        const S* p = (const S*)base + blk_index(i, FVLBM_Q);
        r = jx = jy = 0;
        for (int a = 0; a < FVLBM_Q; a++) {
            const double x = (double)p[a * BLK];
            r += x;
            jx += EXA(a) * x;
            jy += EYA(a) * x;
        }
    }
    static constexpr size_t bytes_per_cell = FVLBM_Q * sizeof(S);
    static constexpr int64_t BLOCK_BYTES = (int64_t)FVLBM_Q * BLK * sizeof(S);
};
template <> struct CellIO<double> : PlainIO<double> {};
template <> struct CellIO<float> : PlainIO<float> {};

// Unbiased (stochastic) rounding of q to the 16-bit format H: the upper of the
// two neighbouring 16-bit values with probability equal to q's distance from
// the lower one in units of their gap, else the lower one.  Round to nearest
// would lose every update smaller than half a 16-bit step, so that a slowly
// relaxing non-equilibrium part could stay up to about 2^-(p+1) tau / dt of
// itself away from its value (p = 10 bits in FP16, 7 in BF16); unbiased
// rounding leaves only zero-mean noise.  It is done on the bits: a uniform
// random integer below one 16-bit step, in units of q's last FP32 bit, is
// added to q's magnitude and the sum is truncated (rounded toward zero) to the
// 16-bit grid, which rounds up exactly when the random number reaches the
// step minus q's remainder.  BF16 (the same exponent range as FP32) drops 16
// bits of every finite FP32 value.  FP16 adds, with one fused multiply-add, a
// uniform fraction of the grid step at |q| (2^(e - 10) for FP16 normals,
// 2^-24 for its subnormals below 2^-14), whose FP32 sum keeps the same ~13
// random bits, and rounds toward zero: one formula for every magnitude, no
// branch.
// The random word of a cell comes from one integer hash of the bits of its
// six rounded values (the "lowbias32" mixing function of C. Wellons'
// hash-prospector, two multiply-xorshift rounds), spread over the directions
// by odd multipliers: it changes whenever the cell's values do, and equal
// cells round alike, so a cell's result does not depend on where it sits
// (batch, alone, partitioned).
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7FEB352Du;
    x ^= x >> 15;
    x *= 0x846CA68Bu;
    x ^= x >> 16;
    return x;
}
// random word of direction a from the cell's hash: the high bits of an odd multiple
__device__ __forceinline__ uint32_t sr_word(uint32_t h, int a) { return h * (0x9E3779B9u + 2u * (uint32_t)a); }
template <typename H> __device__ __forceinline__ uint32_t h_bits_sr(float q, uint32_t rnd);
template <> __device__ __forceinline__ uint32_t h_bits_sr<__half>(float q, uint32_t rnd) {
    const uint32_t b = __float_as_uint(q), mag = b & 0x7FFFFFFFu;
    // FP16 grid step at |q|: 2^(e - 10) for normals, 2^-24 below 2^-14 (subnormals)
    const int e = max((int)(mag >> 23) - 127, -14);
    const float step = __uint_as_float((uint32_t)(e - 10 + 127) << 23);
    const float u = __uint_as_float(0x3F800000u | (rnd >> 9)) - 1.0f;   // uniform in [0, 1)
    const float up = fmaf(u, step, __uint_as_float(mag));
    return __half_as_ushort(__float2half_rz(__uint_as_float(__float_as_uint(up) | (b & 0x80000000u))));
}
template <> __device__ __forceinline__ uint32_t h_bits_sr<__nv_bfloat16>(float q, uint32_t rnd) {
    return (__float_as_uint(q) + (rnd >> 16)) >> 16;
}
template <typename H> __device__ __forceinline__ float h_value(uint32_t bits);
template <> __device__ __forceinline__ float h_value<__half>(uint32_t bits) {
    return __half2float(__ushort_as_half((unsigned short)bits));
}
template <> __device__ __forceinline__ float h_value<__nv_bfloat16>(uint32_t bits) {
    return __bfloat162float(__ushort_as_bfloat16((unsigned short)bits));
}

// Split format: a block of 32 cells holds 3 x 32 floats (rho - 1, rho u_x,
// rho u_y), then 3 x 32 words, word q of a cell packing n_{3+2q} (low 16
// bits) and n_{4+2q} (high 16 bits).
template <typename H> struct SplitIO {
    static_assert(sizeof(H) == 2, "16-bit storage");
    static constexpr int64_t BLOCK_BYTES = BLK * (3 * sizeof(float) + 3 * sizeof(uint32_t));
    __device__ static const float* cptr(const void* base, int64_t i) {
        return (const float*)((const unsigned char*)base + (i >> BLK_SHIFT) * BLOCK_BYTES) + (i & (BLK - 1));
    }
    __device__ static const uint32_t* wptr(const void* base, int64_t i) {
        return (const uint32_t*)((const unsigned char*)base + (i >> BLK_SHIFT) * BLOCK_BYTES + 3 * BLK * sizeof(float)) +
               (i & (BLK - 1));
    }
    // f of one cell from its stored moments and non-equilibrium words
    template <typename T>
    __device__ static void decode(float dr, float jx, float jy, const uint32_t* w, const InstParam& P, T* f) {
        const float inv_rho = 1.0f / (1.0f + dr), ux = jx * inv_rho, uy = jy * inv_rho;
        float n[FVLBM_Q];
        float s = 0, sx = 0, sy = 0;
#pragma unroll
        for (int a = 3; a < FVLBM_Q; a++) {
            const uint32_t word = w[(a - 3) >> 1];
            n[a] = h_value<H>(((a - 3) & 1) ? word >> 16 : word & 0xFFFFu) * P.inv_scale[a];
            s += n[a];
            sx += float(EXA(a)) * n[a];
            sy += float(EYA(a)) * n[a];
        }
        n[1] = -sx;
        n[2] = -sy;
        n[0] = -(s + n[1] + n[2]);
#pragma unroll
        for (int a = 0; a < FVLBM_Q; a++) f[a] = (T)(feqs<float, true>(a, dr, ux, uy) + n[a]);
    }
    template <typename T, bool DEV>
    __device__ static void load(const void* base, int64_t i, const InstParam& P, T* f) {
        const float* c = cptr(base, i);
        const uint32_t* wp = wptr(base, i);
        const uint32_t w[3] = {wp[0], wp[BLK], wp[2 * BLK]};
        decode<T>(c[0], c[BLK], c[2 * BLK], w, P, f);
    }
    template <typename T, bool DEV>
    __device__ static void store(void* base, int64_t i, const InstParam& P, const T* f) {
        float* c = (float*)cptr(base, i);
        uint32_t* wp = (uint32_t*)wptr(base, i);
        float dr = 0, jx = 0, jy = 0;
#pragma unroll
        for (int a = 0; a < FVLBM_Q; a++) {
            dr += (float)f[a];
            jx += float(EXA(a)) * (float)f[a];
            jy += float(EYA(a)) * (float)f[a];
        }
        c[0] = dr;
        c[BLK] = jx;
        c[2 * BLK] = jy;
        const float inv_rho = 1.0f / (1.0f + dr), ux = jx * inv_rho, uy = jy * inv_rho;
        float q[FVLBM_Q];
        uint32_t h = 0x811C9DC5u;
#pragma unroll
        for (int a = 3; a < FVLBM_Q; a++) {
            q[a] = ((float)f[a] - feqs<float, true>(a, dr, ux, uy)) * P.scale[a];
            h = (h ^ __float_as_uint(q[a])) * 0x01000193u;
        }
        h = mix32(h);
        uint32_t bits[FVLBM_Q];
#pragma unroll
        for (int a = 3; a < FVLBM_Q; a++) bits[a] = h_bits_sr<H>(q[a], sr_word(h, a));
#pragma unroll
        for (int q = 0; q < 3; q++) wp[q * BLK] = bits[3 + 2 * q] | (bits[4 + 2 * q] << 16);
    }
    __device__ static void moments64(const void* base, int64_t i, const InstParam&, double& r, double& jx, double& jy) {
        const float* c = cptr(base, i);
        r = c[0];
        jx = c[BLK];
        jy = c[2 * BLK];
    }
    static constexpr size_t bytes_per_cell = 3 * sizeof(float) + 3 * sizeof(uint32_t);
};
template <> struct CellIO<__half> : SplitIO<__half> {};
template <> struct CellIO<__nv_bfloat16> : SplitIO<__nv_bfloat16> {};

// Geometry of one cell (same blocked layout): per face slot k a 64-bit
// descriptor (meta, link) and three 2-vectors of type T: least-squares
// coefficients (component 3k), face midpoint minus centroid (3k + 1) and
// face vector over area (3k + 2).
template <typename T> struct Vec2;
template <> struct Vec2<float> { typedef float2 type; };
template <> struct Vec2<double> { typedef double2 type; };

template <typename T, int MAXF> struct GeoRef {
    typedef typename Vec2<T>::type T2;
    const uint2* d;
    const T2* g;
    __device__ __forceinline__ GeoRef() {}
    template <typename I>
    __device__ __forceinline__ GeoRef(const void* desc, const void* geo, I i)
        : d((const uint2*)desc + blk_index(i, MAXF)), g((const T2*)geo + blk_index(i, 3 * MAXF)) {}
    __device__ __forceinline__ uint2 desc(int k) const { return d[k * BLK]; }
    __device__ __forceinline__ T2 cg(int k) const { return g[(3 * k) * BLK]; }
    __device__ __forceinline__ T2 rv(int k) const { return g[(3 * k + 1) * BLK]; }
    __device__ __forceinline__ T2 nv(int k) const { return g[(3 * k + 2) * BLK]; }
};

}  // namespace fvlbm
