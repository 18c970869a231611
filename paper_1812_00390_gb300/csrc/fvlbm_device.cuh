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

// ------------------------------------------------------------------ storage
template <typename S> struct Store;
// FP64 / FP32 keep the value itself.
template <> struct Store<double> {
    __device__ static double ld(const double* p, int64_t i, float, float) { return p[i]; }
    __device__ static void st(double* p, int64_t i, double v, float, float) { p[i] = v; }
};
template <> struct Store<float> {
    __device__ static float ld(const float* p, int64_t i, float, float) { return p[i]; }
    __device__ static void st(float* p, int64_t i, float v, float, float) { p[i] = v; }
};
// 16-bit storage keeps (g - off) * scale: off is the deviation of the
// instance's initial equilibrium, so the stored number is the departure from
// it and the format's relative precision applies to that departure.
template <> struct Store<__half> {
    __device__ static float ld(const __half* p, int64_t i, float inv_scale, float off) {
        return fmaf(__half2float(p[i]), inv_scale, off);
    }
    __device__ static void st(__half* p, int64_t i, float v, float scale, float off) {
        p[i] = __float2half_rn((v - off) * scale);
    }
};
template <> struct Store<__nv_bfloat16> {
    __device__ static float ld(const __nv_bfloat16* p, int64_t i, float, float off) {
        return __bfloat162float(p[i]) + off;
    }
    __device__ static void st(__nv_bfloat16* p, int64_t i, float v, float, float off) {
        p[i] = __float2bfloat16_rn(v - off);
    }
};

}  // namespace fvlbm
