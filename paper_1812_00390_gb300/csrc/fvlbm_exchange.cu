// Halo exchange of a partitioned solve on one device: after each stage, the
// stored state of every ghost cell is copied from the part that owns it (see
// fvlbm_partition.cpp for which cells and why).  One launch covers every
// message; thread (entry, component) copies one stored component.  Sources are
// owned cells and destinations ghost cells, so no thread reads what another
// writes.
#include <cuda_runtime.h>

#include "fvlbm_device.cuh"
#include "fvlbm_internal.h"

namespace fvlbm {

namespace {

struct PartPtrs {
    void* p[FVLBM_MAX_PARTS];
};

// E: stored component type, C: components per cell in the blocked layout
// (FP64: 9 doubles; FP32: 9 floats; 16-bit split: 3 floats + 3 packed words).
template <typename E, int C>
__global__ void halo_copy_kernel(const int4* __restrict__ ent, int64_t n, PartPtrs ptr) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * C) return;
    const int64_t e = t / C;
    const int c = (int)(t - e * C);
    const int4 x = ent[e];   // src part, src cell, dst part, dst cell
    const E* src = (const E*)ptr.p[x.x];
    E* dst = (E*)ptr.p[x.z];
    dst[blk_index((int64_t)x.w, C) + c * BLK] = src[blk_index((int64_t)x.y, C) + c * BLK];
}

template <typename E, int C>
int launch(cudaStream_t st, const int4* ent, int64_t n, const PartPtrs& p) {
    if (n == 0) return FVLBM_OK;
    const int threads = 256;
    halo_copy_kernel<E, C><<<(unsigned)((n * C + threads - 1) / threads), threads, 0, st>>>(ent, n, p);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FVLBM_OK : fail(FVLBM_ERR_CUDA, "halo exchange: %s", cudaGetErrorString(e));
}

}  // namespace

int launch_halo_copy(int prec, void* stream, const int4* entries, int64_t n, void* const* part_state, int n_parts) {
    if (n_parts < 1 || n_parts > FVLBM_MAX_PARTS) return fail(FVLBM_ERR_ARG, "halo exchange: %d parts", n_parts);
    PartPtrs p{};
    for (int k = 0; k < n_parts; k++) p.p[k] = part_state[k];
    cudaStream_t st = (cudaStream_t)stream;
    switch (prec) {
        case FVLBM_FP64: return launch<double, FVLBM_Q>(st, entries, n, p);
        case FVLBM_FP32_DEV: return launch<float, FVLBM_Q>(st, entries, n, p);
        case FVLBM_FP16_DEV:
        case FVLBM_BF16_DEV: return launch<uint32_t, 6>(st, entries, n, p);
    }
    return fail(FVLBM_ERR_ARG, "halo exchange: unknown precision %d", prec);
}

}  // namespace fvlbm
