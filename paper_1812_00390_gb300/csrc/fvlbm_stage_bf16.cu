// Stage kernels instantiated for the bf16 state.
#include "fvlbm_stage.cuh"

namespace fvlbm {
int stage_bf16(const DevView& v, void* stream, const void* fin, const void* fbase, void* fout, double beta,
               int mode, void* const* ev) {
    return stage_t<float, __nv_bfloat16, true>(v, (cudaStream_t)stream, fin, fbase, fout, beta, mode, ev);
}
}  // namespace fvlbm
