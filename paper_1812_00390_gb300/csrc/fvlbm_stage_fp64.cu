// Stage kernels instantiated for the fp64 state.
#include "fvlbm_stage.cuh"

namespace fvlbm {
int stage_fp64(const DevView& v, void* stream, const void* fin, const void* fbase, void* fout, double beta,
               int mode, void* const* ev) {
    return stage_t<double, double, false>(v, (cudaStream_t)stream, fin, fbase, fout, beta, mode, ev);
}
}  // namespace fvlbm
