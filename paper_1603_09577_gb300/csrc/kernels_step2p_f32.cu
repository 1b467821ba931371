// kernels_step2p_f32.cu -- instantiations of the two-step pair-tile kernel for
// FP32 storage (the other storage compiles in parallel in its own unit).
#include "kernels_step2p.cuh"

namespace lbm {

cudaError_t launch_step2p_f32(const lbm_solver *s, int src, cudaStream_t st)
{
    switch (step_key(s)) {
    case 0: return step2p_t<LBM_F32, 0, 0>(s, src, st);
    case 1: return step2p_t<LBM_F32, 0, 1>(s, src, st);
    case 2: return step2p_t<LBM_F32, 0, 2>(s, src, st);
    case 3: return step2p_t<LBM_F32, 1, 0>(s, src, st);
    case 4: return step2p_t<LBM_F32, 1, 1>(s, src, st);
    case 5: return step2p_t<LBM_F32, 1, 2>(s, src, st);
    case 6: return step2p_t<LBM_F32, kConvNone, 0>(s, src, st);
    case 7: return step2p_t<LBM_F32, kConvNone, 1>(s, src, st);
    case 8: return step2p_t<LBM_F32, kConvNone, 2>(s, src, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbm
