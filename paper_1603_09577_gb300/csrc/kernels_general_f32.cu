// kernels_general_f32.cu -- FP32 instantiations of the general time step.
#include "kernels_general.cuh"

namespace lbm {

cudaError_t launch_general_f32(const lbm_solver *s, int src, const double *bv, const void *phi0, int in_prec,
                               cudaStream_t st)
{
    return general_p<LBM_F32>(s, src, bv, phi0, in_prec, st);
}

}  // namespace lbm
