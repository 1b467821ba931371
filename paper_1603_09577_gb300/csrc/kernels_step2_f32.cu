// kernels_step2_f32.cu -- instantiations of the two-step tile kernel for FP32
// storage, and the two-step dispatch (the BF16S instantiations live in
// kernels_step2_bf16.cu so the two compile in parallel).
#include "kernels_step2.cuh"

namespace lbm {

template <int PREC>
static cudaError_t step2_p(const lbm_solver *s, int src, cudaStream_t st)
{
    switch (step_key(s)) {
    case 0: return step2_t<PREC, 0, 0>(s, src, st);
    case 1: return step2_t<PREC, 0, 1>(s, src, st);
    case 2: return step2_t<PREC, 0, 2>(s, src, st);
    case 3: return step2_t<PREC, 1, 0>(s, src, st);
    case 4: return step2_t<PREC, 1, 1>(s, src, st);
    case 5: return step2_t<PREC, 1, 2>(s, src, st);
    case 6: return step2_t<PREC, kConvNone, 0>(s, src, st);
    case 7: return step2_t<PREC, kConvNone, 1>(s, src, st);
    case 8: return step2_t<PREC, kConvNone, 2>(s, src, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_step2_bf16s(const lbm_solver *s, int src, cudaStream_t st);

cudaError_t launch_step2(const lbm_solver *s, int src, cudaStream_t st)
{
    if (s->d.prec == LBM_F32) return step2_p<LBM_F32>(s, src, st);
    if (s->d.prec == LBM_BF16S) return launch_step2_bf16s(s, src, st);
    return cudaErrorInvalidValue;
}

}  // namespace lbm
