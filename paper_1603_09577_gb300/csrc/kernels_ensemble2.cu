// kernels_ensemble2.cu -- the ensemble with two time steps per sweep through
// HBM: one launch covers the list of 30 x 30 output tiles of every instance and
// runs the shared-memory two-step tile routine of the single-grid kernel on
// each (FP32 storage, periodic walls, constant K per instance). By default one
// block per tile; in persistent mode SMs x resident blocks walk the list.
#include "kernels_step2.cuh"
#include "lbm_ensemble.h"

namespace lbm {

template <int CONV, int DIFF>
__global__ void __launch_bounds__(kT2Threads, Tile2<30>::kMinBlocks)
k_ens_step2(const EnsInst *__restrict__ inst, const int4 *__restrict__ tiles, int ntiles, int parity)
{
    extern __shared__ float sm[];
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = __ldg(tiles + t);
        const EnsInst I = inst[tl.x];
        const Params<float> p = ens_params(I);
        const float *src = parity ? I.pop[1] : I.pop[0];
        float *dst = parity ? I.pop[0] : I.pop[1];
        const int tx0 = tl.y, ty0 = tl.z;
        const bool interior = tx0 >= 2 && tx0 + kTX + 1 <= p.nx - 1 && ty0 >= 2 && ty0 + 30 + 1 <= p.ny - 1;
        if (interior) two_steps<LBM_F32, CONV, DIFF, true, 30, false>(p, src, nullptr, dst, nullptr, sm, tx0, ty0);
        else two_steps<LBM_F32, CONV, DIFF, false, 30, false>(p, src, nullptr, dst, nullptr, sm, tx0, ty0);
        __syncthreads();                 // the next tile overwrites shared memory
    }
}

constexpr size_t kEns2Smem = 9 * Tile2<30>::kRP * sizeof(float);

cudaError_t ens_launch_step2(const lbm_ensemble_s *e, cudaStream_t st)
{
    dim3 block(32, kT2Threads / 32);
    const int grid = e->persistent2 ? e->grid2 : e->ntiles2;
    switch (e->family) {
    case 0: k_ens_step2<0, 0><<<grid, block, kEns2Smem, st>>>(e->d_inst, e->d_tiles2, e->ntiles2, e->parity); break;
    case 1: k_ens_step2<0, 1><<<grid, block, kEns2Smem, st>>>(e->d_inst, e->d_tiles2, e->ntiles2, e->parity); break;
    case 2: k_ens_step2<0, 2><<<grid, block, kEns2Smem, st>>>(e->d_inst, e->d_tiles2, e->ntiles2, e->parity); break;
    case 3: k_ens_step2<1, 0><<<grid, block, kEns2Smem, st>>>(e->d_inst, e->d_tiles2, e->ntiles2, e->parity); break;
    case 4: k_ens_step2<1, 1><<<grid, block, kEns2Smem, st>>>(e->d_inst, e->d_tiles2, e->ntiles2, e->parity); break;
    case 5: k_ens_step2<1, 2><<<grid, block, kEns2Smem, st>>>(e->d_inst, e->d_tiles2, e->ntiles2, e->parity); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int ens2_occupancy_blocks(int family)
{
    int per_sm = 0;
    cudaError_t err;
    switch (family) {
    case 0: err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_step2<0, 0>, kT2Threads, kEns2Smem); break;
    case 1: err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_step2<0, 1>, kT2Threads, kEns2Smem); break;
    case 2: err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_step2<0, 2>, kT2Threads, kEns2Smem); break;
    case 3: err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_step2<1, 0>, kT2Threads, kEns2Smem); break;
    case 4: err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_step2<1, 1>, kT2Threads, kEns2Smem); break;
    default: err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_step2<1, 2>, kT2Threads, kEns2Smem); break;
    }
    return err == cudaSuccess ? per_sm : -1;
}

}  // namespace lbm
