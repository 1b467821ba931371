// kernels_ensemble2.cu -- the ensemble with two time steps per sweep through
// HBM: one launch covers the tile list of every instance and runs a two-step
// tile routine of the single-grid kernels on each (FP32 storage, periodic
// walls, constant K per instance).
//
// Tile shapes: 30 x 30 output tiles with one node per thread (the routine of
// kernels_step2.cuh), or 62 x 14 output tiles with two x-adjacent nodes per
// thread (the routine of kernels_step2p.cuh); both keep 37 KB of shared memory
// per block. Launch modes: one block per tile (the hardware scheduler balances
// the blocks); a persistent grid of SMs x resident blocks walking the list with
// a fixed stride; or a persistent grid whose blocks claim the next tile from an
// atomic counter when they finish one. The claim needs no device-side wait: the
// last block to leave resets the counter for the next launch (it is the last
// one to have claimed), so graph replays find it at zero.
#include "kernels_step2p.cuh"
#include "lbm_ensemble.h"

namespace lbm {

template <int CONV, int DIFF, int SHAPE>
__device__ __forceinline__ void ens_tile2(const EnsInst *__restrict__ inst, int4 tl, int parity, float *sm)
{
    const EnsInst I = inst[tl.x];
    const Params<float> p = ens_params(I);
    const float *src = parity ? I.pop[1] : I.pop[0];
    float *dst = parity ? I.pop[0] : I.pop[1];
    const int tx0 = tl.y, ty0 = tl.z;
    if (SHAPE == 0) {
        const bool interior = tx0 >= 2 && tx0 + kTX + 1 <= p.nx - 1 && ty0 >= 2 && ty0 + 30 + 1 <= p.ny - 1;
        if (interior) two_steps<LBM_F32, CONV, DIFF, true, 30, false>(p, src, nullptr, dst, nullptr, sm, tx0, ty0);
        else two_steps<LBM_F32, CONV, DIFF, false, 30, false>(p, src, nullptr, dst, nullptr, sm, tx0, ty0);
    } else {
        constexpr int TY = kEns2PRows;
        const bool interior = tx0 >= 2 && tx0 + kPRX <= p.nx - 1 && ty0 >= 2 && ty0 + TY + 1 <= p.ny - 1;
        if (interior) two_steps_pair<LBM_F32, CONV, DIFF, true, TY, false>(p, src, nullptr, dst, nullptr, sm, tx0, ty0);
        else two_steps_pair_edge<LBM_F32, CONV, DIFF, TY, false>(p, src, nullptr, dst, nullptr, sm, tx0, ty0);
    }
}

// MODE 0: one block per tile; 1: a persistent grid walking the list with the
// grid's stride; 2: a persistent grid claiming tiles from claim[0], one tile
// ahead (claim[1] counts the blocks that left).
template <int CONV, int DIFF, int SHAPE, int MODE>
__global__ void __launch_bounds__(kT2Threads, 4)
k_ens_step2(const EnsInst *__restrict__ inst, const int4 *__restrict__ tiles, int ntiles, int parity, int *claim)
{
    extern __shared__ __align__(16) float sm_e[];
    __shared__ int next[2];
    if (MODE == 0) {
        ens_tile2<CONV, DIFF, SHAPE>(inst, __ldg(tiles + blockIdx.x), parity, sm_e);
        return;
    }
    const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
    int t = blockIdx.x, b = 0;
    if (MODE == 2) {
        if (lead) next[0] = atomicAdd(claim, 1);
        __syncthreads();
        t = next[0];
    }
    while (t < ntiles) {
        // claim the following tile while this one runs; the barrier that ends
        // the tile publishes it (slot b ^ 1 was last read before the previous
        // barrier)
        if (MODE == 2 && lead) next[b ^ 1] = atomicAdd(claim, 1);
        ens_tile2<CONV, DIFF, SHAPE>(inst, __ldg(tiles + t), parity, sm_e);
        __syncthreads();                 // the next tile overwrites shared memory
        if (MODE == 2) {
            b ^= 1;
            t = next[b];
        } else {
            t += gridDim.x;
        }
    }
    if (MODE == 2 && lead) {
        __threadfence();
        if (atomicAdd(claim + 1, 1) == (int)gridDim.x - 1) {
            atomicExch(claim, 0);
            atomicExch(claim + 1, 0);
        }
    }
}

constexpr size_t kEns2Smem = 9 * Tile2<30>::kRP * sizeof(float);
static_assert(9 * TileP<kEns2PRows>::kRP * sizeof(float) == kEns2Smem, "both tile shapes use the same shared memory");

template <int CONV, int DIFF, int SHAPE>
static cudaError_t ens2_launch_shape(const lbm_ensemble_s *e, cudaStream_t st)
{
    dim3 block(32, kT2Threads / 32);
    const int4 *tiles = SHAPE == 0 ? e->d_tiles2 : e->d_tiles2p;
    const int ntiles = SHAPE == 0 ? e->ntiles2 : e->ntiles2p;
    const int pgrid = SHAPE == 0 ? e->grid2 : e->grid2p;
    if (e->persistent2 == 2)
        k_ens_step2<CONV, DIFF, SHAPE, 2><<<pgrid, block, kEns2Smem, st>>>(e->d_inst, tiles, ntiles, e->parity, e->d_claim);
    else if (e->persistent2 == 1)
        k_ens_step2<CONV, DIFF, SHAPE, 1><<<pgrid, block, kEns2Smem, st>>>(e->d_inst, tiles, ntiles, e->parity, e->d_claim);
    else
        k_ens_step2<CONV, DIFF, SHAPE, 0><<<ntiles, block, kEns2Smem, st>>>(e->d_inst, tiles, ntiles, e->parity, e->d_claim);
    return cudaGetLastError();
}

template <int CONV, int DIFF>
static cudaError_t ens2_launch_f(const lbm_ensemble_s *e, cudaStream_t st)
{
    return e->shape2 ? ens2_launch_shape<CONV, DIFF, 1>(e, st) : ens2_launch_shape<CONV, DIFF, 0>(e, st);
}

cudaError_t ens_launch_step2(const lbm_ensemble_s *e, cudaStream_t st)
{
    switch (e->family) {
    case 0: return ens2_launch_f<0, 0>(e, st);
    case 1: return ens2_launch_f<0, 1>(e, st);
    case 2: return ens2_launch_f<0, 2>(e, st);
    case 3: return ens2_launch_f<1, 0>(e, st);
    case 4: return ens2_launch_f<1, 1>(e, st);
    case 5: return ens2_launch_f<1, 2>(e, st);
    }
    return cudaErrorInvalidValue;
}

template <int CONV, int DIFF>
static int ens2_occ(int shape)
{
    int per_sm = 0;
    const cudaError_t err =
        shape ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_step2<CONV, DIFF, 1, 2>, kT2Threads, kEns2Smem)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_step2<CONV, DIFF, 0, 2>, kT2Threads, kEns2Smem);
    return err == cudaSuccess ? per_sm : -1;
}

int ens2_occupancy_blocks(int family, int shape)
{
    switch (family) {
    case 0: return ens2_occ<0, 0>(shape);
    case 1: return ens2_occ<0, 1>(shape);
    case 2: return ens2_occ<0, 2>(shape);
    case 3: return ens2_occ<1, 0>(shape);
    case 4: return ens2_occ<1, 1>(shape);
    default: return ens2_occ<1, 2>(shape);
    }
}

}  // namespace lbm
