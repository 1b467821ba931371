// kernels_ensemble.cu -- many independent lattices advanced together: one
// persistent launch per time step over a work list of 32 x 8 tiles drawn from
// every instance (FP32 storage, periodic walls, one coefficient family shared,
// per-instance u, K and relaxation rates). Blocks take tiles round-robin (t = blockIdx.x,
// blockIdx.x + gridDim.x, ...): tiles have equal shape, so the static split is
// balanced and no block ever waits on another.
#include "lbm_ensemble.h"

namespace lbm {

template <int CONV, int DIFF>
__device__ __forceinline__ void ens_tile(const EnsInst &I, int tx0, int ty0, int parity)
{
    const Params<float> p = ens_params(I);
    // select with a conditional: a runtime index into the struct's array would
    // put the struct in local memory
    const float *__restrict__ src = parity ? I.pop[1] : I.pop[0];
    float *__restrict__ dst = parity ? I.pop[0] : I.pop[1];
    const int x = tx0 + threadIdx.x;
    const int y = ty0 + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    int xm = x == 0 ? p.nx - 1 : x - 1;
    int xp = x == p.nx - 1 ? 0 : x + 1;
    LBM_CHK(xm, p.nx, p.err, kErrX);
    LBM_CHK(xp, p.nx, p.err, kErrX);
    const long long P = p.plane;
    {
        int ym = y == 0 ? p.ny - 1 : y - 1;
        int yp = y == p.ny - 1 ? 0 : y + 1;
        LBM_CHK(ym, p.ny, p.err, kErrY);
        LBM_CHK(yp, p.ny, p.err, kErrY);
        const long long r0 = (long long)y * p.pitch, rm = (long long)ym * p.pitch, rp = (long long)yp * p.pitch;
        const long long own = r0 + x;
        float f[9];
        f[0] = __ldg(src + own);
        f[1] = __ldg(src + 1 * P + r0 + xm);
        f[2] = __ldg(src + 2 * P + rm + x);
        f[3] = __ldg(src + 3 * P + r0 + xp);
        f[4] = __ldg(src + 4 * P + rp + x);
        f[5] = __ldg(src + 5 * P + rm + xm);
        f[6] = __ldg(src + 6 * P + rm + xp);
        f[7] = __ldg(src + 7 * P + rp + xp);
        f[8] = __ldg(src + 8 * P + rp + xm);
        float phi;
        collide<float, CONV, DIFF, false>(p, f, p.A3, p.A35, p.A5, phi);
#pragma unroll
        for (int k = 0; k < 9; ++k) __stcs(dst + k * P + own, f[k]);
    }
}

template <int CONV, int DIFF>
__global__ void __launch_bounds__(kEnsThreads)
k_ens_step(const EnsInst *__restrict__ inst, const int4 *__restrict__ tiles, int t_begin,
           int t_end, int parity)
{
    for (int t = t_begin + blockIdx.x; t < t_end; t += gridDim.x) {
        const int4 tl = __ldg(tiles + t);
        const EnsInst I = inst[tl.x];
        ens_tile<CONV, DIFF>(I, tl.y, tl.z, parity);
    }
}

// initial condition of every instance (Eq. 40, no source): fbar = feq(phi0),
// then one collision, as for a single lattice
template <int CONV, int DIFF>
__global__ void __launch_bounds__(kEnsThreads)
k_ens_init(const EnsInst *__restrict__ inst, const int4 *__restrict__ tiles, int ntiles,
           const void *__restrict__ phi, int in_prec, int parity)
{
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = __ldg(tiles + t);
        const EnsInst I = inst[tl.x];
        const Params<float> p = ens_params(I);
        const int x = tl.y + threadIdx.x;
        if (x >= I.nx) continue;
        {
            const int y = tl.z + threadIdx.y;
            if (y >= I.ny) continue;
            const long long i = I.phi_off + (long long)y * I.nx + x;
            const float ph = in_prec == LBM_F64 ? (float)((const double *)phi)[i] : ((const float *)phi)[i];
            float f[9], phi_c;
            equilibrium<float, CONV, DIFF>(p, ph, f);
            collide<float, CONV, DIFF, false>(p, f, p.A3, p.A35, p.A5, phi_c);
            const long long own = (long long)y * I.pitch + x;
#pragma unroll
            for (int k = 0; k < 9; ++k) (parity ? I.pop[1] : I.pop[0])[k * I.plane + own] = f[k];
        }
    }
}

__global__ void __launch_bounds__(kEnsThreads)
k_ens_get_phi(const EnsInst *__restrict__ inst, const int4 *__restrict__ tiles, int ntiles, int parity,
              void *__restrict__ out, int out_prec)
{
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = __ldg(tiles + t);
        const EnsInst I = inst[tl.x];
        const int x = tl.y + threadIdx.x;
        if (x >= I.nx) continue;
        {
            const int y = tl.z + threadIdx.y;
            if (y >= I.ny) continue;
            const long long own = (long long)y * I.pitch + x;
            const float *f = parity ? I.pop[1] : I.pop[0];
            float s = f[own];
#pragma unroll
            for (int k = 1; k < 9; ++k) s += f[k * I.plane + own];
            const long long o = I.phi_off + (long long)y * I.nx + x;
            if (out_prec == LBM_F64) ((double *)out)[o] = (double)s;
            else ((float *)out)[o] = s;
        }
    }
}

// ---- per-instance statistics (the eight of lbm_reduce), FP64, fixed order ----
// Pass 1: each 32 x 8 tile's statistics, a block per tile (grid-stride over the
// list), combined by a fixed-order warp-shuffle and shared-memory tree. The
// tiles of an instance are contiguous in the list, so pass 2 (one block per
// instance) combines the instance's tile partials in list order. Every sum is
// taken in the same order on every call: the results are reproducible bit for bit.
constexpr int kEnsAcc = 8;

__device__ __forceinline__ double ens_combine(int j, double a, double b) { return j == 5 ? fmax(a, b) : a + b; }

// fixed-order reduction of v over the block into out (thread 0 writes)
__device__ __forceinline__ void ens_block_reduce(double v[kEnsAcc], double *__restrict__ out)
{
    __shared__ double sh[kEnsThreads / 32][kEnsAcc];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int j = 0; j < kEnsAcc; ++j) v[j] = ens_combine(j, v[j], __shfl_down_sync(0xffffffffu, v[j], off));
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if ((tid & 31) == 0)
#pragma unroll
        for (int j = 0; j < kEnsAcc; ++j) sh[tid >> 5][j] = v[j];
    __syncthreads();
    if (tid == 0)
        for (int j = 0; j < kEnsAcc; ++j) {
            double a = sh[0][j];
            for (int w = 1; w < kEnsThreads / 32; ++w) a = ens_combine(j, a, sh[w][j]);
            out[j] = a;
        }
    __syncthreads();                        // sh is reused by the block's next tile
}

__global__ void __launch_bounds__(kEnsThreads)
k_ens_reduce1(const EnsInst *__restrict__ inst, const int4 *__restrict__ tiles, int ntiles, int parity,
              const double *__restrict__ ref, double *__restrict__ partials)
{
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int4 tl = __ldg(tiles + t);
        const EnsInst I = inst[tl.x];
        const int x = tl.y + threadIdx.x, y = tl.z + threadIdx.y;
        double v[kEnsAcc] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (x < I.nx && y < I.ny) {
            // phi(t_n) exactly as lbm_ensemble_get_phi forms it (FP32 sum in k order)
            const long long own = (long long)y * I.pitch + x;
            const float *f = parity ? I.pop[1] : I.pop[0];
            float s = f[own];
#pragma unroll
            for (int k = 1; k < 9; ++k) s += f[k * I.plane + own];
            const double ph = (double)s;
            if (!isfinite(ph)) {
                v[6] = 1.0;
            } else {
                v[0] = ph;
                v[7] = ph * ph;
                v[5] = fabs(ph);
                if (ref) {
                    const double r = ref[I.phi_off + (long long)y * I.nx + x], d = ph - r;
                    v[1] = fabs(d);
                    v[2] = fabs(r);
                    v[3] = d * d;
                    v[4] = r * r;
                }
            }
        }
        ens_block_reduce(v, partials + (size_t)t * kEnsAcc);
    }
}

__global__ void __launch_bounds__(kEnsThreads)
k_ens_reduce2(const double *__restrict__ partials, const int *__restrict__ tile_begin, double *__restrict__ out)
{
    const int i = blockIdx.x;
    const int b0 = tile_begin[i], b1 = tile_begin[i + 1];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    double v[kEnsAcc] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = b0 + tid; b < b1; b += kEnsThreads)
#pragma unroll
        for (int j = 0; j < kEnsAcc; ++j) v[j] = ens_combine(j, v[j], partials[(size_t)b * kEnsAcc + j]);
    ens_block_reduce(v, out + (size_t)i * kEnsAcc);
}

cudaError_t ens_launch_reduce(const lbm_ensemble_s *e, const double *ref, double *out, cudaStream_t st)
{
    dim3 block(kEnsTile, kEnsRows);
    k_ens_reduce1<<<e->grid, block, 0, st>>>(e->d_inst, e->d_tiles, e->ntiles, e->parity, ref, e->partials);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    k_ens_reduce2<<<e->count, block, 0, st>>>(e->partials, e->d_tile_begin, out);
    return cudaGetLastError();
}

#define LBM_ENS_DISPATCH(KEY, CALL)                    \
    switch (KEY) {                                     \
    case 0: CALL(0, 0); break;                         \
    case 1: CALL(0, 1); break;                         \
    case 2: CALL(0, 2); break;                         \
    case 3: CALL(1, 0); break;                         \
    case 4: CALL(1, 1); break;                         \
    case 5: CALL(1, 2); break;                         \
    default: return cudaErrorInvalidValue;             \
    }

cudaError_t ens_launch_step(const lbm_ensemble_s *e, int t_begin, int t_end, int blocks, cudaStream_t st)
{
    dim3 block(kEnsTile, kEnsRows);
#define CALL(A, B) k_ens_step<A, B><<<blocks, block, 0, st>>>(e->d_inst, e->d_tiles, t_begin, t_end, e->parity)
    LBM_ENS_DISPATCH(e->family, CALL)
#undef CALL
    return cudaGetLastError();
}

cudaError_t ens_launch_init(const lbm_ensemble_s *e, const void *phi, int in_prec, cudaStream_t st)
{
    dim3 block(kEnsTile, kEnsRows);
#define CALL(A, B) k_ens_init<A, B><<<e->grid, block, 0, st>>>(e->d_inst, e->d_tiles, e->ntiles, phi, in_prec, e->parity)
    LBM_ENS_DISPATCH(e->family, CALL)
#undef CALL
    return cudaGetLastError();
}

cudaError_t ens_launch_get_phi(const lbm_ensemble_s *e, void *out, int out_prec, cudaStream_t st)
{
    dim3 block(kEnsTile, kEnsRows);
    k_ens_get_phi<<<e->grid, block, 0, st>>>(e->d_inst, e->d_tiles, e->ntiles, e->parity, out, out_prec);
    return cudaGetLastError();
}

int ens_occupancy_blocks(int family)
{
    int per_sm = 1;
    const int threads = kEnsThreads;
    cudaError_t err;
#define CALL(A, B) err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_step<A, B>, threads, 0)
    switch (family) {
    case 0: CALL(0, 0); break;
    case 1: CALL(0, 1); break;
    case 2: CALL(0, 2); break;
    case 3: CALL(1, 0); break;
    case 4: CALL(1, 1); break;
    default: CALL(1, 2); break;
    }
#undef CALL
    if (err != cudaSuccess) return -1;
    return per_sm;
}

}  // namespace lbm
