// kernels_step2_tma.cu -- the two-step tile kernel with the input region staged
// by the Tensor Memory Accelerator (FP32 storage).
//
// For an interior 30 x 30 output tile, one thread issues a single 3-D tensor
// copy (cp.async.bulk.tensor) of all nine population planes over the rows and
// columns step A pulls from (34 rows x 40 columns; the column start is rounded
// down to a 16-byte boundary) into shared memory; the copy completes on an
// mbarrier. Step A then reads only shared memory, so its global-load latency
// no longer stalls the warps; step B is the shared step of the tile kernel.
// Tiles touching the domain edge take the tile kernel's global-load path.
//
// The wait on the mbarrier is bounded: after kWaitLimit polls the block
// records kErrTimeout in the error word, waits (bounded again) for its copy,
// and returns without computing.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "kernels_step2.cuh"

namespace lbm {

namespace {

constexpr int kSW = 40, kSH = 34, kSPL = kSW * kSH;     // staged box: 40 columns x 34 rows per plane
constexpr unsigned kStageBytes = 9u * kSPL * sizeof(float);
constexpr int kErrTimeout = 16;
constexpr unsigned kWaitLimit = 1u << 22;

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return done != 0;
}

// bounded wait for phase `parity` of the barrier; false when the limit ran out
__device__ __forceinline__ bool mbar_wait_limit(unsigned long long *bar, unsigned parity, unsigned limit)
{
    for (unsigned i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity)
{
    return mbar_wait_limit(bar, parity, kWaitLimit);
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace

template <int CONV, int DIFF, bool KF>
__global__ void __launch_bounds__(kT2Threads, 2)
k_step2_tma(const Params<float> p, const __grid_constant__ CUtensorMap src_map, const float *__restrict__ src,
            float *__restrict__ dst)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    // [staged input 9 x 34 x 40 floats][step-A region 9 x 32 x 32 floats][mbarrier]
    float *stage = reinterpret_cast<float *>(smraw);
    float *sm = stage + 9 * kSPL;
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(sm + 9 * Tile2<30>::kRP);
    constexpr int kRP = Tile2<30>::kRP;
    const int tx0 = blockIdx.x * kTX, ty0 = blockIdx.y * 30;
    const bool interior = tx0 >= 2 && tx0 + kTX + 1 <= p.nx - 1 && ty0 >= 2 && ty0 + 30 + 1 <= p.ny - 1;
    if (!interior) {
        two_steps<LBM_F32, CONV, DIFF, false, 30, KF>(p, src, nullptr, dst, nullptr, sm, tx0, ty0);
        return;
    }
    const int lane = threadIdx.x, warp = threadIdx.y;
    const int tid = warp * 32 + lane;
    if (smem_u32(stage) & 127) {                    // a tensor copy needs a 128-byte aligned destination
        if (tid == 0) atomicOr(p.err, kErrShared);
        two_steps<LBM_F32, CONV, DIFF, true, 30, KF>(p, src, nullptr, dst, nullptr, sm, tx0, ty0);
        return;
    }
    // columns x0 - 2 .. x0 + 31 are pulled; the box starts at the 16-byte
    // boundary at or below x0 - 2 (x0 - 2 >= 0 for an interior tile)
    const int xs = (tx0 - 2) & ~3;
    if (tid == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(bar, kStageBytes);
        tma_load_3d(stage, &src_map, xs, ty0 - 2, 0, bar);
    }
    // The decision to give up is block-wide: if any thread's bounded wait ran
    // out, every thread reports and returns together, so no thread is left
    // behind at a later barrier. The block then waits once more (bounded) for
    // the copy to land before it leaves; if that wait runs out as well, the
    // block leaves with the copy possibly still in flight. Either way its tile's
    // output is not written, and the error word (lbm_debug_flags, 16) tells the
    // host that the results of this launch are not valid.
    const bool landed = mbar_wait_bounded(bar, 0);
    if (__syncthreads_or(!landed)) {
        if (tid == 0) atomicOr(p.err, kErrTimeout);
        mbar_wait_bounded(bar, 0);
        return;
    }

    const Params<F2> pw = widen(p);
    const long long P = p.plane;
    const int off = tx0 - 1 - xs;                   // staged column of region column 0, minus 1
    constexpr int kWarps = kT2Threads / 32;
    // ---- step A from the staged input: region rows hy = warp + 8 j, lane = hx
#pragma unroll 1
    for (int hy0 = warp; hy0 < 32; hy0 += 2 * kWarps) {
        float f[2][9], A3[2] = {p.A3, p.A3}, A35[2] = {p.A35, p.A35}, A5[2] = {p.A5, p.A5}, phi[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int hy = hy0 + h * kWarps;
#pragma unroll
            for (int k = 0; k < 9; ++k) f[h][k] = stage[k * kSPL + (hy + 1 - cy(k)) * kSW + lane + off - cx(k)];
            if (KF) {
                const unsigned own = (unsigned)(ty0 - 1 + hy) * (unsigned)p.pitch + (tx0 - 1 + lane);
                A3[h] = __ldg(p.Afield + own);
                A35[h] = __ldg(p.Afield + P + own);
                A5[h] = __ldg(p.Afield + 2 * P + own);
            }
        }
        collide_pair<CONV, DIFF, KF>(pw, f, A3, A35, A5, phi);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = (hy0 + h * kWarps) * kRX + lane;
#pragma unroll
            for (int k = 0; k < 9; ++k) sm[k * kRP + c] = f[h][k];
        }
    }
    __syncthreads();
    step2_B<LBM_F32, CONV, DIFF, true, 30, KF>(p, pw, dst, nullptr, sm, tx0, ty0);
}

namespace {

constexpr size_t kTmaSmem = kStageBytes + 9 * Tile2<30>::kRP * sizeof(float) + 64;

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    }
    return fn;
}

// 3-D map over one population buffer: x (pitch elements), y (rows), plane
bool make_map(CUtensorMap *map, const lbm_solver *s, const void *base)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)s->L.pitch, (cuuint64_t)s->d.ny, 9};
    const cuuint64_t strides[2] = {(cuuint64_t)s->L.pitch * 4, (cuuint64_t)s->L.plane * 4};
    const cuuint32_t box[3] = {kSW, kSH, 9};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int CONV, int DIFF, bool KF>
cudaError_t step2_tma_t(const lbm_solver *s, int src, cudaStream_t st)
{
    static SmemOptIn once;
    const cudaError_t e = opt_in_smem((const void *)k_step2_tma<CONV, DIFF, KF>, (int)kTmaSmem, once);
    if (e != cudaSuccess) return e;
    CUtensorMap map;
    if (!make_map(&map, s, s->pop[src])) return cudaErrorInvalidValue;
    const Params<float> p = make_params<float>(s);
    dim3 block(32, kT2Threads / 32);
    dim3 grid((s->d.nx + kTX - 1) / kTX, (s->d.ny + 29) / 30);
    k_step2_tma<CONV, DIFF, KF><<<grid, block, kTmaSmem, st>>>(p, map, (const float *)s->pop[src],
                                                              (float *)s->pop[src ^ 1]);
    return cudaGetLastError();
}

template <bool KF>
cudaError_t step2_tma_k(const lbm_solver *s, int src, cudaStream_t st)
{
    switch (s->c.conv * 3 + s->c.diff) {
    case 0: return step2_tma_t<0, 0, KF>(s, src, st);
    case 1: return step2_tma_t<0, 1, KF>(s, src, st);
    case 2: return step2_tma_t<0, 2, KF>(s, src, st);
    case 3: return step2_tma_t<1, 0, KF>(s, src, st);
    case 4: return step2_tma_t<1, 1, KF>(s, src, st);
    case 5: return step2_tma_t<1, 2, KF>(s, src, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_step2_tma(const lbm_solver *s, int src, cudaStream_t st)
{
    if (s->d.prec != LBM_F32) return cudaErrorInvalidValue;
    return s->d.per_cell_K ? step2_tma_k<true>(s, src, st) : step2_tma_k<false>(s, src, st);
}

// ---- failure detection without a fault ----------------------------------------
// The bounded mbarrier wait of the staged kernel, on a barrier that expects 16
// bytes no copy will ever deliver: every thread gives up after `limit` polls and
// the block reports instead of hanging. The barrier never completes, no copy is
// in flight, so the block may leave.
__global__ void k_wait_probe(unsigned limit, int *status)
{
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_expect_tx(&bar, 16);
    __syncthreads();
    const bool done = mbar_wait_limit(&bar, 0, limit);
    if (__syncthreads_or(!done) && threadIdx.x == 0) *status = 1;
    else if (threadIdx.x == 0) *status = 0;
}

}  // namespace lbm

extern "C" int lbm_debug_wait_probe(unsigned polls, int *dev_status, void *stream)
{
    using namespace lbm;
    if (!dev_status) return fail(LBM_EINVAL, "null status word");
    if (polls == 0 || polls > (1u << 24)) return fail(LBM_EINVAL, "polls must be in 1..2^24");
    cudaStream_t st = (cudaStream_t)stream;
    k_wait_probe<<<1, 64, 0, st>>>(polls, dev_status);
    if (int rc = cuda_check(cudaGetLastError(), "lbm_debug_wait_probe")) return rc;
    int timed_out = 0;
    if (int rc = cuda_check(cudaMemcpyAsync(&timed_out, dev_status, sizeof(int), cudaMemcpyDeviceToHost, st),
                            "lbm_debug_wait_probe copy"))
        return rc;
    if (int rc = cuda_check(cudaStreamSynchronize(st), "lbm_debug_wait_probe sync")) return rc;
    if (timed_out) return fail(LBM_ETIMEOUT, "the bounded wait ran out after " + std::to_string(polls) + " polls");
    return LBM_OK;
}
