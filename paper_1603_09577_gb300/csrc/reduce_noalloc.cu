// reduce_noalloc.cu -- the FP64 field reductions for callers that cannot
// allocate device memory at all.
//
// Who needs it: a caller whose host application owns the whole device memory
// budget (a fixed pool handed out by its own manager), or one that may not call
// cudaMalloc/cudaFree because those calls synchronise the device, has no way to
// provide the workspace lbm_reduce takes from a solver. This entry point takes
// only the caller's input and output buffers; the per-block partial sums live
// in a fixed file-scope device array instead of a workspace.
//
// The array (kNaMaxBlocks x 8 doubles = 512 KiB) is part of the library image:
// every GPU that loads the library holds it until the process exits. All calls
// share it and it keeps the last call's contents. Pass 1 writes every slot that
// pass 2 reads, so nothing has to start at zero. Calls whose kernels overlap on
// the GPU (different streams, or several host threads) race on the array: order
// them on one stream.
#include <mutex>
#include <string>

#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaChunk = 8192;                                   // values per block
constexpr int kNaMaxBlocks = 8192;                               // slots in the scratch
constexpr long long kNaMaxValues = (long long)kNaChunk * kNaMaxBlocks;   // 67,108,864
constexpr int kNaAcc = 8;
constexpr int kNaMaxDevices = 64;

static __device__ __align__(256) double g_na_partials[kNaMaxBlocks * kNaAcc];

std::mutex g_na_mu;
double *g_na_ptr[kNaMaxDevices] = {};

__device__ __forceinline__ double na_combine(int j, double a, double b) { return j == 5 ? fmax(a, b) : a + b; }

// fixed-order tree over one block: warp shuffles, then warp 0's lanes in order
__device__ __forceinline__ void na_block_reduce(double v[kNaAcc], double *out)
{
    __shared__ double sh[kNaThreads / 32][kNaAcc];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int j = 0; j < kNaAcc; ++j) v[j] = na_combine(j, v[j], __shfl_down_sync(0xffffffffu, v[j], off));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < kNaAcc; ++j) sh[w][j] = v[j];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int j = 0; j < kNaAcc; ++j) {
            double a = sh[0][j];
            for (int q = 1; q < kNaThreads / 32; ++q) a = na_combine(j, a, sh[q][j]);
            out[j] = a;
        }
}

// pass 1: block b reduces values [b * kNaChunk, (b + 1) * kNaChunk)
__global__ void __launch_bounds__(kNaThreads)
k_na_reduce1(const double *__restrict__ phi, const double *__restrict__ ref, long long n, double *__restrict__ partials)
{
    double v[kNaAcc] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long begin = (long long)blockIdx.x * kNaChunk;
    const long long end = begin + kNaChunk < n ? begin + kNaChunk : n;
    for (long long i = begin + threadIdx.x; i < end; i += kNaThreads) {
        const double ph = phi[i];
        if (!isfinite(ph)) { v[6] += 1.0; continue; }
        v[0] += ph;
        v[7] += ph * ph;
        v[5] = fmax(v[5], fabs(ph));
        if (ref) {
            const double r = ref[i], d = ph - r;
            v[1] += fabs(d);
            v[2] += fabs(r);
            v[3] += d * d;
            v[4] += r * r;
        }
    }
    na_block_reduce(v, partials + (size_t)blockIdx.x * kNaAcc);
}

// pass 2: one block combines the partials in slot order
__global__ void __launch_bounds__(kNaThreads) k_na_reduce2(const double *__restrict__ partials, int nb, double *__restrict__ out)
{
    double v[kNaAcc] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nb; b += kNaThreads)
#pragma unroll
        for (int j = 0; j < kNaAcc; ++j) v[j] = na_combine(j, v[j], partials[(size_t)b * kNaAcc + j]);
    na_block_reduce(v, out);
}

// Device address of the scratch on the current device. Host code may not pass
// g_na_partials itself to a kernel: in host code that name is a host-side
// stand-in. The address is looked up once per device, with that device current.
int na_scratch(double **ptr)
{
    int dev = -1;
    if (int rc = cuda_check(cudaGetDevice(&dev), "lbm_reduce_field_noalloc: cudaGetDevice")) return rc;
    if (dev < 0 || dev >= kNaMaxDevices) return fail(LBM_EUNSUPPORTED, "lbm_reduce_field_noalloc: device ordinal >= 64");
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        if (int rc = cuda_check(cudaGetSymbolAddress(&p, g_na_partials), "lbm_reduce_field_noalloc: cudaGetSymbolAddress"))
            return rc;
        g_na_ptr[dev] = (double *)p;
    }
    *ptr = g_na_ptr[dev];
    return LBM_OK;
}

}  // namespace
}  // namespace lbm

extern "C" int lbm_reduce_field_noalloc(const double *dev_phi, const double *dev_ref, long long n, double *dev_out,
                                        void *stream)
{
    using namespace lbm;
    if (!dev_phi || !dev_out) return fail(LBM_EINVAL, "lbm_reduce_field_noalloc: null field or output");
    if (n < 1) return fail(LBM_EINVAL, "lbm_reduce_field_noalloc: n must be >= 1");
    if (n > kNaMaxValues)
        return fail(LBM_EINVAL, "lbm_reduce_field_noalloc: n = " + std::to_string(n) +
                                    " exceeds the static scratch capacity of " + std::to_string(kNaMaxValues) + " values");
    double *scratch = nullptr;
    if (int rc = na_scratch(&scratch)) return rc;
    const int nb = (int)((n + kNaChunk - 1) / kNaChunk);
    cudaStream_t st = (cudaStream_t)stream;
    k_na_reduce1<<<nb, kNaThreads, 0, st>>>(dev_phi, dev_ref, n, scratch);
    if (int rc = cuda_check(cudaGetLastError(), "lbm_reduce_field_noalloc: pass 1")) return rc;
    k_na_reduce2<<<1, kNaThreads, 0, st>>>(scratch, nb, dev_out);
    return cuda_check(cudaGetLastError(), "lbm_reduce_field_noalloc: pass 2");
}
