// probe_fp64.cu -- measured rate of the FP64 pipe, the roof of the FP64
// stream-collide kernel (whose 118 FP64 instructions per node update keep it
// far from the HBM roof on a GPU with a reduced FP64 rate).
//
// Every thread runs kChains independent fused multiply-add recurrences
// x <- x * b + c for `iters` iterations; with enough resident warps the FP64
// pipe, not the dependency latency, limits the rate. The caller times the
// launch with CUDA events; the launch executes blocks * threads * iters *
// kChains FP64 thread instructions.
#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr int kChains = 8;

__global__ void k_dfma_probe(double b, double c, int iters, double *__restrict__ sink)
{
    double x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = 1.0 + 1e-3 * j + 1e-9 * threadIdx.x;
#pragma unroll 1
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], b, c);
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    // the recurrence converges to c / (1 - b); the store keeps the chains live
    if (s == -1.0) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace lbm

extern "C" int lbm_probe_fp64(int blocks, int threads, int iters, double *dev_sink, long long *fp64_inst,
                              void *stream)
{
    using namespace lbm;
    if (blocks < 1 || threads < 32 || threads > 1024 || threads % 32 || iters < 1 || !dev_sink)
        return fail(LBM_EINVAL, "lbm_probe_fp64: blocks >= 1, threads a multiple of 32 in [32, 1024], iters >= 1, "
                                "a device sink of `blocks` doubles");
    k_dfma_probe<<<blocks, threads, 0, (cudaStream_t)stream>>>(0.999999, 1e-6, iters, dev_sink);
    if (int rc = cuda_check(cudaGetLastError(), "lbm_probe_fp64")) return rc;
    if (fp64_inst) *fp64_inst = (long long)blocks * threads * iters * kChains;
    return LBM_OK;
}
