// kernels_step2.cu -- two fused stream-collide time steps (Eq. 34) per sweep
// through HBM (temporal blocking), FP32 and BF16-shifted storage.
//
// A block owns a 32 x 32 output tile. Step A recomputes the state after the
// first step on the tile plus a one-node halo (34 x 34 nodes), pulling the
// populations straight from global memory, and keeps it in shared memory in
// FP32 (so the intermediate state is never rounded to the storage format).
// Step B pulls from shared memory and writes the state after the second step
// to the tile. Each population is then read and written once per two steps
// (36 B per node update in FP32 instead of 72 B); the halo costs 13% extra
// collisions. Halo reads of the neighbouring tiles' populations come from L2.
// Walls: periodic wrap or anti-bounce-back exactly as in the one-step kernel;
// halo nodes outside an anti-bounce-back wall do not exist and are skipped.
#include "lbm_internal.h"

namespace lbm {

constexpr int kT2 = 32;                 // output tile edge
constexpr int kH2 = kT2 + 2;            // tile plus one-node halo
constexpr int kT2Threads = 256;         // 32 x 8

template <int PREC, int CONV, int DIFF>
__global__ void __launch_bounds__(kT2Threads)
k_step2(const Params<float> p, const typename Store<PREC>::T *__restrict__ src, const float *__restrict__ src_h,
        typename Store<PREC>::T *__restrict__ dst, float *__restrict__ dst_h)
{
    using S = Store<PREC>;
    extern __shared__ float sm[];       // 9 planes of kH2 x kH2
    constexpr int SP = kH2 * kH2;
    const int tx0 = blockIdx.x * kT2, ty0 = blockIdx.y * kT2;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const long long P = p.plane;

    // ---- step A: tile + halo, t_n -> t_{n+1}, into shared memory --------------
    for (int i = tid; i < SP; i += kT2Threads) {
        const int hy = i / kH2, hx = i - hy * kH2;
        int x = tx0 - 1 + hx, y = ty0 - 1 + hy;
        // halo node outside the domain: wrap if periodic, absent if a wall
        if (x < 0 || x >= p.nx) {
            if (p.abb_x) continue;
            x = x < 0 ? x + p.nx : x - p.nx;
        }
        if (y < 0 || y >= p.ny) {
            if (p.abb_y) continue;
            y = y < 0 ? y + p.ny : y - p.ny;
        }
        if (x < 0 || x >= p.nx || y < 0 || y >= p.ny) continue;   // grids narrower than the halo
        const int xm = x == 0 ? p.nx - 1 : x - 1, xp = x == p.nx - 1 ? 0 : x + 1;
        const int ym = y == 0 ? p.ny - 1 : y - 1, yp = y == p.ny - 1 ? 0 : y + 1;
        const long long r0 = (long long)y * p.pitch, rm = (long long)ym * p.pitch, rp = (long long)yp * p.pitch;
        const long long own = r0 + x;
        float f[9];
        f[0] = S::ld(src, own, src_h, wgt<float>(0));
        f[1] = S::ld(src + 1 * P, r0 + xm, src_h, wgt<float>(1));
        f[2] = S::ld(src + 2 * P, rm + x, src_h, wgt<float>(2));
        f[3] = S::ld(src + 3 * P, r0 + xp, src_h, wgt<float>(3));
        f[4] = S::ld(src + 4 * P, rp + x, src_h, wgt<float>(4));
        f[5] = S::ld(src + 5 * P, rm + xm, src_h, wgt<float>(5));
        f[6] = S::ld(src + 6 * P, rm + xp, src_h, wgt<float>(6));
        f[7] = S::ld(src + 7 * P, rp + xp, src_h, wgt<float>(7));
        f[8] = S::ld(src + 8 * P, rp + xm, src_h, wgt<float>(8));
        const bool wall = (p.abb_x && (x == 0 || x == p.nx - 1)) || (p.abb_y && (y == 0 || y == p.ny - 1));
        if (wall) {
#pragma unroll
            for (int k = 1; k < 9; ++k) {
                const int xs = x - cx(k), ys = y - cy(k);
                const bool ox = p.abb_x && (xs < 0 || xs >= p.nx);
                const bool oy = p.abb_y && (ys < 0 || ys >= p.ny);
                if (ox || oy) {
                    const float wx = xs < 0 ? p.phi_wall[0] : p.phi_wall[1];
                    const float wy = ys < 0 ? p.phi_wall[2] : p.phi_wall[3];
                    const float phiw = (ox && oy) ? 0.5f * (wx + wy) : (ox ? wx : wy);
                    f[k] = wall_term<float, CONV, DIFF>(p, k, phiw) - S::ld(src + opp(k) * P, own, src_h, wgt<float>(opp(k)));
                }
            }
        }
        float A3 = p.A3, A35 = p.A35, A5 = p.A5;
        if (p.Afield) {
            A3 = __ldg(p.Afield + own);
            A35 = __ldg(p.Afield + P + own);
            A5 = __ldg(p.Afield + 2 * P + own);
        }
        float phi;
        collide<float, CONV, DIFF>(p, f, A3, A35, A5, phi);
#pragma unroll
        for (int k = 0; k < 9; ++k) sm[k * SP + i] = f[k];
    }
    __syncthreads();

    // ---- step B: tile, t_{n+1} -> t_{n+2}, from shared memory -------------------
    const int x = tx0 + threadIdx.x;
    if (x >= p.nx) return;
#pragma unroll 1
    for (int r = threadIdx.y; r < kT2; r += blockDim.y) {
        const int y = ty0 + r;
        if (y >= p.ny) return;
        const int hx = threadIdx.x + 1, hy = r + 1;
        const int c = hy * kH2 + hx;
        float f[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) f[k] = sm[k * SP + c - cy(k) * kH2 - cx(k)];
        const bool wall = (p.abb_x && (x == 0 || x == p.nx - 1)) || (p.abb_y && (y == 0 || y == p.ny - 1));
        if (wall) {
#pragma unroll
            for (int k = 1; k < 9; ++k) {
                const int xs = x - cx(k), ys = y - cy(k);
                const bool ox = p.abb_x && (xs < 0 || xs >= p.nx);
                const bool oy = p.abb_y && (ys < 0 || ys >= p.ny);
                if (ox || oy) {
                    const float wx = xs < 0 ? p.phi_wall[0] : p.phi_wall[1];
                    const float wy = ys < 0 ? p.phi_wall[2] : p.phi_wall[3];
                    const float phiw = (ox && oy) ? 0.5f * (wx + wy) : (ox ? wx : wy);
                    f[k] = wall_term<float, CONV, DIFF>(p, k, phiw) - sm[opp(k) * SP + c];
                }
            }
        }
        const long long own = (long long)y * p.pitch + x;
        float A3 = p.A3, A35 = p.A35, A5 = p.A5;
        if (p.Afield) {
            A3 = __ldg(p.Afield + own);
            A35 = __ldg(p.Afield + P + own);
            A5 = __ldg(p.Afield + 2 * P + own);
        }
        float phi;
        collide<float, CONV, DIFF>(p, f, A3, A35, A5, phi);
        S::store_cell(dst, dst_h, P, own, f, phi);
    }
}

constexpr size_t kStep2Smem = 9 * kH2 * kH2 * sizeof(float);

template <int PREC, int CONV, int DIFF>
static cudaError_t step2_t(const lbm_solver *s, int src, cudaStream_t st)
{
    using T = typename Store<PREC>::T;
    // opt in to more than 48 KB of dynamic shared memory (per device, so every call)
    cudaError_t e = cudaFuncSetAttribute(k_step2<PREC, CONV, DIFF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kStep2Smem);
    if (e != cudaSuccess) return e;
    const Params<float> p = make_params<float>(s);
    dim3 block(32, kT2Threads / 32);
    dim3 grid((s->d.nx + kT2 - 1) / kT2, (s->d.ny + kT2 - 1) / kT2);
    k_step2<PREC, CONV, DIFF><<<grid, block, kStep2Smem, st>>>(p, (const T *)s->pop[src], s->phi[src],
                                                               (T *)s->pop[src ^ 1], s->phi[src ^ 1]);
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t step2_p(const lbm_solver *s, int src, cudaStream_t st)
{
    switch (s->c.conv * 3 + s->c.diff) {
    case 0: return step2_t<PREC, 0, 0>(s, src, st);
    case 1: return step2_t<PREC, 0, 1>(s, src, st);
    case 2: return step2_t<PREC, 0, 2>(s, src, st);
    case 3: return step2_t<PREC, 1, 0>(s, src, st);
    case 4: return step2_t<PREC, 1, 1>(s, src, st);
    case 5: return step2_t<PREC, 1, 2>(s, src, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_step2(const lbm_solver *s, int src, cudaStream_t st)
{
    if (s->d.prec == LBM_F32) return step2_p<LBM_F32>(s, src, st);
    if (s->d.prec == LBM_BF16S) return step2_p<LBM_BF16S>(s, src, st);
    return cudaErrorInvalidValue;
}

}  // namespace lbm
