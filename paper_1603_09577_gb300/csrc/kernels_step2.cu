// kernels_step2.cu -- two fused stream-collide time steps (Eq. 34) per sweep
// through HBM (temporal blocking), FP32 and BF16-shifted storage.
//
// A block owns a 30 x 62 output tile. Step A recomputes the state after the
// first step on the tile plus a one-node halo (32 x 64 nodes), pulling the
// populations straight from global memory, and keeps it in shared memory in
// FP32 (so the intermediate state is never rounded to the storage format).
// Step B pulls from shared memory and writes the state after the second step
// to the tile. Each population is then read and written once per two steps
// (36 B per node update in FP32 instead of 72 B); the halo costs 10% extra
// collisions. Halo reads of the neighbouring tiles' populations come from L2.
// Blocks whose region lies inside the domain skip all wrap and wall logic.
// Walls: periodic wrap or anti-bounce-back exactly as in the one-step kernel;
// halo nodes outside an anti-bounce-back wall do not exist and are skipped.
#include "lbm_internal.h"

namespace lbm {

// Output tile 30 x 62 nodes; the recomputed region (tile plus one-node halo)
// is then exactly 32 x 64: one warp per region row, every lane busy in step A.
constexpr int kTX = 30, kTY = 62;
constexpr int kRX = kTX + 2, kRY = kTY + 2;      // 32 x 64
constexpr int kT2Threads = 256;                  // 32 x 8
constexpr int kRP = kRX * kRY;                   // shared-memory plane (floats)

// Pull the nine populations of node (x, y) from global memory; INTERIOR: the
// node and its neighbours are inside the domain (no wrap, no wall).
template <int PREC, int CONV, int DIFF, bool INTERIOR>
__device__ __forceinline__ void pull_global(const Params<float> &p, const typename Store<PREC>::T *__restrict__ src,
                                            const float *__restrict__ src_h, int x, int y, float f[9])
{
    using S = Store<PREC>;
    const long long P = p.plane;
    int xm = x - 1, xp = x + 1, ym = y - 1, yp = y + 1;
    if (!INTERIOR) {
        xm = x == 0 ? p.nx - 1 : xm;
        xp = x == p.nx - 1 ? 0 : xp;
        ym = y == 0 ? p.ny - 1 : ym;
        yp = y == p.ny - 1 ? 0 : yp;
    }
    const unsigned pit = (unsigned)p.pitch;
    const unsigned r0 = (unsigned)y * pit, rm = (unsigned)ym * pit, rp = (unsigned)yp * pit;
    f[0] = S::ld(src, r0 + x, src_h, wgt<float>(0));
    f[1] = S::ld(src + 1 * P, r0 + xm, src_h, wgt<float>(1));
    f[2] = S::ld(src + 2 * P, rm + x, src_h, wgt<float>(2));
    f[3] = S::ld(src + 3 * P, r0 + xp, src_h, wgt<float>(3));
    f[4] = S::ld(src + 4 * P, rp + x, src_h, wgt<float>(4));
    f[5] = S::ld(src + 5 * P, rm + xm, src_h, wgt<float>(5));
    f[6] = S::ld(src + 6 * P, rm + xp, src_h, wgt<float>(6));
    f[7] = S::ld(src + 7 * P, rp + xp, src_h, wgt<float>(7));
    f[8] = S::ld(src + 8 * P, rp + xm, src_h, wgt<float>(8));
    if (!INTERIOR) {
        const bool wall = (p.abb_x && (x == 0 || x == p.nx - 1)) || (p.abb_y && (y == 0 || y == p.ny - 1));
        if (wall) {
            const unsigned own = r0 + x;
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
    }
}

template <int PREC, int CONV, int DIFF, bool INTERIOR>
__device__ __forceinline__ void two_steps(const Params<float> &p, const typename Store<PREC>::T *__restrict__ src,
                                          const float *__restrict__ src_h, typename Store<PREC>::T *__restrict__ dst,
                                          float *__restrict__ dst_h, float *sm, int tx0, int ty0)
{
    using S = Store<PREC>;
    const int lane = threadIdx.x, warp = threadIdx.y;
    const long long P = p.plane;

    // ---- step A: region rows hy = warp + 8 j; lane = hx. Two rows per pass keep
    // twice the global loads in flight. -------------------------------------------
    constexpr int kWarps = kT2Threads / 32;
    static_assert(kRY % (2 * kWarps) == 0, "region rows must split into row pairs");
#pragma unroll 1
    for (int hy0 = warp; hy0 < kRY; hy0 += 2 * kWarps) {
        float f[2][9];
        bool ok[2];
        int xs[2], ys[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int x = tx0 - 1 + lane, y = ty0 - 1 + hy0 + h * kWarps;
            bool valid = true;
            if (!INTERIOR) {
                // a halo node outside the domain wraps (periodic) or does not exist (wall)
                if (x < 0 || x >= p.nx) {
                    if (p.abb_x) valid = false;
                    else x = x < 0 ? x + p.nx : x - p.nx;
                }
                if (y < 0 || y >= p.ny) {
                    if (p.abb_y) valid = false;
                    else y = y < 0 ? y + p.ny : y - p.ny;
                }
                if (x < 0 || x >= p.nx || y < 0 || y >= p.ny) valid = false;
                if (!valid) { x = 0; y = 0; }          // any in-domain node; result unused
            }
            ok[h] = valid;
            xs[h] = x;
            ys[h] = y;
            pull_global<PREC, CONV, DIFF, INTERIOR>(p, src, src_h, x, y, f[h]);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float A3 = p.A3, A35 = p.A35, A5 = p.A5;
            if (p.Afield) {
                const unsigned own = (unsigned)ys[h] * (unsigned)p.pitch + xs[h];
                A3 = __ldg(p.Afield + own);
                A35 = __ldg(p.Afield + P + own);
                A5 = __ldg(p.Afield + 2 * P + own);
            }
            float phi;
            collide<float, CONV, DIFF>(p, f[h], A3, A35, A5, phi);
            if (INTERIOR || ok[h]) {
                const int c = (hy0 + h * kWarps) * kRX + lane;
#pragma unroll
                for (int k = 0; k < 9; ++k) sm[k * kRP + c] = f[h][k];
            }
        }
    }
    __syncthreads();

    // ---- step B: output rows r = warp, warp + 8, ...; lanes 0..29 ----------------
    const int x = tx0 + lane;
    if (lane >= kTX || x >= p.nx) return;
#pragma unroll 1
    for (int r = warp; r < kTY; r += kT2Threads / 32) {
        const int y = ty0 + r;
        if (!INTERIOR && y >= p.ny) return;
        const int c = (r + 1) * kRX + lane + 1;
        float f[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) f[k] = sm[k * kRP + c - cy(k) * kRX - cx(k)];
        if (!INTERIOR) {
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
                        f[k] = wall_term<float, CONV, DIFF>(p, k, phiw) - sm[opp(k) * kRP + c];
                    }
                }
            }
        }
        const unsigned own = (unsigned)y * (unsigned)p.pitch + x;
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

template <int PREC, int CONV, int DIFF>
__global__ void __launch_bounds__(kT2Threads, 3)
k_step2(const Params<float> p, const typename Store<PREC>::T *__restrict__ src, const float *__restrict__ src_h,
        typename Store<PREC>::T *__restrict__ dst, float *__restrict__ dst_h)
{
    extern __shared__ float sm[];       // 9 planes of kRY x kRX
    const int tx0 = blockIdx.x * kTX, ty0 = blockIdx.y * kTY;
    // interior block: the region and every node it pulls from lie inside the
    // domain, so no wrap and no wall can occur
    const bool interior = tx0 >= 2 && tx0 + kTX + 1 <= p.nx - 1 && ty0 >= 2 && ty0 + kTY + 1 <= p.ny - 1;
    if (interior) two_steps<PREC, CONV, DIFF, true>(p, src, src_h, dst, dst_h, sm, tx0, ty0);
    else two_steps<PREC, CONV, DIFF, false>(p, src, src_h, dst, dst_h, sm, tx0, ty0);
}

constexpr size_t kStep2Smem = 9 * kRP * sizeof(float);

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
    dim3 grid((s->d.nx + kTX - 1) / kTX, (s->d.ny + kTY - 1) / kTY);
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
