// kernels_step2.cuh -- two fused stream-collide time steps (Eq. 34) per sweep
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
#pragma once

#include "lbm_internal.h"

namespace lbm {

// Output tile 30 x TY nodes; the recomputed region (tile plus one-node halo)
// is then exactly 32 x (TY + 2): one warp per region row, every lane busy in
// step A. TY = 62 (73.7 KB of shared memory, 3 blocks per SM) or TY = 30
// (36.9 KB, registers capped so that 4 blocks fit).
constexpr int kTX = 30;
constexpr int kRX = kTX + 2;                     // 32
constexpr int kT2Threads = 256;                  // 32 x 8
template <int TY> struct Tile2 {
    static constexpr int kTY = TY, kRY = TY + 2, kRP = kRX * kRY;
    static constexpr int kMinBlocks = TY > 32 ? 3 : 4;
};

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
    LBM_CHK(x, p.nx, p.err, kErrX);
    LBM_CHK(y, p.ny, p.err, kErrY);
    LBM_CHK(xm, p.nx, p.err, kErrX);
    LBM_CHK(xp, p.nx, p.err, kErrX);
    LBM_CHK(ym, p.ny, p.err, kErrY);
    LBM_CHK(yp, p.ny, p.err, kErrY);
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

// the coefficients of a Params<float> broadcast to both halves of the packed type
__device__ __forceinline__ Params<F2> widen(const Params<float> &p)
{
    Params<F2> w;
    w.nx = p.nx; w.ny = p.ny; w.pitch = p.pitch; w.plane = p.plane;
    w.abb_x = p.abb_x; w.abb_y = p.abb_y;
    w.s1 = p.s1; w.s2 = p.s2; w.s4 = p.s4; w.s6 = p.s6; w.s7 = p.s7; w.s8 = p.s8;
    w.h1 = p.h1; w.h2 = p.h2; w.h4 = p.h4; w.h6 = p.h6;
    w.A3 = p.A3; w.A35 = p.A35; w.A5 = p.A5;
    w.se1 = p.se1; w.se2 = p.se2; w.sq4 = p.sq4; w.sq6 = p.sq6; w.sp7 = p.sp7; w.sp8 = p.sp8;
    w.he1 = p.he1; w.he2 = p.he2; w.hq4 = p.hq4; w.hq6 = p.hq6;
    w.a3s = p.a3s; w.a35s = p.a35s; w.a5s = p.a5s; w.c3s = p.c3s; w.c35s = p.c35s; w.c5s = p.c5s;
    w.ux = p.ux; w.uy = p.uy; w.uxx = p.uxx; w.uxy = p.uxy; w.uyy = p.uyy;
    w.r0 = p.r0; w.r1 = p.r1; w.half_r0 = p.half_r0; w.inv_den = p.inv_den; w.inv_post = p.inv_post;
    w.has_src = p.has_src;
    w.Afield = nullptr;
    return w;
}

// collide two nodes with one packed instruction stream; NODE_K: A3, A35, A5
// are the nodes' blocks (per-node tensor field), else the constant block of pw
template <int CONV, int DIFF, bool NODE_K>
__device__ __forceinline__ void collide_pair(const Params<F2> &pw, float f[2][9], const float A3[2], const float A35[2],
                                             const float A5[2], float phi[2])
{
    F2 g[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) g[k] = F2(f[0][k], f[1][k]);
    F2 ph;
    collide<F2, CONV, DIFF, NODE_K>(pw, g, F2(A3[0], A3[1]), F2(A35[0], A35[1]), F2(A5[0], A5[1]), ph);
#pragma unroll
    for (int k = 0; k < 9; ++k) { f[0][k] = g[k].v.x; f[1][k] = g[k].v.y; }
    phi[0] = ph.v.x;
    phi[1] = ph.v.y;
}

// Step B of the two-step tile: output rows in pairs from the shared-memory
// region sm (the state after the first step), stored to global memory.
template <int PREC, int CONV, int DIFF, bool INTERIOR, int TY, bool KF>
__device__ __forceinline__ void step2_B(const Params<float> &p, const Params<F2> &pw,
                                        typename Store<PREC>::T *__restrict__ dst, float *__restrict__ dst_h,
                                        const float *sm, int tx0, int ty0)
{
    using S = Store<PREC>;
    constexpr int kTY = Tile2<TY>::kTY, kRP = Tile2<TY>::kRP;
    constexpr int kWarps = kT2Threads / 32;
    const int lane = threadIdx.x, warp = threadIdx.y;
    const long long P = p.plane;
    // ---- step B: output rows in pairs (r, r + 8); lanes 0..29 --------------------
    const int x = tx0 + lane;
    // idle lanes skip step B but do not return: a persistent caller reuses the
    // block for further tiles after a barrier
    if (lane < kTX && x < p.nx) {
#pragma unroll 1
    for (int r0 = warp; r0 < kTY; r0 += 2 * kWarps) {
        float f[2][9], A3[2], A35[2], A5[2], phi[2];
        bool ok[2];
        unsigned own[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = r0 + h * kWarps;
            const int y = ty0 + r;
            ok[h] = r < kTY && (INTERIOR || y < p.ny);
            const int rr = ok[h] ? r : r0;                       // a valid row; result unused
            int c0 = rr * kRX + lane;                             // c - kRX - 1: the region's corner
            LBM_CHK(c0, kRP - 2 * kRX - 1, p.err, kErrShared);
            const int c = c0 + kRX + 1;
#pragma unroll
            for (int k = 0; k < 9; ++k) f[h][k] = sm[k * kRP + c - cy(k) * kRX - cx(k)];
            // an inactive row (beyond the tile or the grid) borrows the tile's first
            // row, which always exists, so every index below stays in bounds
            const int yy = ok[h] ? y : ty0;
            if (!INTERIOR) {
                const bool wall = (p.abb_x && (x == 0 || x == p.nx - 1)) || (p.abb_y && (yy == 0 || yy == p.ny - 1));
                if (wall) {
#pragma unroll
                    for (int k = 1; k < 9; ++k) {
                        const int xs = x - cx(k), ys = yy - cy(k);
                        const bool ox = p.abb_x && (xs < 0 || xs >= p.nx);
                        const bool oy = p.abb_y && (ys < 0 || ys >= p.ny);
                        if (ox || oy) {
                            const float wx = xs < 0 ? p.phi_wall[0] : p.phi_wall[1];
                            const float wy = ys < 0 ? p.phi_wall[2] : p.phi_wall[3];
                            const float phiw = (ox && oy) ? 0.5f * (wx + wy) : (ox ? wx : wy);
                            f[h][k] = wall_term<float, CONV, DIFF>(p, k, phiw) - sm[opp(k) * kRP + c];
                        }
                    }
                }
            }
            int xx = x, yc = yy;
            LBM_CHK(xx, p.nx, p.err, kErrX);
            LBM_CHK(yc, p.ny, p.err, kErrY);
            own[h] = (unsigned)yc * (unsigned)p.pitch + xx;
            A3[h] = p.A3; A35[h] = p.A35; A5[h] = p.A5;
            if (KF) {
                A3[h] = __ldg(p.Afield + own[h]);
                A35[h] = __ldg(p.Afield + P + own[h]);
                A5[h] = __ldg(p.Afield + 2 * P + own[h]);
            }
        }
        collide_pair<CONV, DIFF, KF>(pw, f, A3, A35, A5, phi);
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (ok[h]) S::store_cell(dst, dst_h, P, own[h], f[h], phi[h]);
    }
    }
}

template <int PREC, int CONV, int DIFF, bool INTERIOR, int TY, bool KF>
__device__ __forceinline__ void two_steps(const Params<float> &p, const typename Store<PREC>::T *__restrict__ src,
                                          const float *__restrict__ src_h, typename Store<PREC>::T *__restrict__ dst,
                                          float *__restrict__ dst_h, float *sm, int tx0, int ty0)
{
    using S = Store<PREC>;
    constexpr int kRY = Tile2<TY>::kRY, kRP = Tile2<TY>::kRP;
    const Params<F2> pw = widen(p);
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
        float A3[2] = {p.A3, p.A3}, A35[2] = {p.A35, p.A35}, A5[2] = {p.A5, p.A5}, phi[2];
        if (KF) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const unsigned own = (unsigned)ys[h] * (unsigned)p.pitch + xs[h];
                A3[h] = __ldg(p.Afield + own);
                A35[h] = __ldg(p.Afield + P + own);
                A5[h] = __ldg(p.Afield + 2 * P + own);
            }
        }
        collide_pair<CONV, DIFF, KF>(pw, f, A3, A35, A5, phi);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (INTERIOR || ok[h]) {
                const int c = (hy0 + h * kWarps) * kRX + lane;
#pragma unroll
                for (int k = 0; k < 9; ++k) sm[k * kRP + c] = f[h][k];
            }
        }
    }
    __syncthreads();
    step2_B<PREC, CONV, DIFF, INTERIOR, TY, KF>(p, pw, dst, dst_h, sm, tx0, ty0);
}

template <int PREC, int CONV, int DIFF, int TY, bool KF>
__global__ void __launch_bounds__(kT2Threads, Tile2<TY>::kMinBlocks)
k_step2(const Params<float> p, const typename Store<PREC>::T *__restrict__ src, const float *__restrict__ src_h,
        typename Store<PREC>::T *__restrict__ dst, float *__restrict__ dst_h)
{
    extern __shared__ float sm[];       // 9 planes of kRY x kRX
    constexpr int kTY = Tile2<TY>::kTY;
    const int tx0 = blockIdx.x * kTX, ty0 = blockIdx.y * kTY;
    // interior block: the region and every node it pulls from lie inside the
    // domain, so no wrap and no wall can occur
    const bool interior = tx0 >= 2 && tx0 + kTX + 1 <= p.nx - 1 && ty0 >= 2 && ty0 + kTY + 1 <= p.ny - 1;
    if (interior) two_steps<PREC, CONV, DIFF, true, TY, KF>(p, src, src_h, dst, dst_h, sm, tx0, ty0);
    else two_steps<PREC, CONV, DIFF, false, TY, KF>(p, src, src_h, dst, dst_h, sm, tx0, ty0);
}

template <int PREC, int CONV, int DIFF, int TY, bool KF>
static cudaError_t step2_ty(const lbm_solver *s, int src, cudaStream_t st)
{
    using T = typename Store<PREC>::T;
    constexpr size_t smem = 9 * Tile2<TY>::kRP * sizeof(float);
    if (smem > 48 * 1024) {
        // more than 48 KB of dynamic shared memory: opt in once per device
        static SmemOptIn once;
        const cudaError_t e = opt_in_smem((const void *)k_step2<PREC, CONV, DIFF, TY, KF>, (int)smem, once);
        if (e != cudaSuccess) return e;
    }
    const Params<float> p = make_params<float>(s);
    dim3 block(32, kT2Threads / 32);
    dim3 grid((s->d.nx + kTX - 1) / kTX, (s->d.ny + TY - 1) / TY);
    k_step2<PREC, CONV, DIFF, TY, KF><<<grid, block, smem, st>>>(p, (const T *)s->pop[src], s->phi[src],
                                                                 (T *)s->pop[src ^ 1], s->phi[src ^ 1]);
    return cudaGetLastError();
}

// tile height from the descriptor: block_rows 4 selects 30 x 30 tiles, anything
// else 30 x 62
template <int PREC, int CONV, int DIFF>
static cudaError_t step2_t(const lbm_solver *s, int src, cudaStream_t st)
{
    // per-node tensor field or not: a compile-time choice, so the constant-K
    // kernel carries no field loads or their registers
    if (s->d.per_cell_K) {
        if (s->d.block_rows == 4) return step2_ty<PREC, CONV, DIFF, 30, true>(s, src, st);
        return step2_ty<PREC, CONV, DIFF, 62, true>(s, src, st);
    }
    if (s->d.block_rows == 4) return step2_ty<PREC, CONV, DIFF, 30, false>(s, src, st);
    return step2_ty<PREC, CONV, DIFF, 62, false>(s, src, st);
}

}  // namespace lbm
