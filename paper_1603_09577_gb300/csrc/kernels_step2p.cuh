// kernels_step2p.cuh -- two fused stream-collide time steps (Eq. 34) per sweep
// through HBM with every thread owning two x-adjacent nodes ("pair tiles"),
// FP32 and BF16-shifted storage.
//
// The temporal blocking is that of kernels_step2.cuh: step A recomputes the
// state after the first step on the output tile plus a one-node halo and keeps
// it in shared memory in FP32; step B collides the tile a second time and
// writes it. Here a warp covers a 64-node region row, two nodes per lane, and
// the two nodes of a lane collide together in packed FP32x2 arithmetic.
//
// Alignment is what the pairs buy. The output tile starts at the even column
// X0 = 62 bx and the region at X0 - 1, so
//  - step A's node pairs (x, x + 1) start at odd x: the six directions with
//    c_x != 0 pull an even-aligned source pair (one 64-bit FP32 load, or one
//    32-bit bf16x2 load), the three with c_x = 0 a pair straddling two aligned
//    words; the shift plane of BF16S storage is read as two aligned float2 per
//    source row, which serve all three source pairs of that row;
//  - step B's output pairs start at even x: every population plane (and the
//    shift plane) is written as one aligned word per pair, and the bf16
//    rounding of a pair is one packed conversion.
// Every node's arithmetic is the same sequence of correctly rounded
// operations as in the one-node-per-lane tile kernel, so the two give
// bit-identical results. Tiles whose pulls could leave the domain take a
// per-node path with the periodic wrap and the anti-bounce-back walls.
#pragma once

#include "kernels_step2.cuh"

namespace lbm {

constexpr int kPX = 62;                          // output columns per tile
constexpr int kErrGrid = 32;                     // error-word bit: the launch grid does not cover the lattice
constexpr int kPRX = kPX + 2;                    // region columns: 64, two per lane
template <int TY> struct TileP {
    static constexpr int kTY = TY, kRY = TY + 2, kRP = kPRX * kRY;
    static constexpr int kMinBlocks = TY > 24 ? 3 : 4;
};

__device__ __forceinline__ F2 bf2_unpack(unsigned u)
{
    return F2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}

// Pull the nine population pairs of the interior node pair (x, x + 1), x odd,
// row y, from global memory (no wrap, no wall).
template <int PREC>
__device__ __forceinline__ void pull_pair_interior(const Params<float> &p, const typename Store<PREC>::T *__restrict__ src,
                                                   const float *__restrict__ src_h, int x, int y, F2 g[9])
{
    const long long P = p.plane;
    const unsigned pit = (unsigned)p.pitch;
    // 32-bit element offsets of the three source rows; each pull indexes its
    // plane's base with one of them (64-bit row pointers per direction cost
    // registers the kernel does not have at four blocks per SM)
    const unsigned rr[3] = {(unsigned)(y - 1) * pit, (unsigned)y * pit, (unsigned)(y + 1) * pit};
    if constexpr (PREC == LBM_F32) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const unsigned i = rr[1 - cy(k)] + (unsigned)(x - cx(k));
            const float *pk = src + k * P;
            if (cx(k) == 0) {
                g[k] = F2(__ldg(pk + i), __ldg(pk + i + 1));
            } else {
                g[k] = F2(__ldg(reinterpret_cast<const float2 *>(pk + i)));
            }
        }
    } else {
        // shift pairs of the three source rows: A = (h(x-1), h(x)), B = (h(x+1), h(x+2))
        F2 hA[3], hB[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            hA[j] = F2(__ldg(reinterpret_cast<const float2 *>(src_h + rr[j] + (unsigned)(x - 1))));
            hB[j] = F2(__ldg(reinterpret_cast<const float2 *>(src_h + rr[j] + (unsigned)(x + 1))));
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int j = 1 - cy(k);                       // source row y - cy(k)
            const __nv_bfloat16 *pk = src + k * P;
            unsigned u;
            F2 h;
            if (cx(k) == 0) {
                const unsigned i = rr[j] + (unsigned)(x - 1);
                const unsigned w0 = __ldg(reinterpret_cast<const unsigned *>(pk + i));
                const unsigned w1 = __ldg(reinterpret_cast<const unsigned *>(pk + i + 2));
                u = __byte_perm(w0, w1, 0x5432);          // (elements x, x + 1)
                h = F2(hA[j].v.y, hB[j].v.x);
            } else {
                u = __ldg(reinterpret_cast<const unsigned *>(pk + rr[j] + (unsigned)(x - cx(k))));
                h = cx(k) > 0 ? hA[j] : hB[j];
            }
            g[k] = mad(F2(wgt<float>(k)), h, bf2_unpack(u));
        }
    }
}

// Write the post-collision pair (X, X + 1) of row y, X even; `both`: X + 1 is a
// node of the grid (else only X is written).
template <int PREC>
__device__ __forceinline__ void store_pair(const Params<float> &p, typename Store<PREC>::T *__restrict__ dst,
                                           float *__restrict__ dst_h, unsigned i, const F2 g[9], F2 phi, bool both)
{
    const long long P = p.plane;
    if constexpr (PREC == LBM_F32) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            if (both) __stcs(reinterpret_cast<float2 *>(dst + k * P + i), g[k].v);
            else __stcs(dst + k * P + i, g[k].v.x);
        }
    } else {
        // g_k = bf16(fbar*_k - w_k phi), h = M* - sum_k g_k (the BF16S store of
        // Store<LBM_BF16S>, two nodes per instruction)
        F2 mass(0.f), gsum(0.f);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const F2 dev = mad(F2(-wgt<float>(k)), phi, g[k]);
            const __nv_bfloat162 b = __floats2bfloat162_rn(dev.v.x, dev.v.y);
            const unsigned u = *reinterpret_cast<const unsigned *>(&b);
            mass += g[k];
            gsum += bf2_unpack(u);
            if (both) __stcs(reinterpret_cast<unsigned *>(dst + k * P + i), u);
            else dst[k * P + i] = b.x;
        }
        const F2 h = mass - gsum;
        if (both) __stcs(reinterpret_cast<float2 *>(dst_h + i), h.v);
        else dst_h[i] = h.v.x;
    }
}

template <int PREC, int CONV, int DIFF, bool INTERIOR, int TY, bool KF>
__device__ __forceinline__ void two_steps_pair(const Params<float> &p, const typename Store<PREC>::T *__restrict__ src,
                                               const float *__restrict__ src_h, typename Store<PREC>::T *__restrict__ dst,
                                               float *__restrict__ dst_h, float *sm, int X0, int Y0)
{
    constexpr int kRY = TileP<TY>::kRY, kRP = TileP<TY>::kRP;
    constexpr int kWarps = kT2Threads / 32;
    const Params<F2> pw = widen(p);
    const int lane = threadIdx.x, warp = threadIdx.y;
    const long long P = p.plane;

    // ---- step A: region row hy per warp pass, nodes (X0 - 1 + 2 lane, +1) ----
#pragma unroll 1
    for (int hy = warp; hy < kRY; hy += kWarps) {
        F2 g[9];
        bool ok[2] = {true, true};
        int xs[2], ys[2];
        const int x0 = X0 - 1 + 2 * lane, y0 = Y0 - 1 + hy;
        if (INTERIOR) {
            int xa = x0, ya = y0;
#ifdef LBM_CHECKED
            // the pulls span x0 - 1 .. x0 + 2 and y0 - 1 .. y0 + 1; outside the
            // grid the error word records it and a safe interior pair is used
            if (x0 - 1 < 0 || x0 + 2 >= p.nx || y0 - 1 < 0 || y0 + 1 >= p.ny) {
                if (p.err) atomicOr(p.err, kErrIndex);
                xa = 1;
                ya = 1;
            }
#endif
            pull_pair_interior<PREC>(p, src, src_h, xa, ya, g);
            xs[0] = xa; xs[1] = xa + 1; ys[0] = ys[1] = ya;
        } else {
            float f[2][9];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int x = x0 + h, y = y0;
                bool valid = true;
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
                ok[h] = valid;
                xs[h] = x;
                ys[h] = y;
                pull_global<PREC, CONV, DIFF, false>(p, src, src_h, x, y, f[h]);
            }
#pragma unroll
            for (int k = 0; k < 9; ++k) g[k] = F2(f[0][k], f[1][k]);
        }
        F2 A3(p.A3), A35(p.A35), A5(p.A5), ph;
        if (KF) {
            const unsigned o0 = (unsigned)ys[0] * (unsigned)p.pitch + xs[0];
            const unsigned o1 = (unsigned)ys[1] * (unsigned)p.pitch + xs[1];
            A3 = F2(__ldg(p.Afield + o0), __ldg(p.Afield + o1));
            A35 = F2(__ldg(p.Afield + P + o0), __ldg(p.Afield + P + o1));
            A5 = F2(__ldg(p.Afield + 2 * P + o0), __ldg(p.Afield + 2 * P + o1));
        }
        collide<F2, CONV, DIFF, KF>(pw, g, A3, A35, A5, ph);
        const int c = hy * kPRX + 2 * lane;
        if (INTERIOR || (ok[0] && ok[1])) {
#pragma unroll
            for (int k = 0; k < 9; ++k) *reinterpret_cast<float2 *>(&sm[k * kRP + c]) = g[k].v;
        } else {
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                if (ok[0]) sm[k * kRP + c] = g[k].v.x;
                if (ok[1]) sm[k * kRP + c + 1] = g[k].v.y;
            }
        }
    }
    __syncthreads();

    // ---- step B: output row r per warp pass, nodes (X0 + 2 lane, +1), lanes 0..30 ----
    const int X = X0 + 2 * lane;
    if (lane < kPX / 2 && X < p.nx) {
#pragma unroll 1
        for (int r = warp; r < TY; r += kWarps) {
            const int y = Y0 + r;
            if (!INTERIOR && y >= p.ny) break;
            const int c = (r + 1) * kPRX + 2 * lane + 1;       // region index of node X
            F2 g[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const int s = k * kRP + c - cy(k) * kPRX - cx(k);
                if (cx(k) == 0) g[k] = F2(sm[s], sm[s + 1]);
                else g[k] = F2(*reinterpret_cast<const float2 *>(&sm[s]));
            }
            const bool both = INTERIOR || X + 1 < p.nx;
            if (!INTERIOR) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int x = X + h;
                    const bool wall = (p.abb_x && (x == 0 || x == p.nx - 1)) || (p.abb_y && (y == 0 || y == p.ny - 1));
                    if (wall && x < p.nx) {
#pragma unroll
                        for (int k = 1; k < 9; ++k) {
                            const int xsrc = x - cx(k), ysrc = y - cy(k);
                            const bool ox = p.abb_x && (xsrc < 0 || xsrc >= p.nx);
                            const bool oy = p.abb_y && (ysrc < 0 || ysrc >= p.ny);
                            if (ox || oy) {
                                const float wx = xsrc < 0 ? p.phi_wall[0] : p.phi_wall[1];
                                const float wy = ysrc < 0 ? p.phi_wall[2] : p.phi_wall[3];
                                const float phiw = (ox && oy) ? 0.5f * (wx + wy) : (ox ? wx : wy);
                                const float v = wall_term<float, CONV, DIFF>(p, k, phiw) - sm[opp(k) * kRP + c + h];
                                if (h == 0) g[k].v.x = v;
                                else g[k].v.y = v;
                            }
                        }
                    }
                }
            }
            int xx = X, yy = y;
            LBM_CHK(xx, p.nx, p.err, kErrX);
            LBM_CHK(yy, p.ny, p.err, kErrY);
            const unsigned own = (unsigned)yy * (unsigned)p.pitch + xx;
            F2 A3(p.A3), A35(p.A35), A5(p.A5), ph;
            if (KF) {
                const unsigned o1 = both ? own + 1 : own;
                A3 = F2(__ldg(p.Afield + own), __ldg(p.Afield + o1));
                A35 = F2(__ldg(p.Afield + P + own), __ldg(p.Afield + P + o1));
                A5 = F2(__ldg(p.Afield + 2 * P + own), __ldg(p.Afield + 2 * P + o1));
            }
            collide<F2, CONV, DIFF, KF>(pw, g, A3, A35, A5, ph);
            store_pair<PREC>(p, dst, dst_h, own, g, ph, both);
        }
    }
}

// The per-node path of the tiles along the domain's edges, kept out of line so
// that its register needs (the wrap, the wall terms) do not raise those of the
// interior tiles, which are all but a few per cent of a large grid.
template <int PREC, int CONV, int DIFF, int TY, bool KF>
__device__ __noinline__ void two_steps_pair_edge(const Params<float> &p, const typename Store<PREC>::T *__restrict__ src,
                                                 const float *__restrict__ src_h,
                                                 typename Store<PREC>::T *__restrict__ dst, float *__restrict__ dst_h,
                                                 float *sm, int X0, int Y0)
{
    two_steps_pair<PREC, CONV, DIFF, false, TY, KF>(p, src, src_h, dst, dst_h, sm, X0, Y0);
}

template <int PREC, int CONV, int DIFF, int TY, bool KF>
__global__ void __launch_bounds__(kT2Threads, TileP<TY>::kMinBlocks)
k_step2p(const Params<float> p, const typename Store<PREC>::T *__restrict__ src, const float *__restrict__ src_h,
         typename Store<PREC>::T *__restrict__ dst, float *__restrict__ dst_h)
{
    extern __shared__ __align__(16) float smp[];     // 9 planes of kRY x 64
    // BF16S: check the launch geometry (the grid must tile the whole lattice,
    // else nodes would stay unwritten; such a launch writes nothing and reports
    // kErrGrid in the error word). Besides guarding the launcher, the branch
    // moves ptxas's schedule of the BF16S tile: 163k -> 169k MLUPS on 4096^2.
    // In FP32 the same check measured 0.5 % slower, so FP32 goes without.
    if constexpr (PREC == LBM_BF16S) {
        if ((int)gridDim.x * kPX < p.nx || (int)gridDim.y * TY < p.ny) {
            if (p.err) atomicOr(p.err, kErrGrid);
            return;
        }
    }
    const int X0 = blockIdx.x * kPX, Y0 = blockIdx.y * TY;
    // interior tile: the region and every node it pulls from lie inside the
    // domain, so no wrap and no wall can occur
    const bool interior = X0 >= 2 && X0 + kPRX <= p.nx - 1 && Y0 >= 2 && Y0 + TY + 1 <= p.ny - 1;
    if (interior) two_steps_pair<PREC, CONV, DIFF, true, TY, KF>(p, src, src_h, dst, dst_h, smp, X0, Y0);
    else two_steps_pair_edge<PREC, CONV, DIFF, TY, KF>(p, src, src_h, dst, dst_h, smp, X0, Y0);
}

template <int PREC, int CONV, int DIFF, int TY, bool KF>
static cudaError_t step2p_ty(const lbm_solver *s, int src, cudaStream_t st)
{
    using T = typename Store<PREC>::T;
    constexpr size_t smem = 9 * TileP<TY>::kRP * sizeof(float);
    if (smem > 48 * 1024) {
        static SmemOptIn once;
        const cudaError_t e = opt_in_smem((const void *)k_step2p<PREC, CONV, DIFF, TY, KF>, (int)smem, once);
        if (e != cudaSuccess) return e;
    }
    const Params<float> p = make_params<float>(s);
    dim3 block(32, kT2Threads / 32);
    dim3 grid((s->d.nx + kPX - 1) / kPX, (s->d.ny + TY - 1) / TY);
    k_step2p<PREC, CONV, DIFF, TY, KF><<<grid, block, smem, st>>>(p, (const T *)s->pop[src], s->phi[src],
                                                                  (T *)s->pop[src ^ 1], s->phi[src ^ 1]);
    return cudaGetLastError();
}

// tile height from the descriptor: block_rows 4 selects 62 x 14 tiles (37 KB of
// shared memory, 4 blocks per SM), 2 selects 62 x 22 (55 KB, 4 blocks), anything
// else 62 x 30 (74 KB, 3 blocks)
template <int PREC, int CONV, int DIFF, bool KF>
static cudaError_t step2p_k(const lbm_solver *s, int src, cudaStream_t st)
{
    if (s->d.block_rows == 4) return step2p_ty<PREC, CONV, DIFF, 14, KF>(s, src, st);
    if (s->d.block_rows == 2) return step2p_ty<PREC, CONV, DIFF, 22, KF>(s, src, st);
    return step2p_ty<PREC, CONV, DIFF, 30, KF>(s, src, st);
}

template <int PREC, int CONV, int DIFF>
static cudaError_t step2p_t(const lbm_solver *s, int src, cudaStream_t st)
{
    return s->d.per_cell_K ? step2p_k<PREC, CONV, DIFF, true>(s, src, st) : step2p_k<PREC, CONV, DIFF, false>(s, src, st);
}

}  // namespace lbm
