// kernels_step2m.cu -- two fused stream-collide time steps (Eq. 34) per sweep
// through HBM, kept in registers: each warp marches down a strip of 30 columns.
//
// Lane l holds column xc = x0 - 1 + l (the strip plus one halo column on each
// side). For every row ya the warp
//   A) pulls the populations of row ya at time n (plane k from row ya - cy_k;
//      the +-1 column shift comes from the neighbouring lane by a shuffle, the
//      two edge lanes fetch their missing column from memory) and collides
//      them: G = state at n+1 of row ya;
//   B) assembles the pull of row yb = ya - 1 at time n+1 from G (planes with
//      cy = -1), the previous row's G (cy = 0) and the one before (cy = +1),
//      shifted by shuffles, collides it and stores the state at n+2 (lanes 1-30).
// Every population at time n is loaded once per warp and every population at
// n+2 stored once: 36 B per node update in FP32 (22 B in BF16S), no shared
// memory and no barriers. Halo cost: 32/30 in x, (H+2)/H in y.
#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr unsigned kFullM = 0xffffffffu;
constexpr int kStripW = 30;                   // output columns per warp
constexpr int kWarpsM = 8;                    // warps per block (consecutive row segments)

template <int PREC>
__device__ __forceinline__ float ldp(const typename Store<PREC>::T *__restrict__ plane, long long i)
{
    if constexpr (PREC == LBM_BF16S) return __bfloat162float(plane[i]);
    else return __ldg(plane + i);
}

// Step A of one row: pulled populations of node (xc, ya) at time n. INTERIOR: no
// wrap and no wall anywhere in the loads.
template <int PREC, int CONV, int DIFF, bool INTERIOR>
__device__ __forceinline__ void pull_row(const Params<float> &p, const typename Store<PREC>::T *__restrict__ src,
                                         const float *__restrict__ src_h, int lane, int xc, int xl, int xr, int ya,
                                         float f[9])
{
    const long long P = p.plane;
    int ym = ya - 1, yp = ya + 1;
    if (!INTERIOR) {
        ym = ya == 0 ? p.ny - 1 : ym;
        yp = ya == p.ny - 1 ? 0 : yp;
    }
    LBM_CHK(xc, p.nx, p.err, kErrX);
    LBM_CHK(xl, p.nx, p.err, kErrX);
    LBM_CHK(xr, p.nx, p.err, kErrX);
    LBM_CHK(ya, p.ny, p.err, kErrY);
    LBM_CHK(ym, p.ny, p.err, kErrY);
    LBM_CHK(yp, p.ny, p.err, kErrY);
    const long long r0 = (long long)ya * p.pitch, rm = (long long)ym * p.pitch, rp = (long long)yp * p.pitch;
    // own-column values
    float v[9];
    v[0] = ldp<PREC>(src, r0 + xc);
    v[1] = ldp<PREC>(src + 1 * P, r0 + xc);
    v[2] = ldp<PREC>(src + 2 * P, rm + xc);
    v[3] = ldp<PREC>(src + 3 * P, r0 + xc);
    v[4] = ldp<PREC>(src + 4 * P, rp + xc);
    v[5] = ldp<PREC>(src + 5 * P, rm + xc);
    v[6] = ldp<PREC>(src + 6 * P, rm + xc);
    v[7] = ldp<PREC>(src + 7 * P, rp + xc);
    v[8] = ldp<PREC>(src + 8 * P, rp + xc);
    float hm = 0.f, h0 = 0.f, hp = 0.f;
    if constexpr (PREC == LBM_BF16S) {
        hm = __ldg(src_h + rm + xc);
        h0 = __ldg(src_h + r0 + xc);
        hp = __ldg(src_h + rp + xc);
    }
    // the +-1 column shift: cx = +1 takes lane - 1's value, cx = -1 lane + 1's
    float s1 = __shfl_up_sync(kFullM, v[1], 1), s5 = __shfl_up_sync(kFullM, v[5], 1), s8 = __shfl_up_sync(kFullM, v[8], 1);
    float s3 = __shfl_down_sync(kFullM, v[3], 1), s6 = __shfl_down_sync(kFullM, v[6], 1), s7 = __shfl_down_sync(kFullM, v[7], 1);
    if (lane == 0) {
        s1 = ldp<PREC>(src + 1 * P, r0 + xl);
        s5 = ldp<PREC>(src + 5 * P, rm + xl);
        s8 = ldp<PREC>(src + 8 * P, rp + xl);
    }
    if (lane == 31) {
        s3 = ldp<PREC>(src + 3 * P, r0 + xr);
        s6 = ldp<PREC>(src + 6 * P, rm + xr);
        s7 = ldp<PREC>(src + 7 * P, rp + xr);
    }
    if constexpr (PREC == LBM_BF16S) {
        float hm_l = __shfl_up_sync(kFullM, hm, 1), h0_l = __shfl_up_sync(kFullM, h0, 1), hp_l = __shfl_up_sync(kFullM, hp, 1);
        float hm_r = __shfl_down_sync(kFullM, hm, 1), h0_r = __shfl_down_sync(kFullM, h0, 1), hp_r = __shfl_down_sync(kFullM, hp, 1);
        if (lane == 0) { hm_l = __ldg(src_h + rm + xl); h0_l = __ldg(src_h + r0 + xl); hp_l = __ldg(src_h + rp + xl); }
        if (lane == 31) { hm_r = __ldg(src_h + rm + xr); h0_r = __ldg(src_h + r0 + xr); hp_r = __ldg(src_h + rp + xr); }
        f[0] = fmaf(wgt<float>(0), h0, v[0]);
        f[1] = fmaf(wgt<float>(1), h0_l, s1);
        f[2] = fmaf(wgt<float>(2), hm, v[2]);
        f[3] = fmaf(wgt<float>(3), h0_r, s3);
        f[4] = fmaf(wgt<float>(4), hp, v[4]);
        f[5] = fmaf(wgt<float>(5), hm_l, s5);
        f[6] = fmaf(wgt<float>(6), hm_r, s6);
        f[7] = fmaf(wgt<float>(7), hp_r, s7);
        f[8] = fmaf(wgt<float>(8), hp_l, s8);
    } else {
        f[0] = v[0]; f[1] = s1; f[2] = v[2]; f[3] = s3; f[4] = v[4];
        f[5] = s5; f[6] = s6; f[7] = s7; f[8] = s8;
    }
}

// anti-bounce-back for a wall node: links whose source lies outside take
// -f*_opp(k)(own) + the even equilibrium part at the wall value
template <int CONV, int DIFF, class OwnOpp>
__device__ __forceinline__ void walls(const Params<float> &p, int x, int y, float f[9], OwnOpp own_opp)
{
    const bool wall = (p.abb_x && (x == 0 || x == p.nx - 1)) || (p.abb_y && (y == 0 || y == p.ny - 1));
    if (!wall) return;
#pragma unroll
    for (int k = 1; k < 9; ++k) {
        const int xs = x - cx(k), ys = y - cy(k);
        const bool ox = p.abb_x && (xs < 0 || xs >= p.nx);
        const bool oy = p.abb_y && (ys < 0 || ys >= p.ny);
        if (ox || oy) {
            const float wx = xs < 0 ? p.phi_wall[0] : p.phi_wall[1];
            const float wy = ys < 0 ? p.phi_wall[2] : p.phi_wall[3];
            const float phiw = (ox && oy) ? 0.5f * (wx + wy) : (ox ? wx : wy);
            f[k] = wall_term<float, CONV, DIFF>(p, k, phiw) - own_opp(opp(k));
        }
    }
}

template <int PREC, int CONV, int DIFF, bool INTERIOR>
__device__ __forceinline__ void march(const Params<float> &p, const typename Store<PREC>::T *__restrict__ src,
                                      const float *__restrict__ src_h, typename Store<PREC>::T *__restrict__ dst,
                                      float *__restrict__ dst_h, int x0, int y0, int ylast)
{
    using S = Store<PREC>;
    const int lane = threadIdx.x;
    const long long P = p.plane;
    // step-A column of this lane and its neighbours (wrapped when periodic)
    int xc = x0 - 1 + lane, xl = xc - 1, xr = xc + 1;
    bool colvalid = true;
    if (!INTERIOR) {
        auto wrapx = [&](int x) { return x < 0 ? x + p.nx : (x >= p.nx ? x - p.nx : x); };
        if (xc < 0 || xc >= p.nx) colvalid = !p.abb_x;
        xc = wrapx(xc);
        xl = wrapx(xl);
        xr = wrapx(xr);
        if (xc < 0 || xc >= p.nx) { xc = 0; colvalid = false; }       // grids narrower than the strip
        if (xl < 0 || xl >= p.nx) xl = 0;
        if (xr < 0 || xr >= p.nx) xr = 0;
    }
    const bool out_lane = lane >= 1 && lane <= kStripW && x0 - 1 + lane < p.nx;
    const int xo = x0 - 1 + lane;                                     // output column (lanes 1..30)

    float P1[9], P2[9];                                               // G of rows ya-1 and ya-2
#pragma unroll
    for (int k = 0; k < 9; ++k) { P1[k] = 0.f; P2[k] = 0.f; }

#pragma unroll 1
    for (int ya = y0 - 1; ya <= ylast + 1; ++ya) {
        // ---- step A: row ya at time n+1 ---------------------------------------
        int yrow = ya;
        bool rowvalid = true;
        if (!INTERIOR) {
            if (yrow < 0 || yrow >= p.ny) {
                rowvalid = !p.abb_y;
                yrow = yrow < 0 ? yrow + p.ny : yrow - p.ny;
                if (yrow < 0 || yrow >= p.ny) { yrow = 0; rowvalid = false; }
            }
        }
        float G[9];
        pull_row<PREC, CONV, DIFF, INTERIOR>(p, src, src_h, lane, xc, xl, xr, yrow, G);
        if (!INTERIOR && rowvalid && colvalid)
            walls<CONV, DIFF>(p, xc, yrow, G, [&](int o) {
                return Store<PREC>::ld(src + o * P, (long long)yrow * p.pitch + xc, src_h, wgt<float>(o));
            });
        {
            const long long own = (long long)yrow * p.pitch + xc;
            float phi;
            if (p.Afield)
                collide<float, CONV, DIFF, true>(p, G, __ldg(p.Afield + own), __ldg(p.Afield + P + own),
                                                 __ldg(p.Afield + 2 * P + own), phi);
            else
                collide<float, CONV, DIFF, false>(p, G, p.A3, p.A35, p.A5, phi);
        }
        // ---- step B: row yb = ya - 1 at time n+2 ------------------------------
        const int yb = ya - 1;
        if (yb >= y0) {
            float f[9];
            f[0] = P1[0];
            f[1] = __shfl_up_sync(kFullM, P1[1], 1);
            f[3] = __shfl_down_sync(kFullM, P1[3], 1);
            f[2] = P2[2];
            f[5] = __shfl_up_sync(kFullM, P2[5], 1);
            f[6] = __shfl_down_sync(kFullM, P2[6], 1);
            f[4] = G[4];
            f[7] = __shfl_down_sync(kFullM, G[7], 1);
            f[8] = __shfl_up_sync(kFullM, G[8], 1);
            if (out_lane) {
                if (!INTERIOR) walls<CONV, DIFF>(p, xo, yb, f, [&](int o) { return P1[o]; });
                int xs = xo, ys = yb;
                LBM_CHK(xs, p.nx, p.err, kErrX);
                LBM_CHK(ys, p.ny, p.err, kErrY);
                const long long own = (long long)ys * p.pitch + xs;
                float phi;
                if (p.Afield)
                    collide<float, CONV, DIFF, true>(p, f, __ldg(p.Afield + own), __ldg(p.Afield + P + own),
                                                     __ldg(p.Afield + 2 * P + own), phi);
                else
                    collide<float, CONV, DIFF, false>(p, f, p.A3, p.A35, p.A5, phi);
                S::store_cell(dst, dst_h, P, own, f, phi);
            }
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) { P2[k] = P1[k]; P1[k] = G[k]; }
    }
}

}  // namespace

template <int PREC, int CONV, int DIFF>
__global__ void __launch_bounds__(32 * kWarpsM)
k_step2m(const Params<float> p, const typename Store<PREC>::T *__restrict__ src, const float *__restrict__ src_h,
         typename Store<PREC>::T *__restrict__ dst, float *__restrict__ dst_h, int H)
{
    const int x0 = blockIdx.x * kStripW;
    const int y0 = (blockIdx.y * kWarpsM + threadIdx.y) * H;
    if (y0 >= p.ny) return;                                  // whole warp
    const int ylast = min(y0 + H, p.ny) - 1;
    const bool interior = x0 >= 2 && x0 + kStripW + 1 <= p.nx - 1 && y0 >= 2 && ylast + 2 <= p.ny - 1;
    if (interior) march<PREC, CONV, DIFF, true>(p, src, src_h, dst, dst_h, x0, y0, ylast);
    else march<PREC, CONV, DIFF, false>(p, src, src_h, dst, dst_h, x0, y0, ylast);
}

template <int PREC, int CONV, int DIFF>
static cudaError_t step2m_t(const lbm_solver *s, int src, int H, cudaStream_t st)
{
    using T = typename Store<PREC>::T;
    const Params<float> p = make_params<float>(s);
    dim3 block(32, kWarpsM);
    const int segs = (s->d.ny + H - 1) / H;
    dim3 grid((s->d.nx + kStripW - 1) / kStripW, (segs + kWarpsM - 1) / kWarpsM);
    k_step2m<PREC, CONV, DIFF><<<grid, block, 0, st>>>(p, (const T *)s->pop[src], s->phi[src], (T *)s->pop[src ^ 1],
                                                        s->phi[src ^ 1], H);
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t step2m_p(const lbm_solver *s, int src, int H, cudaStream_t st)
{
    switch (s->c.conv * 3 + s->c.diff) {
    case 0: return step2m_t<PREC, 0, 0>(s, src, H, st);
    case 1: return step2m_t<PREC, 0, 1>(s, src, H, st);
    case 2: return step2m_t<PREC, 0, 2>(s, src, H, st);
    case 3: return step2m_t<PREC, 1, 0>(s, src, H, st);
    case 4: return step2m_t<PREC, 1, 1>(s, src, H, st);
    case 5: return step2m_t<PREC, 1, 2>(s, src, H, st);
    }
    return cudaErrorInvalidValue;
}

// rows per warp segment: 16 * block_rows (0 -> 64)
cudaError_t launch_step2m(const lbm_solver *s, int src, cudaStream_t st)
{
    const int H = s->d.block_rows > 0 ? 16 * s->d.block_rows : 64;
    if (s->d.prec == LBM_F32) return step2m_p<LBM_F32>(s, src, H, st);
    if (s->d.prec == LBM_BF16S) return step2m_p<LBM_BF16S>(s, src, H, st);
    return cudaErrorInvalidValue;
}

}  // namespace lbm
