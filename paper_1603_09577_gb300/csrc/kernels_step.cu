// kernels_step.cu -- the fused pull-stream / collide time step (Eq. 34, Scheme B)
// with periodic or anti-bounce-back boundaries, one thread per lattice node.
//
// Memory: each node reads its 9 incoming populations from the neighbours'
// planes (pull: plane k at (x - c_kx, y - c_ky)) and writes its 9 outgoing
// populations to its own position of the other buffer. Every population is
// read once and written once per step: 72 B per update in FP32, 144 B in FP64,
// 36 B + the phi plane in BF16S.
#include "lbm_internal.h"

namespace lbm {

template <int PREC, int CONV, int DIFF>
__global__ void __launch_bounds__(256)
k_step(const Params<typename Store<PREC>::C> p, const typename Store<PREC>::T *__restrict__ src,
       const float *__restrict__ src_phi, typename Store<PREC>::T *__restrict__ dst, float *__restrict__ dst_phi)
{
    using S = Store<PREC>;
    using C = typename S::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;

    int xm = x == 0 ? p.nx - 1 : x - 1;
    int xp = x == p.nx - 1 ? 0 : x + 1;
    int ym = y == 0 ? p.ny - 1 : y - 1;
    int yp = y == p.ny - 1 ? 0 : y + 1;
    LBM_CHK(xm, p.nx, p.err, kErrX);
    LBM_CHK(xp, p.nx, p.err, kErrX);
    LBM_CHK(ym, p.ny, p.err, kErrY);
    LBM_CHK(yp, p.ny, p.err, kErrY);
    const long long r0 = (long long)y * p.pitch, rm = (long long)ym * p.pitch, rp = (long long)yp * p.pitch;
    const long long own = r0 + x;
    const long long P = p.plane;

    // pull: f_k(x) = f*_k(x - c_k), periodic wrap on both axes
    C f[9];
    f[0] = S::ld(src, own, src_phi, wgt<C>(0));
    f[1] = S::ld(src + 1 * P, r0 + xm, src_phi, wgt<C>(1));
    f[2] = S::ld(src + 2 * P, rm + x, src_phi, wgt<C>(2));
    f[3] = S::ld(src + 3 * P, r0 + xp, src_phi, wgt<C>(3));
    f[4] = S::ld(src + 4 * P, rp + x, src_phi, wgt<C>(4));
    f[5] = S::ld(src + 5 * P, rm + xm, src_phi, wgt<C>(5));
    f[6] = S::ld(src + 6 * P, rm + xp, src_phi, wgt<C>(6));
    f[7] = S::ld(src + 7 * P, rp + xp, src_phi, wgt<C>(7));
    f[8] = S::ld(src + 8 * P, rp + xm, src_phi, wgt<C>(8));

    // anti-bounce-back: a link whose source lies outside a wall takes
    // -f*_opp(k)(x) + the even equilibrium part at the wall value
    const bool wall = (p.abb_x && (x == 0 || x == p.nx - 1)) || (p.abb_y && (y == 0 || y == p.ny - 1));
    if (wall) {
#pragma unroll
        for (int k = 1; k < 9; ++k) {
            const int xs = x - cx(k), ys = y - cy(k);
            const bool ox = p.abb_x && (xs < 0 || xs >= p.nx);
            const bool oy = p.abb_y && (ys < 0 || ys >= p.ny);
            if (ox || oy) {
                const C wx = xs < 0 ? p.phi_wall[0] : p.phi_wall[1];
                const C wy = ys < 0 ? p.phi_wall[2] : p.phi_wall[3];
                const C phiw = (ox && oy) ? C(0.5) * (wx + wy) : (ox ? wx : wy);
                f[k] = wall_term<C, CONV, DIFF>(p, k, phiw) - S::ld(src + opp(k) * P, own, src_phi, wgt<C>(opp(k)));
            }
        }
    }

    C phi;
    if (p.Afield)
        collide<C, CONV, DIFF, true>(p, f, __ldg(p.Afield + own), __ldg(p.Afield + P + own), __ldg(p.Afield + 2 * P + own),
                                     phi);
    else
        collide<C, CONV, DIFF, false>(p, f, p.A3, p.A35, p.A5, phi);
    S::store_cell(dst, dst_phi, P, own, f, phi);
}

template <int PREC, int CONV, int DIFF>
static cudaError_t step_t(const lbm_solver *s, const void *src, const float *src_h, void *dst, float *dst_h,
                          cudaStream_t st)
{
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;
    const Params<C> p = make_params<C>(s);
    const int by = s->d.block_rows > 0 ? s->d.block_rows : 8;
    dim3 block(32, by);
    dim3 grid((s->d.nx + 31) / 32, (s->d.ny + by - 1) / by);
    k_step<PREC, CONV, DIFF><<<grid, block, 0, st>>>(p, (const T *)src, src_h, (T *)dst, dst_h);
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t step_p(const lbm_solver *s, const void *src, const float *src_h, void *dst, float *dst_h,
                          cudaStream_t st)
{
    switch (step_key(s)) {
    case 0: return step_t<PREC, 0, 0>(s, src, src_h, dst, dst_h, st);
    case 1: return step_t<PREC, 0, 1>(s, src, src_h, dst, dst_h, st);
    case 2: return step_t<PREC, 0, 2>(s, src, src_h, dst, dst_h, st);
    case 3: return step_t<PREC, 1, 0>(s, src, src_h, dst, dst_h, st);
    case 4: return step_t<PREC, 1, 1>(s, src, src_h, dst, dst_h, st);
    case 5: return step_t<PREC, 1, 2>(s, src, src_h, dst, dst_h, st);
    case 6: return step_t<PREC, kConvNone, 0>(s, src, src_h, dst, dst_h, st);
    case 7: return step_t<PREC, kConvNone, 1>(s, src, src_h, dst, dst_h, st);
    case 8: return step_t<PREC, kConvNone, 2>(s, src, src_h, dst, dst_h, st);
    }
    return cudaErrorInvalidValue;
}

// one step between explicit state buffers (lbm_save layout; shift planes follow
// the populations for LBM_BF16S)
cudaError_t launch_step_ptr(const lbm_solver *s, const void *src, void *dst, cudaStream_t st)
{
    const float *src_h = s->L.phi_bytes ? (const float *)((const char *)src + s->L.pop_bytes) : nullptr;
    float *dst_h = s->L.phi_bytes ? (float *)((char *)dst + s->L.pop_bytes) : nullptr;
    switch (s->d.prec) {
    case LBM_F64: return step_p<LBM_F64>(s, src, src_h, dst, dst_h, st);
    case LBM_F32: return step_p<LBM_F32>(s, src, src_h, dst, dst_h, st);
    case LBM_BF16S: return step_p<LBM_BF16S>(s, src, src_h, dst, dst_h, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_step(const lbm_solver *s, int src, cudaStream_t st)
{
    switch (s->d.prec) {
    case LBM_F64: return step_p<LBM_F64>(s, s->pop[src], s->phi[src], s->pop[src ^ 1], s->phi[src ^ 1], st);
    case LBM_F32: return step_p<LBM_F32>(s, s->pop[src], s->phi[src], s->pop[src ^ 1], s->phi[src ^ 1], st);
    case LBM_BF16S: return step_p<LBM_BF16S>(s, s->pop[src], s->phi[src], s->pop[src ^ 1], s->phi[src ^ 1], st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbm
