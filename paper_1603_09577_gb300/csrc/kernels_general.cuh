// kernels_general.cuh -- the general fused time step, one thread per node:
// Scheme B (Eq. 34) or Scheme A (Remark II: gamma = 0, theta = 1), the
// power-law flux (Eq. 49-50), the Fisher source (Eq. 46), and periodic,
// anti-bounce-back or non-equilibrium-extrapolation boundaries.
//
// Scheme A keeps phi(t_n) in a plane next to the populations (read at the node,
// written at the node: 2 x 4 B per update in FP32 on top of the 72 B of the
// populations) for the backward difference of R_k. An extrapolated boundary
// node pulls the nine populations of its inward neighbour instead of its own,
// so one launch still reads every population once (plus the boundary nodes'
// neighbour reads, O(perimeter)).
#pragma once

#include "lbm_internal.h"

namespace lbm {

// The Dirichlet record of a step: record min(*cnt + ahead, nrec - 1) of the
// caller's array. *cnt counts the steps since the records were set (or since the
// initial condition) up to the first sweep of the current lbm_step call; `ahead`
// is the step's place within that call. A one-thread launch after the call's
// sweeps advances *cnt, so every block of a launch reads the same value and a
// graph replay of the steps advances the records as a direct run does.
__device__ __forceinline__ const double *record_of(const double *base, const long long *cnt, int nrec, int rec,
                                                   int ahead)
{
    if (!base) return nullptr;
    long long j = (cnt ? *cnt : 0) + ahead;
    if (j > nrec - 1) j = nrec - 1;
    return base + j * (long long)rec;
}

// R(phi): affine (r0 + r1 phi) or Fisher (b phi (1 - phi^delta), Eq. 46)
template <class C>
__device__ __forceinline__ C source_value(const Params<C> &p, C phi)
{
    if (p.fisher) {
        C pd = phi;
        for (int i = 1; i < p.power; ++i) pd = pd * phi;
        return p.b * phi * (C(1) - pd);
    }
    return mad(p.r1, phi, p.r0);
}

// B'(phi) of the flux family
template <class C, int CONV>
__device__ __forceinline__ void bprime(const Params<C> &p, C phi, C &bx, C &by)
{
    constexpr int FAM = conv_family<CONV>();
    if constexpr (FAM == 0) {
        bx = p.ux;
        by = p.uy;
    } else if constexpr (FAM == 1) {
        bx = p.ux * phi;
        by = p.uy * phi;
    } else if constexpr (FAM == 2) {
        C pd = phi;
        for (int i = 1; i < p.power; ++i) pd = pd * phi;
        bx = p.ux * pd;
        by = p.uy * pd;
    } else {
        const Coef<C, CONV, 0> q(p, phi);
        bx = q.Bpx;
        by = q.Bpy;
    }
}

// B(phi) of the flux family (the C-free variant's d_t B)
template <class C, int CONV>
__device__ __forceinline__ void flux_b(const Params<C> &p, C phi, C &bx, C &by)
{
    constexpr int FAM = conv_family<CONV>();
    if constexpr (FAM == 0) {
        bx = p.ux * phi;
        by = p.uy * phi;
    } else if constexpr (FAM == 1) {
        bx = C(0.5) * p.ux * phi * phi;
        by = C(0.5) * p.uy * phi * phi;
    } else {
        const Coef<C, CONV, 0> q(p, phi);
        bx = q.Bx;
        by = q.By;
    }
}

// Scheme A collision in moment space: phi = sum f (Eq. 10a), relaxation of
// Eq. 17, and the source term dt R_k + dt/2 [R_k(t) - R_k(t - dt)], i.e.
// 3/2 M0 R_vec(t) - 1/2 M0 R_vec(t - dt) with M0 R_vec = (R, -2R, R, Bt_x R,
// -Bt_x R, Bt_y R, -Bt_y R, 0, 0) and Bt = (I - A/2) B' (Eq. 28, gamma = 0).
// C-free variant (CONV >= 3, Remark III): + dt G_k of Eq. 37, whose moments are
// (0, 0, 0, G_x, -G_x, G_y, -G_y, 0, 0), G = (I - A/2) [B(phi) - B(phi_prev)].
template <class C, int CONV, int DIFF>
__device__ __forceinline__ void collide_a(const Params<C> &p, C f[9], C A3, C A35, C A5, C phi_prev, C &phi_out)
{
    const Mom<C> mo(f);
    const C phi = mo.rho;
    phi_out = phi;
    const Coef<C, CONV, DIFF> q(p, phi);
    const C C2 = q.Cbxx + q.Cbyy;
    const C e_eq = mad(C(3), C2, C(-4) * phi);
    const C eps_eq = C(3) * (phi - C2);
    const C pxx_eq = q.Cbxx - q.Cbyy;
    C de = -p.s1 * (mo.e - e_eq);
    C deps = -p.s2 * (mo.eps - eps_eq);
    C dqx = -p.s4 * (mo.qx + q.Bx);
    C dqy = -p.s6 * (mo.qy + q.By);
    const C dpxx = -p.s7 * (mo.pxx - pxx_eq);
    const C dpxy = -p.s8 * (mo.pxy - q.Cbxy);
    const C d3 = mo.jx - q.Bx, d5 = mo.jy - q.By;
    C djx = -mad(A3, d3, A35 * d5);
    C djy = -mad(A35, d3, A5 * d5);
    C drho = C(0);
    if (p.has_src) {
        const C R1 = source_value(p, phi), R0 = source_value(p, phi_prev);
        C b0x, b0y;
        bprime<C, CONV>(p, phi_prev, b0x, b0y);
        const C t1x = q.Bpx - C(0.5) * mad(A3, q.Bpx, A35 * q.Bpy);
        const C t1y = q.Bpy - C(0.5) * mad(A35, q.Bpx, A5 * q.Bpy);
        const C t0x = b0x - C(0.5) * mad(A3, b0x, A35 * b0y);
        const C t0y = b0y - C(0.5) * mad(A35, b0x, A5 * b0y);
        const C Rs = C(1.5) * R1 - C(0.5) * R0;
        const C Sx = C(1.5) * t1x * R1 - C(0.5) * t0x * R0;
        const C Sy = C(1.5) * t1y * R1 - C(0.5) * t0y * R0;
        drho = Rs;
        de = mad(C(-2), Rs, de);
        deps += Rs;
        djx += Sx;
        dqx -= Sx;
        djy += Sy;
        dqy -= Sy;
    }
    if constexpr (conv_cfree<CONV>()) {
        C b0x, b0y;
        flux_b<C, CONV>(p, phi_prev, b0x, b0y);
        const C dbx = q.Bx - b0x, dby = q.By - b0y;
        const C gx = dbx - C(0.5) * mad(A3, dbx, A35 * dby);
        const C gy = dby - C(0.5) * mad(A35, dbx, A5 * dby);
        djx += gx;
        dqx -= gx;
        djy += gy;
        dqy -= gy;
    }
    add_moment_change<C>(f, drho, de, deps, djx, dqx, djy, dqy, dpxx, dpxy);
}

// Equilibrium of the stored variable: feq (Scheme A) or feq - R_k/2 (Scheme B, Eq. 33)
template <class C, int CONV, int DIFF, bool SA>
__device__ __forceinline__ void feq_stored(const Params<C> &p, C phi, C out[9])
{
    equilibrium<C, CONV, DIFF>(p, phi, out);
    if (!SA && p.has_src) {
        C Rk[9];
        source_pop<C, CONV, DIFF>(p, phi, mad(p.r1, phi, p.r0), Rk);
#pragma unroll
        for (int k = 0; k < 9; ++k) out[k] -= C(0.5) * Rk[k];
    }
}

// pull the nine populations into node (x, y) with periodic wrap
template <int PREC>
__device__ __forceinline__ void pull_wrap(const Params<typename Store<PREC>::C> &p,
                                          const typename Store<PREC>::T *__restrict__ src, int x, int y,
                                          typename Store<PREC>::C f[9])
{
    using S = Store<PREC>;
    using C = typename S::C;
    int xm = x == 0 ? p.nx - 1 : x - 1;
    int xp = x == p.nx - 1 ? 0 : x + 1;
    int ym = y == 0 ? p.ny - 1 : y - 1;
    int yp = y == p.ny - 1 ? 0 : y + 1;
    LBM_CHK(x, p.nx, p.err, kErrX);
    LBM_CHK(y, p.ny, p.err, kErrY);
    LBM_CHK(xm, p.nx, p.err, kErrX);
    LBM_CHK(xp, p.nx, p.err, kErrX);
    LBM_CHK(ym, p.ny, p.err, kErrY);
    LBM_CHK(yp, p.ny, p.err, kErrY);
    const long long r0 = (long long)y * p.pitch, rm = (long long)ym * p.pitch, rp = (long long)yp * p.pitch;
    const long long P = p.plane;
    f[0] = S::ld(src, r0 + x, nullptr, wgt<C>(0));
    f[1] = S::ld(src + 1 * P, r0 + xm, nullptr, wgt<C>(1));
    f[2] = S::ld(src + 2 * P, rm + x, nullptr, wgt<C>(2));
    f[3] = S::ld(src + 3 * P, r0 + xp, nullptr, wgt<C>(3));
    f[4] = S::ld(src + 4 * P, rp + x, nullptr, wgt<C>(4));
    f[5] = S::ld(src + 5 * P, rm + xm, nullptr, wgt<C>(5));
    f[6] = S::ld(src + 6 * P, rm + xp, nullptr, wgt<C>(6));
    f[7] = S::ld(src + 7 * P, rp + xp, nullptr, wgt<C>(7));
    f[8] = S::ld(src + 8 * P, rp + xm, nullptr, wgt<C>(8));
}

// One time step (SA: Scheme A). src_phi / dst_phi: the phi(t_n) planes of Scheme A.
template <int PREC, int CONV, int DIFF, bool SA>
__global__ void __launch_bounds__(256)
k_step_g(const Params<typename Store<PREC>::C> p, const typename Store<PREC>::T *__restrict__ src,
         const typename Store<PREC>::C *__restrict__ src_phi, typename Store<PREC>::T *__restrict__ dst,
         typename Store<PREC>::C *__restrict__ dst_phi, const long long *__restrict__ rec_cnt, int nrec, int rec_off)
{
    using S = Store<PREC>;
    using C = typename S::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const long long own = (long long)y * p.pitch + x;
    const long long P = p.plane;
    const bool ex = p.nee_x && (x == 0 || x == p.nx - 1);
    const bool ey = p.nee_y && (y == 0 || y == p.ny - 1);
    C f[9];
    if (ex || ey) {
        // extrapolation: f(xb) = feq(phi_b) + [f(xf) - feq(phi(xf))], xf the inward
        // neighbour (diagonal at a corner), all in the stored variable
        const int xf = ex ? (x == 0 ? 1 : p.nx - 2) : x;
        const int yf = ey ? (y == 0 ? 1 : p.ny - 2) : y;
        pull_wrap<PREC>(p, src, xf, yf, f);
        C sum = f[0];
#pragma unroll
        for (int k = 1; k < 9; ++k) sum += f[k];
        const C phif = SA ? sum : (sum + p.half_r0) * p.inv_den;
        const double *bv = record_of(p.bv, rec_cnt, nrec, 2 * (p.nx + p.ny), rec_off);
        const double vb = ex ? bv[x == 0 ? y : p.ny + y] : bv[2 * p.ny + (y == 0 ? x : p.nx + x)];
        C eb[9], ef[9];
        feq_stored<C, CONV, DIFF, SA>(p, (C)vb, eb);
        feq_stored<C, CONV, DIFF, SA>(p, phif, ef);
#pragma unroll
        for (int k = 0; k < 9; ++k) f[k] = eb[k] + (f[k] - ef[k]);
    } else {
        pull_wrap<PREC>(p, src, x, y, f);
        // anti-bounce-back links (an anti-bounce-back axis never meets an
        // extrapolated one)
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
                    f[k] = wall_term<C, CONV, DIFF>(p, k, phiw) - S::ld(src + opp(k) * P, own, nullptr, wgt<C>(opp(k)));
                }
            }
        }
    }
    C A3 = p.A3, A35 = p.A35, A5 = p.A5;
    if (p.Afield) {
        A3 = __ldg(p.Afield + own);
        A35 = __ldg(p.Afield + P + own);
        A5 = __ldg(p.Afield + 2 * P + own);
    }
    C phi;
    if (SA) collide_a<C, CONV, DIFF>(p, f, A3, A35, A5, src_phi[own], phi);
    else collide<C, CONV, DIFF>(p, f, A3, A35, A5, phi);
    S::store_cell(dst, nullptr, P, own, f, phi);
    if (SA) dst_phi[own] = phi;
}

// Initial state of the general path (Eq. 40 in the stored variable, then one
// collision; Scheme A with d_t R_k = 0, i.e. phi_prev = phi0).
template <int PREC, int CONV, int DIFF, bool SA>
__global__ void __launch_bounds__(256)
k_init_g(const Params<typename Store<PREC>::C> p, const void *__restrict__ phi_in, int in_prec,
         typename Store<PREC>::T *__restrict__ dst, typename Store<PREC>::C *__restrict__ dst_phi)
{
    using S = Store<PREC>;
    using C = typename S::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const long long in = (long long)y * p.nx + x;
    const C phi0 = in_prec == LBM_F64 ? C(((const double *)phi_in)[in]) : C(((const float *)phi_in)[in]);
    C f[9];
    feq_stored<C, CONV, DIFF, SA>(p, phi0, f);
    const long long own = (long long)y * p.pitch + x;
    C A3 = p.A3, A35 = p.A35, A5 = p.A5;
    if (p.Afield) {
        A3 = p.Afield[own];
        A35 = p.Afield[p.plane + own];
        A5 = p.Afield[2 * p.plane + own];
    }
    C phi;
    if (SA) collide_a<C, CONV, DIFF>(p, f, A3, A35, A5, phi0, phi);
    else collide<C, CONV, DIFF>(p, f, A3, A35, A5, phi);
    S::store_cell(dst, nullptr, p.plane, own, f, phi);
    if (SA) dst_phi[own] = phi0;
}

template <int PREC, int CONV, int DIFF, bool SA>
static cudaError_t general_t(const lbm_solver *s, int src, const double *bv, const void *phi0, int in_prec,
                             cudaStream_t st)
{
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;
    Params<C> p = make_params<C>(s);
    p.bv = bv;
    const int by = s->d.block_rows > 0 ? s->d.block_rows : 8;
    dim3 block(32, by);
    dim3 grid((s->d.nx + 31) / 32, (s->d.ny + by - 1) / by);
    if (phi0) {
        k_init_g<PREC, CONV, DIFF, SA><<<grid, block, 0, st>>>(p, phi0, in_prec, (T *)s->pop[s->cur],
                                                              (C *)s->phi[s->cur]);
    } else {
        k_step_g<PREC, CONV, DIFF, SA><<<grid, block, 0, st>>>(p, (const T *)s->pop[src], (const C *)s->phi[src],
                                                              (T *)s->pop[src ^ 1], (C *)s->phi[src ^ 1],
                                                              s->dir_counter, s->dir_nrec, s->dir_off);
    }
    return cudaGetLastError();
}

// dispatch over the flux / diffusion families and the scheme; the C-free
// variant (Scheme A only) maps families 0, 1, 2 to codes 4, 5, 6, and the
// Buckley-Leverett flux is code 3
template <int PREC>
static cudaError_t general_p(const lbm_solver *s, int src, const double *bv, const void *phi0, int in_prec,
                             cudaStream_t st)
{
    const bool sa = s->d.scheme == LBM_SCHEME_A;
    if (s->c.cfree) {
        if (!sa) return cudaErrorInvalidValue;
        const int code = s->c.conv == 3 ? 3 : s->c.conv + 4;
#define LBM_GEN_CF(CV, DF) \
    case CV * 4 + DF: return general_t<PREC, CV, DF, true>(s, src, bv, phi0, in_prec, st);
        switch (code * 4 + s->c.diff) {
            LBM_GEN_CF(3, 0)
            LBM_GEN_CF(3, 1)
            LBM_GEN_CF(3, 2)
            LBM_GEN_CF(3, 3)
            LBM_GEN_CF(4, 0)
            LBM_GEN_CF(4, 1)
            LBM_GEN_CF(4, 2)
            LBM_GEN_CF(4, 3)
            LBM_GEN_CF(5, 0)
            LBM_GEN_CF(5, 1)
            LBM_GEN_CF(5, 2)
            LBM_GEN_CF(5, 3)
            LBM_GEN_CF(6, 0)
            LBM_GEN_CF(6, 1)
            LBM_GEN_CF(6, 2)
            LBM_GEN_CF(6, 3)
        }
#undef LBM_GEN_CF
        return cudaErrorInvalidValue;
    }
#define LBM_GEN_CASE(CV, DF)                                                                    \
    case CV * 4 + DF:                                                                           \
        return sa ? general_t<PREC, CV, DF, true>(s, src, bv, phi0, in_prec, st)                \
                  : general_t<PREC, CV, DF, false>(s, src, bv, phi0, in_prec, st);
    switch (s->c.conv * 4 + s->c.diff) {
        LBM_GEN_CASE(0, 0)
        LBM_GEN_CASE(0, 1)
        LBM_GEN_CASE(0, 2)
        LBM_GEN_CASE(0, 3)
        LBM_GEN_CASE(1, 0)
        LBM_GEN_CASE(1, 1)
        LBM_GEN_CASE(1, 2)
        LBM_GEN_CASE(1, 3)
        LBM_GEN_CASE(2, 0)
        LBM_GEN_CASE(2, 1)
        LBM_GEN_CASE(2, 2)
        LBM_GEN_CASE(2, 3)
    }
#undef LBM_GEN_CASE
    return cudaErrorInvalidValue;
}

}  // namespace lbm
