// lbm_device.cuh -- device-side building blocks of the fused D2Q9 MRT
// stream-collide update (arXiv:1603.09577, Sec. 2): lattice constants (Eq. 5),
// storage traits for the three population precisions, the per-cell collision
// in moment space (Eq. 15-17, 34-35) and the anti-bounce-back wall term.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm.h"

namespace lbm {

// ---- D2Q9 lattice (Eq. 5): rest, E, N, W, S, NE, NW, SW, SE -------------
__host__ __device__ constexpr int cx(int k) { return k == 1 || k == 5 || k == 8 ? 1 : (k == 3 || k == 6 || k == 7 ? -1 : 0); }
__host__ __device__ constexpr int cy(int k) { return k == 2 || k == 5 || k == 6 ? 1 : (k == 4 || k == 7 || k == 8 ? -1 : 0); }
__host__ __device__ constexpr int opp(int k) { return k == 0 ? 0 : (k <= 4 ? (k + 1) % 4 + 1 : (k + 1) % 4 + 5); }
template <class C>
__host__ __device__ constexpr C wgt(int k) { return k == 0 ? C(4) / C(9) : (k <= 4 ? C(1) / C(9) : C(1) / C(36)); }

// ---- two nodes per instruction: Blackwell's packed FP32x2 arithmetic ---------
// F2 carries the same quantity of two lattice nodes; its operators issue one
// packed add / multiply / fused multiply-add for both (sm_100 and later).
struct F2 {
    float2 v;
    __device__ __forceinline__ F2() {}
    __device__ __forceinline__ F2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ explicit F2(float2 a) : v(a) {}
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(make_float2(-a.v.x, -a.v.y)); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return F2(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)); }
__device__ __forceinline__ F2 &operator+=(F2 &a, F2 b) { a = a + b; return a; }
__device__ __forceinline__ F2 &operator-=(F2 &a, F2 b) { a = a - b; return a; }

// a * b + c: fused for the packed type, left to contraction for scalars
template <class C> __device__ __forceinline__ C mad(C a, C b, C c) { return a * b + c; }
template <> __device__ __forceinline__ F2 mad<F2>(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }

// ---- kernel parameters (passed by value) -----------------------------------
// Relaxation rates, flux and source coefficients in the compute type C.
template <class C>
struct Params {
    int nx, ny;
    long long pitch;        // elements per row of a population plane
    long long plane;        // elements per plane (ny * pitch)
    int abb_x, abb_y;       // 1: anti-bounce-back walls on that axis
    C s1, s2, s4, s6, s7, s8;
    C h1, h2, h4, h6;       // 1 - s_i / 2
    C A3, A35, A5;          // constant relaxation block (Eq. 17, 26)
    // the rates and the constant block divided by the squared norms of M0's rows
    // (36, 36, 12, 12, 4, 4 and 6), the collision's factors of the source (Eq. 34)
    // likewise: collide<..., false> applies them without rescaling every change
    C se1, se2, sq4, sq6, sp7, sp8;   // s1/36, s2/36, s4/12, s6/12, s7/4, s8/4
    C he1, he2, hq4, hq6;             // -2 h1/36, h2/36, -h4/12, -h6/12
    C a3s, a35s, a5s;                 // A3/6, A35/6, A5/6
    C c3s, c35s, c5s;                 // 1/6 - A3/12, -A35/12, 1/6 - A5/12
    C ux, uy, uxx, uxy, uyy;
    C r0, r1, half_r0, inv_den, inv_post;   // inv_den = 1/(1 - r1/2), inv_post = 1/(1 + r1/2)
    int has_src;
    C phi_wall[4];          // west, east, south, north
    const C *Afield;        // per-cell blocks: 3 planes (A3, A35, A5) or null
    int *err;               // checked builds: device word that records index faults
    // general path: Scheme A, power-law flux, Fisher source, extrapolation walls
    int scheme_a;           // 1: Scheme A (Remark II); phi(t_n) kept in a plane
    int fisher;             // 1: R = b phi (1 - phi^power) (Eq. 46)
    int power;              // delta of the power-law flux (conv 2) and the Fisher source
    C inv_p1, inv_p2;       // 1 / (delta + 1), 1 / (2 delta + 1)
    C dmxx, dmxy, dmyy;     // diff 3: D = Dm phi (the isotropic form of Eq. 62)
    C b;
    int nee_x, nee_y;       // 1: non-equilibrium extrapolation on that axis
    const double *bv;       // Dirichlet record of this step: west, east, south, north
};

// ---- checked builds ------------------------------------------------------------
// Compiled with -DLBM_CHECKED, every node coordinate a kernel derives is tested
// against the grid before it is used to index memory; a coordinate out of range
// sets a bit of a device error word and is replaced by 0, so the access stays in
// bounds and no lane leaves a warp-wide shuffle. Without the macro the checks
// compile to nothing.
#ifdef LBM_CHECKED
__device__ __forceinline__ int lbm_chk(int v, int n, int *err, int code)
{
    if (v < 0 || v >= n) {
        if (err) atomicOr(err, code);
        return 0;
    }
    return v;
}
#define LBM_CHK(v, n, err, code) ((v) = lbm::lbm_chk((v), (n), (err), (code)))
#else
#define LBM_CHK(v, n, err, code) ((void)0)
#endif
constexpr int kErrX = 1, kErrY = 2, kErrShared = 4, kErrIndex = 8;

// ---- storage traits ---------------------------------------------------------
// Populations are structure-of-arrays: plane k at base + k * plane, element
// (x, y) at y * pitch + x.
//
// LBM_BF16S stores g_k = bf16(fbar*_k - w_k phi) and a float shift plane h.
// A population is read back as w_k h + g_k. The shift is written as
// h = M* - sum_k g_k, M* = sum_k fbar*_k, so the nine stored populations of a
// node sum to its post-collision mass up to float rounding: the bf16 rounding
// of the deviations then moves no mass, it only redistributes it over the
// directions of that node in proportion to w_k.
template <int PREC> struct Store;

template <> struct Store<LBM_F64> {
    using T = double;
    using C = double;
    static constexpr bool kPhiPlane = false;
    __device__ static __forceinline__ C ld(const T *__restrict__ f, long long i, const float *, C) { return __ldg(f + i); }
    __device__ static __forceinline__ void store_cell(T *__restrict__ f, float *, long long P, long long i,
                                                      const C v[9], C)
    {
#pragma unroll
        for (int k = 0; k < 9; ++k) __stcs(f + k * P + i, v[k]);
    }
};

template <> struct Store<LBM_F32> {
    using T = float;
    using C = float;
    static constexpr bool kPhiPlane = false;
    __device__ static __forceinline__ C ld(const T *__restrict__ f, long long i, const float *, C) { return __ldg(f + i); }
    __device__ static __forceinline__ void store_cell(T *__restrict__ f, float *, long long P, long long i,
                                                      const C v[9], C)
    {
#pragma unroll
        for (int k = 0; k < 9; ++k) __stcs(f + k * P + i, v[k]);
    }
};

template <> struct Store<LBM_BF16S> {
    using T = __nv_bfloat16;
    using C = float;
    static constexpr bool kPhiPlane = true;
    __device__ static __forceinline__ C ld(const T *__restrict__ f, long long i, const float *__restrict__ h, C w)
    {
        return fmaf(w, __ldg(h + i), __bfloat162float(f[i]));
    }
    __device__ static __forceinline__ void store_cell(T *__restrict__ f, float *__restrict__ h, long long P,
                                                      long long i, const C v[9], C phi)
    {
        C mass = C(0), gsum = C(0);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const T g = __float2bfloat16_rn(fmaf(-wgt_f(k), phi, v[k]));
            mass += v[k];
            gsum += __bfloat162float(g);
            f[k * P + i] = g;
        }
        h[i] = mass - gsum;
    }
    __device__ static __forceinline__ C wgt_f(int k) { return k == 0 ? 4.0f / 9.0f : (k <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f); }
};

// ---- coefficient families (Eq. 1, Eq. 7) ------------------------------------
// Second-moment tensor Cbar = C(phi) + d c_s^2 g(phi) I, flux B and B'.
// CONV codes: 0 linear, 1 Burgers, 2 power law (Eq. 49-50), with C of Eq. 7;
// 3 Buckley-Leverett (Eq. 54) and 4, 5, 6 = families 0, 1, 2 in the C-free
// variant of Remark III (C = 0 in the equilibrium, Eq. 38).
// kConvNone: no convective flux, B = 0 and C = 0 (the linear family with
// u = 0), dispatched at run time so that the collision skips the flux terms,
// which would only add zero products
constexpr int kConvNone = -1;
template <int CONV> constexpr int conv_family() { return CONV >= 4 ? CONV - 4 : CONV; }
template <int CONV> constexpr bool conv_cfree() { return CONV >= 3; }
template <int CONV> constexpr bool has_flux() { return CONV != kConvNone; }

template <class C, int CONV, int DIFF>
struct Coef {
    C Bx, By, Bpx, Bpy, Cbxx, Cbxy, Cbyy;
    __device__ __forceinline__ Coef(const Params<C> &p, C phi)
    {
        constexpr int FAM = conv_family<CONV>();
        C Cxx, Cxy, Cyy;
        const C third = C(1.0 / 3.0);
        if constexpr (FAM == 3) {
            // Eq. 54 scaled per axis: B = (u_x f, u_y f h), f = phi^2 / (phi^2 + (1 - phi)^2),
            // h = 1 - 5 (1 - phi)^2
            const C q = C(1) - phi, den = mad(phi, phi, q * q);
            const C rden = C(1) / den;
            const C f = phi * phi * rden;
            const C fp = C(2) * phi * q * rden * rden;
            const C h = mad(C(-5) * q, q, C(1));
            Bx = p.ux * f; By = p.uy * f * h;
            Bpx = p.ux * fp; Bpy = p.uy * mad(fp, h, f * C(10) * q);
            Cxx = C(0); Cxy = C(0); Cyy = C(0);
        } else if constexpr (FAM == kConvNone) {
            Bx = C(0); By = C(0); Bpx = C(0); Bpy = C(0);
            Cxx = C(0); Cxy = C(0); Cyy = C(0);
        } else if constexpr (FAM == 0) {
            Bx = p.ux * phi; By = p.uy * phi;
            Bpx = p.ux; Bpy = p.uy;
            Cxx = p.uxx * phi; Cxy = p.uxy * phi; Cyy = p.uyy * phi;
        } else if constexpr (FAM == 2) {
            // Eq. 49-50: B = a phi^(d+1)/(d+1), B' = a phi^d, C = a a phi^(2d+1)/(2d+1)
            C pd = phi;
            for (int i = 1; i < p.power; ++i) pd = pd * phi;
            const C pb = pd * phi * p.inv_p1;
            const C pc = pd * pd * phi * p.inv_p2;
            Bx = p.ux * pb; By = p.uy * pb;
            Bpx = p.ux * pd; Bpy = p.uy * pd;
            Cxx = p.uxx * pc; Cxy = p.uxy * pc; Cyy = p.uyy * pc;
        } else {
            const C phi2 = phi * phi;
            Bx = C(0.5) * p.ux * phi2; By = C(0.5) * p.uy * phi2;
            Bpx = p.ux * phi; Bpy = p.uy * phi;
            const C p3 = phi2 * phi * third;
            Cxx = p.uxx * p3; Cxy = p.uxy * p3; Cyy = p.uyy * p3;
        }
        if constexpr (conv_cfree<CONV>()) {
            Cxx = C(0); Cxy = C(0); Cyy = C(0);
        }
        if constexpr (DIFF == 3) {
            // D = Dm phi: d c_s^2 D with d = 1
            const C pt = phi * third;
            Cbxx = mad(p.dmxx, pt, Cxx); Cbxy = mad(p.dmxy, pt, Cxy); Cbyy = mad(p.dmyy, pt, Cyy);
        } else {
            C g;
            if (DIFF == 0) g = phi;
            else if (DIFF == 1) g = mad(C(0.5) * phi, phi, phi);
            else g = mad(phi * phi * third, phi, phi);
            const C cg = g * third;              // d c_s^2 g with d = 1
            if constexpr (FAM == kConvNone) {
                Cbxx = cg; Cbyy = cg; Cbxy = C(0);
            } else {
                Cbxx = Cxx + cg; Cbyy = Cyy + cg; Cbxy = Cxy;
            }
        }
    }
};

// Even part of the equilibrium at a wall value (anti-bounce-back source term):
// feq_k(phi_w) + feq_opp(k)(phi_w) = 2 w_k [phi_w + Q : (c c - c_s^2 I) / (2 c_s^4)],
// Q = Cbar(phi_w) - c_s^2 phi_w I.
template <class C, int CONV, int DIFF>
__device__ __forceinline__ C wall_term(const Params<C> &p, int k, C phiw)
{
    Coef<C, CONV, DIFF> q(p, phiw);
    const C third = C(1) / C(3);
    const C Qxx = q.Cbxx - third * phiw, Qyy = q.Cbyy - third * phiw, Qxy = q.Cbxy;
    const C ex = C(cx(k) * cx(k)) - third, ey = C(cy(k) * cy(k)) - third;
    const C qc = Qxx * ex + C(2 * cx(k) * cy(k)) * Qxy + Qyy * ey;
    return C(2) * wgt<C>(k) * (phiw + C(4.5) * qc);
}

// ---- the collision (Eq. 34 in moment space) ---------------------------------
// In: pre-collision shifted populations f (pulled). Out: f overwritten with the
// post-collision fbar*, phi = Eq. 35. A3, A35, A5: relaxation block of the cell.
// Moments m = M0 f (Eq. 15): rho, e, eps, jx, qx, jy, qy, pxx, pxy.
template <class C>
struct Mom {
    C rho, e, eps, jx, qx, jy, qy, pxx, pxy;
    __device__ __forceinline__ explicit Mom(const C f[9])
    {
        const C ax = f[1] + f[3], ay = f[2] + f[4];
        const C axis = ax + ay;
        const C s57 = f[5] + f[7], s68 = f[6] + f[8];
        const C dg = s57 + s68;
        rho = f[0] + axis + dg;
        e = mad(C(2), dg, mad(C(-4), f[0], -axis));
        eps = mad(C(4), f[0], mad(C(-2), axis, dg));
        const C dx1 = f[1] - f[3], dy1 = f[2] - f[4];
        const C d57 = f[5] - f[7];
        const C dxd = d57 + (f[8] - f[6]);
        const C dyd = d57 + (f[6] - f[8]);
        jx = dx1 + dxd; qx = mad(C(-2), dx1, dxd);
        jy = dy1 + dyd; qy = mad(C(-2), dy1, dyd);
        pxx = ax - ay;
        pxy = s57 - s68;
    }
};

// f += M0^-1 dm with the changes already divided by the squared row norms of M0
// (M0^-1 = M0^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4)): r = drho/9,
// ee = de/36, pp = deps/36, jxn = djx/6, qxn = dqx/12, jyn = djy/6, qyn = dqy/12,
// pxxn = dpxx/4, pxyn = dpxy/4.
template <class C>
__device__ __forceinline__ void add_scaled_change(C f[9], C r, C ee, C pp, C jxn, C qxn, C jyn, C qyn, C pxxn, C pxyn)
{
    f[0] += mad(C(4), pp - ee, r);
    const C base_a = mad(C(-2), pp, r - ee);
    const C X1 = mad(C(-2), qxn, jxn), Y1 = mad(C(-2), qyn, jyn);
    const C ba_p = base_a + pxxn, ba_m = base_a - pxxn;
    f[1] += ba_p + X1;
    f[3] += ba_p - X1;
    f[2] += ba_m + Y1;
    f[4] += ba_m - Y1;
    const C base_d = mad(C(2), ee, r + pp);
    const C X2 = jxn + qxn, Y2 = jyn + qyn;
    const C bd_p = base_d + pxyn, bd_m = base_d - pxyn;
    const C XpY = X2 + Y2, XmY = X2 - Y2;
    f[5] += bd_p + XpY;
    f[6] += bd_m - XmY;
    f[7] += bd_p - XpY;
    f[8] += bd_m + XmY;
}

// f += M0^-1 dm for the unscaled changes dm = m* - m.
template <class C>
__device__ __forceinline__ void add_moment_change(C f[9], C drho, C de, C deps, C djx, C dqx, C djy, C dqy, C dpxx,
                                                  C dpxy)
{
    add_scaled_change<C>(f, drho * C(1.0 / 9.0), de * C(1.0 / 36.0), deps * C(1.0 / 36.0), djx * C(1.0 / 6.0),
                         dqx * C(1.0 / 12.0), djy * C(1.0 / 6.0), dqy * C(1.0 / 12.0), dpxx * C(0.25), dpxy * C(0.25));
}

// NODE_K: A3, A35, A5 are the node's block (per-node tensor field); otherwise
// the block is the constant one of p and its prescaled forms are used.
template <class C, int CONV, int DIFF, bool NODE_K = true>
__device__ __forceinline__ void collide(const Params<C> &p, C f[9], C A3, C A35, C A5, C &phi_out)
{
    const Mom<C> mo(f);
    const C rho = mo.rho, e = mo.e, eps = mo.eps, jx = mo.jx, qx = mo.qx, jy = mo.jy, qy = mo.qy, pxx = mo.pxx,
            pxy = mo.pxy;

    // Eq. 35 for R = r0 + r1 phi
    const C phi = (rho + p.half_r0) * p.inv_den;
    phi_out = phi;
    const Coef<C, CONV, DIFF> q(p, phi);

    // equilibrium moments (Eq. 16 with c = 1)
    constexpr bool FLUX = has_flux<CONV>();
    const C C2 = q.Cbxx + q.Cbyy;
    const C e_eq = mad(C(3), C2, C(-4) * phi);
    const C eps_eq = C(3) * (phi - C2);

    // relaxation (Eq. 17) plus (I - S/2) M0 R (Eq. 34), M0 R = (R, -2R, R,
    // Bt_x R, -Bt_x R, Bt_y R, -Bt_y R, 0, 0) with Bt = B' (Scheme B), written
    // as the change dm = m* - m of every moment, each already divided by the
    // squared norm of its row of M0 (the rates carry the factor). Adding
    // M0^-1 dm to f (instead of rebuilding f from m*) keeps rounding
    // proportional to the departure from equilibrium; with R = 0 the mass
    // change is exactly zero.
    // (without flux B = 0, C = 0: the q and p moments relax toward zero)
    C ee = -p.se1 * (e - e_eq);
    C pp = -p.se2 * (eps - eps_eq);
    C qxn, qyn, pxxn, pxyn;
    if constexpr (FLUX) {
        qxn = -p.sq4 * (qx + q.Bx);
        qyn = -p.sq6 * (qy + q.By);
        pxxn = -p.sp7 * (pxx - (q.Cbxx - q.Cbyy));
        pxyn = -p.sp8 * (pxy - q.Cbxy);
    } else {
        qxn = -p.sq4 * qx;
        qyn = -p.sq6 * qy;
        pxxn = -p.sp7 * pxx;
        pxyn = -p.sp8 * pxy;
    }
    C a3, a35, a5;
    if constexpr (NODE_K) {
        a3 = A3 * C(1.0 / 6.0); a35 = A35 * C(1.0 / 6.0); a5 = A5 * C(1.0 / 6.0);
    } else {
        a3 = p.a3s; a35 = p.a35s; a5 = p.a5s;
    }
    C d3 = jx, d5 = jy;
    if constexpr (FLUX) {
        d3 = jx - q.Bx;
        d5 = jy - q.By;
    }
    C jxn = -mad(a3, d3, a35 * d5);
    C jyn = -mad(a35, d3, a5 * d5);
    C r = C(0);
    if (p.has_src) {
        const C R = mad(p.r1, phi, p.r0);
        r = R * C(1.0 / 9.0);                    // rho* = phi + R/2 = rho + R for every s0
        ee = mad(p.he1, R, ee);
        pp = mad(p.he2, R, pp);
        if constexpr (FLUX) {
            const C sx = q.Bpx * R, sy = q.Bpy * R;
            qxn = mad(p.hq4, sx, qxn);
            qyn = mad(p.hq6, sy, qyn);
            // (I - A/2) B' R of the flux block, divided by 6
            C c3, c35, c5;
            if constexpr (NODE_K) {
                c3 = mad(C(-0.5), a3, C(1.0 / 6.0)); c35 = C(-0.5) * a35; c5 = mad(C(-0.5), a5, C(1.0 / 6.0));
            } else {
                c3 = p.c3s; c35 = p.c35s; c5 = p.c5s;
            }
            jxn = mad(c3, sx, mad(c35, sy, jxn));
            jyn = mad(c35, sx, mad(c5, sy, jyn));
        }
    }

    // f* = f + M0^-1 dm
    add_scaled_change<C>(f, r, ee, pp, jxn, qxn, jyn, qyn, pxxn, pxyn);
}

// Equilibrium populations of Eq. 3 (used only at initialisation).
template <class C, int CONV, int DIFF>
__device__ __forceinline__ void equilibrium(const Params<C> &p, C phi, C feq[9])
{
    const Coef<C, CONV, DIFF> q(p, phi);
    const C third = C(1) / C(3);
    const C Qxx = q.Cbxx - third * phi, Qyy = q.Cbyy - third * phi, Qxy = q.Cbxy;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const C cB = C(cx(k)) * q.Bx + C(cy(k)) * q.By;
        const C qc = Qxx * (C(cx(k) * cx(k)) - third) + C(2 * cx(k) * cy(k)) * Qxy + Qyy * (C(cy(k) * cy(k)) - third);
        feq[k] = wgt<C>(k) * (phi + C(3) * cB + C(4.5) * qc);
    }
}

// Source populations of Eq. 9 with Btilde = B'.
template <class C, int CONV, int DIFF>
__device__ __forceinline__ void source_pop(const Params<C> &p, C phi, C R, C Rk[9])
{
    const Coef<C, CONV, DIFF> q(p, phi);
#pragma unroll
    for (int k = 0; k < 9; ++k) Rk[k] = wgt<C>(k) * (C(1) + C(3) * (C(cx(k)) * q.Bpx + C(cy(k)) * q.Bpy)) * R;
}

}  // namespace lbm
