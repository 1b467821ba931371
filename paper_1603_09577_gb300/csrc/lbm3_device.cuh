// lbm3_device.cuh -- device-side pieces of the three-dimensional (D3Q19)
// extension shared by its kernels: the lattice of Eq. 6, the storage traits,
// the kernel parameters, the coefficient families, the collision in the
// projector form of the moment reading (include/lbm3.h) and the pull of one
// node with periodic wrap and anti-bounce-back walls.
#pragma once

#include <cuda_bf16.h>

#include "lbm3.h"
#include "lbm_internal.h"

namespace lbm {

// Eq. 6: D3Q19 velocities in the paper's order and weights
__host__ __device__ constexpr int c3x(int k)
{
    constexpr int v[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1, 0, 0, 0, 0};
    return v[k];
}
__host__ __device__ constexpr int c3y(int k)
{
    constexpr int v[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return v[k];
}
__host__ __device__ constexpr int c3z(int k)
{
    constexpr int v[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1};
    return v[k];
}
template <class C>
__host__ __device__ constexpr C w3(int k)
{
    return k == 0 ? C(1) / C(3) : (k <= 6 ? C(1) / C(18) : C(1) / C(36));
}
// Eq. 6 lists every velocity next to its opposite: (1, 2), (3, 4), ..., (17, 18)
__host__ __device__ constexpr int opp3(int k) { return k == 0 ? 0 : (k % 2 ? k + 1 : k - 1); }

// Storage of the 19 planes: FP64, FP32, or BF16 deviations g_k = f*_k - w_k phi
// plus an FP32 shift plane h = M* - sum_k g_k (as for D2Q9: the stored node
// sums to its post-collision mass M* up to FP32 rounding). M* is the mass the
// collision hands over, rho + R.
template <int PREC> struct St3;
template <> struct St3<LBM_F64> {
    using T = double;
    using C = double;
    __device__ static __forceinline__ C ld(const T *__restrict__ f, long long i, const float *, C) { return __ldg(f + i); }
    __device__ static __forceinline__ void store(T *__restrict__ f, float *, long long P, long long i, const C v[19], C,
                                                 C)
    {
#pragma unroll
        for (int k = 0; k < 19; ++k) __stcs(f + k * P + i, v[k]);
    }
};
template <> struct St3<LBM_F32> {
    using T = float;
    using C = float;
    __device__ static __forceinline__ C ld(const T *__restrict__ f, long long i, const float *, C) { return __ldg(f + i); }
    __device__ static __forceinline__ void store(T *__restrict__ f, float *, long long P, long long i, const C v[19], C,
                                                 C)
    {
#pragma unroll
        for (int k = 0; k < 19; ++k) __stcs(f + k * P + i, v[k]);
    }
};
template <> struct St3<LBM_BF16S> {
    using T = __nv_bfloat16;
    using C = float;
    __device__ static __forceinline__ C ld(const T *__restrict__ f, long long i, const float *__restrict__ h, C w)
    {
        return fmaf(w, __ldg(h + i), __bfloat162float(f[i]));
    }
    __device__ static __forceinline__ void store(T *__restrict__ f, float *__restrict__ h, long long P, long long i,
                                                 const C v[19], C phi, C mass)
    {
        C gsum = C(0);
#pragma unroll
        for (int k = 0; k < 19; ++k) {
            const T g = __float2bfloat16_rn(fmaf(-w3<float>(k), phi, v[k]));
            gsum += __bfloat162float(g);
            f[k * P + i] = g;
        }
        h[i] = mass - gsum;
    }
};

template <class C>
struct Params3 {
    int nx, ny, nz;
    long long pitch, plane;          // plane = pitch * ny * nz
    C se, hse;                       // s_e and 1 - s_e/2
    C G[6];                          // A - s_e I: xx, xy, xz, yy, yz, zz
    C ux, uy, uz;
    C r0, r1, half_r0, inv_den, inv_post;
    int has_src;
    int abb[3];                      // 1: anti-bounce-back walls on axis x, y, z
    int any_abb;
    C phi_wall[6];                   // x-, x+, y-, y+, z-, z+
    int *err;                        // checked builds: index-fault word
};

// Coefficients at phi (Eq. 7 families, D = g(phi) I): B, B', the tensor
// Q = C + c_s^2 g I - c_s^2 phi I of Eq. 3 and trQ/3, and R = r0 + r1 phi.
template <int CONV, int DIFF, class C>
struct Coef3 {
    C Bx, By, Bz, bpx, bpy, bpz, Qxx, Qyy, Qzz, Qxy, Qxz, Qyz, tr3, R;
    __device__ __forceinline__ Coef3(const Params3<C> &p, C phi)
    {
        C cphi;
        if (CONV == 0) {
            Bx = p.ux * phi; By = p.uy * phi; Bz = p.uz * phi;
            bpx = p.ux; bpy = p.uy; bpz = p.uz;
            cphi = phi;
        } else {
            const C h = C(0.5) * phi * phi;
            Bx = p.ux * h; By = p.uy * h; Bz = p.uz * h;
            bpx = p.ux * phi; bpy = p.uy * phi; bpz = p.uz * phi;
            cphi = phi * phi * phi * C(1.0 / 3.0);
        }
        C g;
        if (DIFF == 0) g = phi;
        else if (DIFF == 1) g = phi + C(0.5) * phi * phi;
        else g = phi + phi * phi * phi * C(1.0 / 3.0);
        const C diag = (g - phi) * C(1.0 / 3.0);
        Qxx = p.ux * p.ux * cphi + diag; Qyy = p.uy * p.uy * cphi + diag; Qzz = p.uz * p.uz * cphi + diag;
        Qxy = p.ux * p.uy * cphi; Qxz = p.ux * p.uz * cphi; Qyz = p.uy * p.uz * cphi;
        tr3 = (Qxx + Qyy + Qzz) * C(1.0 / 3.0);
        R = p.has_src ? p.r1 * phi + p.r0 : C(0);
    }
    // feq_k = w_k [phi + 3 c.B + 4.5 (c Q c - trQ/3)] (Eq. 3)
    __device__ __forceinline__ C feq(int k, C phi) const
    {
        const C cx_ = C(c3x(k)), cy_ = C(c3y(k)), cz_ = C(c3z(k));
        const C cB = cx_ * Bx + cy_ * By + cz_ * Bz;
        const C cQc = cx_ * cx_ * Qxx + cy_ * cy_ * Qyy + cz_ * cz_ * Qzz +
                      C(2) * (cx_ * cy_ * Qxy + cx_ * cz_ * Qxz + cy_ * cz_ * Qyz);
        return w3<C>(k) * (phi + C(3) * cB + C(4.5) * (cQc - tr3));
    }
    // R_k = w_k (1 + 3 c.B') R (Eq. 9, Scheme B)
    __device__ __forceinline__ C source(int k) const
    {
        return w3<C>(k) * (C(1) + C(3) * (C(c3x(k)) * bpx + C(c3y(k)) * bpy + C(c3z(k)) * bpz)) * R;
    }
};

// Eq. 6 pairs each velocity with its opposite (k odd, k + 1); the sign pattern
// the pair form of collide3 is written out for
static_assert(c3x(1) == 1 && c3y(3) == 1 && c3z(5) == 1, "axis velocities");
static_assert(c3x(7) == 1 && c3y(7) == 1 && c3x(9) == 1 && c3y(9) == -1 && c3z(7) == 0 && c3z(9) == 0, "xy");
static_assert(c3x(11) == 1 && c3z(11) == 1 && c3x(13) == -1 && c3z(13) == 1 && c3y(11) == 0 && c3y(13) == 0, "xz");
static_assert(c3y(15) == 1 && c3z(15) == 1 && c3y(17) == 1 && c3z(17) == -1 && c3x(15) == 0 && c3x(17) == 0, "yz");

// The collision f_k - s_e (f_k - feq_k) - c_k.G + (1 - s_e/2) R_k of the moment
// reading, regrouped over each pair (k, opp(k)): with
//   X   = s_e (phi - 9/2 trQ/3) + (1 - s_e/2) R          (even, weight-free)
//   U_w = 3 w (s_e B + (1 - s_e/2) R B') - G             (odd, one per weight)
// the update is f'_k = (1 - s_e) f_k + e_k + c_k.U_w, e_k = w X + (9/2) s_e w c_k Q c_k,
// and f'_opp(k) takes the same even part with the odd part negated. c_k has
// one or two non-zero components, so each pair costs a few additions: the
// zero products of the per-direction form, which IEEE arithmetic keeps, are
// gone. The same arithmetic as Eq. 3 and Eq. 9 in another order of rounding.
template <int CONV, int DIFF, class C>
__device__ __forceinline__ void collide3(const Params3<C> &p, C f[19], C &phi_out, C &mass_out)
{
    C rho = C(0), jx = C(0), jy = C(0), jz = C(0);
#pragma unroll
    for (int k = 0; k < 19; ++k) {
        rho += f[k];
        if (c3x(k)) jx += C(c3x(k)) * f[k];
        if (c3y(k)) jy += C(c3y(k)) * f[k];
        if (c3z(k)) jz += C(c3z(k)) * f[k];
    }
    const C phi = (rho + p.half_r0) * p.inv_den;                 // Eq. 35
    phi_out = phi;
    const Coef3<CONV, DIFF, C> q(p, phi);
    // G = (A - s_e I) [(j - B) + B' R / 2]
    const C vx = (jx - q.Bx) + C(0.5) * q.bpx * q.R, vy = (jy - q.By) + C(0.5) * q.bpy * q.R;
    const C vz = (jz - q.Bz) + C(0.5) * q.bpz * q.R;
    const C Gx = (p.G[0] * vx + p.G[1] * vy + p.G[2] * vz) * C(0.1);
    const C Gy = (p.G[1] * vx + p.G[3] * vy + p.G[4] * vz) * C(0.1);
    const C Gz = (p.G[2] * vx + p.G[4] * vy + p.G[5] * vz) * C(0.1);

    const C omse = C(1) - p.se;
    const C hR = p.has_src ? p.hse * q.R : C(0);
    const C X = p.se * (phi - C(4.5) * q.tr3) + hR;
    C SBx = p.se * q.Bx, SBy = p.se * q.By, SBz = p.se * q.Bz;
    if (p.has_src) { SBx += hR * q.bpx; SBy += hR * q.bpy; SBz += hR * q.bpz; }
    // 3 w: 1/6 for the axis weight 1/18, 1/12 for the diagonal weight 1/36
    const C Ux = C(1.0 / 6.0) * SBx - Gx, Uy = C(1.0 / 6.0) * SBy - Gy, Uz = C(1.0 / 6.0) * SBz - Gz;
    const C Vx = C(1.0 / 12.0) * SBx - Gx, Vy = C(1.0 / 12.0) * SBy - Gy, Vz = C(1.0 / 12.0) * SBz - Gz;
    // (9/2) s_e w: s_e / 4 for w = 1/18 (also 2 (9/2) s_e / 36), s_e / 8 for w = 1/36
    const C q18 = C(0.25) * p.se, q36 = C(0.125) * p.se;
    const C b18 = X * C(1.0 / 18.0), b36 = X * C(1.0 / 36.0);

    // the odd parts cancel over each pair, sum_k e_k = X + (9/2) s_e c_s^2 trQ,
    // and rho - phi = -R/2 (Eq. 35): the node hands over rho + R
    mass_out = p.has_src ? rho + q.R : rho;
    f[0] = omse * f[0] + X * C(1.0 / 3.0);
    C e, o;
    // axis pairs: c Q c = Q_aa
    e = q18 * q.Qxx + b18; f[1] = omse * f[1] + (e + Ux); f[2] = omse * f[2] + (e - Ux);
    e = q18 * q.Qyy + b18; f[3] = omse * f[3] + (e + Uy); f[4] = omse * f[4] + (e - Uy);
    e = q18 * q.Qzz + b18; f[5] = omse * f[5] + (e + Uz); f[6] = omse * f[6] + (e - Uz);
    // diagonal pairs in the plane (a, b): c Q c = Q_aa + Q_bb + 2 c_a c_b Q_ab
    C S = q36 * (q.Qxx + q.Qyy) + b36, D = q18 * q.Qxy;
    e = S + D; o = Vx + Vy; f[7] = omse * f[7] + (e + o); f[8] = omse * f[8] + (e - o);
    e = S - D; o = Vx - Vy; f[9] = omse * f[9] + (e + o); f[10] = omse * f[10] + (e - o);
    S = q36 * (q.Qxx + q.Qzz) + b36; D = q18 * q.Qxz;
    e = S + D; o = Vx + Vz; f[11] = omse * f[11] + (e + o); f[12] = omse * f[12] + (e - o);
    e = S - D; o = Vz - Vx; f[13] = omse * f[13] + (e + o); f[14] = omse * f[14] + (e - o);
    S = q36 * (q.Qyy + q.Qzz) + b36; D = q18 * q.Qyz;
    e = S + D; o = Vy + Vz; f[15] = omse * f[15] + (e + o); f[16] = omse * f[16] + (e - o);
    e = S - D; o = Vy - Vz; f[17] = omse * f[17] + (e + o); f[18] = omse * f[18] + (e - o);
}

// Pull the 19 populations of node (x, y, z) with periodic wrap; WALLS: then
// replace the links that cross an anti-bounce-back wall (at wall nodes only).
// A lattice without walls compiles without the wall code.
template <int PREC, int CONV, int DIFF, bool WALLS>
__device__ __forceinline__ void pull3_node(const Params3<typename St3<PREC>::C> &p,
                                           const typename St3<PREC>::T *__restrict__ src,
                                           const float *__restrict__ src_h, int x, int y, int z,
                                           typename St3<PREC>::C f[19])
{
    using S = St3<PREC>;
    using T = typename S::C;
    int xm = x == 0 ? p.nx - 1 : x - 1, xp = x == p.nx - 1 ? 0 : x + 1;
    int ym = y == 0 ? p.ny - 1 : y - 1, yp = y == p.ny - 1 ? 0 : y + 1;
    int zm = z == 0 ? p.nz - 1 : z - 1, zp = z == p.nz - 1 ? 0 : z + 1;
    LBM_CHK(xm, p.nx, p.err, kErrX);
    LBM_CHK(xp, p.nx, p.err, kErrX);
    LBM_CHK(ym, p.ny, p.err, kErrY);
    LBM_CHK(yp, p.ny, p.err, kErrY);
    LBM_CHK(zm, p.nz, p.err, kErrIndex);
    LBM_CHK(zp, p.nz, p.err, kErrIndex);
    const long long P = p.plane;
#pragma unroll
    for (int k = 0; k < 19; ++k) {
        // source node x - c_k
        const int xs = c3x(k) > 0 ? xm : (c3x(k) < 0 ? xp : x);
        const int ys = c3y(k) > 0 ? ym : (c3y(k) < 0 ? yp : y);
        const int zs = c3z(k) > 0 ? zm : (c3z(k) < 0 ? zp : z);
        f[k] = S::ld(src + k * P, ((long long)zs * p.ny + ys) * p.pitch + xs, src_h, w3<T>(k));
    }
    if constexpr (WALLS) {
        const long long own = ((long long)z * p.ny + y) * p.pitch + x;
        const bool wall = (p.abb[0] && (x == 0 || x == p.nx - 1)) || (p.abb[1] && (y == 0 || y == p.ny - 1)) ||
                          (p.abb[2] && (z == 0 || z == p.nz - 1));
        if (wall) {
            // anti-bounce-back (the rule of the 2-D walls, Sec. 3.6): a link whose
            // source lies beyond a wall takes -fbar*_opp(k) of this node plus
            // feq_k + feq_opp(k) at the wall value (the mean value of the walls
            // the link crosses)
#pragma unroll
            for (int k = 1; k < 19; ++k) {
                const int xs = x - c3x(k), ys = y - c3y(k), zs = z - c3z(k);
                T tot = T(0);
                int cnt = 0;
                if (p.abb[0] && (xs < 0 || xs >= p.nx)) { tot += xs < 0 ? p.phi_wall[0] : p.phi_wall[1]; ++cnt; }
                if (p.abb[1] && (ys < 0 || ys >= p.ny)) { tot += ys < 0 ? p.phi_wall[2] : p.phi_wall[3]; ++cnt; }
                if (p.abb[2] && (zs < 0 || zs >= p.nz)) { tot += zs < 0 ? p.phi_wall[4] : p.phi_wall[5]; ++cnt; }
                if (cnt) {
                    const T phiw = cnt == 1 ? tot : tot / T(cnt);
                    const Coef3<CONV, DIFF, T> q(p, phiw);
                    f[k] = q.feq(k, phiw) + q.feq(opp3(k), phiw) - S::ld(src + opp3(k) * P, own, src_h, w3<T>(opp3(k)));
                }
            }
        }
    }
}

}  // namespace lbm
