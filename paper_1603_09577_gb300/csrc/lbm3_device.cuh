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
// collision hands over, rho + R. A node is addressed by its index within a
// plane (at most 2^31 - 1, checked when the solver is created).
template <int PREC> struct St3;
template <> struct St3<LBM_F64> {
    using T = double;
    using C = double;
    template <class I>
    __device__ static __forceinline__ C ld(const T *__restrict__ f, I i, const float *, I, C) { return __ldg(f + i); }
};
template <> struct St3<LBM_F32> {
    using T = float;
    using C = float;
    template <class I>
    __device__ static __forceinline__ C ld(const T *__restrict__ f, I i, const float *, I, C) { return __ldg(f + i); }
};
template <> struct St3<LBM_BF16S> {
    using T = __nv_bfloat16;
    using C = float;
    template <class I>
    __device__ static __forceinline__ C ld(const T *__restrict__ f, I i, const float *__restrict__ h, I hi, C w)
    {
        return fmaf(w, __ldg(h + hi), __bfloat162float(f[i]));
    }
};

// The two population buffers of one launch (and the BF16S shift planes), a
// kernel argument. Plane k is reached either through its own 64-bit pointer
// (any lattice) or, when 19 planes hold fewer than 2^32 elements, through the
// buffer's pointer and the 32-bit offset k * plane, so that a pull costs 32-bit
// index additions and one address computation from one base register.
template <class T>
struct Planes3 {
    const T *src[19];
    T *dst[19];
    const T *src0;
    T *dst0;
    unsigned poff[19];
    const float *src_h;
    float *dst_h;
};

// store node i's post-collision populations v (and the BF16S shift)
template <int PREC, bool OFF32>
__device__ __forceinline__ void store3(const Planes3<typename St3<PREC>::T> &pl, unsigned i,
                                       const typename St3<PREC>::C v[19], typename St3<PREC>::C phi,
                                       typename St3<PREC>::C mass)
{
    if constexpr (PREC == LBM_BF16S) {
        // g_k = f*_k - w_k phi; the two directions of a pair share w_k, so their
        // shifts, bf16 roundings and sums go two at a time
        const __nv_bfloat16 g0 = __float2bfloat16_rn(fmaf(-w3<float>(0), phi, v[0]));
        if constexpr (OFF32) pl.dst0[i] = g0;
        else pl.dst[0][i] = g0;
        const F2 s18(-w3<float>(1) * phi), s36(-w3<float>(7) * phi);
        F2 gsum(0.f);
#pragma unroll
        for (int m = 0; m < 9; ++m) {
            const int k = 2 * m + 1;
            const F2 gp = F2(v[k], v[k + 1]) + (k < 7 ? s18 : s36);
            const __nv_bfloat162 g = __floats2bfloat162_rn(gp.v.x, gp.v.y);
            gsum = gsum + F2(__low2float(g), __high2float(g));
            if constexpr (OFF32) {
                pl.dst0[i + pl.poff[k]] = __low2bfloat16(g);
                pl.dst0[i + pl.poff[k + 1]] = __high2bfloat16(g);
            } else {
                pl.dst[k][i] = __low2bfloat16(g);
                pl.dst[k + 1][i] = __high2bfloat16(g);
            }
        }
        pl.dst_h[i] = mass - (__bfloat162float(g0) + (gsum.v.x + gsum.v.y));
    } else {
#pragma unroll
        for (int k = 0; k < 19; ++k) {
            if constexpr (OFF32) __stcs(pl.dst0 + (i + pl.poff[k]), v[k]);
            else __stcs(pl.dst[k] + i, v[k]);
        }
    }
}

template <class C>
struct Params3 {
    int nx, ny, nz;
    long long pitch, plane;          // plane = pitch * ny * nz
    C se, hse;                       // s_e and 1 - s_e/2
    C omse, q18, q36;                // 1 - s_e, s_e/4, s_e/8 (the pair form of the collision)
    C G[6];                          // (A - s_e I)/10 (Pi_j = c c^T / 10): xx, xy, xz, yy, yz, zz
    C ux, uy, uz;
    C uu[6];                         // u u^T: xx, xy, xz, yy, yz, zz
    C u2_3;                          // |u|^2 / 3
    C u6[3], u12[3];                 // u/6, u/12
    C ea[3];                         // s_e/4 u_a u_a (a = x, y, z)
    C ep[3], em[3];                  // s_e/8 (u_a u_a + u_b u_b) +/- s_e/4 u_a u_b, (a, b) = xy, xz, yz
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
        Qxx = p.uu[0] * cphi; Qyy = p.uu[3] * cphi; Qzz = p.uu[5] * cphi;
        Qxy = p.uu[1] * cphi; Qxz = p.uu[2] * cphi; Qyz = p.uu[4] * cphi;
        tr3 = p.u2_3 * cphi;
        // the isotropic part c_s^2 (g - phi) I (none for g = phi)
        if constexpr (DIFF != 0) {
            const C diag = DIFF == 1 ? C(0.5) * phi * phi * C(1.0 / 3.0) : phi * phi * phi * C(1.0 / 9.0);
            Qxx += diag; Qyy += diag; Qzz += diag; tr3 += diag;
        }
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

// f'_k = (1 - s_e) f_k + (e + o) and f'_opp = (1 - s_e) f_opp + (e - o): in FP32
// the two as one packed FP32x2 multiply-add
template <class C>
__device__ __forceinline__ void pair_update(C &a, C &b, C omse, C e, C o)
{
    if constexpr (sizeof(C) == 4) {
        const F2 r = mad(F2(a, b), F2(omse), F2(e + o, e - o));
        a = r.v.x;
        b = r.v.y;
    } else {
        a = omse * a + (e + o);
        b = omse * b + (e - o);
    }
}

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
    // rho and j from the pair sums and differences d_m = f_(2m+1) - f_(2m+2)
    C rho, d[9];
    if constexpr (sizeof(C) == 4) {
        // FP32: the pair sums accumulate as one packed FP32x2 sum
        F2 s2 = F2(f[1], f[2]);
#pragma unroll
        for (int m = 1; m < 9; ++m) s2 = s2 + F2(f[2 * m + 1], f[2 * m + 2]);
        rho = f[0] + (s2.v.x + s2.v.y);
    } else {
        rho = f[0];
#pragma unroll
        for (int m = 0; m < 9; ++m) rho += f[2 * m + 1] + f[2 * m + 2];
    }
#pragma unroll
    for (int m = 0; m < 9; ++m) d[m] = f[2 * m + 1] - f[2 * m + 2];
    const C jx = (d[0] + d[3]) + (d[4] + d[5]) - d[6];
    const C jy = (d[1] + d[3]) - d[4] + (d[7] + d[8]);
    const C jz = (d[2] + d[5]) + (d[6] + d[7]) - d[8];
    const C phi = (rho + p.half_r0) * p.inv_den;                 // Eq. 35
    phi_out = phi;
    // Eq. 7 families: B = u beta, B' = u beta', C = u u cphi with beta = phi,
    // beta' = 1, cphi = phi (conv 0) or beta = phi^2/2, beta' = phi, cphi = phi^3/3
    C beta, cphi;
    if constexpr (CONV == 0) { beta = phi; cphi = phi; }
    else { beta = C(0.5) * phi * phi; cphi = phi * phi * phi * C(1.0 / 3.0); }
    const C R = p.has_src ? p.r1 * phi + p.r0 : C(0);
    const C hR = p.has_src ? p.hse * R : C(0);
    // G = (A - s_e I)/10 [(j - B) + B' R / 2], (j - B) + B' R/2 = j - u sv
    C sv = beta, t = p.se * beta;              // s_e B + (1 - s_e/2) R B' = u t
    if (p.has_src) {
        if constexpr (CONV == 0) { sv -= C(0.5) * R; t += hR; }
        else { sv -= C(0.5) * R * phi; t += hR * phi; }
    }
    const C vx = jx - p.ux * sv, vy = jy - p.uy * sv, vz = jz - p.uz * sv;
    const C Gx = p.G[0] * vx + p.G[1] * vy + p.G[2] * vz;
    const C Gy = p.G[1] * vx + p.G[3] * vy + p.G[4] * vz;
    const C Gz = p.G[2] * vx + p.G[4] * vy + p.G[5] * vz;
    // U_w = 3 w u t - G: u/6 for the axis weight 1/18, u/12 for the diagonal weight 1/36
    const C Ux = p.u6[0] * t - Gx, Uy = p.u6[1] * t - Gy, Uz = p.u6[2] * t - Gz;
    const C Vx = p.u12[0] * t - Gx, Vy = p.u12[1] * t - Gy, Vz = p.u12[2] * t - Gz;
    // Q = u u cphi + c_s^2 (g - phi) I; trQ/3 = |u|^2 cphi/3 + the isotropic part
    C tr3 = p.u2_3 * cphi, iso = C(0);
    if constexpr (DIFF == 1) iso = C(0.5) * phi * phi * C(1.0 / 3.0);
    else if constexpr (DIFF == 2) iso = phi * phi * phi * C(1.0 / 9.0);
    if constexpr (DIFF != 0) tr3 += iso;
    const C X = p.se * (phi - C(4.5) * tr3) + hR;
    // even parts: w X + (9/2) s_e w c Q c. Axis: (s_e/4) Q_aa + X/18; diagonal in
    // (a, b): (s_e/8)(Q_aa + Q_bb) +/- (s_e/4) Q_ab + X/36. The products of u u
    // with these factors come from the host (ea, ep, em); the isotropic part
    // adds (s_e/4) iso to both
    C b18 = X * C(1.0 / 18.0), b36 = X * C(1.0 / 36.0);
    if constexpr (DIFF != 0) { b18 += p.q18 * iso; b36 += p.q18 * iso; }
    const C omse = p.omse;

    // the odd parts cancel over each pair, sum_k e_k = X + (9/2) s_e c_s^2 trQ,
    // and rho - phi = -R/2 (Eq. 35): the node hands over rho + R
    mass_out = p.has_src ? rho + R : rho;
    f[0] = omse * f[0] + X * C(1.0 / 3.0);
    pair_update(f[1], f[2], omse, p.ea[0] * cphi + b18, Ux);
    pair_update(f[3], f[4], omse, p.ea[1] * cphi + b18, Uy);
    pair_update(f[5], f[6], omse, p.ea[2] * cphi + b18, Uz);
    pair_update(f[7], f[8], omse, p.ep[0] * cphi + b36, Vx + Vy);
    pair_update(f[9], f[10], omse, p.em[0] * cphi + b36, Vx - Vy);
    pair_update(f[11], f[12], omse, p.ep[1] * cphi + b36, Vx + Vz);
    pair_update(f[13], f[14], omse, p.em[1] * cphi + b36, Vz - Vx);
    pair_update(f[15], f[16], omse, p.ep[2] * cphi + b36, Vy + Vz);
    pair_update(f[17], f[18], omse, p.em[2] * cphi + b36, Vy - Vz);
}

// Pull the 19 populations of node (x, y, z) with periodic wrap; WALLS: then
// replace the links that cross an anti-bounce-back wall (at wall nodes only).
// A lattice without walls compiles without the wall code. The source of
// direction k is the node's own index plus the offsets of its neighbour on
// each axis, in 32-bit arithmetic (a plane holds fewer than 2^31 elements).
template <int PREC, int CONV, int DIFF, bool WALLS, bool OFF32>
__device__ __forceinline__ void pull3_node(const Params3<typename St3<PREC>::C> &p,
                                           const Planes3<typename St3<PREC>::T> &pl, int x, int y, int z,
                                           unsigned own, typename St3<PREC>::C f[19])
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
    // offsets of the neighbours x -/+ 1, y -/+ 1, z -/+ 1 (wrapped)
    const int rowp = (int)p.pitch, slab = (int)p.pitch * p.ny;
    const unsigned ox[2] = {(unsigned)(xm - x), (unsigned)(xp - x)};
    const unsigned oy[2] = {(unsigned)((ym - y) * rowp), (unsigned)((yp - y) * rowp)};
    const unsigned oz[2] = {(unsigned)((zm - z) * slab), (unsigned)((zp - z) * slab)};
    // source node x - c_k of direction k
    auto src_of = [&](int k) {
        unsigned i = own;
        if (c3x(k)) i += ox[c3x(k) > 0 ? 0 : 1];
        if (c3y(k)) i += oy[c3y(k) > 0 ? 0 : 1];
        if (c3z(k)) i += oz[c3z(k) > 0 ? 0 : 1];
        return i;
    };
    if constexpr (PREC == LBM_BF16S) {
        // f_k = g_k + w_k h at the source; a pair (k, opp(k)) shares w_k, so the
        // two reconstructions are one packed multiply-add
        f[0] = OFF32 ? S::ld(pl.src0, own, pl.src_h, own, w3<T>(0)) : S::ld(pl.src[0], own, pl.src_h, own, w3<T>(0));
#pragma unroll
        for (int m = 0; m < 9; ++m) {
            const int k = 2 * m + 1;
            const unsigned ia = src_of(k), ib = src_of(k + 1);
            const __nv_bfloat16 ga = OFF32 ? pl.src0[ia + pl.poff[k]] : pl.src[k][ia];
            const __nv_bfloat16 gb = OFF32 ? pl.src0[ib + pl.poff[k + 1]] : pl.src[k + 1][ib];
            const F2 r = mad(F2(__ldg(pl.src_h + ia), __ldg(pl.src_h + ib)), F2(w3<float>(k)),
                             F2(__bfloat162float(ga), __bfloat162float(gb)));
            f[k] = r.v.x;
            f[k + 1] = r.v.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 19; ++k) {
            const unsigned i = src_of(k);
            if constexpr (OFF32) f[k] = S::ld(pl.src0, i + pl.poff[k], pl.src_h, i, w3<T>(k));
            else f[k] = S::ld(pl.src[k], i, pl.src_h, i, w3<T>(k));
        }
    }
    if constexpr (WALLS) {
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
                    const T back = OFF32 ? S::ld(pl.src0, own + pl.poff[opp3(k)], pl.src_h, own, w3<T>(opp3(k)))
                                         : S::ld(pl.src[opp3(k)], own, pl.src_h, own, w3<T>(opp3(k)));
                    f[k] = q.feq(k, phiw) + q.feq(opp3(k), phiw) - back;
                }
            }
        }
    }
}

}  // namespace lbm
