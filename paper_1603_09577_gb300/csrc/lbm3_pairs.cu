// lbm3_pairs.cu -- the D3Q19 fused stream-collide step with every thread
// owning two x-adjacent nodes (lbm3_desc.kernel_variant 2), FP32 and
// BF16-shifted storage.
//
// A node pair (X, X + 1) starts at an even X, so its output words are aligned:
// each of the 19 population planes (and the shift plane) is written with one
// 64-bit (FP32) or 32-bit (bf16x2) store per pair, the bf16 rounding of a pair
// being one packed conversion. Pulls with c_x = 0 read an aligned source pair;
// those with c_x = +-1 read the pair straddling two aligned words. For BF16S
// the shift plane of each source row is read as aligned float2 words that serve
// all source pairs of that row. Both nodes collide together in packed FP32x2
// arithmetic, with the direction signs resolved at compile time. Pairs whose
// pulls could leave the domain (the first and last node columns, rows and
// layers) take the per-node pull with periodic wrap and walls.
#include "lbm3_device.cuh"

namespace lbm {
namespace {

__device__ __forceinline__ F2 bf2_unpack3(unsigned u)
{
    return F2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}

// s_k . (X, Y, Z) for the velocity of direction k, without multiplications
template <int k>
__device__ __forceinline__ F2 cdot(F2 X, F2 Y, F2 Z)
{
    F2 r(0.f);
    bool any = false;
    if constexpr (c3x(k) != 0) { r = c3x(k) > 0 ? X : -X; any = true; }
    if constexpr (c3y(k) != 0) { r = any ? (c3y(k) > 0 ? r + Y : r - Y) : (c3y(k) > 0 ? Y : -Y); any = true; }
    if constexpr (c3z(k) != 0) { r = any ? (c3z(k) > 0 ? r + Z : r - Z) : (c3z(k) > 0 ? Z : -Z); any = true; }
    return r;
}

// c_k . Q . c_k - tr(Q)/3 for the symmetric Q of Coef3
template <int k>
__device__ __forceinline__ F2 cqc(F2 Qxx, F2 Qyy, F2 Qzz, F2 Qxy, F2 Qxz, F2 Qyz, F2 tr3)
{
    F2 r = -tr3;
    if constexpr (c3x(k) != 0) r += Qxx;
    if constexpr (c3y(k) != 0) r += Qyy;
    if constexpr (c3z(k) != 0) r += Qzz;
    if constexpr (c3x(k) * c3y(k) != 0) r = mad(F2(float(2 * c3x(k) * c3y(k))), Qxy, r);
    if constexpr (c3x(k) * c3z(k) != 0) r = mad(F2(float(2 * c3x(k) * c3z(k))), Qxz, r);
    if constexpr (c3y(k) * c3z(k) != 0) r = mad(F2(float(2 * c3y(k) * c3z(k))), Qyz, r);
    return r;
}

Params3<F2> __device__ __forceinline__ widen3(const Params3<float> &p)
{
    Params3<F2> w;
    w.nx = p.nx; w.ny = p.ny; w.nz = p.nz; w.pitch = p.pitch; w.plane = p.plane;
    w.se = p.se; w.hse = p.hse;
    for (int i = 0; i < 6; ++i) w.G[i] = p.G[i];
    w.ux = p.ux; w.uy = p.uy; w.uz = p.uz;
    w.r0 = p.r0; w.r1 = p.r1; w.half_r0 = p.half_r0; w.inv_den = p.inv_den; w.inv_post = p.inv_post;
    w.has_src = p.has_src;
    w.abb[0] = w.abb[1] = w.abb[2] = 0;           // walls are taken in the per-node pull
    w.any_abb = 0;
    w.err = p.err;
    return w;
}

template <int k>
__device__ __forceinline__ void relax_k(const Params3<F2> &p, F2 f[19], F2 phi, F2 Bx,
                                        F2 By, F2 Bz, F2 bpx, F2 bpy, F2 bpz, F2 Qxx, F2 Qyy, F2 Qzz, F2 Qxy, F2 Qxz,
                                        F2 Qyz, F2 tr3, F2 R, F2 Gx, F2 Gy, F2 Gz)
{
    const F2 w(w3<float>(k));
    F2 fe;
    if constexpr (k == 0) fe = w * mad(F2(4.5f), -tr3, phi);
    else fe = w * mad(F2(4.5f), cqc<k>(Qxx, Qyy, Qzz, Qxy, Qxz, Qyz, tr3), mad(F2(3.f), cdot<k>(Bx, By, Bz), phi));
    F2 v = f[k] - p.se * (f[k] - fe);
    if constexpr (k != 0) v = v - cdot<k>(Gx, Gy, Gz);
    if (p.has_src) {
        F2 src;
        if constexpr (k == 0) src = w * R;
        else src = w * mad(F2(3.f), cdot<k>(bpx, bpy, bpz), F2(1.f)) * R;
        v = mad(p.hse, src, v);
    }
    f[k] = v;
}

template <int k0>
__device__ __forceinline__ void relax_all(const Params3<F2> &p, F2 f[19], F2 phi, F2 Bx,
                                          F2 By, F2 Bz, F2 bpx, F2 bpy, F2 bpz, F2 Qxx, F2 Qyy, F2 Qzz, F2 Qxy, F2 Qxz,
                                          F2 Qyz, F2 tr3, F2 R, F2 Gx, F2 Gy, F2 Gz)
{
    relax_k<k0>(p, f, phi, Bx, By, Bz, bpx, bpy, bpz, Qxx, Qyy, Qzz, Qxy, Qxz, Qyz, tr3, R, Gx, Gy, Gz);
    if constexpr (k0 + 1 < 19)
        relax_all<k0 + 1>(p, f, phi, Bx, By, Bz, bpx, bpy, bpz, Qxx, Qyy, Qzz, Qxy, Qxz, Qyz, tr3, R, Gx, Gy, Gz);
}

template <int k0>
__device__ __forceinline__ void moments(const F2 f[19], F2 &rho, F2 &jx, F2 &jy, F2 &jz)
{
    if constexpr (k0 > 0) {
        rho += f[k0];
        if constexpr (c3x(k0) > 0) jx += f[k0];
        if constexpr (c3x(k0) < 0) jx -= f[k0];
        if constexpr (c3y(k0) > 0) jy += f[k0];
        if constexpr (c3y(k0) < 0) jy -= f[k0];
        if constexpr (c3z(k0) > 0) jz += f[k0];
        if constexpr (c3z(k0) < 0) jz -= f[k0];
    }
    if constexpr (k0 + 1 < 19) moments<k0 + 1>(f, rho, jx, jy, jz);
}

// The collision of collide3 (projector form of the moment reading, Scheme B)
// for two nodes at once.
template <int CONV, int DIFF>
__device__ __forceinline__ void collide3p(const Params3<F2> &p, F2 f[19], F2 &phi_out)
{
    F2 rho = f[0], jx(0.f), jy(0.f), jz(0.f);
    moments<0>(f, rho, jx, jy, jz);
    const F2 phi = (rho + p.half_r0) * p.inv_den;                  // Eq. 35
    phi_out = phi;
    const Coef3<CONV, DIFF, F2> q(p, phi);
    const F2 half(0.5f);
    const F2 vx = mad(half * q.bpx, q.R, jx - q.Bx), vy = mad(half * q.bpy, q.R, jy - q.By);
    const F2 vz = mad(half * q.bpz, q.R, jz - q.Bz);
    const F2 tenth(0.1f);
    const F2 Gx = mad(p.G[0], vx, mad(p.G[1], vy, p.G[2] * vz)) * tenth;
    const F2 Gy = mad(p.G[1], vx, mad(p.G[3], vy, p.G[4] * vz)) * tenth;
    const F2 Gz = mad(p.G[2], vx, mad(p.G[4], vy, p.G[5] * vz)) * tenth;
    relax_all<0>(p, f, phi, q.Bx, q.By, q.Bz, q.bpx, q.bpy, q.bpz, q.Qxx, q.Qyy, q.Qzz, q.Qxy, q.Qxz, q.Qyz,
                 q.tr3, q.R, Gx, Gy, Gz);
}

// interior pair (X, X + 1), X even: every pull inside the domain
template <int PREC>
__device__ __forceinline__ void pull3_pair(const Params3<float> &p, const typename St3<PREC>::T *__restrict__ src,
                                           const float *__restrict__ src_h, int X, int y, int z, F2 f[19])
{
    const long long P = p.plane;
    const unsigned pit = (unsigned)p.pitch, ny = (unsigned)p.ny;
#pragma unroll
    for (int k = 0; k < 19; ++k) {
        const unsigned i = ((unsigned)(z - c3z(k)) * ny + (unsigned)(y - c3y(k))) * pit + (unsigned)X;
        if constexpr (PREC == LBM_F32) {
            const float *pk = src + k * P;
            if (c3x(k) == 0) f[k] = F2(__ldg(reinterpret_cast<const float2 *>(pk + i)));
            else f[k] = F2(__ldg(pk + i - c3x(k)), __ldg(pk + i + 1 - c3x(k)));
        } else {
            const __nv_bfloat16 *pk = src + k * P;
            unsigned u;
            F2 h;
            const float2 hc = __ldg(reinterpret_cast<const float2 *>(src_h + i));
            if (c3x(k) == 0) {
                u = __ldg(reinterpret_cast<const unsigned *>(pk + i));
                h = F2(hc);
            } else if (c3x(k) > 0) {                                // source pair (X - 1, X)
                const unsigned w0 = __ldg(reinterpret_cast<const unsigned *>(pk + i - 2));
                const unsigned w1 = __ldg(reinterpret_cast<const unsigned *>(pk + i));
                u = __byte_perm(w0, w1, 0x5432);
                h = F2(__ldg(src_h + i - 1), hc.x);
            } else {                                                // source pair (X + 1, X + 2)
                const unsigned w0 = __ldg(reinterpret_cast<const unsigned *>(pk + i));
                const unsigned w1 = __ldg(reinterpret_cast<const unsigned *>(pk + i + 2));
                u = __byte_perm(w0, w1, 0x5432);
                h = F2(hc.y, __ldg(src_h + i + 2));
            }
            f[k] = mad(F2(w3<float>(k)), h, bf2_unpack3(u));
        }
    }
}

template <int PREC>
__device__ __forceinline__ void store3_pair(const Params3<float> &p, typename St3<PREC>::T *__restrict__ dst,
                                            float *__restrict__ dst_h, long long i, const F2 f[19], F2 phi, bool both)
{
    const long long P = p.plane;
    if constexpr (PREC == LBM_F32) {
#pragma unroll
        for (int k = 0; k < 19; ++k) {
            if (both) __stcs(reinterpret_cast<float2 *>(dst + k * P + i), f[k].v);
            else __stcs(dst + k * P + i, f[k].v.x);
        }
    } else {
        F2 mass(0.f), gsum(0.f);
#pragma unroll
        for (int k = 0; k < 19; ++k) {
            const F2 dev = mad(F2(-w3<float>(k)), phi, f[k]);
            const __nv_bfloat162 b = __floats2bfloat162_rn(dev.v.x, dev.v.y);
            const unsigned u = *reinterpret_cast<const unsigned *>(&b);
            mass += f[k];
            gsum += bf2_unpack3(u);
            if (both) __stcs(reinterpret_cast<unsigned *>(dst + k * P + i), u);
            else dst[k * P + i] = b.x;
        }
        const F2 h = mass - gsum;
        if (both) __stcs(reinterpret_cast<float2 *>(dst_h + i), h.v);
        else dst_h[i] = h.v.x;
    }
}

// the per-node pull of the two nodes of an edge pair, out of line so that its
// wrap and wall logic does not add to the registers of the interior pairs
template <int PREC, int CONV, int DIFF>
__device__ __noinline__ void pull3_pair_edge(const Params3<float> &p, const typename St3<PREC>::T *__restrict__ src,
                                             const float *__restrict__ src_h, int X, int y, int z, bool both, F2 f[19])
{
    float a[19], b[19];
    pull3_node<PREC, CONV, DIFF>(p, src, src_h, X, y, z, a);
    pull3_node<PREC, CONV, DIFF>(p, src, src_h, both ? X + 1 : X, y, z, b);
#pragma unroll
    for (int k = 0; k < 19; ++k) f[k] = F2(a[k], b[k]);
}

template <int PREC, int CONV, int DIFF>
__global__ void __launch_bounds__(256)
k_step3p(const Params3<float> p, const typename St3<PREC>::T *__restrict__ src, const float *__restrict__ src_h,
         typename St3<PREC>::T *__restrict__ dst, float *__restrict__ dst_h)
{
    const int X = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (X >= p.nx || y >= p.ny) return;
    const bool both = X + 1 < p.nx;
    const bool interior = X >= 1 && X + 2 <= p.nx - 1 && y >= 1 && y + 1 <= p.ny - 1 && z >= 1 && z + 1 <= p.nz - 1;
    F2 f[19];
    if (interior) {
        pull3_pair<PREC>(p, src, src_h, X, y, z, f);
    } else {
        pull3_pair_edge<PREC, CONV, DIFF>(p, src, src_h, X, y, z, both, f);
    }
    F2 phi;
    collide3p<CONV, DIFF>(widen3(p), f, phi);
    store3_pair<PREC>(p, dst, dst_h, ((long long)z * p.ny + y) * p.pitch + X, f, phi, both);
}

template <int PREC, int CONV, int DIFF>
cudaError_t launch_t(const Params3<float> &p, int block_rows, const void *src, const float *src_h, void *dst,
                     float *dst_h, cudaStream_t st)
{
    using T = typename St3<PREC>::T;
    const dim3 block(32, block_rows > 0 ? block_rows : 8);
    const dim3 grid((p.nx + 63) / 64, (p.ny + block.y - 1) / block.y, p.nz);
    k_step3p<PREC, CONV, DIFF><<<grid, block, 0, st>>>(p, (const T *)src, src_h, (T *)dst, dst_h);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_p(int family, const Params3<float> &p, int block_rows, const void *src, const float *src_h,
                     void *dst, float *dst_h, cudaStream_t st)
{
    switch (family) {
    case 0: return launch_t<PREC, 0, 0>(p, block_rows, src, src_h, dst, dst_h, st);
    case 1: return launch_t<PREC, 0, 1>(p, block_rows, src, src_h, dst, dst_h, st);
    case 2: return launch_t<PREC, 0, 2>(p, block_rows, src, src_h, dst, dst_h, st);
    case 3: return launch_t<PREC, 1, 0>(p, block_rows, src, src_h, dst, dst_h, st);
    case 4: return launch_t<PREC, 1, 1>(p, block_rows, src, src_h, dst, dst_h, st);
    case 5: return launch_t<PREC, 1, 2>(p, block_rows, src, src_h, dst, dst_h, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch3_pairs(int prec, int family, const Params3<float> &p, int block_rows, const void *src,
                          const float *src_h, void *dst, float *dst_h, cudaStream_t st)
{
    if (prec == LBM_F32) return launch_p<LBM_F32>(family, p, block_rows, src, src_h, dst, dst_h, st);
    if (prec == LBM_BF16S) return launch_p<LBM_BF16S>(family, p, block_rows, src, src_h, dst, dst_h, st);
    return cudaErrorInvalidValue;
}

}  // namespace lbm
