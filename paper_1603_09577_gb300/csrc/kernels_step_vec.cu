// kernels_step_vec.cu -- the fused pull-stream / collide step (Eq. 34) with four
// x-adjacent nodes per thread, for FP32 and BF16-shifted storage.
//
// A warp covers 128 consecutive nodes of one row. Every plane is read with one
// aligned vector load per thread (16 B of FP32 or 8 B of bf16); the +-1 x-shift
// of the pull comes from the neighbouring lane by a warp shuffle, and only the
// lane at a warp's or row's end fetches its missing element from memory. The
// nine outgoing planes are written with aligned vector stores. Compared with one
// node per thread this removes most of the per-node address arithmetic and
// load/store instructions, which bound the one-node kernel's issue rate.
// Requires nx % 4 == 0 (rows are padded to 64 elements, so vectors are aligned).
#include "lbm_internal.h"

namespace lbm {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// four consecutive values starting at element x0 of a row (x0 % 4 == 0)
__device__ __forceinline__ void load4(const float *__restrict__ row, int x0, float v[4])
{
    const float4 a = __ldg(reinterpret_cast<const float4 *>(row + x0));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}

__device__ __forceinline__ void load4(const __nv_bfloat16 *__restrict__ row, int x0, float v[4])
{
    const uint2 a = __ldg(reinterpret_cast<const uint2 *>(row + x0));
    v[0] = __uint_as_float(a.x << 16); v[1] = __uint_as_float(a.x & 0xffff0000u);
    v[2] = __uint_as_float(a.y << 16); v[3] = __uint_as_float(a.y & 0xffff0000u);
}

__device__ __forceinline__ float load1(const float *__restrict__ row, int x) { return __ldg(row + x); }
__device__ __forceinline__ float load1(const __nv_bfloat16 *__restrict__ row, int x) { return __bfloat162float(row[x]); }

// Lane geometry of the +-1 shifts: the left neighbour element x0 - 1 comes from
// lane - 1 unless this lane starts a warp or the row (then from memory at xl);
// likewise the right element x0 + 4 (memory at xr).
struct Lanes {
    int x0;            // first node of this thread (clamped into the row for idle lanes)
    bool left_mem, right_mem;
    int xl, xr;
};

// Values of one plane at source nodes (x - CX) for the four nodes of this thread.
template <int CX, class T>
__device__ __forceinline__ void fetch(const T *__restrict__ row, const Lanes &L, float out[4])
{
    float v[4];
    load4(row, L.x0, v);
    if (CX == 0) {
        out[0] = v[0]; out[1] = v[1]; out[2] = v[2]; out[3] = v[3];
    } else if (CX == 1) {
        float left = __shfl_up_sync(kFull, v[3], 1);
        if (L.left_mem) left = load1(row, L.xl);
        out[0] = left; out[1] = v[0]; out[2] = v[1]; out[3] = v[2];
    } else {
        float right = __shfl_down_sync(kFull, v[0], 1);
        if (L.right_mem) right = load1(row, L.xr);
        out[0] = v[1]; out[1] = v[2]; out[2] = v[3]; out[3] = right;
    }
}

template <int PREC> struct VecIO;

template <> struct VecIO<LBM_F32> {
    using T = float;
    template <int CX>
    __device__ static __forceinline__ void pull(const T *__restrict__ plane, const float *, long long row, const Lanes &L,
                                                float, float out[4])
    {
        fetch<CX>(plane + row, L, out);
    }
    __device__ static __forceinline__ void store(T *__restrict__ f, float *, long long P, long long i, float v[4][9],
                                                 const float *)
    {
#pragma unroll
        for (int k = 0; k < 9; ++k)
            __stcs(reinterpret_cast<float4 *>(f + k * P + i), make_float4(v[0][k], v[1][k], v[2][k], v[3][k]));
    }
};

template <> struct VecIO<LBM_BF16S> {
    using T = __nv_bfloat16;
    // hv: the shift plane of the source row at x0 - 1 .. x0 + 4 (fetched once per row)
    template <int CX>
    __device__ static __forceinline__ void pull(const T *__restrict__ plane, const float hv[6], long long row,
                                                const Lanes &L, float w, float out[4])
    {
        float g[4];
        fetch<CX>(plane + row, L, g);
#pragma unroll
        for (int c = 0; c < 4; ++c) out[c] = fmaf(w, hv[c + 1 - CX], g[c]);
    }
    // g_k = bf16(f*_k - w_k phi); shift h = M* - sum_k g_k (mass-exact storage)
    __device__ static __forceinline__ void store(T *__restrict__ f, float *__restrict__ h, long long P, long long i,
                                                 float v[4][9], const float *phi)
    {
        float mass[4], gsum[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) { mass[c] = 0.f; gsum[c] = 0.f; }
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float w = wgt<float>(k);
            __nv_bfloat162 lo = __floats2bfloat162_rn(fmaf(-w, phi[0], v[0][k]), fmaf(-w, phi[1], v[1][k]));
            __nv_bfloat162 hi = __floats2bfloat162_rn(fmaf(-w, phi[2], v[2][k]), fmaf(-w, phi[3], v[3][k]));
            const float2 flo = __bfloat1622float2(lo), fhi = __bfloat1622float2(hi);
            gsum[0] += flo.x; gsum[1] += flo.y; gsum[2] += fhi.x; gsum[3] += fhi.y;
#pragma unroll
            for (int c = 0; c < 4; ++c) mass[c] += v[c][k];
            uint2 packed;
            packed.x = *reinterpret_cast<unsigned *>(&lo);
            packed.y = *reinterpret_cast<unsigned *>(&hi);
            *reinterpret_cast<uint2 *>(f + k * P + i) = packed;
        }
        __stcs(reinterpret_cast<float4 *>(h + i),
               make_float4(mass[0] - gsum[0], mass[1] - gsum[1], mass[2] - gsum[2], mass[3] - gsum[3]));
    }
};

}  // namespace

template <int PREC, int CONV, int DIFF>
__global__ void __launch_bounds__(256)
k_step_v4(const Params<float> p, const typename VecIO<PREC>::T *__restrict__ src, const float *__restrict__ src_h,
          typename VecIO<PREC>::T *__restrict__ dst, float *__restrict__ dst_h)
{
    using IO = VecIO<PREC>;
    using S = Store<PREC>;
    const int lane = threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (y >= p.ny) return;                       // whole warp: one row per warp
    const int xq = (blockIdx.x * 32 + lane) * 4;
    const bool active = xq < p.nx;
    Lanes L;
    L.x0 = active ? xq : p.nx - 4;
    L.left_mem = lane == 0 || L.x0 == 0;
    L.right_mem = lane == 31 || L.x0 + 4 >= p.nx;
    L.xl = L.x0 == 0 ? p.nx - 1 : L.x0 - 1;
    L.xr = L.x0 + 4 >= p.nx ? 0 : L.x0 + 4;

    int ym = y == 0 ? p.ny - 1 : y - 1;
    int yp = y == p.ny - 1 ? 0 : y + 1;
    LBM_CHK(L.x0, p.nx - 3, p.err, kErrX);
    LBM_CHK(L.xl, p.nx, p.err, kErrX);
    LBM_CHK(L.xr, p.nx, p.err, kErrX);
    LBM_CHK(ym, p.ny, p.err, kErrY);
    LBM_CHK(yp, p.ny, p.err, kErrY);
    const long long r0 = (long long)y * p.pitch, rm = (long long)ym * p.pitch, rp = (long long)yp * p.pitch;
    const long long P = p.plane;

    // BF16S: shift plane of rows y - 1, y, y + 1 at x0 - 1 .. x0 + 4, once per row
    float hm[6], h0[6], hp[6];
    if (PREC == LBM_BF16S) {
        const long long rows[3] = {rm, r0, rp};
        float *hs[3] = {hm, h0, hp};
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            float v[4];
            load4(src_h + rows[r], L.x0, v);
            float left = __shfl_up_sync(kFull, v[3], 1);
            float right = __shfl_down_sync(kFull, v[0], 1);
            if (L.left_mem) left = __ldg(src_h + rows[r] + L.xl);
            if (L.right_mem) right = __ldg(src_h + rows[r] + L.xr);
            hs[r][0] = left;
#pragma unroll
            for (int c = 0; c < 4; ++c) hs[r][c + 1] = v[c];
            hs[r][5] = right;
        }
    }

    float f[4][9];
    {
        float t[4];
#define LBM_PULL(K, CXV, ROW, HV)                                                    \
    IO::template pull<CXV>(src + (K) * P, HV, ROW, L, wgt<float>(K), t);             \
    _Pragma("unroll") for (int c = 0; c < 4; ++c) f[c][K] = t[c];
        LBM_PULL(0, 0, r0, h0)
        LBM_PULL(1, 1, r0, h0)
        LBM_PULL(2, 0, rm, hm)
        LBM_PULL(3, -1, r0, h0)
        LBM_PULL(4, 0, rp, hp)
        LBM_PULL(5, 1, rm, hm)
        LBM_PULL(6, -1, rm, hm)
        LBM_PULL(7, -1, rp, hp)
        LBM_PULL(8, 1, rp, hp)
#undef LBM_PULL
    }

    // anti-bounce-back on the wall nodes of this quad (see kernels_step.cu)
    const bool wall_quad = active && ((p.abb_x && (L.x0 == 0 || L.x0 + 4 >= p.nx)) ||
                                      (p.abb_y && (y == 0 || y == p.ny - 1)));
    if (wall_quad) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int x = L.x0 + c;
            const long long own = r0 + x;
#pragma unroll
            for (int k = 1; k < 9; ++k) {
                const int xs = x - cx(k), ys = y - cy(k);
                const bool ox = p.abb_x && (xs < 0 || xs >= p.nx);
                const bool oy = p.abb_y && (ys < 0 || ys >= p.ny);
                if (ox || oy) {
                    const float wx = xs < 0 ? p.phi_wall[0] : p.phi_wall[1];
                    const float wy = ys < 0 ? p.phi_wall[2] : p.phi_wall[3];
                    const float phiw = (ox && oy) ? 0.5f * (wx + wy) : (ox ? wx : wy);
                    f[c][k] = wall_term<float, CONV, DIFF>(p, k, phiw) -
                              S::ld(src + opp(k) * P, own, src_h, wgt<float>(opp(k)));
                }
            }
        }
    }

    float A3[4], A35[4], A5[4];
    if (p.Afield) {
        float t[4];
        load4(p.Afield + r0, L.x0, t);
#pragma unroll
        for (int c = 0; c < 4; ++c) A3[c] = t[c];
        load4(p.Afield + P + r0, L.x0, t);
#pragma unroll
        for (int c = 0; c < 4; ++c) A35[c] = t[c];
        load4(p.Afield + 2 * P + r0, L.x0, t);
#pragma unroll
        for (int c = 0; c < 4; ++c) A5[c] = t[c];
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) { A3[c] = p.A3; A35[c] = p.A35; A5[c] = p.A5; }
    }

    float phi[4];
    if (p.Afield) {
#pragma unroll
        for (int c = 0; c < 4; ++c) collide<float, CONV, DIFF, true>(p, f[c], A3[c], A35[c], A5[c], phi[c]);
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) collide<float, CONV, DIFF, false>(p, f[c], A3[c], A35[c], A5[c], phi[c]);
    }
    if (active) IO::store(dst, dst_h, P, r0 + L.x0, f, phi);
}

template <int PREC, int CONV, int DIFF>
static cudaError_t step_v4_t(const lbm_solver *s, int src, cudaStream_t st)
{
    using T = typename VecIO<PREC>::T;
    const Params<float> p = make_params<float>(s);
    const int by = s->d.block_rows > 0 ? s->d.block_rows : 8;
    dim3 block(32, by);
    dim3 grid((s->d.nx + 127) / 128, (s->d.ny + by - 1) / by);
    k_step_v4<PREC, CONV, DIFF><<<grid, block, 0, st>>>(p, (const T *)s->pop[src], s->phi[src], (T *)s->pop[src ^ 1],
                                                         s->phi[src ^ 1]);
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t step_v4_p(const lbm_solver *s, int src, cudaStream_t st)
{
    switch (s->c.conv * 3 + s->c.diff) {
    case 0: return step_v4_t<PREC, 0, 0>(s, src, st);
    case 1: return step_v4_t<PREC, 0, 1>(s, src, st);
    case 2: return step_v4_t<PREC, 0, 2>(s, src, st);
    case 3: return step_v4_t<PREC, 1, 0>(s, src, st);
    case 4: return step_v4_t<PREC, 1, 1>(s, src, st);
    case 5: return step_v4_t<PREC, 1, 2>(s, src, st);
    }
    return cudaErrorInvalidValue;
}

bool step_v4_supported(const lbm_solver *s)
{
    return (s->d.prec == LBM_F32 || s->d.prec == LBM_BF16S) && s->d.nx % 4 == 0 && s->d.nx >= 4;
}

// Automatic choice: the four-node kernel where it is measured faster (BF16S,
// whose one-node form is issue-bound); FP32 keeps one node per thread, which
// already runs at the HBM roof with higher occupancy.
bool step_v4_preferred(const lbm_solver *s) { return s->d.prec == LBM_BF16S && step_v4_supported(s); }

cudaError_t launch_step_v4(const lbm_solver *s, int src, cudaStream_t st)
{
    if (s->d.prec == LBM_F32) return step_v4_p<LBM_F32>(s, src, st);
    if (s->d.prec == LBM_BF16S) return step_v4_p<LBM_BF16S>(s, src, st);
    return cudaErrorInvalidValue;
}

}  // namespace lbm
