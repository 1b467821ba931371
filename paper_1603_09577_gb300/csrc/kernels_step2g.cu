// kernels_step2g.cu -- two time steps per sweep through HBM for the general
// path (FP32): Scheme A (Remark II) or B, the power-law flux (Eq. 49-50), the
// tensor diffusion function of Eq. 62, affine or Fisher sources (Eq. 46), and
// periodic, anti-bounce-back or non-equilibrium-extrapolation walls.
//
// The tile scheme is that of the two-step tile kernel: a block owns a 30 x 30
// output tile, step A recomputes the state after the first step on the 32 x 32
// region (tile plus one-node halo) into shared memory, step B pulls from there.
// Scheme A also keeps phi(t_{n+1}) of the region in shared memory (the previous
// level of step B's backward difference). An extrapolated Dirichlet node pulls
// its inward neighbour: from global memory in step A, from the region in step B.
// On an extrapolated axis the last tile is shifted to end at the last node
// (overlapping its neighbour, whose shared outputs it writes with identical
// values), so that the inward neighbour of every output node and that
// neighbour's own sources lie inside the region.
#include "kernels_general.cuh"
#include "kernels_step2.cuh"

namespace lbm {

namespace {

constexpr int kRPg = Tile2<30>::kRP;              // 32 x 32 region

__device__ __forceinline__ Params<F2> widen_g(const Params<float> &p)
{
    Params<F2> w = widen(p);
    w.scheme_a = p.scheme_a;
    w.fisher = p.fisher;
    w.power = p.power;
    w.inv_p1 = p.inv_p1;
    w.inv_p2 = p.inv_p2;
    w.b = p.b;
    w.dmxx = p.dmxx;
    w.dmxy = p.dmxy;
    w.dmyy = p.dmyy;
    w.nee_x = p.nee_x;
    w.nee_y = p.nee_y;
    w.bv = nullptr;
    return w;
}

__device__ __forceinline__ int tile_origin(int b, int n, int nee)
{
    const int t0 = b * kTX;
    return (nee && n >= kTX && t0 > n - kTX) ? n - kTX : t0;
}

// The caller's Dirichlet records and the place of this sweep's first step
// (kernel parameters; the record is looked up where a Dirichlet node needs it,
// so no pointer stays live in registers across the sweep)
struct Records {
    const double *base;
    const long long *cnt;
    int nrec, off;
};

// Dirichlet value of an extrapolated node at the level `lvl` (0: step A,
// 1: step B) from its record (west, east, south, north)
__device__ __forceinline__ float dirichlet(const Params<float> &p, const Records &r, int lvl, bool ex, int x, int y)
{
    const double *bv = record_of(r.base, r.cnt, r.nrec, 2 * (p.nx + p.ny), r.off + lvl);
    return (float)(ex ? bv[x == 0 ? y : p.ny + y] : bv[2 * p.ny + (y == 0 ? x : p.nx + x)]);
}

template <int CONV, int DIFF, bool SA>
__device__ __forceinline__ void collide_pair_g(const Params<F2> &pw, float f[2][9], const float prev[2], float phi[2])
{
    F2 g[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) g[k] = F2(f[0][k], f[1][k]);
    F2 ph;
    if (SA) collide_a<F2, CONV, DIFF>(pw, g, pw.A3, pw.A35, pw.A5, F2(prev[0], prev[1]), ph);
    else collide<F2, CONV, DIFF, false>(pw, g, pw.A3, pw.A35, pw.A5, ph);
#pragma unroll
    for (int k = 0; k < 9; ++k) { f[0][k] = g[k].v.x; f[1][k] = g[k].v.y; }
    phi[0] = ph.v.x;
    phi[1] = ph.v.y;
}

// Step A input of one region node: the pulled populations (extrapolated on a
// Dirichlet node) and phi(t_n); false for a node outside the domain.
template <int CONV, int DIFF, bool SA, bool INTERIOR>
__device__ __forceinline__ bool node_A(const Params<float> &p, const float *__restrict__ src,
                                       const float *__restrict__ src_phi, const Records &rec, int x, int y, float f[9],
                                       float &prev)
{
    if (INTERIOR) {
        pull_global<LBM_F32, CONV, DIFF, true>(p, src, nullptr, x, y, f);
        prev = SA ? src_phi[(unsigned)y * (unsigned)p.pitch + x] : 0.0f;
        return true;
    }
    bool valid = true;
    if (x < 0 || x >= p.nx) {
        if (p.abb_x || p.nee_x) valid = false;
        else x = x < 0 ? x + p.nx : x - p.nx;
    }
    if (y < 0 || y >= p.ny) {
        if (p.abb_y || p.nee_y) valid = false;
        else y = y < 0 ? y + p.ny : y - p.ny;
    }
    if (x < 0 || x >= p.nx || y < 0 || y >= p.ny) valid = false;
    if (!valid) { x = 0; y = 0; }                  // any in-domain node; result unused
    const bool ex = p.nee_x && (x == 0 || x == p.nx - 1);
    const bool ey = p.nee_y && (y == 0 || y == p.ny - 1);
    if (valid && (ex || ey)) {
        const int xf = ex ? (x == 0 ? 1 : p.nx - 2) : x;
        const int yf = ey ? (y == 0 ? 1 : p.ny - 2) : y;
        pull_global<LBM_F32, CONV, DIFF, false>(p, src, nullptr, xf, yf, f);
        float sum = f[0];
#pragma unroll
        for (int k = 1; k < 9; ++k) sum += f[k];
        const float phif = SA ? sum : (sum + p.half_r0) * p.inv_den;
        float eb[9], ef[9];
        feq_stored<float, CONV, DIFF, SA>(p, dirichlet(p, rec, 0, ex, x, y), eb);
        feq_stored<float, CONV, DIFF, SA>(p, phif, ef);
#pragma unroll
        for (int k = 0; k < 9; ++k) f[k] = eb[k] + (f[k] - ef[k]);
    } else {
        pull_global<LBM_F32, CONV, DIFF, false>(p, src, nullptr, x, y, f);
    }
    int xx = x, yy = y;
    LBM_CHK(xx, p.nx, p.err, kErrX);
    LBM_CHK(yy, p.ny, p.err, kErrY);
    prev = SA ? src_phi[(unsigned)yy * (unsigned)p.pitch + xx] : 0.0f;
    return valid;
}

template <int CONV, int DIFF, bool SA, bool INTERIOR>
__device__ __forceinline__ void two_steps_g(const Params<float> &p, const float *__restrict__ src,
                                            const float *__restrict__ src_phi, float *__restrict__ dst,
                                            float *__restrict__ dst_phi, const Records &rec,
                                            float *sm, int tx0, int ty0)
{
    constexpr int kWarps = kT2Threads / 32;
    const Params<F2> pw = widen_g(p);
    float *smphi = sm + 9 * kRPg;
    const int lane = threadIdx.x, warp = threadIdx.y;
    const long long P = p.plane;

    // ---- step A: region rows hy0 + 8 h, two rows per pass
#pragma unroll 1
    for (int hy0 = warp; hy0 < 32; hy0 += 2 * kWarps) {
        float f[2][9], prev[2], phi[2];
        bool ok[2];
#pragma unroll
        for (int h = 0; h < 2; ++h)
            ok[h] = node_A<CONV, DIFF, SA, INTERIOR>(p, src, src_phi, rec, tx0 - 1 + lane, ty0 - 1 + hy0 + h * kWarps,
                                                     f[h], prev[h]);
        collide_pair_g<CONV, DIFF, SA>(pw, f, prev, phi);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (INTERIOR || ok[h]) {
                const int c = (hy0 + h * kWarps) * kRX + lane;
#pragma unroll
                for (int k = 0; k < 9; ++k) sm[k * kRPg + c] = f[h][k];
                if (SA) smphi[c] = phi[h];
            }
        }
    }
    __syncthreads();

    // ---- step B: output rows in pairs (r, r + 8); lanes 0..29
    const int x = tx0 + lane;
    if (lane < kTX && x < p.nx) {
#pragma unroll 1
        for (int r0 = warp; r0 < 30; r0 += 2 * kWarps) {
            float f[2][9], prev[2], phi[2];
            bool ok[2];
            unsigned own[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = r0 + h * kWarps;
                const int y = ty0 + r;
                ok[h] = r < 30 && (INTERIOR || y < p.ny);
                const int rr = ok[h] ? r : r0;                   // a valid row; result unused
                int c0 = rr * kRX + lane;
                LBM_CHK(c0, kRPg - 2 * kRX - 1, p.err, kErrShared);
                const int c = c0 + kRX + 1;
                const int yy = ok[h] ? y : ty0;
                const bool ex = !INTERIOR && p.nee_x && (x == 0 || x == p.nx - 1);
                const bool ey = !INTERIOR && p.nee_y && (yy == 0 || yy == p.ny - 1);
                if (ex || ey) {
                    // extrapolation from the inward neighbour, pulled from the region
                    const int dx = ex ? (x == 0 ? 1 : -1) : 0, dy = ey ? (yy == 0 ? 1 : -1) : 0;
                    int cf = c + dy * kRX + dx;
                    LBM_CHK(cf, kRPg - kRX - 1, p.err, kErrShared);
                    if (cf < kRX + 1) cf = kRX + 1;                // keeps every read in bounds
                    float sum = 0.0f;
#pragma unroll
                    for (int k = 0; k < 9; ++k) {
                        f[h][k] = sm[k * kRPg + cf - cy(k) * kRX - cx(k)];
                        sum += f[h][k];
                    }
                    const float phif = SA ? sum : (sum + p.half_r0) * p.inv_den;
                    float eb[9], ef[9];
                    feq_stored<float, CONV, DIFF, SA>(p, dirichlet(p, rec, 1, ex, x, yy), eb);
                    feq_stored<float, CONV, DIFF, SA>(p, phif, ef);
#pragma unroll
                    for (int k = 0; k < 9; ++k) f[h][k] = eb[k] + (f[h][k] - ef[k]);
                } else {
#pragma unroll
                    for (int k = 0; k < 9; ++k) f[h][k] = sm[k * kRPg + c - cy(k) * kRX - cx(k)];
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
                                    f[h][k] = wall_term<float, CONV, DIFF>(p, k, phiw) - sm[opp(k) * kRPg + c];
                                }
                            }
                        }
                    }
                }
                prev[h] = SA ? smphi[c] : 0.0f;
                int xx = x, yc = yy;
                LBM_CHK(xx, p.nx, p.err, kErrX);
                LBM_CHK(yc, p.ny, p.err, kErrY);
                own[h] = (unsigned)yc * (unsigned)p.pitch + xx;
            }
            collide_pair_g<CONV, DIFF, SA>(pw, f, prev, phi);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (ok[h]) {
#pragma unroll
                    for (int k = 0; k < 9; ++k) __stcs(dst + k * P + own[h], f[h][k]);
                    if (SA) dst_phi[own[h]] = phi[h];
                }
            }
        }
    }
}

}  // namespace

template <int CONV, int DIFF, bool SA>
__global__ void __launch_bounds__(kT2Threads, 4)
k_step2g(const Params<float> p, const float *__restrict__ src, const float *__restrict__ src_phi,
         float *__restrict__ dst, float *__restrict__ dst_phi, const double *records, const long long *rec_cnt,
         int nrec, int rec_off)
{
    extern __shared__ float sm[];       // 9 planes (+ phi for Scheme A) of 32 x 32
    const Records rec{records, rec_cnt, nrec, rec_off};
    const int tx0 = tile_origin(blockIdx.x, p.nx, p.nee_x), ty0 = tile_origin(blockIdx.y, p.ny, p.nee_y);
    // interior tile: no wrap, wall or Dirichlet node in the region or its sources
    const bool interior = tx0 >= 2 && tx0 + kTX + 1 <= p.nx - 1 && ty0 >= 2 && ty0 + 30 + 1 <= p.ny - 1;
    if (interior) two_steps_g<CONV, DIFF, SA, true>(p, src, src_phi, dst, dst_phi, rec, sm, tx0, ty0);
    else two_steps_g<CONV, DIFF, SA, false>(p, src, src_phi, dst, dst_phi, rec, sm, tx0, ty0);
}

namespace {

template <int CONV, int DIFF, bool SA>
cudaError_t step2g_t(const lbm_solver *s, int src, const double *records, cudaStream_t st)
{
    const size_t smem = (9 + (SA ? 1 : 0)) * kRPg * sizeof(float);
    Params<float> p = make_params<float>(s);
    dim3 block(32, kT2Threads / 32);
    dim3 grid((s->d.nx + kTX - 1) / kTX, (s->d.ny + 29) / 30);
    k_step2g<CONV, DIFF, SA><<<grid, block, smem, st>>>(p, (const float *)s->pop[src], s->phi[src],
                                                        (float *)s->pop[src ^ 1], s->phi[src ^ 1], records,
                                                        s->dir_counter, s->dir_nrec, s->dir_off);
    return cudaGetLastError();
}

template <bool SA>
cudaError_t step2g_s(const lbm_solver *s, int src, const double *records, cudaStream_t st)
{
#define LBM_G2(CV, DF) \
    case CV * 4 + DF: return step2g_t<CV, DF, SA>(s, src, records, st);
    switch (s->c.conv * 4 + s->c.diff) {
        LBM_G2(0, 0)
        LBM_G2(0, 1)
        LBM_G2(0, 2)
        LBM_G2(0, 3)
        LBM_G2(1, 0)
        LBM_G2(1, 1)
        LBM_G2(1, 2)
        LBM_G2(1, 3)
        LBM_G2(2, 0)
        LBM_G2(2, 1)
        LBM_G2(2, 2)
        LBM_G2(2, 3)
    }
#undef LBM_G2
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_step2_general(const lbm_solver *s, int src, const double *records, cudaStream_t st)
{
    if (s->d.prec != LBM_F32 || s->c.cfree || s->c.conv > 2 || s->d.per_cell_K) return cudaErrorInvalidValue;
    return s->d.scheme == LBM_SCHEME_A ? step2g_s<true>(s, src, records, st) : step2g_s<false>(s, src, records, st);
}

}  // namespace lbm
