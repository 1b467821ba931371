// kernels_aux.cu -- initialisation (Eq. 40), phi read-out (Eq. 35), the per-cell
// relaxation blocks of a tensor field (Eq. 26) and the deterministic FP64
// reductions (Eq. 39 and norms).
#include "lbm_internal.h"

namespace lbm {

// ---- initialisation: fbar = feq(phi0) - R_k/2 (Eq. 40, 33), then one collision
template <int PREC, int CONV, int DIFF>
__global__ void __launch_bounds__(256)
k_init(const Params<typename Store<PREC>::C> p, const void *__restrict__ phi_in, int in_prec,
       typename Store<PREC>::T *__restrict__ dst, float *__restrict__ dst_phi)
{
    using S = Store<PREC>;
    using C = typename S::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const long long in = (long long)y * p.nx + x;
    const C phi0 = in_prec == LBM_F64 ? C(((const double *)phi_in)[in]) : C(((const float *)phi_in)[in]);
    C f[9], Rk[9];
    equilibrium<C, CONV, DIFF>(p, phi0, f);
    if (p.has_src) {
        source_pop<C, CONV, DIFF>(p, phi0, p.r0 + p.r1 * phi0, Rk);
#pragma unroll
        for (int k = 0; k < 9; ++k) f[k] -= C(0.5) * Rk[k];
    }
    const long long own = (long long)y * p.pitch + x;
    C A3 = p.A3, A35 = p.A35, A5 = p.A5;
    if (p.Afield) {
        A3 = p.Afield[own];
        A35 = p.Afield[p.plane + own];
        A5 = p.Afield[2 * p.plane + own];
    }
    C phi;
    collide<C, CONV, DIFF>(p, f, A3, A35, A5, phi);
    S::store_cell(dst, dst_phi, p.plane, own, f, phi);
}

template <int PREC, int CONV, int DIFF>
static cudaError_t init_t(const lbm_solver *s, const void *phi, int in_prec, cudaStream_t st)
{
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;
    const Params<C> p = make_params<C>(s);
    dim3 block(32, 8), grid((s->d.nx + 31) / 32, (s->d.ny + 7) / 8);
    k_init<PREC, CONV, DIFF><<<grid, block, 0, st>>>(p, phi, in_prec, (T *)s->pop[s->cur], s->phi[s->cur]);
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t init_p(const lbm_solver *s, const void *phi, int in_prec, cudaStream_t st)
{
    switch (s->c.conv * 3 + s->c.diff) {
    case 0: return init_t<PREC, 0, 0>(s, phi, in_prec, st);
    case 1: return init_t<PREC, 0, 1>(s, phi, in_prec, st);
    case 2: return init_t<PREC, 0, 2>(s, phi, in_prec, st);
    case 3: return init_t<PREC, 1, 0>(s, phi, in_prec, st);
    case 4: return init_t<PREC, 1, 1>(s, phi, in_prec, st);
    case 5: return init_t<PREC, 1, 2>(s, phi, in_prec, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_init(const lbm_solver *s, const void *phi, int in_prec, cudaStream_t st)
{
    switch (s->d.prec) {
    case LBM_F64: return init_p<LBM_F64>(s, phi, in_prec, st);
    case LBM_F32: return init_p<LBM_F32>(s, phi, in_prec, st);
    case LBM_BF16S: return init_p<LBM_BF16S>(s, phi, in_prec, st);
    }
    return cudaErrorInvalidValue;
}

// ---- phi(t_n) of the stored post-collision state ---------------------------
// The collision raises the zeroth moment by R/2 (Eq. 34-35): sum fbar* = phi + R/2,
// so phi = (sum fbar* - r0/2) / (1 + r1/2).
template <int PREC>
__device__ __forceinline__ double node_phi(const Params<typename Store<PREC>::C> &p,
                                           const typename Store<PREC>::T *__restrict__ f,
                                           const float *__restrict__ phiplane, long long own)
{
    using S = Store<PREC>;
    using C = typename S::C;
    if (!S::kPhiPlane && p.scheme_a) return (double)((const C *)phiplane)[own];   // Scheme A keeps phi(t_n)
    C sum = S::ld(f, own, phiplane, wgt<C>(0));
#pragma unroll
    for (int k = 1; k < 9; ++k) sum += S::ld(f + k * p.plane, own, phiplane, wgt<C>(k));
    return (double)((sum - p.half_r0) * p.inv_post);
}

template <int PREC>
__global__ void __launch_bounds__(256)
k_get_phi(const Params<typename Store<PREC>::C> p, const typename Store<PREC>::T *__restrict__ f,
          const float *__restrict__ phiplane, void *__restrict__ out, int out_prec)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const double v = node_phi<PREC>(p, f, phiplane, (long long)y * p.pitch + x);
    const long long o = (long long)y * p.nx + x;
    if (out_prec == LBM_F64) ((double *)out)[o] = v;
    else ((float *)out)[o] = (float)v;
}

template <int PREC>
static cudaError_t get_phi_p(const lbm_solver *s, void *out, int out_prec, cudaStream_t st)
{
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;
    const Params<C> p = make_params<C>(s);
    dim3 block(32, 8), grid((s->d.nx + 31) / 32, (s->d.ny + 7) / 8);
    k_get_phi<PREC><<<grid, block, 0, st>>>(p, (const T *)s->pop[s->cur], s->phi[s->cur], out, out_prec);
    return cudaGetLastError();
}

cudaError_t launch_get_phi(const lbm_solver *s, void *out, int out_prec, cudaStream_t st)
{
    switch (s->d.prec) {
    case LBM_F64: return get_phi_p<LBM_F64>(s, out, out_prec, st);
    case LBM_F32: return get_phi_p<LBM_F32>(s, out, out_prec, st);
    case LBM_BF16S: return get_phi_p<LBM_BF16S>(s, out, out_prec, st);
    }
    return cudaErrorInvalidValue;
}

// ---- per-cell relaxation blocks from a tensor field (Eq. 26) -----------------
// A = (K / (d c_s^2) + I/2)^-1 per node; a node whose K is not positive definite
// raises *flag and gets the block A = I so the state stays finite.
template <class C>
__global__ void k_kfield(int nx, int ny, long long pitch, long long plane, const double *__restrict__ K,
                         C *__restrict__ A, int *__restrict__ flag)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const long long n = (long long)nx * ny, i = (long long)y * nx + x, o = (long long)y * pitch + x;
    const double a = 3.0 * K[i] + 0.5, b = 3.0 * K[n + i], c = 3.0 * K[2 * n + i] + 0.5;
    double det = a * c - b * b;
    double A3 = c / det, A35 = -b / det, A5 = a / det;
    if (!(K[i] > 0.0) || !(K[i] * K[2 * n + i] - K[n + i] * K[n + i] > 0.0) || !(det > 0.0)) {
        atomicAdd(flag, 1);
        A3 = 1.0; A35 = 0.0; A5 = 1.0;
    }
    A[o] = (C)A3;
    A[plane + o] = (C)A35;
    A[2 * plane + o] = (C)A5;
}

cudaError_t launch_kfield(const lbm_solver *s, const double *K, cudaStream_t st)
{
    dim3 block(32, 8), grid((s->d.nx + 31) / 32, (s->d.ny + 7) / 8);
    if (s->d.prec == LBM_F64)
        k_kfield<double><<<grid, block, 0, st>>>(s->d.nx, s->d.ny, s->L.pitch, s->L.plane, K, (double *)s->afield, s->flag);
    else
        k_kfield<float><<<grid, block, 0, st>>>(s->d.nx, s->d.ny, s->L.pitch, s->L.plane, K, (float *)s->afield, s->flag);
    return cudaGetLastError();
}

// ---- deterministic FP64 reductions ---------------------------------------------
// Pass 1: a fixed grid of kReduceBlocks blocks; each thread accumulates a fixed
// grid-stride subset, then a fixed-order warp-shuffle and shared-memory tree.
// Pass 2: one block combines the per-block partials in index order.
constexpr int kNacc = 8;

__device__ __forceinline__ void warp_reduce(double v[kNacc])
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int j = 0; j < kNacc; ++j) {
            const double o = __shfl_down_sync(0xffffffffu, v[j], off);
            v[j] = j == 5 ? fmax(v[j], o) : v[j] + o;
        }
}

__device__ __forceinline__ void block_reduce(double v[kNacc], double *out)
{
    __shared__ double sh[kReduceThreads / 32][kNacc];
    warp_reduce(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < kNacc; ++j) sh[w][j] = v[j];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 0; j < kNacc; ++j) {
            double a = sh[0][j];
            for (int q = 1; q < kReduceThreads / 32; ++q) a = j == 5 ? fmax(a, sh[q][j]) : a + sh[q][j];
            out[j] = a;
        }
    }
}

template <int PREC>
__global__ void __launch_bounds__(kReduceThreads)
k_reduce1(const Params<typename Store<PREC>::C> p, const typename Store<PREC>::T *__restrict__ f,
          const float *__restrict__ phiplane, const double *__restrict__ ref, double *__restrict__ partials)
{
    double v[kNacc] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long n = (long long)p.nx * p.ny;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / p.nx), x = (int)(i - (long long)y * p.nx);
        const double ph = node_phi<PREC>(p, f, phiplane, (long long)y * p.pitch + x);
        if (!isfinite(ph)) { v[6] += 1.0; continue; }
        v[0] += ph;
        v[7] += ph * ph;
        v[5] = fmax(v[5], fabs(ph));
        if (ref) {
            const double r = ref[i], d = ph - r;
            v[1] += fabs(d);
            v[2] += fabs(r);
            v[3] += d * d;
            v[4] += r * r;
        }
    }
    block_reduce(v, partials + (size_t)blockIdx.x * kNacc);
}

__global__ void __launch_bounds__(kReduceThreads) k_reduce2(const double *__restrict__ partials, int nb, double *__restrict__ out)
{
    double v[kNacc] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
        for (int j = 0; j < kNacc; ++j) {
            const double a = partials[(size_t)b * kNacc + j];
            v[j] = j == 5 ? fmax(v[j], a) : v[j] + a;
        }
    block_reduce(v, out);
}

// the same statistics over a plain FP64 field (the D3Q19 solver's phi)
__global__ void __launch_bounds__(kReduceThreads)
k_reduce_field1(const double *__restrict__ field, long long n, const double *__restrict__ ref,
                double *__restrict__ partials)
{
    double v[kNacc] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double ph = field[i];
        if (!isfinite(ph)) { v[6] += 1.0; continue; }
        v[0] += ph;
        v[7] += ph * ph;
        v[5] = fmax(v[5], fabs(ph));
        if (ref) {
            const double r = ref[i], d = ph - r;
            v[1] += fabs(d);
            v[2] += fabs(r);
            v[3] += d * d;
            v[4] += r * r;
        }
    }
    block_reduce(v, partials + (size_t)blockIdx.x * kNacc);
}

cudaError_t launch_reduce_field(const double *field, long long n, const double *ref, double *partials, double *out,
                                cudaStream_t st)
{
    k_reduce_field1<<<kReduceBlocks, kReduceThreads, 0, st>>>(field, n, ref, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce2<<<1, kReduceThreads, 0, st>>>(partials, kReduceBlocks, out);
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t reduce_p(const lbm_solver *s, const double *ref, double *out, cudaStream_t st)
{
    using S = Store<PREC>;
    using T = typename S::T;
    using C = typename S::C;
    const Params<C> p = make_params<C>(s);
    k_reduce1<PREC><<<kReduceBlocks, kReduceThreads, 0, st>>>(p, (const T *)s->pop[s->cur], s->phi[s->cur], ref, s->partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce2<<<1, kReduceThreads, 0, st>>>(s->partials, kReduceBlocks, out);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const lbm_solver *s, const double *ref, double *out, cudaStream_t st)
{
    switch (s->d.prec) {
    case LBM_F64: return reduce_p<LBM_F64>(s, ref, out, st);
    case LBM_F32: return reduce_p<LBM_F32>(s, ref, out, st);
    case LBM_BF16S: return reduce_p<LBM_BF16S>(s, ref, out, st);
    }
    return cudaErrorInvalidValue;
}

// ---- Dirichlet record count -----------------------------------------------------
__global__ void k_tick(long long *counter, int by) { *counter += by; }

cudaError_t launch_tick(long long *counter, int by, cudaStream_t st)
{
    k_tick<<<1, 1, 0, st>>>(counter, by);
    return cudaGetLastError();
}

}  // namespace lbm
