// lbm3_d3q19.cu -- the three-dimensional (D3Q19) fused stream-collide step,
// its initialisation and read-out, and the lbm3_* C ABI (include/lbm3.h).
//
// One thread per node, x fastest (warps of 32 along x), a grid of
// (x tiles, y tiles, z). Every step pulls the 19 populations f_k(x) =
// f*_k(x - c_k) with periodic wrap (19 reads and 19 writes per update: 152 B
// in FP32), replaces the links that cross an anti-bounce-back wall at wall
// nodes, then collides in the projector form of the moment reading (see
// lbm3.h): feq of Eq. 3 per direction, the flux block acting on j - B, and the
// Scheme B source.
#include <math.h>
#include <string.h>

#include <new>
#include <string>

#include <cuda_bf16.h>

#include "lbm3.h"
#include "lbm_internal.h"

#include "lbm3_device.cuh"

namespace lbm {

template <int PREC, int CONV, int DIFF, bool WALLS, bool OFF32>
__global__ void __launch_bounds__(256)
k_step3(const Params3<typename St3<PREC>::C> p, const Planes3<typename St3<PREC>::T> pl)
{
    using S = St3<PREC>;
    using T = typename S::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const unsigned own = ((unsigned)z * (unsigned)p.ny + (unsigned)y) * (unsigned)p.pitch + (unsigned)x;
    T f[19];
    pull3_node<PREC, CONV, DIFF, WALLS, OFF32>(p, pl, x, y, z, own, f);
    T phi, mass;
    collide3<CONV, DIFF, T>(p, f, phi, mass);
    store3<PREC, OFF32>(pl, own, f, phi, mass);
}

template <int PREC, int CONV, int DIFF>
__global__ void __launch_bounds__(256)
k_init3(const Params3<typename St3<PREC>::C> p, const void *__restrict__ phi_in, int in_prec,
        const Planes3<typename St3<PREC>::T> pl)
{
    using T = typename St3<PREC>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const long long in = ((long long)z * p.ny + y) * p.nx + x;
    const T phi0 = in_prec == LBM_F64 ? T(((const double *)phi_in)[in]) : T(((const float *)phi_in)[in]);
    // fbar = feq(phi0) - R_k/2 (Eq. 40, 33), then one collision
    T f[19];
    {
        const Coef3<CONV, DIFF, T> q(p, phi0);
#pragma unroll
        for (int k = 0; k < 19; ++k) f[k] = q.feq(k, phi0) - T(0.5) * q.source(k);
    }
    T phi, mass;
    collide3<CONV, DIFF, T>(p, f, phi, mass);
    const unsigned own = ((unsigned)z * (unsigned)p.ny + (unsigned)y) * (unsigned)p.pitch + (unsigned)x;
    store3<PREC, false>(pl, own, f, phi, mass);
}

// phi(t_n) = (sum fbar* - r0/2) / (1 + r1/2) into an FP64 or FP32 field
template <int PREC>
__global__ void __launch_bounds__(256)
k_get_phi3(const Params3<typename St3<PREC>::C> p, const typename St3<PREC>::T *__restrict__ f,
           const float *__restrict__ h, void *__restrict__ out, int out_prec)
{
    using S = St3<PREC>;
    using T = typename S::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const long long own = ((long long)z * p.ny + y) * p.pitch + x;
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 19; ++k) s += S::ld(f + k * p.plane, own, h, own, w3<T>(k));
    const double v = (double)((s - p.half_r0) * p.inv_post);
    const long long o = ((long long)z * p.ny + y) * p.nx + x;
    if (out_prec == LBM_F64) ((double *)out)[o] = v;
    else ((float *)out)[o] = (float)v;
}

}  // namespace lbm

struct lbm3_solver {
    lbm3_desc d;
    lbm3_coeffs c;
    int coeffs_set = 0, phi_set = 0;
    long long pitch = 0, plane = 0;
    size_t esize = 0;
    void *pop[2] = {nullptr, nullptr};
    float *hpl[2] = {nullptr, nullptr};   // BF16S shift planes
    double *staging = nullptr;
    double *partials = nullptr;
    int *err = nullptr;
    int cur = 0;
    size_t state_bytes = 0;               // populations, then the BF16S shift plane (contiguous)
    double G[6] = {0, 0, 0, 0, 0, 0};
};

namespace lbm {
namespace {

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

int check_desc3(const lbm3_desc *d)
{
    if (!d) return fail(LBM_EINVAL, "null lbm3_desc");
    if (d->nx < 2 || d->ny < 2 || d->nz < 2) return fail(LBM_EINVAL, "nx, ny and nz must be >= 2");
    if ((long long)d->nx * d->ny * d->nz > (1LL << 31)) return fail(LBM_EINVAL, "grid larger than 2^31 nodes");
    // node indices within a plane (rows padded to the pitch) are 32-bit
    const long long pitch = ((long long)d->nx + kPitchAlign - 1) / kPitchAlign * kPitchAlign;
    if (pitch * d->ny * d->nz > (1LL << 31) - 1) return fail(LBM_EINVAL, "population plane larger than 2^31 - 1 elements");
    if (d->prec != LBM_F64 && d->prec != LBM_F32 && d->prec != LBM_BF16S)
        return fail(LBM_EINVAL, "D3Q19 storage is LBM_F64, LBM_F32 or LBM_BF16S");
    const int b = d->block_rows;
    if (!(b == 0 || b == 1 || b == 2 || b == 4 || b == 8)) return fail(LBM_EINVAL, "block_rows must be 0, 1, 2, 4 or 8");
    if (d->ny > 65535 * 8 || d->nz > 65535) return fail(LBM_EINVAL, "ny or nz exceeds the launch grid");
    for (int a = 0; a < 3; ++a)
        if (d->bc[a] != LBM_PERIODIC && d->bc[a] != LBM_ABB)
            return fail(LBM_EINVAL, "D3Q19 boundaries are LBM_PERIODIC or LBM_ABB per axis");
    for (int i = 0; i < 6; ++i)
        if (!isfinite(d->phi_wall[i])) return fail(LBM_EINVAL, "non-finite wall value");
    return LBM_OK;
}

struct Layout3 {
    long long pitch, plane;
    size_t esize, pop_bytes, h_bytes, off_stage, off_part, off_err, total;
};

Layout3 layout3(const lbm3_desc *d)
{
    Layout3 L;
    L.pitch = ((long long)d->nx + kPitchAlign - 1) / kPitchAlign * kPitchAlign;
    L.plane = L.pitch * d->ny * d->nz;
    L.esize = d->prec == LBM_F64 ? 8 : (d->prec == LBM_F32 ? 4 : 2);
    L.pop_bytes = up256(19 * (size_t)L.plane * L.esize);
    L.h_bytes = d->prec == LBM_BF16S ? up256((size_t)L.plane * 4) : 0;
    L.off_stage = 2 * (L.pop_bytes + L.h_bytes);
    L.off_part = L.off_stage + up256((size_t)d->nx * d->ny * d->nz * 8);
    L.off_err = L.off_part + up256((size_t)kReduceBlocks * 8 * sizeof(double));
    L.total = L.off_err + 256;
    return L;
}

// Eq. 26 in 3-D: A = (K / (d c_s^2) + I/2)^-1 (Cholesky test of K, adjugate inverse)
bool relax_block3(const double K[6], double A[6])
{
    const double kxx = K[0], kxy = K[1], kxz = K[2], kyy = K[3], kyz = K[4], kzz = K[5];
    const double m1 = kxx, m2 = kxx * kyy - kxy * kxy;
    const double m3 = kxx * (kyy * kzz - kyz * kyz) - kxy * (kxy * kzz - kyz * kxz) + kxz * (kxy * kyz - kyy * kxz);
    if (!(m1 > 0.0 && m2 > 0.0 && m3 > 0.0)) return false;
    const double a = 3 * kxx + 0.5, b = 3 * kxy, c = 3 * kxz, d = 3 * kyy + 0.5, e = 3 * kyz, f = 3 * kzz + 0.5;
    const double det = a * (d * f - e * e) - b * (b * f - e * c) + c * (b * e - d * c);
    A[0] = (d * f - e * e) / det;    // xx
    A[1] = (c * e - b * f) / det;    // xy
    A[2] = (b * e - c * d) / det;    // xz
    A[3] = (a * f - c * c) / det;    // yy
    A[4] = (b * c - a * e) / det;    // yz
    A[5] = (a * d - b * b) / det;    // zz
    return true;
}

template <class T>
Params3<T> params3(const lbm3_solver *s)
{
    Params3<T> p;
    p.nx = s->d.nx; p.ny = s->d.ny; p.nz = s->d.nz;
    p.pitch = s->pitch; p.plane = s->plane;
    p.se = (T)s->c.se;
    p.hse = (T)(1.0 - 0.5 * s->c.se);
    p.omse = (T)(1.0 - s->c.se);
    p.q18 = (T)(0.25 * s->c.se);
    p.q36 = (T)(0.125 * s->c.se);
    for (int i = 0; i < 6; ++i) p.G[i] = (T)(0.1 * s->G[i]);
    const double *u = s->c.u;
    p.ux = (T)u[0]; p.uy = (T)u[1]; p.uz = (T)u[2];
    p.uu[0] = (T)(u[0] * u[0]); p.uu[1] = (T)(u[0] * u[1]); p.uu[2] = (T)(u[0] * u[2]);
    p.uu[3] = (T)(u[1] * u[1]); p.uu[4] = (T)(u[1] * u[2]); p.uu[5] = (T)(u[2] * u[2]);
    p.u2_3 = (T)((u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) / 3.0);
    const double q18 = 0.25 * s->c.se, q36 = 0.125 * s->c.se;
    const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};   // planes xy, xz, yz
    for (int a = 0; a < 3; ++a) {
        p.u6[a] = (T)(u[a] / 6.0);
        p.u12[a] = (T)(u[a] / 12.0);
        p.ea[a] = (T)(q18 * u[a] * u[a]);
        const double sq = u[pa[a]] * u[pa[a]] + u[pb[a]] * u[pb[a]], cr = u[pa[a]] * u[pb[a]];
        p.ep[a] = (T)(q36 * sq + q18 * cr);
        p.em[a] = (T)(q36 * sq - q18 * cr);
    }
    p.r0 = (T)s->c.r0; p.r1 = (T)s->c.r1;
    p.half_r0 = (T)(0.5 * s->c.r0);
    p.inv_den = (T)(1.0 / (1.0 - 0.5 * s->c.r1));
    p.inv_post = (T)(1.0 / (1.0 + 0.5 * s->c.r1));
    p.has_src = s->c.r0 != 0.0 || s->c.r1 != 0.0;
    for (int a = 0; a < 3; ++a) p.abb[a] = s->d.bc[a] == LBM_ABB;
    p.any_abb = p.abb[0] || p.abb[1] || p.abb[2];
    for (int i = 0; i < 6; ++i) p.phi_wall[i] = (T)s->d.phi_wall[i];
    p.err = s->err;
    return p;
}

dim3 block3(const lbm3_solver *s) { return dim3(32, s->d.block_rows > 0 ? s->d.block_rows : 8); }
dim3 grid3(const lbm3_solver *s)
{
    const dim3 b = block3(s);
    return dim3((s->d.nx + 31) / 32, (s->d.ny + b.y - 1) / b.y, s->d.nz);
}

template <class T>
Planes3<T> planes3(const lbm3_solver *s)
{
    Planes3<T> pl;
    const T *src = (const T *)s->pop[s->cur];
    T *dst = (T *)s->pop[s->cur ^ 1];
    for (int k = 0; k < 19; ++k) {
        pl.src[k] = src + k * s->plane;
        pl.dst[k] = dst + k * s->plane;
        pl.poff[k] = (unsigned)(k * s->plane);   // used only when 19 * plane < 2^32
    }
    pl.src0 = src;
    pl.dst0 = dst;
    pl.src_h = s->hpl[s->cur];
    pl.dst_h = s->hpl[s->cur ^ 1];
    return pl;
}

template <int PREC, int CONV, int DIFF>
cudaError_t launch3_t(const lbm3_solver *s, const void *phi0, int in_prec, cudaStream_t st)
{
    using T = typename St3<PREC>::T;
    const auto p = params3<typename St3<PREC>::C>(s);
    if (phi0) {
        // the initial state goes to the current buffer
        Planes3<T> pl = planes3<T>(s);
        for (int k = 0; k < 19; ++k) pl.dst[k] = (T *)pl.src[k];
        pl.dst_h = s->hpl[s->cur];
        k_init3<PREC, CONV, DIFF><<<grid3(s), block3(s), 0, st>>>(p, phi0, in_prec, pl);
    } else {
        const bool off32 = 19 * s->plane < (1LL << 32);
        const Planes3<T> pl = planes3<T>(s);
        if (p.any_abb && off32) k_step3<PREC, CONV, DIFF, true, true><<<grid3(s), block3(s), 0, st>>>(p, pl);
        else if (p.any_abb) k_step3<PREC, CONV, DIFF, true, false><<<grid3(s), block3(s), 0, st>>>(p, pl);
        else if (off32) k_step3<PREC, CONV, DIFF, false, true><<<grid3(s), block3(s), 0, st>>>(p, pl);
        else k_step3<PREC, CONV, DIFF, false, false><<<grid3(s), block3(s), 0, st>>>(p, pl);
    }
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch3_p(const lbm3_solver *s, const void *phi0, int in_prec, cudaStream_t st)
{
    switch (s->c.conv * 3 + s->c.diff) {
    case 0: return launch3_t<PREC, 0, 0>(s, phi0, in_prec, st);
    case 1: return launch3_t<PREC, 0, 1>(s, phi0, in_prec, st);
    case 2: return launch3_t<PREC, 0, 2>(s, phi0, in_prec, st);
    case 3: return launch3_t<PREC, 1, 0>(s, phi0, in_prec, st);
    case 4: return launch3_t<PREC, 1, 1>(s, phi0, in_prec, st);
    case 5: return launch3_t<PREC, 1, 2>(s, phi0, in_prec, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch3(const lbm3_solver *s, const void *phi0, int in_prec, cudaStream_t st)
{
    switch (s->d.prec) {
    case LBM_F64: return launch3_p<LBM_F64>(s, phi0, in_prec, st);
    case LBM_F32: return launch3_p<LBM_F32>(s, phi0, in_prec, st);
    case LBM_BF16S: return launch3_p<LBM_BF16S>(s, phi0, in_prec, st);
    }
    return cudaErrorInvalidValue;
}

template <int PREC>
cudaError_t get_phi3_p(const lbm3_solver *s, void *out, int out_prec, cudaStream_t st)
{
    using T = typename St3<PREC>::T;
    k_get_phi3<PREC><<<grid3(s), block3(s), 0, st>>>(params3<typename St3<PREC>::C>(s), (const T *)s->pop[s->cur],
                                                     s->hpl[s->cur], out, out_prec);
    return cudaGetLastError();
}

cudaError_t get_phi3(const lbm3_solver *s, void *out, int out_prec, cudaStream_t st)
{
    switch (s->d.prec) {
    case LBM_F64: return get_phi3_p<LBM_F64>(s, out, out_prec, st);
    case LBM_F32: return get_phi3_p<LBM_F32>(s, out, out_prec, st);
    case LBM_BF16S: return get_phi3_p<LBM_BF16S>(s, out, out_prec, st);
    }
    return cudaErrorInvalidValue;
}

int ready3(lbm3_handle h)
{
    if (!h) return fail(LBM_EINVAL, "null handle");
    if (!h->coeffs_set) return fail(LBM_EINVAL, "lbm3_set_coeffs has not been called");
    return LBM_OK;
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" {

int lbm3_workspace_size(const lbm3_desc *desc, size_t *bytes)
{
    if (int rc = check_desc3(desc)) return rc;
    if (!bytes) return fail(LBM_EINVAL, "null size pointer");
    *bytes = layout3(desc).total;
    return LBM_OK;
}

int lbm3_create(lbm3_handle *h, const lbm3_desc *desc, void *dev_workspace, size_t bytes)
{
    if (!h) return fail(LBM_EINVAL, "null handle pointer");
    *h = nullptr;
    if (int rc = check_desc3(desc)) return rc;
    const Layout3 L = layout3(desc);
    if (!dev_workspace || ((uintptr_t)dev_workspace & 255) != 0)
        return fail(LBM_EINVAL, "workspace null or not 256-byte aligned");
    if (bytes < L.total) return fail(LBM_EINVAL, "workspace smaller than lbm3_workspace_size");
    lbm3_solver *s = new (std::nothrow) lbm3_solver();
    if (!s) return fail(LBM_EINVAL, "out of host memory");
    char *ws = (char *)dev_workspace;
    s->d = *desc;
    s->pitch = L.pitch;
    s->plane = L.plane;
    s->esize = L.esize;
    s->pop[0] = ws;
    s->pop[1] = ws + L.pop_bytes + L.h_bytes;
    if (L.h_bytes) {
        s->hpl[0] = (float *)(ws + L.pop_bytes);
        s->hpl[1] = (float *)(ws + 2 * L.pop_bytes + L.h_bytes);
    }
    s->staging = (double *)(ws + L.off_stage);
    s->partials = (double *)(ws + L.off_part);
    s->err = (int *)(ws + L.off_err);
    s->state_bytes = L.pop_bytes + L.h_bytes;
    *h = s;
    return LBM_OK;
}

int lbm3_destroy(lbm3_handle h)
{
    delete h;
    return LBM_OK;
}

int lbm3_set_coeffs(lbm3_handle h, const lbm3_coeffs *c)
{
    if (!h) return fail(LBM_EINVAL, "null handle");
    if (!c) return fail(LBM_EINVAL, "null lbm3_coeffs");
    if (c->conv != 0 && c->conv != 1) return fail(LBM_EINVAL, "conv must be 0 or 1");
    if (c->diff < 0 || c->diff > 2) return fail(LBM_EINVAL, "diff must be 0, 1 or 2");
    if (!(c->se > 0.0 && c->se < 2.0)) return fail(LBM_EINVAL, "s_e must lie in (0, 2)");
    if (!(c->s0 >= 0.0 && c->s0 < 2.0)) return fail(LBM_EINVAL, "s0 must lie in [0, 2)");
    for (int i = 0; i < 3; ++i)
        if (!isfinite(c->u[i])) return fail(LBM_EINVAL, "non-finite coefficient");
    if (!isfinite(c->r0) || !isfinite(c->r1) || !(c->r1 > -2.0 && c->r1 < 2.0))
        return fail(LBM_EINVAL, "source coefficients must be finite with |r1| < 2");
    double A[6];
    if (!relax_block3(c->K, A)) return fail(LBM_EINVAL, "K is not symmetric positive definite");
    h->c = *c;
    // G = A - s_e I
    h->G[0] = A[0] - c->se; h->G[1] = A[1]; h->G[2] = A[2];
    h->G[3] = A[3] - c->se; h->G[4] = A[4]; h->G[5] = A[5] - c->se;
    h->coeffs_set = 1;
    return LBM_OK;
}

int lbm3_set_phi(lbm3_handle h, const void *dev_phi, int prec, void *stream)
{
    if (int rc = ready3(h)) return rc;
    if (!dev_phi) return fail(LBM_EINVAL, "null phi");
    if (prec != LBM_F64 && prec != LBM_F32) return fail(LBM_EINVAL, "phi must be LBM_F64 or LBM_F32");
    if (int rc = cuda_check(cudaMemsetAsync(h->err, 0, sizeof(int), (cudaStream_t)stream), "lbm3_set_phi")) return rc;
    if (int rc = cuda_check(launch3(h, dev_phi, prec, (cudaStream_t)stream), "lbm3_set_phi")) return rc;
    h->phi_set = 1;
    return LBM_OK;
}

int lbm3_step(lbm3_handle h, int nsteps, void *stream)
{
    if (int rc = ready3(h)) return rc;
    if (!h->phi_set) return fail(LBM_EINVAL, "lbm3_set_phi has not been called");
    if (nsteps < 0) return fail(LBM_EINVAL, "negative step count");
    for (int i = 0; i < nsteps; ++i) {
        if (int rc = cuda_check(launch3(h, nullptr, 0, (cudaStream_t)stream), "lbm3_step")) return rc;
        h->cur ^= 1;
    }
    return LBM_OK;
}

int lbm3_state_bytes(lbm3_handle h, size_t *bytes)
{
    if (!h) return fail(LBM_EINVAL, "null lbm3 handle");
    if (!bytes) return fail(LBM_EINVAL, "null size pointer");
    *bytes = h->state_bytes;
    return LBM_OK;
}

int lbm3_save(lbm3_handle h, void *dev_dst, void *stream)
{
    if (!h) return fail(LBM_EINVAL, "null lbm3 handle");
    if (!h->phi_set) return fail(LBM_EINVAL, "lbm3_set_phi has not been called");
    if (!dev_dst) return fail(LBM_EINVAL, "null destination");
    return cuda_check(cudaMemcpyAsync(dev_dst, h->pop[h->cur], h->state_bytes, cudaMemcpyDeviceToDevice,
                                      (cudaStream_t)stream), "lbm3_save");
}

int lbm3_load(lbm3_handle h, const void *dev_src, void *stream)
{
    if (!h) return fail(LBM_EINVAL, "null lbm3 handle");
    if (!dev_src) return fail(LBM_EINVAL, "null source");
    if (int rc = cuda_check(cudaMemcpyAsync(h->pop[h->cur], dev_src, h->state_bytes, cudaMemcpyDeviceToDevice,
                                            (cudaStream_t)stream), "lbm3_load"))
        return rc;
    h->phi_set = 1;
    return LBM_OK;
}

int lbm3_get_phi(lbm3_handle h, void *dev_out, int prec, void *stream)
{
    if (int rc = ready3(h)) return rc;
    if (!h->phi_set) return fail(LBM_EINVAL, "lbm3_set_phi has not been called");
    if (!dev_out) return fail(LBM_EINVAL, "null output");
    if (prec != LBM_F64 && prec != LBM_F32) return fail(LBM_EINVAL, "output must be LBM_F64 or LBM_F32");
    return cuda_check(get_phi3(h, dev_out, prec, (cudaStream_t)stream), "lbm3_get_phi");
}

int lbm3_reduce(lbm3_handle h, const double *dev_ref, double *dev_out, void *stream)
{
    if (int rc = ready3(h)) return rc;
    if (!h->phi_set) return fail(LBM_EINVAL, "lbm3_set_phi has not been called");
    if (!dev_out) return fail(LBM_EINVAL, "null output");
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = cuda_check(get_phi3(h, h->staging, LBM_F64, st), "lbm3_reduce")) return rc;
    const long long n = (long long)h->d.nx * h->d.ny * h->d.nz;
    return cuda_check(launch_reduce_field(h->staging, n, dev_ref, h->partials, dev_out, st), "lbm3_reduce");
}

int lbm3_debug_flags(lbm3_handle h, int *flags, void *stream)
{
    if (!h) return fail(LBM_EINVAL, "null handle");
    if (!flags) return fail(LBM_EINVAL, "null flags pointer");
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = cuda_check(cudaMemcpyAsync(flags, h->err, sizeof(int), cudaMemcpyDeviceToHost, st), "lbm3_debug_flags"))
        return rc;
    return cuda_check(cudaStreamSynchronize(st), "lbm3_debug_flags sync");
}

}  // extern "C"
