// kernels_adjoint.cu -- discrete adjoint of the fused stream-collide step for the
// linear family (B = u phi, C = u u^T phi, D = phi I, no source, periodic walls)
// with a per-node or constant diffusion tensor.
//
// Forward, per step: G = pull(F_n), F_{n+1} = collide(G). The collision is
// F = G + M0^-1 dm with dm = -S (M0 G - E phi), phi = 1^T G, E = m_eq per unit
// phi (Eq. 16), so its Jacobian is J = I - M0^-1 S (I - E e0^T) M0 (Eq. 17-19).
// One reverse step maps Lambda_{n+1} = dL/dF_{n+1} to Lambda_n = dL/dF_n:
//   mu    = M0^-T Lambda = diag(1/|row_i|^2) M0 Lambda
//   sigma = S^T mu                              (sigma_0 = 0: rho is not relaxed)
//   nu    = J^T Lambda = Lambda + M0^-1 dm',  dm'_i = -|row_i|^2 sigma_i (i >= 1),
//                                             dm'_0 = 9 E^T sigma
//   Lambda_n,k(x - c_k) = nu_k(x)            (adjoint of the pull: a push)
// and the parameter gradients of the step, accumulated in FP64:
//   dL/dA_ij += -mu_i (m - m_eq)_j, i, j in {3, 5} (block A of Eq. 17, 21)
//   dL/du    += sum_i sigma_i d m_eq,i / du   (m_eq of Eq. 16)
// The last reverse step ends at F_0 = feq(phi0) (Eq. 40): dL/dphi0 = sum_k a_k
// Lambda_0,k with a = feq per unit phi, and dL/du += mu^T d m_eq/du at phi0.
// Finally A = (K / (d c_s^2) + I/2)^-1 (Eq. 26) gives dL/dK = -A G A / (d c_s^2).
#include "lbm_internal.h"

namespace lbm {

constexpr int kAdjBX = 32, kAdjBY = 8;

// E = m_eq per unit phi for the linear family (Eq. 16, c = 1, g = phi)
template <class C>
struct LinEq {
    C E1, E2, E7, E8;        // e, eps, pxx, pxy entries (E0 = 1, E3 = ux, E4 = -ux, E5 = uy, E6 = -uy)
    __device__ __forceinline__ explicit LinEq(const Params<C> &p)
    {
        const C C2 = p.uxx + p.uyy + C(2) / C(3);
        E1 = C(3) * C2 - C(4);
        E2 = C(3) - C(3) * C2;
        E7 = p.uxx - p.uyy;
        E8 = p.uxy;
    }
};

template <class C>
__device__ __forceinline__ void moments(const C f[9], C m[9])
{
    const C ax = f[1] + f[3], ay = f[2] + f[4];
    const C axis = ax + ay;
    const C dg = (f[5] + f[7]) + (f[6] + f[8]);
    m[0] = f[0] + axis + dg;
    m[1] = C(2) * dg - axis - C(4) * f[0];
    m[2] = C(4) * f[0] - C(2) * axis + dg;
    const C dx1 = f[1] - f[3], dy1 = f[2] - f[4];
    const C dxd = (f[5] - f[7]) + (f[8] - f[6]);
    const C dyd = (f[5] - f[7]) + (f[6] - f[8]);
    m[3] = dx1 + dxd;
    m[4] = dxd - C(2) * dx1;
    m[5] = dy1 + dyd;
    m[6] = dyd - C(2) * dy1;
    m[7] = ax - ay;
    m[8] = (f[5] + f[7]) - (f[6] + f[8]);
}

// f += M0^-1 dm
template <class C>
__device__ __forceinline__ void add_inverse(const C dm[9], C f[9])
{
    const C r = dm[0] * (C(1) / C(9));
    const C ee = dm[1] * (C(1) / C(36)), pp = dm[2] * (C(1) / C(36));
    const C jxn = dm[3] * (C(1) / C(6)), qxn = dm[4] * (C(1) / C(12));
    const C jyn = dm[5] * (C(1) / C(6)), qyn = dm[6] * (C(1) / C(12));
    const C pxxn = dm[7] * C(0.25), pxyn = dm[8] * C(0.25);
    f[0] += r - C(4) * ee + C(4) * pp;
    const C base_a = r - ee - C(2) * pp;
    const C X1 = jxn - C(2) * qxn, Y1 = jyn - C(2) * qyn;
    f[1] += base_a + X1 + pxxn;
    f[3] += base_a - X1 + pxxn;
    f[2] += base_a + Y1 - pxxn;
    f[4] += base_a - Y1 - pxxn;
    const C base_d = r + C(2) * ee + pp;
    const C X2 = jxn + qxn, Y2 = jyn + qyn;
    f[5] += base_d + X2 + Y2 + pxyn;
    f[6] += base_d - X2 + Y2 - pxyn;
    f[7] += base_d - X2 - Y2 + pxyn;
    f[8] += base_d + X2 - Y2 - pxyn;
}

// fixed-order block sum of two values, added in FP64 to partial[0..1]
template <class C>
__device__ __forceinline__ void block_add2(C a, C b, double *partial)
{
    __shared__ C sh[kAdjBX * kAdjBY / 32][2];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
    }
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = t & 31, w = t >> 5;
    if (lane == 0) { sh[w][0] = a; sh[w][1] = b; }
    __syncthreads();
    if (t == 0) {
        C sa = sh[0][0], sb = sh[0][1];
        for (int q = 1; q < (int)(blockDim.x * blockDim.y) / 32; ++q) { sa += sh[q][0]; sb += sh[q][1]; }
        partial[0] += (double)sa;
        partial[1] += (double)sb;
    }
}

template <class C>
__global__ void __launch_bounds__(kAdjBX * kAdjBY)
k_adjoint_step(const Params<C> p, const C *__restrict__ F, const C *__restrict__ lam_in, C *__restrict__ lam_out,
               double *__restrict__ gA, double *__restrict__ partials)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const bool in = x < p.nx && y < p.ny;
    C dux = C(0), duy = C(0);
    if (in) {
        int xm = x == 0 ? p.nx - 1 : x - 1, xp = x == p.nx - 1 ? 0 : x + 1;
        int ym = y == 0 ? p.ny - 1 : y - 1, yp = y == p.ny - 1 ? 0 : y + 1;
        LBM_CHK(xm, p.nx, p.err, kErrX);
        LBM_CHK(xp, p.nx, p.err, kErrX);
        LBM_CHK(ym, p.ny, p.err, kErrY);
        LBM_CHK(yp, p.ny, p.err, kErrY);
        const long long r0 = (long long)y * p.pitch, rm = (long long)ym * p.pitch, rp = (long long)yp * p.pitch;
        const long long own = r0 + x, P = p.plane;
        C G[9], L[9];
        G[0] = __ldg(F + own);
        G[1] = __ldg(F + 1 * P + r0 + xm);
        G[2] = __ldg(F + 2 * P + rm + x);
        G[3] = __ldg(F + 3 * P + r0 + xp);
        G[4] = __ldg(F + 4 * P + rp + x);
        G[5] = __ldg(F + 5 * P + rm + xm);
        G[6] = __ldg(F + 6 * P + rm + xp);
        G[7] = __ldg(F + 7 * P + rp + xp);
        G[8] = __ldg(F + 8 * P + rp + xm);
#pragma unroll
        for (int k = 0; k < 9; ++k) L[k] = __ldg(lam_in + k * P + own);
        C A3 = p.A3, A35 = p.A35, A5 = p.A5;
        if (p.Afield) {
            A3 = __ldg(p.Afield + own);
            A35 = __ldg(p.Afield + P + own);
            A5 = __ldg(p.Afield + 2 * P + own);
        }
        const LinEq<C> E(p);
        C mL[9], m[9];
        moments(L, mL);
        moments(G, m);
        // mu = M0^-T Lambda, sigma = S^T mu (S symmetric in the (3, 5) block)
        const C mu3 = mL[3] * (C(1) / C(6)), mu5 = mL[5] * (C(1) / C(6));
        C sg[9];
        sg[0] = C(0);
        sg[1] = p.s1 * mL[1] * (C(1) / C(36));
        sg[2] = p.s2 * mL[2] * (C(1) / C(36));
        sg[3] = A3 * mu3 + A35 * mu5;
        sg[4] = p.s4 * mL[4] * (C(1) / C(12));
        sg[5] = A35 * mu3 + A5 * mu5;
        sg[6] = p.s6 * mL[6] * (C(1) / C(12));
        sg[7] = p.s7 * mL[7] * C(0.25);
        sg[8] = p.s8 * mL[8] * C(0.25);
        C dm[9];
        dm[0] = C(9) * (E.E1 * sg[1] + E.E2 * sg[2] + p.ux * (sg[3] - sg[4]) + p.uy * (sg[5] - sg[6]) +
                        E.E7 * sg[7] + E.E8 * sg[8]);
        dm[1] = C(-36) * sg[1];
        dm[2] = C(-36) * sg[2];
        dm[3] = C(-6) * sg[3];
        dm[4] = C(-12) * sg[4];
        dm[5] = C(-6) * sg[5];
        dm[6] = C(-12) * sg[6];
        dm[7] = C(-4) * sg[7];
        dm[8] = C(-4) * sg[8];
        add_inverse(dm, L);
        // adjoint of the pull: Lambda_n,k(x - c_k) = nu_k(x)
        lam_out[own] = L[0];
        lam_out[1 * P + r0 + xm] = L[1];
        lam_out[2 * P + rm + x] = L[2];
        lam_out[3 * P + r0 + xp] = L[3];
        lam_out[4 * P + rp + x] = L[4];
        lam_out[5 * P + rm + xm] = L[5];
        lam_out[6 * P + rm + xp] = L[6];
        lam_out[7 * P + rp + xp] = L[7];
        lam_out[8 * P + rp + xm] = L[8];
        // parameter gradients of this step: products in the compute type, the
        // running sums over steps in FP64
        const C phi = m[0];
        const C d3 = m[3] - p.ux * phi, d5 = m[5] - p.uy * phi;
        gA[own] -= (double)(mu3 * d3);
        gA[P + own] -= (double)(mu3 * d5 + mu5 * d3);
        gA[2 * P + own] -= (double)(mu5 * d5);
        dux = phi * (C(6) * p.ux * (sg[1] - sg[2]) + sg[3] - sg[4] + C(2) * p.ux * sg[7] + p.uy * sg[8]);
        duy = phi * (C(6) * p.uy * (sg[1] - sg[2]) + sg[5] - sg[6] - C(2) * p.uy * sg[7] + p.ux * sg[8]);
    }
    block_add2(dux, duy, partials + 2 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x));
}

// Lambda_N = dL/dphi_N on every population (phi = sum_k F_k)
template <class C>
__global__ void k_adjoint_begin(const Params<C> p, const void *__restrict__ dphi, int in_prec, C *__restrict__ lam)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const long long i = (long long)y * p.nx + x, own = (long long)y * p.pitch + x;
    const C g = in_prec == LBM_F64 ? (C)((const double *)dphi)[i] : (C)((const float *)dphi)[i];
#pragma unroll
    for (int k = 0; k < 9; ++k) lam[k * p.plane + own] = g;
}

// dL/dphi0, dL/dK per node and the u-gradient of the initial equilibrium
template <class C>
__global__ void __launch_bounds__(kAdjBX * kAdjBY)
k_adjoint_end(const Params<C> p, const void *__restrict__ phi0, int in_prec, const C *__restrict__ lam,
              const double *__restrict__ gA, double *__restrict__ dphi0, double *__restrict__ dK,
              double *__restrict__ partials)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const bool in = x < p.nx && y < p.ny;
    double dux = 0.0, duy = 0.0;
    if (in) {
        const long long i = (long long)y * p.nx + x, own = (long long)y * p.pitch + x, P = p.plane;
        const long long n = (long long)p.nx * p.ny;
        const double ph = in_prec == LBM_F64 ? ((const double *)phi0)[i] : (double)((const float *)phi0)[i];
        double L[9], mL[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) L[k] = (double)lam[k * P + own];
        moments(L, mL);
        // a_k = feq_k per unit phi (Eq. 3, linear family): dL/dphi0 = sum a_k Lambda_k = E^T mu
        const double ux = p.ux, uy = p.uy;
        const double C2 = ux * ux + uy * uy + 2.0 / 3.0;
        const double mu[9] = {mL[0] / 9.0, mL[1] / 36.0, mL[2] / 36.0, mL[3] / 6.0, mL[4] / 12.0,
                              mL[5] / 6.0, mL[6] / 12.0, mL[7] / 4.0, mL[8] / 4.0};
        dphi0[i] = mu[0] + (3.0 * C2 - 4.0) * mu[1] + (3.0 - 3.0 * C2) * mu[2] + ux * (mu[3] - mu[4]) +
                   uy * (mu[5] - mu[6]) + (ux * ux - uy * uy) * mu[7] + ux * uy * mu[8];
        dux = ph * (6.0 * ux * (mu[1] - mu[2]) + mu[3] - mu[4] + 2.0 * ux * mu[7] + uy * mu[8]);
        duy = ph * (6.0 * uy * (mu[1] - mu[2]) + mu[5] - mu[6] - 2.0 * uy * mu[7] + ux * mu[8]);
        // dL/dK = -A Gs A / (d c_s^2), Gs = [[G33, G35/2], [G35/2, G55]], with the
        // relaxation block the forward steps used
        double A00 = p.A3, A01 = p.A35, A11 = p.A5;
        if (p.Afield) { A00 = p.Afield[own]; A01 = p.Afield[P + own]; A11 = p.Afield[2 * P + own]; }
        const double G00 = gA[own], G01 = 0.5 * gA[P + own], G11 = gA[2 * P + own];
        const double T00 = A00 * G00 + A01 * G01, T01 = A00 * G01 + A01 * G11;
        const double T10 = A01 * G00 + A11 * G01, T11 = A01 * G01 + A11 * G11;
        const double H00 = -3.0 * (T00 * A00 + T01 * A01), H01 = -3.0 * (T00 * A01 + T01 * A11);
        const double H10 = -3.0 * (T10 * A00 + T11 * A01), H11 = -3.0 * (T10 * A01 + T11 * A11);
        dK[i] = H00;
        dK[n + i] = H01 + H10;
        dK[2 * n + i] = H11;
    }
    block_add2(dux, duy, partials + 2 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x));
}

// sum of the per-block u-gradient partials in block order
__global__ void k_adjoint_du(const double *__restrict__ partials, int nb, double *__restrict__ du)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < nb; ++q) { a += partials[2 * q]; b += partials[2 * q + 1]; }
        du[0] = a;
        du[1] = b;
    }
}

static dim3 adj_grid(const lbm_solver *s) { return dim3((s->d.nx + kAdjBX - 1) / kAdjBX, (s->d.ny + kAdjBY - 1) / kAdjBY); }

int adjoint_blocks(const lbm_solver *s)
{
    const dim3 g = adj_grid(s);
    return (int)(g.x * g.y);
}

cudaError_t launch_adjoint_begin(const lbm_solver *s, const void *dphi, int in_prec, void *lam, cudaStream_t st)
{
    dim3 block(kAdjBX, kAdjBY), grid = adj_grid(s);
    if (s->d.prec == LBM_F64)
        k_adjoint_begin<double><<<grid, block, 0, st>>>(make_params<double>(s), dphi, in_prec, (double *)lam);
    else
        k_adjoint_begin<float><<<grid, block, 0, st>>>(make_params<float>(s), dphi, in_prec, (float *)lam);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_step(const lbm_solver *s, const void *F, const void *lam_in, void *lam_out, double *gA,
                                double *partials, cudaStream_t st)
{
    dim3 block(kAdjBX, kAdjBY), grid = adj_grid(s);
    if (s->d.prec == LBM_F64)
        k_adjoint_step<double><<<grid, block, 0, st>>>(make_params<double>(s), (const double *)F, (const double *)lam_in,
                                                       (double *)lam_out, gA, partials);
    else
        k_adjoint_step<float><<<grid, block, 0, st>>>(make_params<float>(s), (const float *)F, (const float *)lam_in,
                                                      (float *)lam_out, gA, partials);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_end(const lbm_solver *s, const void *phi0, int in_prec, const void *lam, const double *gA,
                               double *dphi0, double *dK, double *du, double *partials, cudaStream_t st)
{
    dim3 block(kAdjBX, kAdjBY), grid = adj_grid(s);
    if (s->d.prec == LBM_F64)
        k_adjoint_end<double><<<grid, block, 0, st>>>(make_params<double>(s), phi0, in_prec, (const double *)lam, gA,
                                                      dphi0, dK, partials);
    else
        k_adjoint_end<float><<<grid, block, 0, st>>>(make_params<float>(s), phi0, in_prec, (const float *)lam, gA,
                                                     dphi0, dK, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_adjoint_du<<<1, 32, 0, st>>>(partials, adjoint_blocks(s), du);
    return cudaGetLastError();
}

}  // namespace lbm
