// lbm_api.cu -- the extern "C" boundary of liblbm: handle life cycle, workspace
// layout, argument validation, coefficient set-up and dispatch to the kernels.
// The library never allocates device memory: every buffer is a slice of the
// caller's workspace.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>

#include "lbm_internal.h"

namespace lbm {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

int cuda_check(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return LBM_OK;
    return fail(LBM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

cudaError_t opt_in_smem(const void *kernel, int bytes, SmemOptIn &flags)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (flags.done[dev].load(std::memory_order_acquire)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) flags.done[dev].store(1, std::memory_order_release);
    return e;
}

static size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

int make_layout(const lbm_desc *d, Layout *L)
{
    L->pitch = ((long long)d->nx + kPitchAlign - 1) / kPitchAlign * kPitchAlign;
    L->plane = L->pitch * d->ny;
    L->esize = d->prec == LBM_F64 ? 8 : (d->prec == LBM_F32 ? 4 : 2);
    L->csize = d->prec == LBM_F64 ? 8 : 4;
    L->pop_bytes = up256(9 * (size_t)L->plane * L->esize);
    // BF16S: the float shift plane; Scheme A: the plane phi(t_n) in the compute type
    L->phi_bytes = d->prec == LBM_BF16S          ? up256((size_t)L->plane * 4)
                   : d->scheme == LBM_SCHEME_A ? up256((size_t)L->plane * L->csize)
                                               : 0;
    size_t off = 0;
    for (int b = 0; b < 2; ++b) {
        L->off_pop[b] = off;
        off += L->pop_bytes;
        L->off_phi[b] = off;
        off += L->phi_bytes;
    }
    L->off_afield = off;
    if (d->per_cell_K) off += up256(3 * (size_t)L->plane * L->csize);
    L->off_staging = off;
    off += up256((size_t)d->nx * d->ny * 8);
    L->off_partials = off;
    off += up256((size_t)kReduceBlocks * 8 * sizeof(double));
    L->off_flag = off;
    off += 256;
    L->off_check = off;
    off += 256;
    L->off_err = off;
    off += 256;
    L->off_cnt = off;
    off += 256;
    L->total = off;
    return LBM_OK;
}

static int check_desc(const lbm_desc *d)
{
    if (!d) return fail(LBM_EINVAL, "null lbm_desc");
    if (d->nx < 2 || d->ny < 2) return fail(LBM_EINVAL, "nx and ny must be >= 2");
    if ((long long)d->nx * d->ny > (1LL << 31)) return fail(LBM_EINVAL, "grid larger than 2^31 nodes");
    if (d->prec != LBM_F64 && d->prec != LBM_F32 && d->prec != LBM_BF16S) return fail(LBM_EINVAL, "unknown precision");
    if (d->bc_x < LBM_PERIODIC || d->bc_x > LBM_NEE || d->bc_y < LBM_PERIODIC || d->bc_y > LBM_NEE)
        return fail(LBM_EINVAL, "unknown boundary kind");
    if (d->scheme != LBM_SCHEME_B && d->scheme != LBM_SCHEME_A) return fail(LBM_EINVAL, "unknown scheme");
    if ((d->bc_x == LBM_NEE && (d->nx < 3 || d->bc_y == LBM_ABB)) || (d->bc_y == LBM_NEE && (d->ny < 3 || d->bc_x == LBM_ABB)))
        return fail(LBM_EINVAL, "extrapolation needs >= 3 nodes on its axis and a periodic or extrapolated other axis");
    if (d->scheme == LBM_SCHEME_A || d->bc_x == LBM_NEE || d->bc_y == LBM_NEE) {
        if (d->prec == LBM_BF16S) return fail(LBM_EUNSUPPORTED, "Scheme A and extrapolation are built for LBM_F64 and LBM_F32");
        if (d->steps_per_pass == 2 && (d->prec != LBM_F32 || d->kernel_variant != 0 || d->per_cell_K))
            return fail(LBM_EUNSUPPORTED,
                        "two steps per pass with Scheme A or extrapolation: LBM_F32, kernel_variant 0, constant K");
        if (d->kernel_variant > 1) return fail(LBM_EUNSUPPORTED, "Scheme A and extrapolation run kernel_variant 0 or 1");
    }
    for (int i = 0; i < 4; ++i)
        if (!isfinite(d->phi_wall[i])) return fail(LBM_EINVAL, "non-finite wall value");
    if (d->steps_per_pass != 1 && d->steps_per_pass != 2) return fail(LBM_EINVAL, "steps_per_pass must be 1 or 2");
    if (d->steps_per_pass == 2 && d->prec == LBM_F64)
        return fail(LBM_EUNSUPPORTED, "two steps per pass is built for LBM_F32 and LBM_BF16S");
    if (d->kernel_variant < 0 || d->kernel_variant > 5) return fail(LBM_EINVAL, "kernel_variant must be 0 to 5");
    if (d->kernel_variant == 5 && (d->steps_per_pass != 2 || d->prec == LBM_F64))
        return fail(LBM_EINVAL, "kernel_variant 5 (pair tiles) needs steps_per_pass 2 and LBM_F32 or LBM_BF16S");
    if (d->kernel_variant == 3 && d->steps_per_pass != 2)
        return fail(LBM_EINVAL, "kernel_variant 3 (column march) needs steps_per_pass 2");
    if (d->kernel_variant == 4 && (d->steps_per_pass != 2 || d->prec != LBM_F32))
        return fail(LBM_EINVAL, "kernel_variant 4 (tensor-copy staging) needs steps_per_pass 2 and LBM_F32");
    if (d->kernel_variant == 2 && !(d->prec != LBM_F64 && d->nx % 4 == 0))
        return fail(LBM_EUNSUPPORTED, "kernel_variant 2 needs LBM_F32 or LBM_BF16S and nx % 4 == 0");
    {
        const int b = d->block_rows;
        if (!(b == 0 || b == 1 || b == 2 || b == 4 || b == 8))
            return fail(LBM_EINVAL, "block_rows must be 0, 1, 2, 4 or 8");
    }
    return LBM_OK;
}

// Eq. 26 solved for the relaxation block: A = (K / (d c_s^2) + I/2)^-1, d = 1.
static bool relax_block(const double K[3], double *A3, double *A35, double *A5)
{
    if (!(K[0] > 0.0) || !(K[0] * K[2] - K[1] * K[1] > 0.0)) return false;
    const double a = 3.0 * K[0] + 0.5, b = 3.0 * K[1], c = 3.0 * K[2] + 0.5;
    const double det = a * c - b * b;
    *A3 = c / det;
    *A35 = -b / det;
    *A5 = a / det;
    return true;
}

template <class C>
Params<C> make_params(const lbm_solver *s)
{
    Params<C> p;
    const lbm_coeffs &c = s->c;
    p.nx = s->d.nx;
    p.ny = s->d.ny;
    p.pitch = s->L.pitch;
    p.plane = s->L.plane;
    p.abb_x = s->d.bc_x == LBM_ABB;
    p.abb_y = s->d.bc_y == LBM_ABB;
    p.s1 = (C)c.s[1]; p.s2 = (C)c.s[2]; p.s4 = (C)c.s[4];
    p.s6 = (C)c.s[6]; p.s7 = (C)c.s[7]; p.s8 = (C)c.s[8];
    p.h1 = (C)(1.0 - 0.5 * c.s[1]); p.h2 = (C)(1.0 - 0.5 * c.s[2]);
    p.h4 = (C)(1.0 - 0.5 * c.s[4]); p.h6 = (C)(1.0 - 0.5 * c.s[6]);
    double A3 = 1, A35 = 0, A5 = 1;
    relax_block(c.K, &A3, &A35, &A5);
    p.A3 = (C)A3; p.A35 = (C)A35; p.A5 = (C)A5;
    set_scaled_rates<C>(c.s, A3, A35, A5, &p);
    p.ux = (C)c.u[0]; p.uy = (C)c.u[1];
    p.uxx = (C)(c.u[0] * c.u[0]); p.uxy = (C)(c.u[0] * c.u[1]); p.uyy = (C)(c.u[1] * c.u[1]);
    p.r0 = (C)c.r0; p.r1 = (C)c.r1;
    p.half_r0 = (C)(0.5 * c.r0);
    p.inv_den = (C)(1.0 / (1.0 - 0.5 * c.r1));
    p.inv_post = (C)(1.0 / (1.0 + 0.5 * c.r1));
    p.has_src = (c.r0 != 0.0 || c.r1 != 0.0);
    for (int i = 0; i < 4; ++i) p.phi_wall[i] = (C)s->d.phi_wall[i];
    p.Afield = s->d.per_cell_K ? (const C *)s->afield : nullptr;
    p.err = s->err;
    p.scheme_a = s->d.scheme == LBM_SCHEME_A;
    p.fisher = c.src_family == 1;
    p.power = c.power > 0 ? c.power : 1;
    p.inv_p1 = (C)(1.0 / (p.power + 1));
    p.inv_p2 = (C)(1.0 / (2 * p.power + 1));
    p.dmxx = (C)c.Dm[0];
    p.dmxy = (C)c.Dm[1];
    p.dmyy = (C)c.Dm[2];
    p.b = (C)c.b;
    p.nee_x = s->d.bc_x == LBM_NEE;
    p.nee_y = s->d.bc_y == LBM_NEE;
    p.bv = nullptr;
    if (p.fisher) p.has_src = 1;
    return p;
}

template Params<float> make_params<float>(const lbm_solver *);
template Params<double> make_params<double>(const lbm_solver *);

// the general kernel serves Scheme A, extrapolation walls and the power-law flux
static bool general_path(const lbm_solver *s)
{
    return s->d.scheme == LBM_SCHEME_A || s->d.bc_x == LBM_NEE || s->d.bc_y == LBM_NEE || s->c.conv >= 2 ||
           s->c.diff == 3;
}

static cudaError_t launch_general(const lbm_solver *s, int src, const double *bv, const void *phi0, int in_prec,
                                  cudaStream_t st)
{
    if (s->d.prec == LBM_F64) return launch_general_f64(s, src, bv, phi0, in_prec, st);
    if (s->d.prec == LBM_F32) return launch_general_f32(s, src, bv, phi0, in_prec, st);
    return cudaErrorInvalidValue;
}

static int check_handle(lbm_handle h)
{
    if (!h) return fail(LBM_EINVAL, "null handle");
    return LBM_OK;
}

static int check_ready(lbm_handle h)
{
    if (check_handle(h)) return LBM_EINVAL;
    if (!h->coeffs_set) return fail(LBM_EINVAL, "lbm_set_coeffs has not been called");
    if (h->d.per_cell_K && !h->kfield_set) return fail(LBM_EINVAL, "lbm_set_K_field has not been called");
    return LBM_OK;
}

}  // namespace lbm

using namespace lbm;

extern "C" {

const char *lbm_last_error(void) { return g_err.c_str(); }

int lbm_workspace_size(const lbm_desc *desc, size_t *bytes)
{
    if (int rc = check_desc(desc)) return rc;
    if (!bytes) return fail(LBM_EINVAL, "null size pointer");
    Layout L;
    make_layout(desc, &L);
    *bytes = L.total;
    return LBM_OK;
}

int lbm_create(lbm_handle *h, const lbm_desc *desc, void *dev_workspace, size_t bytes)
{
    if (!h) return fail(LBM_EINVAL, "null handle pointer");
    *h = nullptr;
    if (int rc = check_desc(desc)) return rc;
    Layout L;
    make_layout(desc, &L);
    if (!dev_workspace) return fail(LBM_EINVAL, "null workspace");
    if (((uintptr_t)dev_workspace & 255) != 0) return fail(LBM_EINVAL, "workspace must be 256-byte aligned");
    if (bytes < L.total) return fail(LBM_EINVAL, "workspace smaller than lbm_workspace_size");
    lbm_solver *s = new (std::nothrow) lbm_solver();
    if (!s) return fail(LBM_EINVAL, "out of host memory");
    s->d = *desc;
    s->L = L;
    s->ws = (char *)dev_workspace;
    s->ws_bytes = bytes;
    for (int b = 0; b < 2; ++b) {
        s->pop[b] = s->ws + L.off_pop[b];
        s->phi[b] = L.phi_bytes ? (float *)(s->ws + L.off_phi[b]) : nullptr;
    }
    s->afield = desc->per_cell_K ? (void *)(s->ws + L.off_afield) : nullptr;
    s->staging = s->ws + L.off_staging;
    s->partials = (double *)(s->ws + L.off_partials);
    s->flag = (int *)(s->ws + L.off_flag);
    s->check = (double *)(s->ws + L.off_check);
    s->err = (int *)(s->ws + L.off_err);
    s->dir_counter = (long long *)(s->ws + L.off_cnt);
    *h = s;
    return LBM_OK;
}

int lbm_destroy(lbm_handle h)
{
    delete h;
    return LBM_OK;
}

int lbm_set_coeffs(lbm_handle h, const lbm_coeffs *c)
{
    if (check_handle(h)) return LBM_EINVAL;
    if (!c) return fail(LBM_EINVAL, "null lbm_coeffs");
    if (c->conv < 0 || c->conv > 3) return fail(LBM_EINVAL, "conv must be 0, 1, 2 or 3");
    if (c->cfree != 0 && c->cfree != 1) return fail(LBM_EINVAL, "cfree must be 0 or 1");
    if (c->cfree && h->d.scheme != LBM_SCHEME_A)
        return fail(LBM_EINVAL, "the C-free variant needs Scheme A (its d_t B uses the phi(t_n) plane)");
    if (c->conv == 3 && !c->cfree) return fail(LBM_EINVAL, "the Buckley-Leverett flux (conv 3) needs cfree = 1");
    if (c->src_family != 0 && c->src_family != 1) return fail(LBM_EINVAL, "src_family must be 0 or 1");
    if ((c->conv == 2 || c->src_family == 1) && (c->power < 1 || c->power > 16))
        return fail(LBM_EINVAL, "power (delta) must be in 1..16");
    if (!isfinite(c->b)) return fail(LBM_EINVAL, "non-finite coefficient");
    if (c->src_family == 1) {
        if (h->d.scheme != LBM_SCHEME_A) return fail(LBM_EINVAL, "the Fisher source needs Scheme A (Eq. 35 has no closed form)");
        if (c->r0 != 0.0 || c->r1 != 0.0) return fail(LBM_EINVAL, "src_family 1 takes b; r0 and r1 must be 0");
    }
    // the general kernels: one step per pass (kernel_variant 0 or 1), or two
    // (FP32, kernel_variant 0, constant K, not the C-free variant)
    const bool general2_ok = h->d.prec == LBM_F32 && h->d.kernel_variant == 0 && !h->d.per_cell_K && !c->cfree &&
                             c->conv <= 2;
    if (c->conv >= 2) {
        if (h->d.prec == LBM_BF16S) return fail(LBM_EUNSUPPORTED, "conv 2 and 3 are built for LBM_F64 and LBM_F32");
        if (h->d.steps_per_pass == 1 ? h->d.kernel_variant > 1 : !general2_ok)
            return fail(LBM_EUNSUPPORTED, "conv 2 and 3: one step per pass with kernel_variant 0 or 1, or conv 2 "
                                          "with two steps per pass (LBM_F32, kernel_variant 0, constant K)");
    }
    if ((c->cfree || c->src_family == 1) && h->d.steps_per_pass == 2 && !general2_ok)
        return fail(LBM_EUNSUPPORTED, "the C-free variant runs one step per pass");
    if (c->diff < 0 || c->diff > 3) return fail(LBM_EINVAL, "diff must be 0, 1, 2 or 3");
    if (c->diff == 3) {
        if (!isfinite(c->Dm[0]) || !isfinite(c->Dm[1]) || !isfinite(c->Dm[2]))
            return fail(LBM_EINVAL, "non-finite diffusion tensor Dm");
        if (h->d.prec == LBM_BF16S) return fail(LBM_EUNSUPPORTED, "diff 3 is built for LBM_F64 and LBM_F32");
        if (h->d.steps_per_pass == 1 ? h->d.kernel_variant > 1 : !general2_ok)
            return fail(LBM_EUNSUPPORTED, "diff 3: one step per pass with kernel_variant 0 or 1, or two steps per "
                                          "pass with LBM_F32, kernel_variant 0 and constant K");
    }
    for (int i = 0; i < 9; ++i) {
        if (i == 3 || i == 5) continue;
        if (!(c->s[i] > 0.0 && c->s[i] < 2.0) && !(i == 0 && c->s[i] == 0.0))
            return fail(LBM_EINVAL, "relaxation rates must lie in (0, 2)");
    }
    if (!isfinite(c->u[0]) || !isfinite(c->u[1]) || !isfinite(c->r0) || !isfinite(c->r1))
        return fail(LBM_EINVAL, "non-finite coefficient");
    if (!(c->r1 < 2.0 && c->r1 > -2.0)) return fail(LBM_EINVAL, "|r1| must be < 2 for Eq. 35 to be solvable");
    if (!h->d.per_cell_K) {
        double a, b, d;
        if (!relax_block(c->K, &a, &b, &d)) return fail(LBM_EINVAL, "K is not symmetric positive definite");
    }
    h->c = *c;
    h->coeffs_set = 1;
    return LBM_OK;
}

int lbm_set_K_field(lbm_handle h, const double *dev_K, void *stream)
{
    if (check_handle(h)) return LBM_EINVAL;
    if (!h->d.per_cell_K) return fail(LBM_EINVAL, "solver was created without per_cell_K");
    if (!dev_K) return fail(LBM_EINVAL, "null tensor field");
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = cuda_check(cudaMemsetAsync(h->flag, 0, sizeof(int), st), "lbm_set_K_field memset")) return rc;
    if (int rc = cuda_check(launch_kfield(h, dev_K, st), "lbm_set_K_field launch")) return rc;
    int bad = 0;
    if (int rc = cuda_check(cudaMemcpyAsync(&bad, h->flag, sizeof(int), cudaMemcpyDeviceToHost, st), "lbm_set_K_field copy"))
        return rc;
    if (int rc = cuda_check(cudaStreamSynchronize(st), "lbm_set_K_field sync")) return rc;
    if (bad) return fail(LBM_EINVAL, std::to_string(bad) + " nodes have a tensor that is not positive definite");
    h->kfield_set = 1;
    return LBM_OK;
}

static bool is_nee(const lbm_solver *h) { return h->d.bc_x == LBM_NEE || h->d.bc_y == LBM_NEE; }

// bytes of a saved state: populations, the phi plane, and for extrapolated
// walls a 256-byte tail holding the device count of the Dirichlet records
static size_t state_size(const lbm_solver *h) { return h->L.pop_bytes + h->L.phi_bytes + (is_nee(h) ? 256 : 0); }

// a pending restart of the record count, issued on `st`
static int flush_record_reset(lbm_solver *h, cudaStream_t st)
{
    if (!h->dir_reset) return LBM_OK;
    if (int rc = cuda_check(cudaMemsetAsync(h->dir_counter, 0, sizeof(long long), st), "Dirichlet record count"))
        return rc;
    h->dir_reset = 0;
    return LBM_OK;
}

int lbm_set_phi(lbm_handle h, const void *dev_phi, int prec, void *stream)
{
    if (int rc = check_ready(h)) return rc;
    if (!dev_phi) return fail(LBM_EINVAL, "null phi");
    if (prec != LBM_F64 && prec != LBM_F32) return fail(LBM_EINVAL, "phi must be LBM_F64 or LBM_F32");
    if (int rc = cuda_check(cudaMemsetAsync(h->err, 0, sizeof(int), (cudaStream_t)stream), "lbm_set_phi")) return rc;
    const cudaError_t e = general_path(h) ? launch_general(h, h->cur, nullptr, dev_phi, prec, (cudaStream_t)stream)
                                          : launch_init(h, dev_phi, prec, (cudaStream_t)stream);
    if (int rc = cuda_check(e, "lbm_set_phi")) return rc;
    if (is_nee(h)) {                     // the Dirichlet records restart with the initial condition
        if (int rc = cuda_check(cudaMemsetAsync(h->dir_counter, 0, sizeof(long long), (cudaStream_t)stream),
                                "lbm_set_phi (records)"))
            return rc;
        h->dir_reset = 0;
    }
    h->phi_set = 1;
    h->t = 0;
    return LBM_OK;
}

int lbm_set_phi_host(lbm_handle h, const void *host_phi, int prec, void *stream)
{
    if (int rc = check_ready(h)) return rc;
    if (!host_phi) return fail(LBM_EINVAL, "null phi");
    if (prec != LBM_F64 && prec != LBM_F32) return fail(LBM_EINVAL, "phi must be LBM_F64 or LBM_F32");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)h->d.nx * h->d.ny * (prec == LBM_F64 ? 8 : 4);
    if (int rc = cuda_check(cudaMemcpyAsync(h->staging, host_phi, n, cudaMemcpyHostToDevice, st), "lbm_set_phi_host copy"))
        return rc;
    return lbm_set_phi(h, h->staging, prec, stream);
}

int lbm_step(lbm_handle h, int nsteps, void *stream)
{
    if (int rc = check_ready(h)) return rc;
    if (!h->phi_set) return fail(LBM_EINVAL, "lbm_set_phi has not been called");
    if (nsteps < 0) return fail(LBM_EINVAL, "negative step count");
    cudaStream_t st = (cudaStream_t)stream;
    int done = 0;
    if (general_path(h)) {
        const bool nee = is_nee(h);
        if (nee && !h->dir_vals) return fail(LBM_EINVAL, "lbm_set_dirichlet has not been called");
        // the kernels pick the record from the device count of steps since the
        // records were set plus the sweep's place in this call (dir_off); one
        // one-thread launch advances the count after the call's sweeps
        const double *records = nee ? h->dir_vals : nullptr;
        if (nee)
            if (int rc = flush_record_reset(h, st)) return rc;
        if (h->d.steps_per_pass == 2) {
            for (; done + 2 <= nsteps; done += 2) {
                h->dir_off = done;
                if (int rc = cuda_check(launch_step2_general(h, h->cur, records, st),
                                        "lbm_step (general, two steps per pass)"))
                    return rc;
                h->cur ^= 1;
                h->t += 2;
            }
        }
        for (; done < nsteps; ++done) {
            h->dir_off = done;
            if (int rc = cuda_check(launch_general(h, h->cur, records, nullptr, 0, st), "lbm_step (general)"))
                return rc;
            h->cur ^= 1;
            h->t += 1;
        }
        h->dir_off = 0;
        if (nee && h->dir_nrec > 1 && nsteps > 0)
            if (int rc = cuda_check(launch_tick(h->dir_counter, nsteps, st), "lbm_step (records)")) return rc;
        return LBM_OK;
    }
    if (h->d.steps_per_pass == 2) {
        for (; done + 2 <= nsteps; done += 2) {
            const cudaError_t e = h->d.kernel_variant == 3   ? launch_step2m(h, h->cur, st)
                                  : h->d.kernel_variant == 4 ? launch_step2_tma(h, h->cur, st)
                                  : h->d.kernel_variant == 5 ? (h->d.prec == LBM_F32 ? launch_step2p_f32(h, h->cur, st)
                                                                                     : launch_step2p_bf16s(h, h->cur, st))
                                                             : launch_step2(h, h->cur, st);
            if (int rc = cuda_check(e, "lbm_step (two steps per pass)")) return rc;
            h->cur ^= 1;
            h->t += 2;
        }
    }
    const bool vec = h->d.kernel_variant == 2 || (h->d.kernel_variant == 0 && step_v4_preferred(h));
    for (; done < nsteps; ++done) {
        if (int rc = cuda_check(vec ? launch_step_v4(h, h->cur, st) : launch_step(h, h->cur, st), "lbm_step")) return rc;
        h->cur ^= 1;
        h->t += 1;
    }
    return LBM_OK;
}

int lbm_set_dirichlet(lbm_handle h, const double *dev_values, int nrec)
{
    if (check_handle(h)) return LBM_EINVAL;
    if (h->d.bc_x != LBM_NEE && h->d.bc_y != LBM_NEE) return fail(LBM_EINVAL, "no axis uses LBM_NEE");
    if (!dev_values || nrec < 1) return fail(LBM_EINVAL, "need a device array of nrec >= 1 records");
    h->dir_vals = dev_values;
    h->dir_nrec = nrec;
    h->dir_reset = 1;                    // record 0 serves the next step (count cleared on its stream)
    return LBM_OK;
}

int lbm_get_phi(lbm_handle h, void *dev_out, int prec, void *stream)
{
    if (int rc = check_ready(h)) return rc;
    if (!h->phi_set) return fail(LBM_EINVAL, "lbm_set_phi has not been called");
    if (!dev_out) return fail(LBM_EINVAL, "null output");
    if (prec != LBM_F64 && prec != LBM_F32) return fail(LBM_EINVAL, "output must be LBM_F64 or LBM_F32");
    return cuda_check(launch_get_phi(h, dev_out, prec, (cudaStream_t)stream), "lbm_get_phi");
}

int lbm_get_phi_host(lbm_handle h, void *host_out, int prec, void *stream)
{
    if (!host_out) return fail(LBM_EINVAL, "null output");
    if (int rc = lbm_get_phi(h, h ? h->staging : nullptr, prec, stream)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)h->d.nx * h->d.ny * (prec == LBM_F64 ? 8 : 4);
    if (int rc = cuda_check(cudaMemcpyAsync(host_out, h->staging, n, cudaMemcpyDeviceToHost, st), "lbm_get_phi_host copy"))
        return rc;
    return cuda_check(cudaStreamSynchronize(st), "lbm_get_phi_host sync");
}

int lbm_reduce(lbm_handle h, const double *dev_ref, double *dev_out, void *stream)
{
    if (int rc = check_ready(h)) return rc;
    if (!h->phi_set) return fail(LBM_EINVAL, "lbm_set_phi has not been called");
    if (!dev_out) return fail(LBM_EINVAL, "null output");
    return cuda_check(launch_reduce(h, dev_ref, dev_out, (cudaStream_t)stream), "lbm_reduce");
}

int lbm_check_finite(lbm_handle h, long long *nonfinite, void *stream)
{
    if (int rc = check_ready(h)) return rc;
    if (!h->phi_set) return fail(LBM_EINVAL, "lbm_set_phi has not been called");
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = cuda_check(launch_reduce(h, nullptr, h->check, st), "lbm_check_finite")) return rc;
    double out[8];
    if (int rc = cuda_check(cudaMemcpyAsync(out, h->check, sizeof(out), cudaMemcpyDeviceToHost, st), "lbm_check_finite copy"))
        return rc;
    if (int rc = cuda_check(cudaStreamSynchronize(st), "lbm_check_finite sync")) return rc;
    const long long bad = (long long)out[6];
    if (nonfinite) *nonfinite = bad;
    if (bad) return fail(LBM_ENONFINITE, std::to_string(bad) + " nodes have a non-finite phi at step " + std::to_string(h->t));
    return LBM_OK;
}

int lbm_debug_flags(lbm_handle h, int *flags, void *stream)
{
    if (check_handle(h)) return LBM_EINVAL;
    if (!flags) return fail(LBM_EINVAL, "null flags pointer");
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = cuda_check(cudaMemcpyAsync(flags, h->err, sizeof(int), cudaMemcpyDeviceToHost, st), "lbm_debug_flags"))
        return rc;
    return cuda_check(cudaStreamSynchronize(st), "lbm_debug_flags sync");
}

int lbm_build_checked(void)
{
#ifdef LBM_CHECKED
    return 1;
#else
    return 0;
#endif
}

int lbm_state_bytes(lbm_handle h, size_t *bytes)
{
    if (check_handle(h)) return LBM_EINVAL;
    if (!bytes) return fail(LBM_EINVAL, "null size pointer");
    *bytes = state_size(h);
    return LBM_OK;
}

int lbm_save(lbm_handle h, void *dev_dst, void *stream)
{
    if (check_handle(h)) return LBM_EINVAL;
    if (!dev_dst) return fail(LBM_EINVAL, "null destination");
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = cuda_check(cudaMemcpyAsync(dev_dst, h->pop[h->cur], h->L.pop_bytes, cudaMemcpyDeviceToDevice, st), "lbm_save"))
        return rc;
    if (h->L.phi_bytes)
        if (int rc = cuda_check(cudaMemcpyAsync((char *)dev_dst + h->L.pop_bytes, h->phi[h->cur], h->L.phi_bytes,
                                                cudaMemcpyDeviceToDevice, st), "lbm_save phi"))
            return rc;
    if (is_nee(h)) {
        if (int rc = flush_record_reset(h, st)) return rc;
        return cuda_check(cudaMemcpyAsync((char *)dev_dst + h->L.pop_bytes + h->L.phi_bytes, h->dir_counter,
                                          sizeof(long long), cudaMemcpyDeviceToDevice, st), "lbm_save records");
    }
    return LBM_OK;
}

int lbm_load(lbm_handle h, const void *dev_src, void *stream)
{
    if (check_handle(h)) return LBM_EINVAL;
    if (!dev_src) return fail(LBM_EINVAL, "null source");
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = cuda_check(cudaMemcpyAsync(h->pop[h->cur], dev_src, h->L.pop_bytes, cudaMemcpyDeviceToDevice, st), "lbm_load"))
        return rc;
    if (h->L.phi_bytes)
        if (int rc = cuda_check(cudaMemcpyAsync(h->phi[h->cur], (const char *)dev_src + h->L.pop_bytes, h->L.phi_bytes,
                                                cudaMemcpyDeviceToDevice, st), "lbm_load phi"))
            return rc;
    if (is_nee(h)) {
        if (int rc = cuda_check(cudaMemcpyAsync(h->dir_counter, (const char *)dev_src + h->L.pop_bytes + h->L.phi_bytes,
                                                sizeof(long long), cudaMemcpyDeviceToDevice, st), "lbm_load records"))
            return rc;
        h->dir_reset = 0;
    }
    h->phi_set = 1;
    return LBM_OK;
}

// ---- adjoint -----------------------------------------------------------------

static int adjoint_supported(lbm_handle h)
{
    if (check_ready(h)) return LBM_EINVAL;
    if (h->d.prec == LBM_BF16S) return fail(LBM_EUNSUPPORTED, "the adjoint is built for LBM_F64 and LBM_F32");
    if (h->d.bc_x != LBM_PERIODIC || h->d.bc_y != LBM_PERIODIC)
        return fail(LBM_EUNSUPPORTED, "the adjoint is built for periodic boundaries");
    if (h->c.conv != 0 || h->c.diff != 0 || h->c.r0 != 0.0 || h->c.r1 != 0.0 || h->c.src_family != 0 || h->c.cfree)
        return fail(LBM_EUNSUPPORTED, "the adjoint is built for the linear family (conv 0, diff 0) without source");
    if (h->d.scheme != LBM_SCHEME_B) return fail(LBM_EUNSUPPORTED, "the adjoint is built for Scheme B");
    return LBM_OK;
}

static size_t adj_lam_bytes(lbm_handle h) { return up256(9 * (size_t)h->L.plane * h->L.csize); }

int lbm_adjoint_workspace_size(lbm_handle h, size_t *bytes)
{
    if (int rc = adjoint_supported(h)) return rc;
    if (!bytes) return fail(LBM_EINVAL, "null size pointer");
    *bytes = 2 * adj_lam_bytes(h) + up256(3 * (size_t)h->L.plane * 8) + up256((size_t)adjoint_blocks(h) * 2 * 8);
    return LBM_OK;
}

int lbm_adjoint_begin(lbm_handle h, void *dev_ws, size_t bytes, const void *dev_dphiN, int prec, void *stream)
{
    if (int rc = adjoint_supported(h)) return rc;
    size_t need = 0;
    lbm_adjoint_workspace_size(h, &need);
    if (!dev_ws || ((uintptr_t)dev_ws & 255) != 0) return fail(LBM_EINVAL, "adjoint workspace null or not 256-byte aligned");
    if (bytes < need) return fail(LBM_EINVAL, "adjoint workspace smaller than lbm_adjoint_workspace_size");
    if (!dev_dphiN) return fail(LBM_EINVAL, "null dL/dphi");
    if (prec != LBM_F64 && prec != LBM_F32) return fail(LBM_EINVAL, "dL/dphi must be LBM_F64 or LBM_F32");
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)dev_ws;
    const size_t lb = adj_lam_bytes(h), gb = up256(3 * (size_t)h->L.plane * 8);
    h->adj = w;
    h->lam[0] = w;
    h->lam[1] = w + lb;
    h->gA = (double *)(w + 2 * lb);
    h->adj_partials = (double *)(w + 2 * lb + gb);
    h->adj_cur = 0;
    if (int rc = cuda_check(cudaMemsetAsync(h->gA, 0, gb + up256((size_t)adjoint_blocks(h) * 16), st), "lbm_adjoint_begin"))
        return rc;
    if (int rc = cuda_check(launch_adjoint_begin(h, dev_dphiN, prec, h->lam[0], st), "lbm_adjoint_begin")) return rc;
    h->adj_active = 1;
    return LBM_OK;
}

int lbm_adjoint_step(lbm_handle h, const void *dev_state_n, void *stream)
{
    if (int rc = adjoint_supported(h)) return rc;
    if (!h->adj_active) return fail(LBM_EINVAL, "lbm_adjoint_begin has not been called");
    if (!dev_state_n) return fail(LBM_EINVAL, "null forward state");
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = cuda_check(launch_adjoint_step(h, dev_state_n, h->lam[h->adj_cur], h->lam[h->adj_cur ^ 1], h->gA,
                                                h->adj_partials, st), "lbm_adjoint_step"))
        return rc;
    h->adj_cur ^= 1;
    return LBM_OK;
}

int lbm_adjoint_segment(lbm_handle h, const void *dev_ckpt, int nsteps, void *dev_states, size_t bytes, void *stream)
{
    if (int rc = adjoint_supported(h)) return rc;
    if (!h->adj_active) return fail(LBM_EINVAL, "lbm_adjoint_begin has not been called");
    if (!dev_ckpt) return fail(LBM_EINVAL, "null checkpoint");
    if (nsteps < 1) return fail(LBM_EINVAL, "segment length must be >= 1");
    const size_t sb = state_size(h);
    if (nsteps > 1 && (!dev_states || bytes < (size_t)(nsteps - 1) * sb))
        return fail(LBM_EINVAL, "state scratch smaller than (nsteps - 1) * lbm_state_bytes");
    cudaStream_t st = (cudaStream_t)stream;
    auto state = [&](int j) -> const void * { return j == 0 ? dev_ckpt : (const char *)dev_states + (size_t)(j - 1) * sb; };
    // recompute F_{t0+1} .. F_{t0+nsteps-1} from the checkpoint
    for (int j = 1; j < nsteps; ++j)
        if (int rc = cuda_check(launch_step_ptr(h, state(j - 1), (void *)state(j), st), "lbm_adjoint_segment recompute"))
            return rc;
    // reverse steps over the segment, last state first
    for (int j = nsteps - 1; j >= 0; --j) {
        if (int rc = cuda_check(launch_adjoint_step(h, state(j), h->lam[h->adj_cur], h->lam[h->adj_cur ^ 1], h->gA,
                                                    h->adj_partials, st), "lbm_adjoint_segment reverse step"))
            return rc;
        h->adj_cur ^= 1;
    }
    return LBM_OK;
}

int lbm_adjoint_end(lbm_handle h, const void *dev_phi0, int prec, double *dev_dphi0, double *dev_dK, double *dev_du,
                    void *stream)
{
    if (int rc = adjoint_supported(h)) return rc;
    if (!h->adj_active) return fail(LBM_EINVAL, "lbm_adjoint_begin has not been called");
    if (!dev_phi0 || !dev_dphi0 || !dev_dK || !dev_du) return fail(LBM_EINVAL, "null argument");
    if (prec != LBM_F64 && prec != LBM_F32) return fail(LBM_EINVAL, "phi0 must be LBM_F64 or LBM_F32");
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = cuda_check(launch_adjoint_end(h, dev_phi0, prec, h->lam[h->adj_cur], h->gA, dev_dphi0, dev_dK, dev_du,
                                               h->adj_partials, st), "lbm_adjoint_end"))
        return rc;
    h->adj_active = 0;
    return LBM_OK;
}

}  // extern "C"
