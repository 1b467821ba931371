// lbm_internal.h -- host-side solver state, workspace layout and the kernel
// launchers shared by the translation units of liblbm.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <atomic>
#include <string>

#include "lbm.h"
#include "lbm_device.cuh"

namespace lbm {

constexpr int kReduceBlocks = 1024;     // fixed: deterministic reduction order
constexpr int kReduceThreads = 256;
constexpr int kPitchAlign = 64;         // row pitch in elements (>= 128 B rows)

struct Layout {
    long long pitch = 0, plane = 0;
    size_t esize = 0, csize = 0;
    size_t off_pop[2] = {0, 0}, off_phi[2] = {0, 0};
    size_t off_afield = 0, off_staging = 0, off_partials = 0, off_flag = 0, off_check = 0, off_err = 0, off_cnt = 0;
    size_t pop_bytes = 0, phi_bytes = 0, total = 0;
};

int make_layout(const lbm_desc *d, Layout *L);

}  // namespace lbm

struct lbm_solver {
    lbm_desc d;
    lbm_coeffs c;
    lbm::Layout L;
    int coeffs_set = 0, phi_set = 0, kfield_set = 0;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    void *pop[2] = {nullptr, nullptr};
    float *phi[2] = {nullptr, nullptr};
    void *afield = nullptr;
    void *staging = nullptr;
    double *partials = nullptr;
    int *flag = nullptr;
    double *check = nullptr;        // 8 doubles: reduction output of lbm_check_finite
    int *err = nullptr;             // index-fault word of checked builds
    int cur = 0;
    long long t = 0;
    // Dirichlet records of the extrapolated axes (caller-owned device memory)
    const double *dir_vals = nullptr;
    int dir_nrec = 0;
    long long *dir_counter = nullptr;   // device: steps since the records' count restarted
    int dir_reset = 0;                  // 1: clear dir_counter before the next step
    int dir_off = 0;                    // place of the next sweep's first step within its lbm_step call
    // adjoint (caller-provided second workspace)
    char *adj = nullptr;
    void *lam[2] = {nullptr, nullptr};
    double *gA = nullptr;
    double *adj_partials = nullptr;
    int adj_cur = 0, adj_active = 0;
};

namespace lbm {

// Per-device record of a kernel's opt-in to more than 48 KB of dynamic shared
// memory. The flags are atomic, so first launches from several host threads do
// not race on them (cudaFuncSetAttribute is idempotent and may then run twice).
// The opt-in happens at the first launch on a device, which must therefore come
// before any stream capture on that device.
struct SmemOptIn {
    std::atomic<int> done[64];
};
cudaError_t opt_in_smem(const void *kernel, int bytes, SmemOptIn &flags);

void set_error(const std::string &msg);
int fail(int code, const std::string &msg);
int cuda_check(cudaError_t e, const char *what);

// kernel parameters in the compute type of the solver
template <class C>
Params<C> make_params(const lbm_solver *s);

// Family key of the step launchers: conv * 3 + diff, or 6 + diff for the linear
// family without a flux (conv 0 with u = 0), which runs the collision without
// the flux terms (kConvNone).
inline int step_key(const lbm_solver *s)
{
    if (s->c.conv == 0 && s->c.u[0] == 0.0 && s->c.u[1] == 0.0 && s->c.diff >= 0 && s->c.diff <= 2)
        return 6 + s->c.diff;
    return s->c.conv * 3 + s->c.diff;
}

// the prescaled rates, source factors and block of the collision (Params),
// from the rates s0..s8 and the block A (computed in double, rounded once)
template <class C>
inline void set_scaled_rates(const double s[9], double A3, double A35, double A5, Params<C> *p)
{
    const double h1 = 1.0 - 0.5 * s[1], h2 = 1.0 - 0.5 * s[2], h4 = 1.0 - 0.5 * s[4], h6 = 1.0 - 0.5 * s[6];
    p->se1 = (C)(s[1] / 36.0); p->se2 = (C)(s[2] / 36.0);
    p->sq4 = (C)(s[4] / 12.0); p->sq6 = (C)(s[6] / 12.0);
    p->sp7 = (C)(s[7] / 4.0); p->sp8 = (C)(s[8] / 4.0);
    p->he1 = (C)(-2.0 * h1 / 36.0); p->he2 = (C)(h2 / 36.0);
    p->hq4 = (C)(-h4 / 12.0); p->hq6 = (C)(-h6 / 12.0);
    p->a3s = (C)(A3 / 6.0); p->a35s = (C)(A35 / 6.0); p->a5s = (C)(A5 / 6.0);
    p->c3s = (C)(1.0 / 6.0 - A3 / 12.0); p->c35s = (C)(-A35 / 12.0); p->c5s = (C)(1.0 / 6.0 - A5 / 12.0);
}

cudaError_t launch_init(const lbm_solver *s, const void *phi, int in_prec, cudaStream_t st);
cudaError_t launch_step(const lbm_solver *s, int src, cudaStream_t st);
cudaError_t launch_step2(const lbm_solver *s, int src, cudaStream_t st);
cudaError_t launch_step2m(const lbm_solver *s, int src, cudaStream_t st);
cudaError_t launch_step2_tma(const lbm_solver *s, int src, cudaStream_t st);
// two steps per pass, two x-adjacent nodes per thread (kernel_variant 5)
cudaError_t launch_step2p_f32(const lbm_solver *s, int src, cudaStream_t st);
cudaError_t launch_step2p_bf16s(const lbm_solver *s, int src, cudaStream_t st);
cudaError_t launch_step_ptr(const lbm_solver *s, const void *src, void *dst, cudaStream_t st);
// general path (Scheme A, extrapolation walls, power-law flux): a step when
// phi0 is null, else the initialisation from phi0
cudaError_t launch_general_f64(const lbm_solver *s, int src, const double *bv, const void *phi0, int in_prec,
                               cudaStream_t st);
cudaError_t launch_general_f32(const lbm_solver *s, int src, const double *bv, const void *phi0, int in_prec,
                               cudaStream_t st);
// two general steps per pass (FP32); records: the caller's Dirichlet records
cudaError_t launch_step2_general(const lbm_solver *s, int src, const double *records, cudaStream_t st);
// advance the device record count by `by` steps (one thread, after a call's sweeps)
cudaError_t launch_tick(long long *counter, int by, cudaStream_t st);
bool step_v4_supported(const lbm_solver *s);
bool step_v4_preferred(const lbm_solver *s);
cudaError_t launch_step_v4(const lbm_solver *s, int src, cudaStream_t st);
cudaError_t launch_get_phi(const lbm_solver *s, void *out, int out_prec, cudaStream_t st);
cudaError_t launch_reduce(const lbm_solver *s, const double *ref, double *out, cudaStream_t st);
cudaError_t launch_kfield(const lbm_solver *s, const double *K, cudaStream_t st);
// the eight deterministic FP64 statistics of a plain FP64 field (partials:
// kReduceBlocks * 8 doubles)
cudaError_t launch_reduce_field(const double *field, long long n, const double *ref, double *partials, double *out,
                                cudaStream_t st);

int adjoint_blocks(const lbm_solver *s);
cudaError_t launch_adjoint_begin(const lbm_solver *s, const void *dphi, int in_prec, void *lam, cudaStream_t st);
cudaError_t launch_adjoint_step(const lbm_solver *s, const void *F, const void *lam_in, void *lam_out, double *gA,
                                double *partials, cudaStream_t st);
cudaError_t launch_adjoint_end(const lbm_solver *s, const void *phi0, int in_prec, const void *lam, const double *gA,
                               double *dphi0, double *dK, double *du, double *partials, cudaStream_t st);

}  // namespace lbm
