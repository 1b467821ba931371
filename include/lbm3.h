/*
 * lbm3.h -- C ABI of the three-dimensional (D3Q19) extension of the MRT
 * lattice Boltzmann model for nonlinear anisotropic convection-diffusion
 * equations (Chai, Shi & Guo, arXiv:1603.09577: lattice of Eq. 6, equilibrium
 * of Eq. 3, source of Eq. 9, Scheme B of Eq. 33-35, relaxation block of
 * Eq. 26 in three dimensions).
 *
 * The paper gives no D3Q19 moment matrix. This library uses a moment basis
 * whose rows are mutually orthogonal and include rho = sum_k f_k and
 * j = sum_k c_k f_k; rho relaxes with s0 (immaterial in Scheme B), j with the
 * 3 x 3 block A = (K / (d c_s^2) + I/2)^-1, every other moment with the one
 * rate s_e, so that the collision is
 *     fbar*_k = fbar_k - s_e (fbar_k - feq_k) - c_k . G / 10 + (1 - s_e/2) R_k,
 *     G = (A - s_e I) [(j - B) + B' R / 2],
 * independent of how the other 15 rows are chosen. Lattice units c = 1,
 * c_s^2 = 1/3, d = 1; periodic boundaries or anti-bounce-back Dirichlet walls
 * per axis.
 *
 * Conventions as in lbm.h: int status (LBM_OK or an LBM_E* code, message from
 * lbm_last_error()), caller-owned device workspace (256-byte aligned) and
 * streams (cudaStream_t passed as void*), fields row-major with x fastest:
 * element (x, y, z) at (z * ny + y) * nx + x. The stored state is the
 * post-collision shifted population fbar*(x, t_n).
 */
#ifndef LBM3_H
#define LBM3_H

#include <stddef.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm3_solver *lbm3_handle;

typedef struct {
    int nx, ny, nz;         /* nodes per axis, each >= 2                          */
    int prec;               /* LBM_F64, LBM_F32 or LBM_BF16S (bf16 deviations
                               g_k = fbar*_k - w_k phi plus an FP32 shift plane
                               h = M* - sum_k g_k, float arithmetic, as in lbm.h) */
    int block_rows;         /* rows of 32-thread warps per block: 0 (= 8), 1, 2,
                               4 or 8                                             */
    int bc[3];              /* per axis x, y, z: LBM_PERIODIC or LBM_ABB
                               (anti-bounce-back walls half-way beyond the first
                               and last node, the rule of Sec. 3.6: a link whose
                               source lies beyond a wall takes -fbar*_opp(k) of
                               the node plus feq_k + feq_opp(k) at the wall
                               value; a link crossing two or three walls takes
                               their mean value)                                  */
    double phi_wall[6];     /* wall values: x-, x+, y-, y+, z-, z+               */
} lbm3_desc;

typedef struct {
    int conv;               /* 0: B = u phi, C = u u^T phi; 1: B = a phi^2/2,
                               C = a a^T phi^3/3 (Eq. 7)                          */
    double u[3];            /* u (conv 0) or a (conv 1)                          */
    int diff;               /* D = g(phi) I, g = 0: phi, 1: phi + phi^2/2,
                               2: phi + phi^3/3                                   */
    double K[6];            /* Kxx, Kxy, Kxz, Kyy, Kyz, Kzz: symmetric positive
                               definite; A follows from Eq. 26                    */
    double s0, se;          /* rate of rho (any value in [0, 2)) and of every
                               moment other than rho and j, in (0, 2)            */
    double r0, r1;          /* source R = r0 + r1 phi (|r1| < 2)                  */
} lbm3_coeffs;

/* Bytes of device workspace for this description. LBM_EINVAL for a lattice of
   more than 2^31 nodes, or whose population plane (rows padded to a multiple of
   64 elements) holds more than 2^31 - 1 elements: the kernels index a node
   within a plane in 32-bit arithmetic. A lattice whose 19 planes hold 2^32
   elements or more is addressed through one 64-bit pointer per plane, a
   smaller one through 32-bit offsets from one base pointer (same results). */
int lbm3_workspace_size(const lbm3_desc *desc, size_t *bytes);
/* Create a solver on a caller-owned device workspace (kept until destroy). */
int lbm3_create(lbm3_handle *h, const lbm3_desc *desc, void *dev_workspace, size_t bytes);
int lbm3_destroy(lbm3_handle h);
/* Coefficients; validates the rates and K (host only). */
int lbm3_set_coeffs(lbm3_handle h, const lbm3_coeffs *c);
/* Initial condition (Eq. 40 in the shifted variable of Eq. 33, then one
   collision). dev_phi: nx*ny*nz values of `prec` (LBM_F64 or LBM_F32). */
int lbm3_set_phi(lbm3_handle h, const void *dev_phi, int prec, void *stream);
/* Advance nsteps fused pull-stream / collide steps (asynchronous). The kernels
   alternate between the two population buffers and need no function
   attributes, so a stream capture of an even nsteps replays consistently. */
int lbm3_step(lbm3_handle h, int nsteps, void *stream);
/* Checkpoint / resume: the state is lbm3_state_bytes bytes (the 19 population
   planes and, for LBM_BF16S, the shift plane). dev_dst / dev_src: device
   buffers of that size, owned by the caller. Asynchronous on `stream`.
   lbm3_load also serves as the initial condition (no lbm3_set_phi needed). */
int lbm3_state_bytes(lbm3_handle h, size_t *bytes);
int lbm3_save(lbm3_handle h, void *dev_dst, void *stream);
int lbm3_load(lbm3_handle h, const void *dev_src, void *stream);
/* phi(t_n) into dev_out (nx*ny*nz values of `prec`). */
int lbm3_get_phi(lbm3_handle h, void *dev_out, int prec, void *stream);
/* The eight FP64 statistics of lbm_reduce over phi(t_n) (dev_ref: nx*ny*nz
   doubles or NULL; dev_out: 8 doubles on the device); deterministic. */
int lbm3_reduce(lbm3_handle h, const double *dev_ref, double *dev_out, void *stream);
/* Index-fault word of the bounds-checked build (see lbm_debug_flags): 0 when
   every neighbour coordinate stayed in range since lbm3_set_phi; always 0 in
   the release build. Synchronises `stream`. */
int lbm3_debug_flags(lbm3_handle h, int *flags, void *stream);

#ifdef __cplusplus
}
#endif
#endif
