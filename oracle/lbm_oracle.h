/*
 * lbm_oracle.h -- plain FP64 CPU oracle of the D2Q9 multiple-relaxation-time
 * lattice Boltzmann model for nonlinear anisotropic convection-diffusion
 * equations (Chai, Shi & Guo, arXiv:1603.09577, Sec. 2).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library. It shares no code, header,
 * table or helper with the CUDA library; the product path never calls it.
 *
 * Units: lattice units, c = dx/dt = 1, c_s^2 = 1/3, d = 1 (Sec. 3 default).
 * Storage: populations are structure-of-arrays, f[(k*ny + y)*nx + x].
 * The stored state after every call is the post-collision population
 * fbar*(x, t_n) of Scheme B (Eq. 33-34).
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Problem description (Eq. 1 with the closed coefficient families used here). */
typedef struct {
    int nx, ny;
    int bc_x, bc_y;         /* 0: periodic, 1: anti-bounce-back Dirichlet wall    */
    double phi_wall[4];     /* wall values: west, east, south, north              */
    int conv;               /* 0: B = u phi, C = u u phi; 1: B = a phi^2/2,
                               C = a a phi^3/3 (Eq. 7); 2: power law (Eq. 49-50);
                               3: Buckley-Leverett B = (u_x f, u_y g) of Eq. 54
                               (C-free variant only)                              */
    double u[2];            /* u (conv 0) or a (conv 1)                           */
    int diff;               /* D = g(phi) I with g = 0: phi, 1: phi + phi^2/2,
                               2: phi + phi^3/3; 3: D = Dm phi, a constant
                               symmetric tensor (the isotropic form of Eq. 62,
                               D = K phi / kappa; general path only)              */
    double K[3];            /* constant diffusion tensor Kxx, Kxy, Kyy            */
    const double *Kfield;   /* optional per-cell tensor, 3 planes of nx*ny
                               (Kxx, Kxy, Kyy); overrides K when not NULL         */
    double s[9];            /* s0..s8 of Eq. 17; s3, s5, s35 come from K (Eq. 26) */
    double r0, r1;          /* affine source R = r0 + r1 phi (Eq. 35 solved)      */
    int src;                /* explicit source: 0 none, 1 Eq. 43, 2 Eq. 66        */
    double src_par[8];      /* x0, y0, dx, dt, kappa, ux, uy (physical units)     */
    int collision;          /* 0: moment form, 1: P-form, 2: single-rate BGK loop */
    /* Scheme A, the power-law flux, the Fisher source and the non-equilibrium
       extrapolation boundary (bc_x / bc_y = 2); used by the *_x functions.    */
    int scheme;             /* 0: Scheme B (Eq. 33-35); 1: Scheme A (gamma = 0,
                               Remark II: Btilde = (I - A/2) B', dt R_k by a
                               backward difference)                               */
    int power;              /* delta >= 1 of conv 2, B = a phi^(delta+1)/(delta+1),
                               C = a a phi^(2 delta+1)/(2 delta+1) (Eq. 49-50),
                               and of the Fisher source                           */
    int src_family;         /* 0: R = r0 + r1 phi; 1: R = b phi (1 - phi^delta)
                               (Eq. 46; Scheme A only)                            */
    double b;               /* Fisher source coefficient                          */
    double Dm[3];           /* Dm_xx, Dm_xy, Dm_yy of diff 3                      */
    int cfree;              /* 1: Remark III variant (Scheme A only): C = 0 in the
                               equilibrium (Eq. 38) and the extra source G_k of
                               Eq. 37 with d_t B by a backward difference          */
} oracle_problem;

/* Status: 0 ok, nonzero invalid argument. */
int oracle_num_threads(void);

/* Equilibrium populations (Eq. 3) for one value of phi. */
int oracle_feq(const oracle_problem *p, double phi, double feq[9]);
/* Discrete source populations (Eq. 9, Scheme B: Btilde = B'). */
int oracle_source_pop(const oracle_problem *p, double phi, double R, double Rk[9]);
/* Relaxation block A = [[s3, s35], [s53, s5]] from K (Eq. 26 solved for A). */
int oracle_relax_block(const double K[3], double A[4]);
/* One collision of one cell with a given tensor K; returns phi in *phi_out. */
int oracle_collide_cell(const oracle_problem *p, const double K[3], const double f[9],
                        double Rexp, double fout[9], double *phi_out);
/* P = M0^-1 S M0 and Q = M0^-1 (I - S/2) M0 for one cell (row-major 9x9). */
int oracle_pform_matrices(const oracle_problem *p, const double K[3], double P[81], double Q[81]);

/* Initial state (Eq. 40 in the shifted variable of Eq. 33, then one collision). */
int oracle_init(const oracle_problem *p, const double *phi0, double *F);
/* One time step n -> n+1: pull streaming with boundaries, then collision.
   phi_out (nullable) receives phi(t_{n+1}) computed from the streamed state. */
int oracle_step(const oracle_problem *p, const double *F_in, double *F_out, int n, double *phi_out);
/* phi(t_n) from a stored post-collision state (inverts the collision's mass gain). */
int oracle_phi_from_post(const oracle_problem *p, const double *F, int n, double *phi);
/* Whole run: init from phi0, nsteps steps, phi(t_N) out, optional final state. */
int oracle_run(const oracle_problem *p, const double *phi0, int nsteps, double *phi_out, double *F_out);

/* General stepping: Scheme A or B, periodic, anti-bounce-back (1) or
   non-equilibrium extrapolation (2) boundaries, every flux and source family.
   The state is the post-collision populations F plus the plane Phi = phi(t_n)
   (Scheme A needs phi(t_n) for the backward difference of R_k).
   bvals: the Dirichlet values phi_b of the time level being computed, laid
   out west[ny], east[ny], south[nx], north[nx]; a node on two edges (a corner)
   takes the west/east value. NULL when no axis uses extrapolation. */
int oracle_init_x(const oracle_problem *p, const double *phi0, double *F, double *Phi);
int oracle_step_x(const oracle_problem *p, const double *F_in, const double *Phi_in, const double *bvals,
                  double *F_out, double *Phi_out);
/* nsteps steps from phi0; bvals_all: nsteps records of 2 (nx + ny) values
   (record n for the step that produces t_{n+1}) or NULL. */
int oracle_run_x(const oracle_problem *p, const double *phi0, int nsteps, const double *bvals_all, double *phi_out);
/* One collision of one cell for the general path (phi_prev: phi(t_{n-1}) of the
   cell, used by Scheme A only). */
int oracle_collide_cell_x(const oracle_problem *p, const double K[3], const double f[9], double phi_prev,
                          double fout[9], double *phi_out);

/* Discrete adjoint of a run for the linear family (conv 0, diff 0, no source),
   loss = 1/2 sum (phi_N - target)^2. dK: 3 planes (dKxx, dKxy, dKyy) per cell. */
int oracle_adjoint(const oracle_problem *p, const double *phi0, const double *target, int nsteps,
                   double *loss, double *dphi0, double *dK, double *du);
#ifdef __cplusplus
}
#endif
#endif
