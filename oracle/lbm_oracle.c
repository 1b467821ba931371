/*
 * lbm_oracle.c -- plain FP64 CPU oracle of the D2Q9 MRT lattice Boltzmann
 * model for nonlinear anisotropic convection-diffusion equations
 * (Chai, Shi & Guo, arXiv:1603.09577).
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
 * CPU-baseline leg are its only users. It is written for reading, not speed:
 * every cell is collided by the textbook matrix products of the paper, in the
 * paper's order, and streamed by an explicit pull loop. Built with
 * -ffp-contract=off so that x86 and Arm give the same bits.
 *
 * What each function follows:
 *   lattice, weights ............ Eq. 5 (D2Q9), c = 1, c_s^2 = c^2/3
 *   equilibrium .................. Eq. 3 with D = g(phi) I or D = Dm phi (Eq. 62),
 *                                  d = 1 (Sec. 3)
 *   C(phi) from B'(phi) .......... Eq. 7
 *   discrete source .............. Eq. 9 with Btilde = B' (Scheme B, Eq. 28)
 *   M0, moments .................. Eq. 8, Eq. 14-15 (M^-1 S M = M0^-1 S M0, Eq. 18)
 *   relaxation matrix ............ Eq. 17, block A of Eq. 21 from K by Eq. 26
 *   collision + source ........... Eq. 34 (Scheme B, shifted variable Eq. 33)
 *   macroscopic phi .............. Eq. 35, closed form for affine R = r0 + r1 phi
 *   initialisation ............... Eq. 40
 *   walls ........................ anti-bounce-back, half-way wall (Sec. 3.6)
 *   explicit sources ............. Eq. 43 (Sec. 3.1), Eq. 66 (Sec. 3.5)
 *   power-law flux ............... Eq. 49-50 (conv 2), C from Eq. 7
 *   Fisher source ................ Eq. 46, R = b phi (1 - phi^delta)
 *   Scheme A ..................... Remark II: gamma = 0, theta = 1 (Eq. 28), so
 *                                  Btilde = (I - A/2) B' and the source term of
 *                                  Eq. 2 is dt R_k + dt^2/2 d_t R_k with the
 *                                  backward difference of Remark II
 *   C-free variant ............... Remark III: C = 0 in the equilibrium (Eq. 38) and
 *                                  the source G_k of Eq. 36-37, d_t B by the backward
 *                                  difference of Remark II
 *   Buckley-Leverett flux ........ Eq. 54 (conv 3, scaled by u = dt/dx per axis)
 *   extrapolation boundary ....... non-equilibrium extrapolation (cited in Sec. 3,
 *                                  Guo, Zheng & Shi 2002): a boundary node takes
 *                                  feq(phi_b) plus the non-equilibrium part of
 *                                  its inward neighbour, then collides
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9

/* Eq. 5: D2Q9 velocities in the paper's order and their weights. */
static const int CX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WK[Q] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0; /* c_s^2 = c^2 / 3 with c = 1 */
static const double DPAR = 1.0;      /* d = 1, the default of Sec. 3 */

/* Eq. 15: M0, rows (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy). */
static const int M0[Q][Q] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-4, -1, -1, -1, -1, 2, 2, 2, 2},
    {4, -2, -2, -2, -2, 1, 1, 1, 1},
    {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 1, -1, 1, -1},
};

/* Squared row norms of M0; the rows are mutually orthogonal, so
   M0^-1 = M0^T diag(1 / |row_i|^2). */
static int row_norm2(int i)
{
    int s = 0;
    for (int j = 0; j < Q; ++j) s += M0[i][j] * M0[i][j];
    return s;
}

static int opposite(int k)
{
    for (int j = 0; j < Q; ++j)
        if (CX[j] == -CX[k] && CY[j] == -CY[k]) return j;
    return -1;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- coefficient functions of Eq. 1 ------------------------------------ */

/* B(phi), B'(phi) and C(phi) with C' = B' B'^T (Eq. 7). C is (xx, xy, yy). */
static double ipow(double v, int n)
{
    double r = 1.0;
    for (int i = 0; i < n; ++i) r *= v;
    return r;
}

static void flux(const oracle_problem *p, double phi, double B[2], double Bp[2], double C[3])
{
    const double ax = p->u[0], ay = p->u[1];
    if (p->conv == 0) {
        B[0] = ax * phi;            B[1] = ay * phi;
        Bp[0] = ax;                 Bp[1] = ay;
        C[0] = ax * ax * phi;       C[1] = ax * ay * phi;      C[2] = ay * ay * phi;
    } else if (p->conv == 2) {
        /* Eq. 49: B = a phi^(delta+1) / (delta+1); B' = a phi^delta;
           Eq. 7 / Eq. 50: C = a a^T phi^(2 delta+1) / (2 delta+1) */
        const int dl = p->power;
        const double pb = ipow(phi, dl + 1) / (dl + 1);
        const double pd = ipow(phi, dl);
        const double pc = ipow(phi, 2 * dl + 1) / (2 * dl + 1);
        B[0] = ax * pb;             B[1] = ay * pb;
        Bp[0] = ax * pd;            Bp[1] = ay * pd;
        C[0] = ax * ax * pc;        C[1] = ax * ay * pc;       C[2] = ay * ay * pc;
    } else if (p->conv == 3) {
        /* Eq. 54: f = phi^2 / (phi^2 + (1 - phi)^2), g = f (1 - 5 (1 - phi)^2);
           no closed-form C is used (Remark III variant) */
        const double q = 1.0 - phi, den = phi * phi + q * q;
        const double f = phi * phi / den;
        const double fp = 2.0 * phi * q / (den * den);
        const double h = 1.0 - 5.0 * q * q;
        B[0] = ax * f;              B[1] = ay * f * h;
        Bp[0] = ax * fp;            Bp[1] = ay * (fp * h + f * 10.0 * q);
        C[0] = C[1] = C[2] = 0.0;
    } else {
        B[0] = ax * phi * phi / 2;  B[1] = ay * phi * phi / 2;
        Bp[0] = ax * phi;           Bp[1] = ay * phi;
        double p3 = phi * phi * phi / 3;
        C[0] = ax * ax * p3;        C[1] = ax * ay * p3;       C[2] = ay * ay * p3;
    }
    if (p->cfree) C[0] = C[1] = C[2] = 0.0;       /* Eq. 38 */
}

/* Diffusion function D(phi) = g(phi) I. */
static double gdiff(const oracle_problem *p, double phi)
{
    switch (p->diff) {
    case 1: return phi + phi * phi / 2;
    case 2: return phi + phi * phi * phi / 3;
    default: return phi;
    }
}

int oracle_feq(const oracle_problem *p, double phi, double feq[9])
{
    double B[2], Bp[2], C[3];
    flux(p, phi, B, Bp, C);
    /* D(phi): g(phi) I, or Dm phi (diff 3, the isotropic form of Eq. 62) */
    double Dxx, Dxy, Dyy;
    if (p->diff == 3) {
        Dxx = p->Dm[0] * phi; Dxy = p->Dm[1] * phi; Dyy = p->Dm[2] * phi;
    } else {
        Dxx = Dyy = gdiff(p, phi); Dxy = 0.0;
    }
    /* (C + d c_s^2 D - c_s^2 phi I), Eq. 3 */
    double Qxx = C[0] + DPAR * CS2 * Dxx - CS2 * phi;
    double Qxy = C[1] + DPAR * CS2 * Dxy;
    double Qyy = C[2] + DPAR * CS2 * Dyy - CS2 * phi;
    for (int k = 0; k < Q; ++k) {
        double cx = CX[k], cy = CY[k];
        double cB = cx * B[0] + cy * B[1];
        double QC = Qxx * (cx * cx - CS2) + 2.0 * Qxy * cx * cy + Qyy * (cy * cy - CS2);
        feq[k] = WK[k] * (phi + cB / CS2 + QC / (2.0 * CS2 * CS2));
    }
    return 0;
}

int oracle_source_pop(const oracle_problem *p, double phi, double R, double Rk[9])
{
    double B[2], Bp[2], C[3];
    flux(p, phi, B, Bp, C);
    /* Eq. 9 with Btilde = B' (Scheme B, gamma = 1, Eq. 28) */
    for (int k = 0; k < Q; ++k) {
        double cBt = CX[k] * Bp[0] + CY[k] * Bp[1];
        Rk[k] = WK[k] * (1.0 + cBt / CS2) * R;
    }
    return 0;
}

int oracle_relax_block(const double K[3], double A[4])
{
    /* Eq. 26 with dt = 1: A^-1 = K / (d c_s^2) + I/2. */
    double a = K[0] / (DPAR * CS2) + 0.5;
    double b = K[1] / (DPAR * CS2);
    double c = K[2] / (DPAR * CS2) + 0.5;
    double det = a * c - b * b;
    if (!(det > 0) || !(a > 0)) return 1;
    A[0] = c / det;  A[1] = -b / det;
    A[2] = -b / det; A[3] = a / det;
    return 0;
}

/* Full 9x9 relaxation matrix of Eq. 17. */
static int relax_matrix(const oracle_problem *p, const double K[3], double S[Q][Q])
{
    double A[4];
    if (oracle_relax_block(K, A)) return 1;
    memset(S, 0, sizeof(double) * Q * Q);
    for (int i = 0; i < Q; ++i) S[i][i] = p->s[i];
    S[3][3] = A[0]; S[3][5] = A[1];
    S[5][3] = A[2]; S[5][5] = A[3];
    return 0;
}

/* ---- explicit source terms of the test problems ------------------------ */

/* Returns R * dt (lattice units) at node (i, j), time level n. */
static double explicit_source(const oracle_problem *p, int i, int j, int n)
{
    if (p->src == 0) return 0.0;
    const double *q = p->src_par;
    double x = q[0] + i * q[2], y = q[1] + j * q[2], t = n * q[3];
    double kap = q[4], ux = q[5], uy = q[6];
    const double pi = 3.14159265358979323846;
    if (p->src == 1) { /* Eq. 43 */
        double e = exp((1.0 - 2.0 * pi * pi * kap) * t);
        return q[3] * e * (sin(pi * (x + y)) + pi * (ux + uy) * cos(pi * (x + y)));
    }
    /* Eq. 66 */
    double e = exp((1.0 - 12.0 * pi * pi * kap) * t);
    double s2x = sin(2 * pi * x), s2y = sin(2 * pi * y), c2x = cos(2 * pi * x), c2y = cos(2 * pi * y);
    return q[3] * e * (s2x * s2y + 4.0 * kap * pi * pi * cos(4 * pi * x) * s2y * s2y
                       + 2.0 * pi * (ux * c2x * s2y + uy * s2x * c2y));
}

/* ---- collision ---------------------------------------------------------- */

/* phi from the shifted populations (Eq. 35) for R = r0 + r1 phi + Rexp. */
static double phi_from_pre(const oracle_problem *p, const double f[Q], double Rexp)
{
    double sum = 0.0;
    for (int k = 0; k < Q; ++k) sum += f[k];
    return (sum + 0.5 * (p->r0 + Rexp)) / (1.0 - 0.5 * p->r1);
}

static void matvec_M0(const double v[Q], double out[Q])
{
    for (int i = 0; i < Q; ++i) {
        double s = 0.0;
        for (int j = 0; j < Q; ++j) s += M0[i][j] * v[j];
        out[i] = s;
    }
}

static void matvec_M0inv(const double m[Q], double out[Q])
{
    double mn[Q];
    for (int i = 0; i < Q; ++i) mn[i] = m[i] / row_norm2(i);
    for (int k = 0; k < Q; ++k) {
        double s = 0.0;
        for (int i = 0; i < Q; ++i) s += M0[i][k] * mn[i];
        out[k] = s;
    }
}

/* Collision in moment space (Eq. 34 multiplied by M0):
   m* = m - S (m - m_eq) + (I - S/2) M0 R_vec. */
static void collide_moment(const double S[Q][Q], const double f[Q], const double feq[Q],
                           const double Rk[Q], double out[Q])
{
    double m[Q], meq[Q], mR[Q], ms[Q];
    matvec_M0(f, m);
    matvec_M0(feq, meq);
    matvec_M0(Rk, mR);
    for (int i = 0; i < Q; ++i) {
        double relax = 0.0, half = 0.0;
        for (int j = 0; j < Q; ++j) {
            relax += S[i][j] * (m[j] - meq[j]);
            half += S[i][j] * mR[j];
        }
        ms[i] = m[i] - relax + (mR[i] - 0.5 * half);
    }
    matvec_M0inv(ms, out);
}

/* P = M0^-1 S M0 and Q = M0^-1 (I - S/2) M0. Each entry is
   sum_i sum_l (M0_ik / n_i) X_il M0_lj; every n_i divides 36, so an entry is
   (1/36) sum over the distinct values v of X of v * (integer). Grouping equal
   values first keeps the integer parts exact, so S = s I gives P = s I and
   Q = (1 - s/2) I exactly, as in exact rational arithmetic. */
static void pform_entry_matrix(const double X[Q][Q], double out[Q][Q])
{
    for (int k = 0; k < Q; ++k)
        for (int j = 0; j < Q; ++j) {
            double vals[Q * Q];
            long coef[Q * Q];
            int nv = 0;
            for (int i = 0; i < Q; ++i)
                for (int l = 0; l < Q; ++l) {
                    if (X[i][l] == 0.0) continue;
                    long c = (long)M0[i][k] * M0[l][j] * (36 / row_norm2(i));
                    int g = 0;
                    while (g < nv && vals[g] != X[i][l]) ++g;
                    if (g == nv) { vals[nv] = X[i][l]; coef[nv] = 0; ++nv; }
                    coef[g] += c;
                }
            double s = 0.0;
            for (int g = 0; g < nv; ++g) s += vals[g] * ((double)coef[g] / 36.0);
            out[k][j] = s;
        }
}

int oracle_pform_matrices(const oracle_problem *p, const double K[3], double P[81], double Qm[81])
{
    double S[Q][Q], H[Q][Q], Pm[Q][Q], Qq[Q][Q];
    if (relax_matrix(p, K, S)) return 1;
    for (int i = 0; i < Q; ++i)
        for (int l = 0; l < Q; ++l) H[i][l] = (i == l ? 1.0 : 0.0) - 0.5 * S[i][l];
    /* the diagonal of I - S/2 written as 1 - s/2 with one rounding */
    for (int i = 0; i < Q; ++i) H[i][i] = 1.0 - 0.5 * S[i][i];
    pform_entry_matrix(S, Pm);
    pform_entry_matrix(H, Qq);
    for (int k = 0; k < Q; ++k)
        for (int j = 0; j < Q; ++j) { P[k * Q + j] = Pm[k][j]; Qm[k * Q + j] = Qq[k][j]; }
    return 0;
}

/* Eq. 34 in population space with the matrices above. */
static void collide_pform(const double P[Q * Q], const double Qm[Q * Q], const double f[Q],
                          const double feq[Q], const double Rk[Q], double out[Q])
{
    for (int k = 0; k < Q; ++k) {
        double x = 0.0, y = 0.0;
        for (int j = 0; j < Q; ++j) x += P[k * Q + j] * (f[j] - feq[j]);
        for (int j = 0; j < Q; ++j) y += Qm[k * Q + j] * Rk[j];
        out[k] = f[k] - x + y;
    }
}

/* Single-relaxation-time (BGK) form, valid when S = s I. */
static void collide_bgk(double s, const double f[Q], const double feq[Q], const double Rk[Q],
                        double out[Q])
{
    for (int k = 0; k < Q; ++k) {
        double x = s * (f[k] - feq[k]);
        double y = (1.0 - 0.5 * s) * Rk[k];
        out[k] = f[k] - x + y;
    }
}

int oracle_collide_cell(const oracle_problem *p, const double K[3], const double f[9],
                        double Rexp, double fout[9], double *phi_out)
{
    double phi = phi_from_pre(p, f, Rexp);
    double R = p->r0 + p->r1 * phi + Rexp;
    double feq[Q], Rk[Q];
    oracle_feq(p, phi, feq);
    oracle_source_pop(p, phi, R, Rk);
    if (p->collision == 0) {
        double S[Q][Q];
        if (relax_matrix(p, K, S)) return 1;
        collide_moment(S, f, feq, Rk, fout);
    } else if (p->collision == 1) {
        double P[Q * Q], Qm[Q * Q];
        if (oracle_pform_matrices(p, K, P, Qm)) return 1;
        collide_pform(P, Qm, f, feq, Rk, fout);
    } else {
        double A[4];
        if (oracle_relax_block(K, A)) return 1;
        collide_bgk(A[0], f, feq, Rk, fout);
    }
    if (phi_out) *phi_out = phi;
    return 0;
}

/* ---- lattice ------------------------------------------------------------ */

static void cell_K(const oracle_problem *p, int x, int y, double K[3])
{
    if (p->Kfield) {
        size_t n = (size_t)p->nx * p->ny, c = (size_t)y * p->nx + x;
        K[0] = p->Kfield[c]; K[1] = p->Kfield[n + c]; K[2] = p->Kfield[2 * n + c];
    } else {
        K[0] = p->K[0]; K[1] = p->K[1]; K[2] = p->K[2];
    }
}

static int check_problem(const oracle_problem *p)
{
    if (p->nx < 1 || p->ny < 1) return 1;
    if (p->collision == 2) {
        /* the BGK loop needs S = s I */
        double A[4];
        if (p->Kfield || oracle_relax_block(p->K, A)) return 1;
        if (A[1] != 0.0 || A[0] != A[3]) return 1;
        for (int i = 0; i < Q; ++i)
            if (i != 3 && i != 5 && p->s[i] != A[0]) return 1;
    }
    return 0;
}

#define IDX(p, k, x, y) (((size_t)(k) * (p)->ny + (size_t)(y)) * (p)->nx + (size_t)(x))

int oracle_init(const oracle_problem *p, const double *phi0, double *F)
{
    if (check_problem(p)) return 1;
    int bad = 0;
#pragma omp parallel for reduction(| : bad)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            double phi = phi0[(size_t)y * p->nx + x];
            double Rexp = explicit_source(p, x, y, 0);
            double R = p->r0 + p->r1 * phi + Rexp;
            double feq[Q], Rk[Q], fb[Q], out[Q], K[3];
            oracle_feq(p, phi, feq);         /* Eq. 40 */
            oracle_source_pop(p, phi, R, Rk);
            for (int k = 0; k < Q; ++k) fb[k] = feq[k] - 0.5 * Rk[k]; /* Eq. 33 */
            cell_K(p, x, y, K);
            bad |= oracle_collide_cell(p, K, fb, Rexp, out, NULL);
            for (int k = 0; k < Q; ++k) F[IDX(p, k, x, y)] = out[k];
        }
    return bad;
}

/* Pull one population into (x, y): periodic wrap or anti-bounce-back from the
   half-way wall. The wall term is the even part of the equilibrium at the wall
   value, feq_k(phi_w) + feq_opp(k)(phi_w) = 2 w_k [phi_w + Q_w : (c c - c_s^2 I) / (2 c_s^4)]. */
static double pull(const oracle_problem *p, const double *F, int k, int x, int y)
{
    int xs = x - CX[k], ys = y - CY[k];
    int out_x = 0, out_y = 0;
    if (xs < 0 || xs >= p->nx) {
        if (p->bc_x == 0) xs = (xs + p->nx) % p->nx;
        else out_x = 1;
    }
    if (ys < 0 || ys >= p->ny) {
        if (p->bc_y == 0) ys = (ys + p->ny) % p->ny;
        else out_y = 1;
    }
    if (!out_x && !out_y) return F[IDX(p, k, xs, ys)];
    double wx = (x - CX[k] < 0) ? p->phi_wall[0] : p->phi_wall[1];
    double wy = (y - CY[k] < 0) ? p->phi_wall[2] : p->phi_wall[3];
    double phiw = (out_x && out_y) ? 0.5 * (wx + wy) : (out_x ? wx : wy);
    double feq[Q];
    oracle_feq(p, phiw, feq);
    int o = opposite(k);
    return -F[IDX(p, o, x, y)] + (feq[k] + feq[o]);
}

int oracle_step(const oracle_problem *p, const double *F_in, double *F_out, int n, double *phi_out)
{
    if (check_problem(p)) return 1;
    int bad = 0;
#pragma omp parallel for reduction(| : bad)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            double f[Q], out[Q], K[3], phi;
            for (int k = 0; k < Q; ++k) f[k] = pull(p, F_in, k, x, y);
            cell_K(p, x, y, K);
            bad |= oracle_collide_cell(p, K, f, explicit_source(p, x, y, n + 1), out, &phi);
            for (int k = 0; k < Q; ++k) F_out[IDX(p, k, x, y)] = out[k];
            if (phi_out) phi_out[(size_t)y * p->nx + x] = phi;
        }
    return bad;
}

int oracle_phi_from_post(const oracle_problem *p, const double *F, int n, double *phi)
{
    /* The collision adds R/2 to the zeroth moment (Eq. 34-35), so
       sum_k fbar*_k = phi + R/2 with R = r0 + r1 phi + Rexp. */
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            double s = 0.0;
            for (int k = 0; k < Q; ++k) s += F[IDX(p, k, x, y)];
            double Rexp = explicit_source(p, x, y, n);
            phi[(size_t)y * p->nx + x] = (s - 0.5 * (p->r0 + Rexp)) / (1.0 + 0.5 * p->r1);
        }
    return 0;
}

int oracle_run(const oracle_problem *p, const double *phi0, int nsteps, double *phi_out, double *F_out)
{
    size_t n = (size_t)Q * p->nx * p->ny;
    double *a = malloc(n * sizeof(double)), *b = malloc(n * sizeof(double));
    if (!a || !b) { free(a); free(b); return 2; }
    int rc = oracle_init(p, phi0, a);
    if (nsteps == 0 && !rc) {
        memcpy(phi_out, phi0, sizeof(double) * p->nx * p->ny);
    }
    for (int s = 0; s < nsteps && !rc; ++s) {
        rc = oracle_step(p, a, b, s, s == nsteps - 1 ? phi_out : NULL);
        double *t = a; a = b; b = t;
    }
    if (!rc && F_out) memcpy(F_out, a, n * sizeof(double));
    free(a); free(b);
    return rc;
}

/* ---- general path: Scheme A, Fisher source, extrapolation boundary -------- */

/* Source value R(phi) of the general path. */
static double source_value(const oracle_problem *p, double phi)
{
    if (p->src_family == 1) return p->b * phi * (1.0 - ipow(phi, p->power)); /* Eq. 46 */
    return p->r0 + p->r1 * phi;
}

/* Discrete source populations (Eq. 9) with the scheme's Btilde (Eq. 28):
   Scheme B (gamma = 1) Btilde = B'; Scheme A (gamma = 0) Btilde = (I - A/2) B'. */
static void source_pop_x(const oracle_problem *p, const double A[4], double phi, double R, double Rk[Q])
{
    double B[2], Bp[2], C[3], Bt[2];
    flux(p, phi, B, Bp, C);
    if (p->scheme == 1) {
        Bt[0] = Bp[0] - 0.5 * (A[0] * Bp[0] + A[1] * Bp[1]);
        Bt[1] = Bp[1] - 0.5 * (A[2] * Bp[0] + A[3] * Bp[1]);
    } else {
        Bt[0] = Bp[0];
        Bt[1] = Bp[1];
    }
    for (int k = 0; k < Q; ++k) Rk[k] = WK[k] * (1.0 + (CX[k] * Bt[0] + CY[k] * Bt[1]) / CS2) * R;
}

int oracle_collide_cell_x(const oracle_problem *p, const double K[3], const double f[9], double phi_prev,
                          double fout[9], double *phi_out)
{
    double S[Q][Q], A[4];
    if (relax_matrix(p, K, S) || oracle_relax_block(K, A)) return 1;
    double feq[Q], Rk[Q], phi = 0.0;
    if (p->scheme == 1) {
        /* Scheme A: phi = sum_k phi_k (Eq. 10a); Eq. 2 with theta = 1, gamma = 0:
           phi*_k = phi_k - (M^-1 S M)(phi - phi_eq) + dt R_k(t) + dt^2/2 d_t R_k,
           d_t R_k = [R_k(t) - R_k(t - dt)] / dt (Remark II). */
        for (int k = 0; k < Q; ++k) phi += f[k];
        double Rk0[Q], m[Q], meq[Q], ms[Q], relaxed[Q];
        oracle_feq(p, phi, feq);
        source_pop_x(p, A, phi, source_value(p, phi), Rk);
        source_pop_x(p, A, phi_prev, source_value(p, phi_prev), Rk0);
        matvec_M0(f, m);
        matvec_M0(feq, meq);
        for (int i = 0; i < Q; ++i) {
            double r = 0.0;
            for (int j = 0; j < Q; ++j) r += S[i][j] * (m[j] - meq[j]);
            ms[i] = m[i] - r;
        }
        matvec_M0inv(ms, relaxed);
        for (int k = 0; k < Q; ++k) fout[k] = relaxed[k] + Rk[k] + 0.5 * (Rk[k] - Rk0[k]);
        if (p->cfree) {
            /* Eq. 36-37: + dt G_k, G_k = w_k c_k . (I - A/2) d_t B / c_s^2 with
               d_t B = [B(phi) - B(phi_prev)] / dt */
            double B1[2], B0[2], Bp[2], C[3], dB[2], G[2];
            flux(p, phi, B1, Bp, C);
            flux(p, phi_prev, B0, Bp, C);
            dB[0] = B1[0] - B0[0];
            dB[1] = B1[1] - B0[1];
            G[0] = dB[0] - 0.5 * (A[0] * dB[0] + A[1] * dB[1]);
            G[1] = dB[1] - 0.5 * (A[2] * dB[0] + A[3] * dB[1]);
            for (int k = 0; k < Q; ++k) fout[k] += WK[k] * (CX[k] * G[0] + CY[k] * G[1]) / CS2;
        }
    } else {
        /* Scheme B (Eq. 34-35), affine source only */
        if (p->src_family != 0) return 1;
        phi = phi_from_pre(p, f, 0.0);
        oracle_feq(p, phi, feq);
        source_pop_x(p, A, phi, source_value(p, phi), Rk);
        collide_moment(S, f, feq, Rk, fout);
    }
    if (phi_out) *phi_out = phi;
    return 0;
}

static int check_problem_x(const oracle_problem *p)
{
    if (p->nx < 1 || p->ny < 1 || p->src != 0 || p->collision != 0) return 1;
    if (p->scheme != 0 && p->scheme != 1) return 1;
    if (p->src_family == 1 && p->scheme != 1) return 1;
    if (p->cfree && p->scheme != 1) return 1;       /* d_t B needs phi(t_n): Scheme A's plane */
    if (p->conv == 3 && !p->cfree) return 1;
    if (p->diff < 0 || p->diff > 3) return 1;
    if ((p->conv == 2 || p->src_family == 1) && p->power < 1) return 1;
    if (p->bc_x < 0 || p->bc_x > 2 || p->bc_y < 0 || p->bc_y > 2) return 1;
    /* extrapolation needs an inward neighbour inside the domain, and the other
       axis periodic or extrapolated (no anti-bounce-back link at that node) */
    if (p->bc_x == 2 && (p->nx < 3 || p->bc_y == 1)) return 1;
    if (p->bc_y == 2 && (p->ny < 3 || p->bc_x == 1)) return 1;
    return 0;
}

/* feq minus the Scheme B shift (Eq. 33): the equilibrium of the stored variable. */
static void feq_stored(const oracle_problem *p, double phi, double out[Q])
{
    oracle_feq(p, phi, out);
    if (p->scheme == 0) {
        double Rk[Q], A[4] = {0, 0, 0, 0};
        source_pop_x(p, A, phi, source_value(p, phi), Rk);
        for (int k = 0; k < Q; ++k) out[k] -= 0.5 * Rk[k];
    }
}

int oracle_init_x(const oracle_problem *p, const double *phi0, double *F, double *Phi)
{
    if (check_problem_x(p)) return 1;
    int bad = 0;
#pragma omp parallel for reduction(| : bad)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            double phi = phi0[(size_t)y * p->nx + x];
            double f[Q], out[Q], K[3];
            /* Eq. 40 (Scheme A: phi_k = feq; Scheme B: its shifted form, Eq. 33);
               Scheme A takes d_t R_k = 0 at t = 0 (phi_prev = phi0) */
            feq_stored(p, phi, f);
            cell_K(p, x, y, K);
            bad |= oracle_collide_cell_x(p, K, f, phi, out, NULL);
            for (int k = 0; k < Q; ++k) F[IDX(p, k, x, y)] = out[k];
            Phi[(size_t)y * p->nx + x] = phi;
        }
    return bad;
}

/* Dirichlet value of an extrapolated boundary node (corners: west/east first). */
static double boundary_value(const oracle_problem *p, const double *bv, int x, int y)
{
    if (p->bc_x == 2 && x == 0) return bv[y];
    if (p->bc_x == 2 && x == p->nx - 1) return bv[p->ny + y];
    if (p->bc_y == 2 && y == 0) return bv[2 * p->ny + x];
    return bv[2 * p->ny + p->nx + x];
}

int oracle_step_x(const oracle_problem *p, const double *F_in, const double *Phi_in, const double *bvals,
                  double *F_out, double *Phi_out)
{
    if (check_problem_x(p)) return 1;
    if ((p->bc_x == 2 || p->bc_y == 2) && !bvals) return 1;
    int bad = 0;
#pragma omp parallel for reduction(| : bad)
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            double f[Q], out[Q], K[3], phi;
            const int ex = p->bc_x == 2 && (x == 0 || x == p->nx - 1);
            const int ey = p->bc_y == 2 && (y == 0 || y == p->ny - 1);
            if (ex || ey) {
                /* non-equilibrium extrapolation: pull the inward neighbour xf,
                   f(xb) = feq(phi_b) + [f(xf) - feq(phi(xf))] in the stored variable */
                const int xf = ex ? (x == 0 ? 1 : p->nx - 2) : x;
                const int yf = ey ? (y == 0 ? 1 : p->ny - 2) : y;
                double ff[Q], eb[Q], ef[Q], phif = 0.0;
                for (int k = 0; k < Q; ++k) ff[k] = pull(p, F_in, k, xf, yf);
                if (p->scheme == 1) {
                    for (int k = 0; k < Q; ++k) phif += ff[k];
                } else {
                    phif = phi_from_pre(p, ff, 0.0);
                }
                feq_stored(p, boundary_value(p, bvals, x, y), eb);
                feq_stored(p, phif, ef);
                for (int k = 0; k < Q; ++k) f[k] = eb[k] + (ff[k] - ef[k]);
            } else {
                for (int k = 0; k < Q; ++k) f[k] = pull(p, F_in, k, x, y);
            }
            cell_K(p, x, y, K);
            const double prev = Phi_in ? Phi_in[(size_t)y * p->nx + x] : 0.0;
            bad |= oracle_collide_cell_x(p, K, f, prev, out, &phi);
            for (int k = 0; k < Q; ++k) F_out[IDX(p, k, x, y)] = out[k];
            Phi_out[(size_t)y * p->nx + x] = phi;
        }
    return bad;
}

int oracle_run_x(const oracle_problem *p, const double *phi0, int nsteps, const double *bvals_all, double *phi_out)
{
    const size_t cells = (size_t)p->nx * p->ny, n = (size_t)Q * cells, rec = 2 * ((size_t)p->nx + p->ny);
    double *a = malloc(n * sizeof(double)), *b = malloc(n * sizeof(double));
    double *pa = malloc(cells * sizeof(double)), *pb = malloc(cells * sizeof(double));
    if (!a || !b || !pa || !pb) { free(a); free(b); free(pa); free(pb); return 2; }
    int rc = oracle_init_x(p, phi0, a, pa);
    for (int s = 0; s < nsteps && !rc; ++s) {
        rc = oracle_step_x(p, a, pa, bvals_all ? bvals_all + (size_t)s * rec : NULL, b, pb);
        double *t = a; a = b; b = t;
        t = pa; pa = pb; pb = t;
    }
    if (!rc) memcpy(phi_out, pa, cells * sizeof(double));
    free(a); free(b); free(pa); free(pb);
    return rc;
}

/* ---- discrete adjoint (linear family) ----------------------------------- */

/* Collision of the linear family with no source, as a function of f only. */
static void collide_linear(const oracle_problem *p, const double K[3], const double f[Q], double out[Q])
{
    oracle_collide_cell(p, K, f, 0.0, out, NULL);
}

/* Jacobian J[k][j] = d collide_k / d f_j: the collision is linear in f here,
   so column j is the collision of the j-th unit vector. */
static void jacobian(const oracle_problem *p, const double K[3], double J[Q][Q])
{
    for (int j = 0; j < Q; ++j) {
        double e[Q] = {0}, col[Q];
        e[j] = 1.0;
        collide_linear(p, K, e, col);
        for (int k = 0; k < Q; ++k) J[k][j] = col[k];
    }
}

/* d feq_k / d u_alpha for B = u phi, C = u u phi, D = phi I (Eq. 3, 61). */
static void dfeq_du(const oracle_problem *p, double phi, double d[2][Q])
{
    double ux = p->u[0], uy = p->u[1];
    for (int k = 0; k < Q; ++k) {
        double cu = CX[k] * ux + CY[k] * uy;
        /* Q = phi u u; Q:(cc - cs2 I) = phi ((c.u)^2 - cs2 |u|^2) */
        d[0][k] = WK[k] * phi * (CX[k] / CS2 + (2.0 * cu * CX[k] - 2.0 * CS2 * ux) / (2.0 * CS2 * CS2));
        d[1][k] = WK[k] * phi * (CY[k] / CS2 + (2.0 * cu * CY[k] - 2.0 * CS2 * uy) / (2.0 * CS2 * CS2));
    }
}

int oracle_adjoint(const oracle_problem *p, const double *phi0, const double *target, int nsteps,
                   double *loss, double *dphi0, double *dK, double *du)
{
    if (p->conv != 0 || p->diff != 0 || p->r0 != 0.0 || p->r1 != 0.0 || p->src != 0 ||
        p->bc_x != 0 || p->bc_y != 0 || nsteps < 1 || p->collision != 0)
        return 1;
    const int nx = p->nx, ny = p->ny;
    const size_t ncell = (size_t)nx * ny, nst = Q * ncell;
    /* G[n]: pre-collision states, n = 0..N (G[0] = feq(phi0)); F = collide(G). */
    double *G = malloc(nst * (nsteps + 1) * sizeof(double));
    double *F = malloc(nst * sizeof(double));
    double *lamF = malloc(nst * sizeof(double));
    double *lamG = malloc(nst * sizeof(double));
    double *gA = calloc(3 * ncell, sizeof(double));
    if (!G || !F || !lamF || !lamG || !gA) { free(G); free(F); free(lamF); free(lamG); free(gA); return 2; }

    /* forward, keeping every pre-collision state */
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double feq[Q];
            oracle_feq(p, phi0[(size_t)y * nx + x], feq);
            for (int k = 0; k < Q; ++k) G[IDX(p, k, x, y)] = feq[k];
        }
    for (int n = 0; n < nsteps; ++n) {
        const double *Gn = G + nst * n;
        double *Gn1 = G + nst * (n + 1);
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double f[Q], out[Q], K[3];
                for (int k = 0; k < Q; ++k) f[k] = Gn[IDX(p, k, x, y)];
                cell_K(p, x, y, K);
                collide_linear(p, K, f, out);
                for (int k = 0; k < Q; ++k) F[IDX(p, k, x, y)] = out[k];
            }
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                for (int k = 0; k < Q; ++k) Gn1[IDX(p, k, x, y)] = pull(p, F, k, x, y);
    }
    /* loss on phi_N = sum_k G[N]_k */
    double L = 0.0;
    const double *GN = G + nst * nsteps;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double s = 0.0;
            for (int k = 0; k < Q; ++k) s += GN[IDX(p, k, x, y)];
            double r = s - target[(size_t)y * nx + x];
            L += 0.5 * r * r;
            for (int k = 0; k < Q; ++k) lamG[IDX(p, k, x, y)] = r;
        }
    *loss = L;
    du[0] = du[1] = 0.0;

    for (int n = nsteps - 1; n >= 0; --n) {
        /* adjoint of the pull: lamF_k(y) = lamG_k(y + c_k) (periodic) */
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                for (int k = 0; k < Q; ++k) {
                    int xd = (x + CX[k] + nx) % nx, yd = (y + CY[k] + ny) % ny;
                    lamF[IDX(p, k, x, y)] = lamG[IDX(p, k, xd, yd)];
                }
        const double *Gn = G + nst * n;
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double K[3], J[Q][Q], S[Q][Q], lf[Q], g[Q], m[Q], meq[Q], feq[Q], phi = 0.0;
                cell_K(p, x, y, K);
                jacobian(p, K, J);
                relax_matrix(p, K, S);
                for (int k = 0; k < Q; ++k) { lf[k] = lamF[IDX(p, k, x, y)]; g[k] = Gn[IDX(p, k, x, y)]; phi += g[k]; }
                /* lamG = J^T lamF */
                for (int j = 0; j < Q; ++j) {
                    double s = 0.0;
                    for (int k = 0; k < Q; ++k) s += J[k][j] * lf[k];
                    lamG[IDX(p, j, x, y)] = s;
                }
                /* d collide / d A_ij = -M0^-1 e_i (m - m_eq)_j, i, j in {3, 5} */
                oracle_feq(p, phi, feq);
                matvec_M0(g, m);
                matvec_M0(feq, meq);
                double mu[Q]; /* M0^-T lamF: mu_i = (M0 lamF)_i / n_i */
                matvec_M0(lf, mu);
                for (int i = 0; i < Q; ++i) mu[i] /= row_norm2(i);
                double d3 = m[3] - meq[3], d5 = m[5] - meq[5];
                double *ga = gA + (size_t)y * nx + x;
                ga[0] += -mu[3] * d3;
                ga[ncell] += -mu[3] * d5 - mu[5] * d3;
                ga[2 * ncell] += -mu[5] * d5;
                /* d collide / d u at fixed f = M0^-1 S M0 dfeq/du */
                double dfu[2][Q];
                dfeq_du(p, phi, dfu);
                for (int a = 0; a < 2; ++a) {
                    double dm[Q], sdm[Q], acc = 0.0;
                    matvec_M0(dfu[a], dm);
                    for (int i = 0; i < Q; ++i) {
                        double s = 0.0;
                        for (int j = 0; j < Q; ++j) s += S[i][j] * dm[j];
                        sdm[i] = s;
                    }
                    for (int i = 0; i < Q; ++i) acc += mu[i] * sdm[i];
                    du[a] += acc;
                }
            }
    }
    /* G[0] = feq(phi0): dphi0 = a^T lamG with a = dfeq/dphi; u enters feq too */
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double a1[Q], dfu[2][Q], s = 0.0;
            oracle_feq(p, 1.0, a1); /* linear family: feq = phi * feq(1) */
            dfeq_du(p, phi0[(size_t)y * nx + x], dfu);
            for (int k = 0; k < Q; ++k) {
                double l = lamG[IDX(p, k, x, y)];
                s += a1[k] * l;
                du[0] += dfu[0][k] * l;
                du[1] += dfu[1][k] * l;
            }
            dphi0[(size_t)y * nx + x] = s;
        }
    /* chain A = (K / (d c_s^2) + I/2)^-1: dA = -A dK A / (d c_s^2) */
    for (size_t c = 0; c < ncell; ++c) {
        double K[3], A[4];
        int x = (int)(c % nx), y = (int)(c / nx);
        cell_K(p, x, y, K);
        oracle_relax_block(K, A);
        double G33 = gA[c], G35 = gA[ncell + c], G55 = gA[2 * ncell + c];
        /* symmetric gradient matrix Gs with off-diagonal G35/2 */
        double Gs[2][2] = {{G33, 0.5 * G35}, {0.5 * G35, G55}};
        double Am[2][2] = {{A[0], A[1]}, {A[2], A[3]}};
        double T[2][2], Hm[2][2];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) T[i][j] = Am[i][0] * Gs[0][j] + Am[i][1] * Gs[1][j];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) Hm[i][j] = -(T[i][0] * Am[0][j] + T[i][1] * Am[1][j]) / (DPAR * CS2);
        dK[c] = Hm[0][0];
        dK[ncell + c] = Hm[0][1] + Hm[1][0];
        dK[2 * ncell + c] = Hm[1][1];
    }
    free(G); free(F); free(lamF); free(lamG); free(gA);
    return 0;
}
