/*
 * lbm.h -- C ABI of the GB300 (sm_103a) library for the D2Q9 multiple-
 * relaxation-time lattice Boltzmann model of nonlinear anisotropic
 * convection-diffusion equations (Chai, Shi & Guo, arXiv:1603.09577).
 *
 * The equation solved is Eq. 1,
 *     d_t phi + div B(phi) = div[K . (div D(phi))] + R,
 * with D(phi) = g(phi) I and the closed coefficient families of lbm_coeffs.
 * Every time step is one fused pull-stream / collide sweep on the D2Q9
 * lattice (Eq. 5), in lattice units c = dx/dt = 1, c_s^2 = 1/3, d = 1: Scheme B
 * (Eq. 34, the default) or Scheme A (Remark II: gamma = 0, theta = 1,
 * Btilde = (I - A/2) B', the time derivative of R_k by a backward difference).
 *
 * Conventions for every entry point:
 *  - Return value: LBM_OK (0) or an error code; lbm_last_error() gives a
 *    thread-local message. No C++ exception crosses this boundary.
 *  - Memory: the caller owns all device memory. The library never allocates
 *    device memory; lbm_create receives a workspace of lbm_workspace_size()
 *    bytes (device, 256-byte aligned) and keeps pointers into it until
 *    lbm_destroy. Host-side handle memory is the library's.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *    default stream). Calls are asynchronous on that stream unless stated.
 *  - Fields: phi arrays are row-major (ny rows of nx), element (x, y) at
 *    y * nx + x, no padding. Precision tags: LBM_F64 = double, LBM_F32 = float.
 *  - State: after lbm_set_phi and after every lbm_step the stored state is the
 *    post-collision shifted population fbar*(x, t_n) (Eq. 33-34); with Scheme A
 *    the post-collision phi*_k(x, t_n) of Eq. 2 plus the plane phi(x, t_n).
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LBM_OK 0
#define LBM_EINVAL 1        /* invalid argument or handle                       */
#define LBM_ECUDA 2         /* a CUDA runtime call failed                        */
#define LBM_ENONFINITE 3    /* a non-finite value was detected                   */
#define LBM_ETIMEOUT 4      /* a bounded device-side wait ran out                */
#define LBM_EUNSUPPORTED 5  /* valid request this build does not implement      */

/* population storage precision */
#define LBM_F64 0           /* double populations, double arithmetic            */
#define LBM_F32 1           /* float populations, float arithmetic              */
#define LBM_BF16S 2         /* bf16 equilibrium-shifted deviations g_k =
                               fbar*_k - w_k phi plus a float shift plane h with
                               sum_k (w_k h + g_k) = the node's post-collision
                               mass; float arithmetic                            */

/* boundary kinds per axis */
#define LBM_PERIODIC 0
#define LBM_ABB 1           /* anti-bounce-back Dirichlet wall half-way between
                               the boundary node and its missing neighbour
                               (Sec. 3.6)                                        */
#define LBM_NEE 2           /* non-equilibrium extrapolation (cited in Sec. 3 as
                               the default boundary): the first and last node
                               rows of the axis are Dirichlet nodes; each takes
                               feq(phi_b) plus the non-equilibrium part of its
                               inward neighbour (stored variable), then collides.
                               phi_b per step from lbm_set_dirichlet. The other
                               axis must be LBM_PERIODIC or LBM_NEE; the axis
                               needs >= 3 nodes                                  */

/* time-stepping scheme (lbm_desc.scheme) */
#define LBM_SCHEME_B 0      /* gamma = 1 (Eq. 31-35), affine sources             */
#define LBM_SCHEME_A 1      /* gamma = 0 (Remark II), any source family          */

typedef struct lbm_solver *lbm_handle;

/* Grid, storage and boundaries. */
typedef struct {
    int nx, ny;             /* nodes per axis, each >= 2                          */
    int prec;               /* LBM_F64, LBM_F32 or LBM_BF16S                      */
    int bc_x, bc_y;         /* LBM_PERIODIC, LBM_ABB or LBM_NEE per axis          */
    double phi_wall[4];     /* Dirichlet values: west, east, south, north         */
    int steps_per_pass;     /* 1, or 2: two time steps per sweep through memory
                               (F32 and BF16S with periodic or ABB walls)         */
    int per_cell_K;         /* 1: K comes from lbm_set_K_field                    */
    int kernel_variant;     /* 0: automatic; 1: one node per thread; 2: four
                               x-adjacent nodes per thread with vector loads
                               (LBM_F32 / LBM_BF16S, nx % 4 == 0); 3: with
                               steps_per_pass 2, the register column march (each
                               warp walks a 30-column strip) instead of the
                               shared-memory tile kernel; 4: with steps_per_pass
                               2 and LBM_F32, the tile kernel with each interior
                               tile's input staged by a TMA tensor copy; 5: with
                               steps_per_pass 2 (LBM_F32 / LBM_BF16S), the tile
                               kernel with two x-adjacent nodes per thread and
                               paired (vector) loads and stores               */
    int block_rows;         /* rows of 32-thread warps per thread block: 0 (= 8),
                               1, 2, 4 or 8; for kernel_variant 3 the rows each
                               warp marches are 16 * block_rows (0: 64); for the
                               two-step tile kernel 4 selects 30 x 30 tiles,
                               other values 30 x 62; for kernel_variant 5, 4
                               selects 62 x 14 tiles, 2 62 x 22, other values
                               62 x 30                                            */
    int scheme;             /* LBM_SCHEME_B (0) or LBM_SCHEME_A. Scheme A, LBM_NEE,
                               conv 2 / 3 and diff 3 run the general kernels:
                               one node per thread (LBM_F64 or LBM_F32,
                               steps_per_pass 1, kernel_variant 0 or 1), or two
                               steps per pass on 30 x 30 tiles (LBM_F32,
                               kernel_variant 0, constant K, not conv 3 / cfree) */
} lbm_desc;

/* Coefficient families of Eq. 1 (Sec. 2.1), source and relaxation rates. */
typedef struct {
    int conv;               /* 0: B = u phi, C = u u^T phi;
                               1: B = a phi^2/2, C = a a^T phi^3/3 (Eq. 7);
                               2: B = a phi^(delta+1)/(delta+1),
                                  C = a a^T phi^(2 delta+1)/(2 delta+1)
                                  (Eq. 49-50), delta = power;
                               3: Buckley-Leverett B = (u_x f, u_y f h),
                                  f = phi^2/(phi^2 + (1-phi)^2), h = 1 - 5(1-phi)^2
                                  (Eq. 54), only with cfree = 1                   */
    double u[2];            /* u (conv 0), a (conv 1, 2) or the per-axis scale
                               dt/dx (conv 3)                                    */
    int diff;               /* D = g(phi) I, g = 0: phi, 1: phi + phi^2/2,
                               2: phi + phi^3/3; 3: D = Dm phi with the constant
                               symmetric tensor Dm (the isotropic form of Eq. 62,
                               Dm = K / kappa with K = kappa I here)              */
    double K[3];            /* constant tensor (Kxx, Kxy, Kyy), symmetric positive
                               definite; the block A = [[s3, s35], [s53, s5]] of
                               Eq. 17 follows from Eq. 26:
                               A = (K / (d c_s^2) + I/2)^-1                       */
    double s[9];            /* s0..s8 of Eq. 17; entries 3 and 5 are ignored
                               (they come from K); all others in (0, 2)           */
    double r0, r1;          /* source R = r0 + r1 phi (src_family 0); Scheme B
                               takes phi from Eq. 35 in closed form
                               phi = (sum fbar + r0/2) / (1 - r1/2)               */
    int src_family;         /* 0: R = r0 + r1 phi; 1: R = b phi (1 - phi^delta)
                               (Eq. 46, Scheme A only; r0 = r1 = 0)               */
    int power;              /* delta in 1..16 for conv 2 and src_family 1        */
    double b;               /* Fisher source coefficient (src_family 1)          */
    double Dm[3];           /* Dm_xx, Dm_xy, Dm_yy of diff 3                     */
    int cfree;              /* 1: Remark III variant, Scheme A only: C = 0 in the
                               equilibrium (Eq. 38) plus dt G_k (Eq. 36-37),
                               G_k = w_k c_k . (I - A/2) d_t B / c_s^2 with d_t B
                               by the backward difference of Remark II           */
} lbm_coeffs;

/* Bytes of device workspace lbm_create needs for this description. */
int lbm_workspace_size(const lbm_desc *desc, size_t *bytes);

/* Create a solver. dev_workspace: device pointer, >= lbm_workspace_size bytes,
   256-byte aligned, owned by the caller and kept alive until lbm_destroy. */
int lbm_create(lbm_handle *h, const lbm_desc *desc, void *dev_workspace, size_t bytes);
int lbm_destroy(lbm_handle h);

/* Set the coefficient families, the constant tensor K, rates and source.
   Validates s_i in (0, 2) and K positive definite (Eq. 26 needs A^-1 - I/2
   positive definite). Host-only; takes effect for later launches. */
int lbm_set_coeffs(lbm_handle h, const lbm_coeffs *c);

/* Per-cell tensor field (requires desc.per_cell_K): dev_K holds three planes of
   nx*ny doubles (Kxx, Kxy, Kyy). A kernel converts it by Eq. 26 into per-cell
   relaxation blocks stored in the workspace. */
int lbm_set_K_field(lbm_handle h, const double *dev_K, void *stream);

/* Initial condition phi(x, 0) (Eq. 40): fbar = feq(phi0) - R_k/2 (Eq. 33), then
   one collision, so that the stored state is fbar*(x, t_0); Scheme A: phi_k =
   feq(phi0), then one collision with d_t R_k = 0. dev_phi: nx*ny values of
   precision `prec` (LBM_F64 or LBM_F32). */
int lbm_set_phi(lbm_handle h, const void *dev_phi, int prec, void *stream);

/* Advance nsteps time steps (fused pull-stream + collide of Eq. 34 with the
   boundaries of lbm_desc). Asynchronous; no host synchronisation. The kernels
   alternate between the two population buffers; a stream capture of an even
   number of launches (nsteps even, or with steps_per_pass 2 a multiple of 4)
   therefore replays consistently. The first call on a device configures kernel
   attributes: make it before any stream capture. */
int lbm_step(lbm_handle h, int nsteps, void *stream);

/* Dirichlet data of the LBM_NEE axes. dev_values: device array of nrec >= 1
   records, each 2 (nx + ny) doubles laid out west[ny], east[ny], south[nx],
   north[nx] (a corner node takes its west/east value); the caller owns it and
   keeps it alive while steps run. Record j serves the (j + 1)-th step after
   this call or after the latest lbm_set_phi, whichever came last; after the
   last record the last one is reused (nrec = 1: constant values). lbm_set_phi
   itself takes the boundary values from phi0. The step count lives on the
   device and advances with the steps (one one-thread launch per lbm_step call
   when nrec > 1), so a CUDA graph of captured steps walks through the records
   on every replay as direct steps would. This call restarts the count on the
   stream of the next lbm_step or lbm_save (a capture of that lbm_step records
   the restart too, and every replay then starts the records over: step or
   save once before capturing); lbm_set_phi restarts it on its own stream;
   lbm_save stores it with the state and lbm_load restores it. */
int lbm_set_dirichlet(lbm_handle h, const double *dev_values, int nrec);

/* phi(t_n) of the current state into dev_out (nx*ny values of `prec`). */
int lbm_get_phi(lbm_handle h, void *dev_out, int prec, void *stream);

/* Host-buffer variants of lbm_set_phi / lbm_get_phi: the copy between host
   memory (pinned for asynchronous copies) and a staging area of the workspace
   is part of the call. lbm_get_phi_host synchronises `stream` before returning. */
int lbm_set_phi_host(lbm_handle h, const void *host_phi, int prec, void *stream);
int lbm_get_phi_host(lbm_handle h, void *host_out, int prec, void *stream);

/* Reductions over phi(t_n) (Eq. 39 and norms), FP64, deterministic order.
   dev_ref: nx*ny doubles or NULL. dev_out: 8 doubles on the device:
   [0] sum phi, [1] sum |phi - ref|, [2] sum |ref|, [3] sum (phi - ref)^2,
   [4] sum ref^2, [5] max |phi|, [6] number of non-finite phi, [7] sum phi^2.
   Entries 1-4 are 0 when dev_ref is NULL. GRE (Eq. 39) = out[1] / out[2]. */
int lbm_reduce(lbm_handle h, const double *dev_ref, double *dev_out, void *stream);

/* Failure detection: counts the nodes whose phi(t_n) is not finite (a blown-up
   run, a NaN in the input). Synchronises `stream`. Returns LBM_ENONFINITE (and
   the count in *nonfinite, which may be NULL) if there is any, else LBM_OK. */
int lbm_check_finite(lbm_handle h, long long *nonfinite, void *stream);

/* Checked builds (liblbm_checked.so, compiled with LBM_CHECKED): every node
   coordinate the kernels derive is tested before it indexes memory; one out of
   range sets a bit (1: x, 2: y, 4: shared-memory region, 8: linear index) of a
   device word and is replaced by 0. lbm_debug_flags reads the word (cleared by
   lbm_set_phi), synchronising `stream`; lbm_build_checked returns 1 in a checked
   build, 0 otherwise. In every build, a BF16S pair-tile launch (kernel_variant 5)
   whose grid would not cover the lattice writes nothing and sets 32, and the
   TMA-staged kernel's bounded wait sets 16 (below); otherwise the word stays 0
   in normal builds. */
int lbm_debug_flags(lbm_handle h, int *flags, void *stream);
int lbm_build_checked(void);

/* Failure detection without a GPU fault: runs the bounded mbarrier wait that the
   TMA-staged kernel (kernel_variant 4) uses on a barrier that expects bytes no
   copy will deliver. The wait gives up after `polls` polls (1..2^24; 2^12 takes
   well under a millisecond), writes 1 to *dev_status (a caller-owned device int)
   and the call returns LBM_ETIMEOUT; the context stays usable. Synchronises
   `stream`. The staged kernel reports the same condition by OR-ing 16 into the
   word lbm_debug_flags reads. */
int lbm_debug_wait_probe(unsigned polls, int *dev_status, void *stream);

/* Rate probe of the FP64 pipe, the roof of the LBM_F64 step kernel (the paper has
   no counterpart: it is a measurement aid). Launches blocks x threads threads,
   each running 8 independent FP64 fused multiply-add recurrences for `iters`
   iterations, asynchronously on `stream`; the caller times the launch (CUDA
   events on the same stream) and divides *fp64_inst (host, may be NULL: the
   FP64 thread instructions the launch executes) by the time. dev_sink: caller-
   owned device memory of `blocks` doubles, never written in practice (it keeps
   the recurrences live). Returns LBM_EINVAL for blocks < 1, threads not a
   multiple of 32 in [32, 1024], iters < 1 or a null sink. */
int lbm_probe_fp64(int blocks, int threads, int iters, double *dev_sink, long long *fp64_inst, void *stream);

/* Checkpoint / resume: the state is lbm_state_bytes bytes (populations; the phi
   plane for LBM_BF16S and Scheme A; with LBM_NEE walls, a 256-byte tail holding
   the Dirichlet record count). dev_dst / dev_src: device buffers of that size. */
int lbm_state_bytes(lbm_handle h, size_t *bytes);
int lbm_save(lbm_handle h, void *dev_dst, void *stream);
int lbm_load(lbm_handle h, const void *dev_src, void *stream);

/* ---- discrete adjoint (gradients through the time steps) --------------------
   Built for LBM_F64 and LBM_F32 with periodic boundaries and the linear family
   (conv 0, diff 0, r0 = r1 = 0), constant or per-node K; other solvers return
   LBM_EUNSUPPORTED. The forward step is F_{n+1} = collide(pull(F_n)) (Eq. 34);
   one reverse step applies the transposed collision Jacobian in moment space
   (Eq. 15-17, 19) and the transposed pull, and accumulates in FP64 the gradient
   with respect to the relaxation block A of every node (Eq. 17, 21) and to u
   (through m_eq, Eq. 16). lbm_adjoint_end chains A to K by Eq. 26.
   Usage: lbm_adjoint_begin with dL/dphi(t_N); then for n = N-1 down to 0 one
   lbm_adjoint_step with the forward state F_n (lbm_save layout, e.g. restored
   from checkpoints and recomputed); then lbm_adjoint_end. */

/* Bytes of the adjoint's own device workspace (two adjoint population buffers
   of the solver's precision, FP64 gradient planes, FP64 per-block partials). */
int lbm_adjoint_workspace_size(lbm_handle h, size_t *bytes);

/* Start a reverse sweep: dev_ws (device, 256-byte aligned, caller-owned, kept
   until lbm_adjoint_end) holds the adjoint state; dev_dphiN: nx*ny values of
   dL/dphi(t_N) in precision `prec`. Zeroes the gradient accumulators. */
int lbm_adjoint_begin(lbm_handle h, void *dev_ws, size_t bytes, const void *dev_dphiN, int prec, void *stream);

/* One reverse step through the update F_{n+1} = collide(pull(F_n)); dev_state_n
   is the forward post-collision state F_n in lbm_save layout. */
int lbm_adjoint_step(lbm_handle h, const void *dev_state_n, void *stream);

/* A whole checkpoint segment in one call: from the forward state F_t0
   (dev_ckpt, lbm_save layout) recompute F_{t0+1} .. F_{t0+nsteps-1} into
   dev_states ((nsteps - 1) * lbm_state_bytes bytes, caller-owned scratch), then
   run the nsteps reverse steps over them, last first. Equivalent to nsteps
   lbm_adjoint_step calls with the recomputed states. */
int lbm_adjoint_segment(lbm_handle h, const void *dev_ckpt, int nsteps, void *dev_states, size_t bytes, void *stream);

/* Finish at the initial condition F_0 = feq(phi0) (Eq. 40): dev_phi0 (nx*ny of
   `prec`); outputs dL/dphi0 (nx*ny doubles), dL/dK (3 planes of nx*ny doubles:
   dKxx, dKxy, dKyy per node, Kxy counted once) and dL/du (2 doubles). */
int lbm_adjoint_end(lbm_handle h, const void *dev_phi0, int prec, double *dev_dphi0, double *dev_dK, double *dev_du,
                    void *stream);

/* ---- batched ensemble of independent lattices ---------------------------------
   Many lattices of different sizes and coefficients advanced together with one
   persistent launch per time step over a work list of 32 x 8 tiles taken from
   every instance (each step is Eq. 34 per instance, FP32 storage, periodic
   walls). All instances share the coefficient family; u, K and the relaxation
   rates are per instance; no source term. Fields of all instances are
   packed one after another (instance i's nx_i*ny_i values, row-major). */
typedef struct lbm_ensemble_s *lbm_ensemble;

/* Device workspace bytes for `count` instances of sizes nx[i] x ny[i]. */
int lbm_ensemble_workspace_size(int count, const int *nx, const int *ny, size_t *bytes);
/* Create; coeffs: `count` entries (per-instance u and K). A synchronous set-up
   call: it enqueues the copies of the instance and tile tables into the caller's
   workspace on `stream` and waits for `stream` (no other stream is touched), so
   the tables are in place when it returns. */
int lbm_ensemble_create(lbm_ensemble *e, int count, const int *nx, const int *ny, const lbm_coeffs *coeffs,
                        void *dev_workspace, size_t bytes, void *stream);
int lbm_ensemble_destroy(lbm_ensemble e);
/* Total nodes, number of tiles and the persistent grid size (blocks). */
int lbm_ensemble_info(lbm_ensemble e, long long *nodes, int *tiles, int *grid);
/* Initial condition of every instance (Eq. 40) from the packed phi array. */
int lbm_ensemble_set_phi(lbm_ensemble e, const void *dev_phi, int prec, void *stream);
/* Persistent launches advance 1 (default) or 2 time steps each; with 2, every
   launch runs a two-step shared-memory tile routine on the tiles of all
   instances (two steps per sweep through HBM). Set before capturing a graph. */
int lbm_ensemble_configure(lbm_ensemble e, int steps_per_pass);
/* Grid of the two-step launches: persistent = 0 (default) launches one block
   per tile of the union tile list (all instances in one launch, the hardware
   scheduler balancing the blocks); persistent = 1 launches SMs x resident
   blocks that walk the list with a fixed stride; persistent = 2 launches the
   same grid, each block claiming the next tile from a counter in the workspace
   when it finishes one (no device-side waits; the last block to leave resets
   the counter, so launches on one stream and graph replays each start from
   zero; launches of one ensemble must not overlap). The two-step lists hold the
   largest instances' tiles first. One-step launches always use the persistent
   grid over their 32 x 8 tiles (faster for tiles that small). Set before
   capturing a graph. Results are identical bit for bit in every mode. */
int lbm_ensemble_set_persistent(lbm_ensemble e, int persistent);
/* Tiles of the two-step launches: pair_tiles = 0 (default) 30 x 30 output tiles
   with one node per thread, 1 62 x 14 output tiles with two x-adjacent nodes
   per thread (paired loads and stores; the routine of kernel_variant 5). The
   results are identical bit for bit. Set before capturing a graph. */
int lbm_ensemble_set_tiles(lbm_ensemble e, int pair_tiles);
/* nsteps time steps; mode 0: one launch over all tiles per step (two steps per
   launch when configured, an odd remainder with one); mode 1: one launch per
   instance per step (one-step arithmetic, for comparison). */
int lbm_ensemble_step(lbm_ensemble e, int nsteps, int mode, void *stream);
/* Capture nsteps persistent steps (a positive multiple of 2 * steps per
   launch) on a non-default stream into a CUDA graph held by the ensemble;
   lbm_ensemble_replay launches it (advancing the state by nsteps). */
int lbm_ensemble_capture(lbm_ensemble e, int nsteps, void *stream);
int lbm_ensemble_replay(lbm_ensemble e, void *stream);
/* phi(t_n) of every instance into the packed array dev_out. */
int lbm_ensemble_get_phi(lbm_ensemble e, void *dev_out, int prec, void *stream);
/* The statistics of lbm_reduce (Eq. 39 and norms) for every instance: dev_ref
   is the packed FP64 reference (one value per node, lbm_ensemble_get_phi's
   order) or NULL; dev_out receives count x 8 doubles on the device, instance
   i's eight at dev_out[8 i], in lbm_reduce's order and meaning, phi(t_n) being
   the FP32 value lbm_ensemble_get_phi returns. FP64, summed in a fixed order
   (per 32 x 8 tile, then the tiles in order): bit-reproducible. Asynchronous;
   uses a scratch area of the ensemble's workspace, so calls on different
   streams must not overlap. */
int lbm_ensemble_reduce(lbm_ensemble e, const double *dev_ref, double *dev_out, void *stream);
/* Index-fault word of checked builds (see lbm_debug_flags); synchronises. */
int lbm_ensemble_debug_flags(lbm_ensemble e, int *flags, void *stream);

/* The reductions of lbm_reduce over a caller-given field, for callers that
   cannot allocate device memory (the paper has no counterpart: this serves
   programs whose host application owns the whole device memory pool, or that
   may not call cudaMalloc/cudaFree because those calls synchronise the device,
   and so cannot provide a solver workspace).
   dev_phi: n doubles on the device; dev_ref: n doubles or NULL; dev_out: 8
   doubles on the device, same meaning as lbm_reduce's. n <= 67,108,864.
   No device memory is allocated: the partial sums use a fixed 512 KiB array in
   the library's device image, present on every device that loads the library
   until the process exits. The first call on a device looks up that array's
   address (cudaGetSymbolAddress) with the device current; make the first call
   on each device before any stream capture. The address is kept per device
   ordinal for the life of the process and is valid only in the context that was
   current at that first call: cudaDeviceReset, or making another context current
   for the device through the driver API, is not supported afterwards. All calls
   share the array, so calls whose kernels overlap on the GPU race: order them on
   one stream. Returns LBM_EINVAL for n < 1, n > 67,108,864 or a null field or
   output, and LBM_EUNSUPPORTED on a device ordinal of 64 or more. */
int lbm_reduce_field_noalloc(const double *dev_phi, const double *dev_ref, long long n, double *dev_out,
                             void *stream);

/* Thread-local message of the last failing call on this thread. */
const char *lbm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
