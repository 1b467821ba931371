// lbm_ensemble.h -- internal state of a batched ensemble of independent lattices.
#pragma once

#include "lbm_internal.h"

namespace lbm {

constexpr int kEnsTile = 32;        // tile width (nodes along x)
constexpr int kEnsRows = 8;         // tile height: one node per thread
constexpr int kEnsThreads = kEnsTile * kEnsRows;

// Per-instance data read by the kernels (device table).
struct __align__(16) EnsInst {
    float *pop[2];          // A/B population buffers (9 planes each)
    long long pitch, plane;
    long long phi_off;      // offset of this instance in the packed phi arrays
    int nx, ny;
    float A3, A35, A5;
    float se1, se2, sq4, sq6, sp7, sp8, he1, he2, hq4, hq6;   // prescaled collision factors (Params)
    float a3s, a35s, a5s, c3s, c35s, c5s;
    float ux, uy, uxx, uxy, uyy;
    float s1, s2, s4, s6, s7, s8, h1, h2, h4, h6;
    int *err;               // checked builds: shared index-fault word
};

__device__ __forceinline__ Params<float> ens_params(const EnsInst &I)
{
    Params<float> p;
    p.nx = I.nx; p.ny = I.ny; p.pitch = I.pitch; p.plane = I.plane;
    p.abb_x = 0; p.abb_y = 0;
    p.s1 = I.s1; p.s2 = I.s2; p.s4 = I.s4; p.s6 = I.s6; p.s7 = I.s7; p.s8 = I.s8;
    p.h1 = I.h1; p.h2 = I.h2; p.h4 = I.h4; p.h6 = I.h6;
    p.A3 = I.A3; p.A35 = I.A35; p.A5 = I.A5;
    p.se1 = I.se1; p.se2 = I.se2; p.sq4 = I.sq4; p.sq6 = I.sq6; p.sp7 = I.sp7; p.sp8 = I.sp8;
    p.he1 = I.he1; p.he2 = I.he2; p.hq4 = I.hq4; p.hq6 = I.hq6;
    p.a3s = I.a3s; p.a35s = I.a35s; p.a5s = I.a5s; p.c3s = I.c3s; p.c35s = I.c35s; p.c5s = I.c5s;
    p.ux = I.ux; p.uy = I.uy; p.uxx = I.uxx; p.uxy = I.uxy; p.uyy = I.uyy;
    p.r0 = 0.f; p.r1 = 0.f; p.half_r0 = 0.f; p.inv_den = 1.f; p.inv_post = 1.f;
    p.has_src = 0;
    for (int i = 0; i < 4; ++i) p.phi_wall[i] = 0.f;
    p.Afield = nullptr;
    p.err = I.err;
    return p;
}

}  // namespace lbm

struct lbm_ensemble_s {
    int count = 0, family = 0, ntiles = 0, grid = 0, parity = 0;
    int spp = 1;                    // time steps per persistent launch (1 or 2)
    int ntiles2 = 0, grid2 = 0;     // 30 x 30 tiles of the two-step kernel
    int ntiles2p = 0, grid2p = 0;   // 62 x 14 pair tiles of the two-step kernel
    int shape2 = 0;                 // two-step tiles: 0 30 x 30 (one node per thread), 1 62 x 14 (two)
    int persistent2 = 0;            // two-step launch: 0 a block per tile, 1 persistent with a fixed
                                    // stride, 2 persistent with tiles claimed from a counter
    int4 *d_tiles2 = nullptr;
    int4 *d_tiles2p = nullptr;
    int *d_claim = nullptr;         // tile counter and departed-block counter of mode 2
    lbm::EnsInst *d_inst = nullptr;
    int4 *d_tiles = nullptr;
    int *tile_begin = nullptr;      // host: first tile of each instance (count + 1)
    long long total_nodes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_steps = 0, graph_parity = 0;
    int *err = nullptr;             // index-fault word of checked builds
    double *partials = nullptr;     // per-tile statistics (8 doubles per 32 x 8 tile)
    int *d_tile_begin = nullptr;    // device copy of tile_begin
};

namespace lbm {
cudaError_t ens_launch_step(const lbm_ensemble_s *e, int t_begin, int t_end, int blocks, cudaStream_t st);
cudaError_t ens_launch_step2(const lbm_ensemble_s *e, cudaStream_t st);
int ens2_occupancy_blocks(int family, int shape);
constexpr int kEns2Tile = 30;       // two-step tiles: 30 x 30 outputs
constexpr int kEns2PCols = 62;      // two-step pair tiles: 62 x 14 outputs
constexpr int kEns2PRows = 14;
cudaError_t ens_launch_init(const lbm_ensemble_s *e, const void *phi, int in_prec, cudaStream_t st);
cudaError_t ens_launch_get_phi(const lbm_ensemble_s *e, void *out, int out_prec, cudaStream_t st);
// the eight statistics of every instance into out (count x 8 doubles)
cudaError_t ens_launch_reduce(const lbm_ensemble_s *e, const double *ref, double *out, cudaStream_t st);
int ens_occupancy_blocks(int family);
}  // namespace lbm
