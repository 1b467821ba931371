// ensemble_api.cu -- extern "C" entry points of the batched ensemble: layout of
// the caller's workspace, the tile work list, persistent or per-instance
// launches, and CUDA-graph capture / replay of many persistent steps.
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "lbm_ensemble.h"

namespace lbm {
namespace {

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

struct EnsLayout {
    size_t off_inst = 0, off_tiles = 0, off_tiles2 = 0, off_tiles2p = 0, off_err = 0, off_partials = 0, off_tbegin = 0,
           total = 0;
    int ntiles = 0, ntiles2 = 0, ntiles2p = 0;
    std::vector<size_t> off_pop;    // per instance: buffer A offset (B follows)
    std::vector<long long> pitch;
};

int ens_layout(int count, const int *nx, const int *ny, EnsLayout *L)
{
    if (count < 1) return fail(LBM_EINVAL, "ensemble count must be >= 1");
    if (!nx || !ny) return fail(LBM_EINVAL, "null size arrays");
    long long tiles = 0, tiles2 = 0, tiles2p = 0;
    for (int i = 0; i < count; ++i) {
        if (nx[i] < 2 || ny[i] < 2) return fail(LBM_EINVAL, "instance " + std::to_string(i) + ": nx and ny must be >= 2");
        tiles += (long long)((nx[i] + kEnsTile - 1) / kEnsTile) * ((ny[i] + kEnsRows - 1) / kEnsRows);
        tiles2 += (long long)((nx[i] + kEns2Tile - 1) / kEns2Tile) * ((ny[i] + kEns2Tile - 1) / kEns2Tile);
        tiles2p += (long long)((nx[i] + kEns2PCols - 1) / kEns2PCols) * ((ny[i] + kEns2PRows - 1) / kEns2PRows);
    }
    if (tiles > (1LL << 30)) return fail(LBM_EINVAL, "too many tiles");
    L->ntiles = (int)tiles;
    L->ntiles2 = (int)tiles2;
    L->ntiles2p = (int)tiles2p;
    size_t off = 0;
    L->off_inst = off;
    off += up256(sizeof(EnsInst) * (size_t)count);
    L->off_tiles = off;
    off += up256(sizeof(int4) * (size_t)tiles);
    L->off_tiles2 = off;
    off += up256(sizeof(int4) * (size_t)tiles2);
    L->off_tiles2p = off;
    off += up256(sizeof(int4) * (size_t)tiles2p);
    L->off_err = off;                   // error word at +0, tile-claim counters at +128
    off += 256;
    L->off_partials = off;
    off += up256(8 * sizeof(double) * (size_t)tiles);
    L->off_tbegin = off;
    off += up256(sizeof(int) * ((size_t)count + 1));
    L->off_pop.resize(count);
    L->pitch.resize(count);
    for (int i = 0; i < count; ++i) {
        L->pitch[i] = ((long long)nx[i] + kPitchAlign - 1) / kPitchAlign * kPitchAlign;
        L->off_pop[i] = off;
        off += 2 * up256(9 * (size_t)L->pitch[i] * ny[i] * sizeof(float));
    }
    L->total = off;
    return LBM_OK;
}

bool relax_block_k(const double K[3], double *A3, double *A35, double *A5)
{
    if (!(K[0] > 0.0) || !(K[0] * K[2] - K[1] * K[1] > 0.0)) return false;
    const double a = 3.0 * K[0] + 0.5, b = 3.0 * K[1], c = 3.0 * K[2] + 0.5, det = a * c - b * b;
    *A3 = c / det;
    *A35 = -b / det;
    *A5 = a / det;
    return true;
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" {

int lbm_ensemble_workspace_size(int count, const int *nx, const int *ny, size_t *bytes)
{
    if (!bytes) return fail(LBM_EINVAL, "null size pointer");
    EnsLayout L;
    if (int rc = ens_layout(count, nx, ny, &L)) return rc;
    *bytes = L.total;
    return LBM_OK;
}

int lbm_ensemble_create(lbm_ensemble *out, int count, const int *nx, const int *ny, const lbm_coeffs *coeffs,
                        void *dev_ws, size_t bytes, void *stream)
{
    if (!out) return fail(LBM_EINVAL, "null ensemble pointer");
    *out = nullptr;
    EnsLayout L;
    if (int rc = ens_layout(count, nx, ny, &L)) return rc;
    if (!coeffs) return fail(LBM_EINVAL, "null coefficient array");
    if (!dev_ws || ((uintptr_t)dev_ws & 255) != 0) return fail(LBM_EINVAL, "workspace null or not 256-byte aligned");
    if (bytes < L.total) return fail(LBM_EINVAL, "workspace smaller than lbm_ensemble_workspace_size");
    const lbm_coeffs &c0 = coeffs[0];
    if (c0.conv < 0 || c0.conv > 1 || c0.diff < 0 || c0.diff > 2) return fail(LBM_EINVAL, "unknown coefficient family");
    std::vector<EnsInst> inst(count);
    char *ws = (char *)dev_ws;
    for (int i = 0; i < count; ++i) {
        const lbm_coeffs &c = coeffs[i];
        if (c.conv != c0.conv || c.diff != c0.diff)
            return fail(LBM_EINVAL, "every instance must use the same coefficient family");
        for (int j = 1; j < 9; ++j)
            if (j != 3 && j != 5 && !(c.s[j] > 0.0 && c.s[j] < 2.0))
                return fail(LBM_EINVAL, "instance " + std::to_string(i) + ": relaxation rates must lie in (0, 2)");
        if (c.cfree) return fail(LBM_EUNSUPPORTED, "ensemble instances use the exact-C equilibrium");
        if (c.r0 != 0.0 || c.r1 != 0.0 || c.src_family != 0)
            return fail(LBM_EUNSUPPORTED, "ensemble instances carry no source term");
        double A3, A35, A5;
        if (!relax_block_k(c.K, &A3, &A35, &A5))
            return fail(LBM_EINVAL, "instance " + std::to_string(i) + ": K is not symmetric positive definite");
        EnsInst &I = inst[i];
        const size_t half = up256(9 * (size_t)L.pitch[i] * ny[i] * sizeof(float));
        I.pop[0] = (float *)(ws + L.off_pop[i]);
        I.pop[1] = (float *)(ws + L.off_pop[i] + half);
        I.pitch = L.pitch[i];
        I.plane = L.pitch[i] * ny[i];
        I.nx = nx[i];
        I.ny = ny[i];
        I.A3 = (float)A3; I.A35 = (float)A35; I.A5 = (float)A5;
        {
            Params<float> sc;
            set_scaled_rates<float>(c.s, A3, A35, A5, &sc);
            I.se1 = sc.se1; I.se2 = sc.se2; I.sq4 = sc.sq4; I.sq6 = sc.sq6; I.sp7 = sc.sp7; I.sp8 = sc.sp8;
            I.he1 = sc.he1; I.he2 = sc.he2; I.hq4 = sc.hq4; I.hq6 = sc.hq6;
            I.a3s = sc.a3s; I.a35s = sc.a35s; I.a5s = sc.a5s; I.c3s = sc.c3s; I.c35s = sc.c35s; I.c5s = sc.c5s;
        }
        I.ux = (float)c.u[0]; I.uy = (float)c.u[1];
        I.uxx = (float)(c.u[0] * c.u[0]); I.uxy = (float)(c.u[0] * c.u[1]); I.uyy = (float)(c.u[1] * c.u[1]);
        I.s1 = (float)c.s[1]; I.s2 = (float)c.s[2]; I.s4 = (float)c.s[4];
        I.s6 = (float)c.s[6]; I.s7 = (float)c.s[7]; I.s8 = (float)c.s[8];
        I.h1 = (float)(1.0 - 0.5 * c.s[1]); I.h2 = (float)(1.0 - 0.5 * c.s[2]);
        I.h4 = (float)(1.0 - 0.5 * c.s[4]); I.h6 = (float)(1.0 - 0.5 * c.s[6]);
        I.err = (int *)(ws + L.off_err);
    }
    lbm_ensemble_s *e = new (std::nothrow) lbm_ensemble_s();
    if (!e) return fail(LBM_EINVAL, "out of host memory");
    e->count = count;
    e->family = c0.conv * 3 + c0.diff;
    e->ntiles = L.ntiles;
    e->tile_begin = new (std::nothrow) int[count + 1];
    if (!e->tile_begin) {
        delete e;
        return fail(LBM_EINVAL, "out of host memory");
    }
    std::vector<int4> tiles;
    tiles.reserve(L.ntiles);
    long long phi_off = 0;
    for (int i = 0; i < count; ++i) {
        e->tile_begin[i] = (int)tiles.size();
        inst[i].phi_off = phi_off;
        phi_off += (long long)nx[i] * ny[i];
        for (int ty = 0; ty < ny[i]; ty += kEnsRows)
            for (int tx = 0; tx < nx[i]; tx += kEnsTile) tiles.push_back(make_int4(i, tx, ty, 0));
    }
    e->tile_begin[count] = (int)tiles.size();
    e->total_nodes = phi_off;
    // two-step tile lists: largest instances first (the small instances' tiles,
    // all along their wrapped edges, then fill the end of a launch), each
    // instance's tiles row by row
    std::vector<int> by_size(count);
    for (int i = 0; i < count; ++i) by_size[i] = i;
    std::stable_sort(by_size.begin(), by_size.end(), [&](int a, int b) {
        return (long long)nx[a] * ny[a] > (long long)nx[b] * ny[b];
    });
    std::vector<int4> tiles2, tiles2p;
    tiles2.reserve(L.ntiles2);
    tiles2p.reserve(L.ntiles2p);
    for (int i : by_size) {
        for (int ty = 0; ty < ny[i]; ty += kEns2Tile)
            for (int tx = 0; tx < nx[i]; tx += kEns2Tile) tiles2.push_back(make_int4(i, tx, ty, 0));
        for (int ty = 0; ty < ny[i]; ty += kEns2PRows)
            for (int tx = 0; tx < nx[i]; tx += kEns2PCols) tiles2p.push_back(make_int4(i, tx, ty, 0));
    }
    e->ntiles2 = (int)tiles2.size();
    e->d_tiles2 = (int4 *)(ws + L.off_tiles2);
    e->ntiles2p = (int)tiles2p.size();
    e->d_tiles2p = (int4 *)(ws + L.off_tiles2p);
    e->d_claim = (int *)(ws + L.off_err + 128);
    e->d_inst = (EnsInst *)(ws + L.off_inst);
    e->d_tiles = (int4 *)(ws + L.off_tiles);
    e->err = (int *)(ws + L.off_err);
    e->partials = (double *)(ws + L.off_partials);
    e->d_tile_begin = (int *)(ws + L.off_tbegin);
    // the tables go through the caller's stream; the call waits for that stream
    // alone, so the host vectors may go and the tables are in place on return
    cudaStream_t st = (cudaStream_t)stream;
    int rc = cuda_check(cudaMemcpyAsync(e->d_inst, inst.data(), sizeof(EnsInst) * count, cudaMemcpyHostToDevice, st),
                        "lbm_ensemble_create instance table");
    if (!rc) rc = cuda_check(cudaMemcpyAsync(e->d_tiles2, tiles2.data(), sizeof(int4) * tiles2.size(),
                                             cudaMemcpyHostToDevice, st), "lbm_ensemble_create two-step tile table");
    if (!rc) rc = cuda_check(cudaMemcpyAsync(e->d_tiles2p, tiles2p.data(), sizeof(int4) * tiles2p.size(),
                                             cudaMemcpyHostToDevice, st), "lbm_ensemble_create pair tile table");
    if (!rc) rc = cuda_check(cudaMemsetAsync(e->err, 0, 256, st), "lbm_ensemble_create error word and counters");
    if (!rc) rc = cuda_check(cudaMemcpyAsync(e->d_tiles, tiles.data(), sizeof(int4) * tiles.size(),
                                             cudaMemcpyHostToDevice, st), "lbm_ensemble_create tile table");
    if (!rc) rc = cuda_check(cudaMemcpyAsync(e->d_tile_begin, e->tile_begin, sizeof(int) * ((size_t)count + 1),
                                             cudaMemcpyHostToDevice, st), "lbm_ensemble_create tile offsets");
    if (!rc) rc = cuda_check(cudaStreamSynchronize(st), "lbm_ensemble_create: waiting for the table copies");
    int dev = 0, sms = 0;
    if (!rc) rc = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (!rc) rc = cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    const int per_sm = rc ? 0 : ens_occupancy_blocks(e->family);
    if (!rc && per_sm <= 0) rc = fail(LBM_ECUDA, "occupancy query failed");
    const int per_sm2 = rc ? 0 : ens2_occupancy_blocks(e->family, 0);
    if (!rc && per_sm2 <= 0) rc = fail(LBM_ECUDA, "occupancy query failed (two-step kernel)");
    const int per_sm2p = rc ? 0 : ens2_occupancy_blocks(e->family, 1);
    if (!rc && per_sm2p <= 0) rc = fail(LBM_ECUDA, "occupancy query failed (two-step pair kernel)");
    if (rc) {
        delete[] e->tile_begin;
        delete e;
        return rc;
    }
    e->grid = sms * per_sm;
    e->grid2 = sms * per_sm2;
    e->grid2p = sms * per_sm2p;
    *out = e;
    return LBM_OK;
}

int lbm_ensemble_destroy(lbm_ensemble e)
{
    if (!e) return LBM_OK;
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    delete[] e->tile_begin;
    delete e;
    return LBM_OK;
}

int lbm_ensemble_info(lbm_ensemble e, long long *nodes, int *tiles, int *grid)
{
    if (!e) return fail(LBM_EINVAL, "null ensemble");
    if (nodes) *nodes = e->total_nodes;
    if (tiles) *tiles = e->ntiles;
    if (grid) *grid = e->grid;
    return LBM_OK;
}

int lbm_ensemble_set_phi(lbm_ensemble e, const void *dev_phi, int prec, void *stream)
{
    if (!e || !dev_phi) return fail(LBM_EINVAL, "null ensemble or phi");
    if (prec != LBM_F64 && prec != LBM_F32) return fail(LBM_EINVAL, "phi must be LBM_F64 or LBM_F32");
    return cuda_check(ens_launch_init(e, dev_phi, prec, (cudaStream_t)stream), "lbm_ensemble_set_phi");
}

int lbm_ensemble_step(lbm_ensemble e, int nsteps, int mode, void *stream)
{
    if (!e) return fail(LBM_EINVAL, "null ensemble");
    if (nsteps < 0) return fail(LBM_EINVAL, "negative step count");
    if (mode != 0 && mode != 1) return fail(LBM_EINVAL, "mode must be 0 (persistent) or 1 (one launch per instance)");
    cudaStream_t st = (cudaStream_t)stream;
    int n = 0;
    if (mode == 0 && e->spp == 2)
        for (; n + 2 <= nsteps; n += 2) {
            if (int rc = cuda_check(ens_launch_step2(e, st), "lbm_ensemble_step (two steps per pass)")) return rc;
            e->parity ^= 1;
        }
    for (; n < nsteps; ++n) {
        if (mode == 0) {
            if (int rc = cuda_check(ens_launch_step(e, 0, e->ntiles, e->grid, st), "lbm_ensemble_step")) return rc;
        } else {
            for (int i = 0; i < e->count; ++i) {
                const int b = e->tile_begin[i], t = e->tile_begin[i + 1];
                if (int rc = cuda_check(ens_launch_step(e, b, t, t - b, st), "lbm_ensemble_step")) return rc;
            }
        }
        e->parity ^= 1;
    }
    return LBM_OK;
}

int lbm_ensemble_configure(lbm_ensemble e, int steps_per_pass)
{
    if (!e) return fail(LBM_EINVAL, "null ensemble");
    if (steps_per_pass != 1 && steps_per_pass != 2) return fail(LBM_EINVAL, "steps_per_pass must be 1 or 2");
    if (e->exec) return fail(LBM_EINVAL, "configure before capturing a graph");
    e->spp = steps_per_pass;
    return LBM_OK;
}

int lbm_ensemble_set_persistent(lbm_ensemble e, int persistent)
{
    if (!e) return fail(LBM_EINVAL, "null ensemble");
    if (persistent < 0 || persistent > 2) return fail(LBM_EINVAL, "persistent must be 0, 1 or 2");
    if (e->exec) return fail(LBM_EINVAL, "choose the grid before capturing a graph");
    e->persistent2 = persistent;
    return LBM_OK;
}

int lbm_ensemble_set_tiles(lbm_ensemble e, int pair_tiles)
{
    if (!e) return fail(LBM_EINVAL, "null ensemble");
    if (pair_tiles != 0 && pair_tiles != 1) return fail(LBM_EINVAL, "pair_tiles must be 0 or 1");
    if (e->exec) return fail(LBM_EINVAL, "choose the tiles before capturing a graph");
    e->shape2 = pair_tiles;
    return LBM_OK;
}

int lbm_ensemble_capture(lbm_ensemble e, int nsteps, void *stream)
{
    if (!e) return fail(LBM_EINVAL, "null ensemble");
    if (!stream) return fail(LBM_EINVAL, "capture needs a non-default stream");
    if (nsteps < 2 || nsteps % (2 * e->spp))
        return fail(LBM_EINVAL, "captured step count must be a positive multiple of 2 * steps per pass");
    cudaStream_t st = (cudaStream_t)stream;
    if (e->exec) { cudaGraphExecDestroy(e->exec); e->exec = nullptr; }
    if (e->graph) { cudaGraphDestroy(e->graph); e->graph = nullptr; }
    const int parity0 = e->parity;
    if (int rc = cuda_check(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture"))
        return rc;
    int rc = LBM_OK;
    for (int n = 0; n < nsteps && !rc; n += e->spp) {
        rc = cuda_check(e->spp == 2 ? ens_launch_step2(e, st) : ens_launch_step(e, 0, e->ntiles, e->grid, st),
                        "captured step");
        e->parity ^= 1;
    }
    cudaGraph_t g = nullptr;
    const int rc_end = cuda_check(cudaStreamEndCapture(st, &g), "cudaStreamEndCapture");
    e->parity = parity0;
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (rc_end) return rc_end;
    e->graph = g;
    if (int rc2 = cuda_check(cudaGraphInstantiate(&e->exec, g, 0), "cudaGraphInstantiate")) return rc2;
    e->graph_steps = nsteps;
    e->graph_parity = parity0;
    return LBM_OK;
}

int lbm_ensemble_replay(lbm_ensemble e, void *stream)
{
    if (!e || !e->exec) return fail(LBM_EINVAL, "no captured graph");
    if (e->parity != e->graph_parity) return fail(LBM_EINVAL, "state parity differs from the captured graph's");
    return cuda_check(cudaGraphLaunch(e->exec, (cudaStream_t)stream), "cudaGraphLaunch");
}

int lbm_ensemble_debug_flags(lbm_ensemble e, int *flags, void *stream)
{
    if (!e || !flags) return fail(LBM_EINVAL, "null ensemble or flags pointer");
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = cuda_check(cudaMemcpyAsync(flags, e->err, sizeof(int), cudaMemcpyDeviceToHost, st), "lbm_ensemble_debug_flags"))
        return rc;
    return cuda_check(cudaStreamSynchronize(st), "lbm_ensemble_debug_flags sync");
}

int lbm_ensemble_reduce(lbm_ensemble e, const double *dev_ref, double *dev_out, void *stream)
{
    if (!e || !dev_out) return fail(LBM_EINVAL, "null ensemble or output");
    return cuda_check(ens_launch_reduce(e, dev_ref, dev_out, (cudaStream_t)stream), "lbm_ensemble_reduce");
}

int lbm_ensemble_get_phi(lbm_ensemble e, void *dev_out, int prec, void *stream)
{
    if (!e || !dev_out) return fail(LBM_EINVAL, "null ensemble or output");
    if (prec != LBM_F64 && prec != LBM_F32) return fail(LBM_EINVAL, "output must be LBM_F64 or LBM_F32");
    return cuda_check(ens_launch_get_phi(e, dev_out, prec, (cudaStream_t)stream), "lbm_ensemble_get_phi");
}

}  // extern "C"
