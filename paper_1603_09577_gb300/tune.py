"""Autotuner of the launch configuration of one lattice.

For a problem (grid, storage precision, walls, coefficient family) it times the
candidate configurations on the current device -- kernel variant (one node or
four x-adjacent nodes per thread), rows per thread block, one or two time steps
per sweep through memory (shared-memory tiles of one or two nodes per thread,
the register column march with 16 to 128 rows per warp, the TMA-staged tile) --
on a synthetic field, and
keeps the fastest in a JSON cache keyed by device name and problem, so later
runs reuse it. Problems on the general path (Scheme A, extrapolated walls, the
power-law flux, the tensor diffusion function) choose between the general
one-step kernel (rows per block) and the general two-step tile kernel.

    cfg = tune(4096, 4096, "f32", bc=("abb", "abb"), conv=0, diff=2)
    s = Solver(4096, 4096, prec="f32", bc=("abb", "abb"), **cfg)

For a batched ensemble, tune_ensemble chooses the two-step launch: the tile
shape (30 x 30 nodes, or 62 x 14 with two nodes per thread) and the grid (one
block per tile, or a persistent grid walking the tiles with a fixed stride or
claiming them from a counter), keyed by the instances' sizes and family:

    cfg = tune_ensemble(instances, conv=0, diff=1)
    e = Ensemble(instances, steps_per_pass=2, **cfg)
"""
from __future__ import annotations

import hashlib
import json
import os
import threading

import torch

from .solver import Solver

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("LBM_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "lbm_gb300", "tune.json"))


def _key(nx, ny, prec, bc, conv, diff, per_cell_K, scheme="B"):
    dev = torch.cuda.get_device_name()
    return f"{dev}|{nx}x{ny}|{prec}|{bc[0]},{bc[1]}|c{conv}d{diff}|K{int(per_cell_K)}|s{scheme}"


def _general(bc, conv, diff, scheme) -> bool:
    return scheme == "A" or "nee" in bc or conv >= 2 or diff == 3


def general_candidates(prec: str, per_cell_K: bool):
    """The general kernels: one node per thread (rows per block), and for FP32
    with constant K the two-step tile kernel."""
    out = [dict(kernel_variant=1, block_rows=b, steps_per_pass=1) for b in (1, 2, 4, 8)]
    if prec == "f32" and not per_cell_K:
        out.append(dict(kernel_variant=0, block_rows=0, steps_per_pass=2))
    return out


def candidates(nx: int, prec: str):
    out = [dict(kernel_variant=1, block_rows=b, steps_per_pass=1) for b in (1, 2, 4, 8)]
    if prec != "f64" and nx % 4 == 0:
        out += [dict(kernel_variant=2, block_rows=b, steps_per_pass=1) for b in (1, 2, 4, 8)]
    if prec != "f64":
        out.append(dict(kernel_variant=0, block_rows=0, steps_per_pass=2))
        out.append(dict(kernel_variant=0, block_rows=4, steps_per_pass=2))
        out += [dict(kernel_variant=5, block_rows=b, steps_per_pass=2) for b in (0, 2, 4)]
        out += [dict(kernel_variant=3, block_rows=b, steps_per_pass=2) for b in (1, 2, 4, 8)]
    if prec == "f32":
        out.append(dict(kernel_variant=4, block_rows=0, steps_per_pass=2))
    return out


def _time(cfg, nx, ny, prec, bc, conv, diff, per_cell_K, steps, reps, scheme="B"):
    s = Solver(nx, ny, prec=prec, bc=bc, per_cell_K=per_cell_K, scheme=scheme, **cfg)
    s.set_coeffs(conv=conv, u=(0.02, 0.01), diff=diff, K=(0.02, 0.004, 0.015), power=1)
    if "nee" in bc:
        s.set_dirichlet(torch.full((1, 2 * (nx + ny)), 0.5, dtype=torch.float64, device="cuda"))
    if per_cell_K:
        K = torch.zeros((3, ny, nx), dtype=torch.float64, device="cuda")
        K[0] = 0.02
        K[2] = 0.015
        s.set_K_field(K)
    g = torch.Generator(device="cuda").manual_seed(0)
    phi0 = 0.5 + 0.1 * torch.rand((ny, nx), generator=g, device="cuda", dtype=torch.float64)
    s.set_phi(phi0)
    st = torch.cuda.current_stream()
    s.step(steps)                                    # warm-up
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        s.step(steps)
        b.record(st)
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b) / steps)
    del s
    return best


def tune(nx: int, ny: int, prec: str = "f32", bc=("periodic", "periodic"), conv: int = 0, diff: int = 0,
         per_cell_K: bool = False, steps: int = 20, reps: int = 3, use_cache: bool = True, scheme: str = "B") -> dict:
    """Fastest launch configuration (kwargs for Solver) for this problem. Problems
    on the general path (Scheme A, extrapolated walls, conv 2, diff 3) choose
    among the general kernels."""
    key = _key(nx, ny, prec, bc, conv, diff, per_cell_K, scheme)
    path = cache_path()
    with _lock:
        cache = {}
        if use_cache and os.path.exists(path):
            try:
                with open(path) as f:
                    cache = json.load(f)
            except (OSError, ValueError):
                cache = {}
        if use_cache and key in cache:
            return dict(cache[key]["config"])
        timings = []
        cands = (general_candidates(prec, per_cell_K) if _general(bc, conv, diff, scheme)
                 else candidates(nx, prec))
        for cfg in cands:
            ms = _time(cfg, nx, ny, prec, bc, conv, diff, per_cell_K, steps, reps, scheme)
            timings.append((ms, cfg))
        ms, best = min(timings, key=lambda t: t[0])
        cache[key] = {"config": best, "ms_per_step": ms,
                      "all": [{"config": c, "ms_per_step": t} for t, c in timings]}
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, path)
        return dict(best)


def ensemble_candidates():
    """Two-step ensemble launches: tile shape x grid (0 one block per tile, 1
    persistent with a fixed stride, 2 persistent claiming tiles)."""
    return [dict(pair_tiles=pt, persistent=m) for pt in (False, True) for m in (0, 1, 2)]


def _ensemble_key(instances, conv, diff):
    sig = hashlib.sha256(json.dumps([[int(d["nx"]), int(d["ny"])] for d in instances]).encode()).hexdigest()[:16]
    dev = torch.cuda.get_device_name()
    return f"{dev}|ensemble|{len(instances)}|{sig}|c{conv}d{diff}"


def _load(path):
    if os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f)
        except (OSError, ValueError):
            pass
    return {}


def _save(path, cache):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, path)


def tune_ensemble(instances, conv: int = 0, diff: int = 1, steps: int = 20, reps: int = 3,
                  use_cache: bool = True) -> dict:
    """Fastest two-step launch (kwargs pair_tiles, persistent for Ensemble) for
    these instances; every candidate computes the same state bit for bit."""
    from .ensemble import Ensemble
    key = _ensemble_key(instances, conv, diff)
    path = cache_path()
    with _lock:
        cache = _load(path) if use_cache else {}
        if use_cache and key in cache:
            return dict(cache[key]["config"])
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        timings = []
        with torch.cuda.stream(side):
            phi = None
            for cfg in ensemble_candidates():
                e = Ensemble(instances, conv=conv, diff=diff, steps_per_pass=2, **cfg)
                if phi is None:
                    g = torch.Generator(device="cuda").manual_seed(0)
                    phi = 0.5 + 0.1 * torch.rand(e.nodes, generator=g, device="cuda", dtype=torch.float32)
                e.set_phi(phi)
                e.step(steps)                                # warm-up
                best = float("inf")
                for _ in range(reps):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(side)
                    e.step(steps)
                    b.record(side)
                    b.synchronize()
                    best = min(best, a.elapsed_time(b) / steps)
                timings.append((best, cfg))
                del e
        torch.cuda.current_stream().wait_stream(side)
        ms, best = min(timings, key=lambda t: t[0])
        cache[key] = {"config": best, "ms_per_step": ms,
                      "all": [{"config": c, "ms_per_step": t} for t, c in timings]}
        _save(path, cache)
        return dict(best)
