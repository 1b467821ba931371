"""A batched ensemble of independent lattices (see lbm.h): torch supplies the
workspace and streams, liblbm runs every step."""
from __future__ import annotations

import ctypes

import torch

from . import _lib as C
from .solver import REDUCE_KEYS, _prec_of, _ptr, _stream


class Ensemble:
    """instances: list of dicts with nx, ny, u (2), K (3) and optionally s (9
    rates; default `s`); the coefficient family (conv, diff) is shared."""

    def __init__(self, instances, conv=0, diff=1, s=(1.0, 1.2, 1.2, 0.0, 1.0, 0.0, 1.0, 1.1, 1.1), device=None,
                 steps_per_pass: int = 1, persistent: int = 0, pair_tiles: bool = False):
        self.lib = C.lib()
        self.device = torch.device(device if device is not None else "cuda")
        n = len(instances)
        self.sizes = [(int(d["nx"]), int(d["ny"])) for d in instances]
        self.nx = (ctypes.c_int * n)(*[a for a, _ in self.sizes])
        self.ny = (ctypes.c_int * n)(*[b for _, b in self.sizes])
        co = (C.Coeffs * n)()
        for i, d in enumerate(instances):
            co[i].conv, co[i].diff = int(conv), int(diff)
            co[i].u[:] = [float(v) for v in d["u"]]
            co[i].K[:] = [float(v) for v in d["K"]]
            co[i].s[:] = [float(v) for v in d.get("s", s)]
            co[i].r0 = co[i].r1 = 0.0
        self.coeffs = co
        size = ctypes.c_size_t()
        C.check(self.lib.lbm_ensemble_workspace_size(n, self.nx, self.ny, ctypes.byref(size)))
        self.workspace = torch.empty(size.value, dtype=torch.uint8, device=self.device)
        self.h = ctypes.c_void_p()
        C.check(self.lib.lbm_ensemble_create(ctypes.byref(self.h), n, self.nx, self.ny, co, _ptr(self.workspace),
                                             size.value, _stream()))
        C.check(self.lib.lbm_ensemble_configure(self.h, int(steps_per_pass)))
        # two-step launches: one block per tile (0, default), a persistent grid
        # walking the tiles with a fixed stride (1) or claiming them (2); tiles of
        # 30 x 30 nodes, or 62 x 14 with two nodes per thread (pair_tiles)
        C.check(self.lib.lbm_ensemble_set_persistent(self.h, int(persistent)))
        C.check(self.lib.lbm_ensemble_set_tiles(self.h, int(bool(pair_tiles))))
        self.persistent, self.pair_tiles = int(persistent), bool(pair_tiles)
        self.steps_per_pass = int(steps_per_pass)
        nodes, tiles, grid = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_int()
        C.check(self.lib.lbm_ensemble_info(self.h, ctypes.byref(nodes), ctypes.byref(tiles), ctypes.byref(grid)))
        self.nodes, self.tiles, self.grid = nodes.value, tiles.value, grid.value
        self.offsets = [0]
        for a, b in self.sizes:
            self.offsets.append(self.offsets[-1] + a * b)

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            try:
                self.lib.lbm_ensemble_destroy(h)
            except Exception:
                pass
            self.h = None

    def pack(self, fields, dtype=torch.float64) -> torch.Tensor:
        return torch.cat([torch.as_tensor(f, dtype=dtype).reshape(-1) for f in fields]).to(self.device)

    def unpack(self, flat: torch.Tensor):
        return [flat[self.offsets[i]:self.offsets[i + 1]].reshape(b, a) for i, (a, b) in enumerate(self.sizes)]

    def set_phi(self, packed: torch.Tensor, stream=None):
        assert packed.is_cuda and packed.numel() == self.nodes and packed.is_contiguous()
        C.check(self.lib.lbm_ensemble_set_phi(self.h, _ptr(packed), _prec_of(packed), _stream(stream)))
        return self

    def step(self, n: int = 1, mode: int = 0, stream=None):
        C.check(self.lib.lbm_ensemble_step(self.h, int(n), int(mode), _stream(stream)))
        return self

    def capture(self, n: int, stream=None):
        C.check(self.lib.lbm_ensemble_capture(self.h, int(n), _stream(stream)))
        return self

    def replay(self, stream=None):
        C.check(self.lib.lbm_ensemble_replay(self.h, _stream(stream)))
        return self

    def phi(self, dtype=torch.float64, stream=None) -> torch.Tensor:
        out = torch.empty(self.nodes, dtype=dtype, device=self.device)
        C.check(self.lib.lbm_ensemble_get_phi(self.h, _ptr(out), _prec_of(out), _stream(stream)))
        return out

    def reduce_async(self, ref: torch.Tensor | None = None, out: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
        """Per-instance statistics (sum, abs_err, abs_ref, sq_err, sq_ref, max_abs,
        nonfinite, sum_sq) as a (count, 8) float64 tensor on the device; ref: the
        packed reference field (FP64) or None."""
        if out is None:
            out = torch.empty((len(self.sizes), 8), dtype=torch.float64, device=self.device)
        assert out.is_cuda and out.dtype == torch.float64 and out.is_contiguous() and out.numel() == 8 * len(self.sizes)
        if ref is not None:
            ref = ref.to(device=self.device, dtype=torch.float64).contiguous()
            assert ref.numel() == self.nodes
            self._ref = ref
        C.check(self.lib.lbm_ensemble_reduce(self.h, _ptr(ref) if ref is not None else None, _ptr(out),
                                             _stream(stream)))
        return out

    def reduce(self, ref: torch.Tensor | None = None) -> list[dict]:
        """reduce_async, read back: one dict per instance (keys of Solver.reduce)."""
        return [dict(zip(REDUCE_KEYS, row)) for row in self.reduce_async(ref).cpu().tolist()]


def shard(instances, rank: int, world: int) -> list[int]:
    """Indices of the instances that rank `rank` of `world` runs when an ensemble
    is split across GPUs (instances are independent: no exchange between ranks).
    Largest instances first, each to the rank with the fewest nodes so far, so
    every rank gets nearly the same number of node updates per step; the result
    is deterministic and the ranks' lists partition range(len(instances))."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    order = sorted(range(len(instances)), key=lambda i: (-instances[i]["nx"] * instances[i]["ny"], i))
    load = [0] * world
    mine = []
    for i in order:
        r = min(range(world), key=lambda j: (load[j], j))
        load[r] += instances[i]["nx"] * instances[i]["ny"]
        if r == rank:
            mine.append(i)
    return sorted(mine)
