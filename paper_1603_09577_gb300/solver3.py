"""Python front end of the D3Q19 lattice (include/lbm3.h): torch provides
device memory and streams, every computation runs in liblbm's CUDA kernels."""
from __future__ import annotations

import ctypes

import torch

from . import _lib as C
from .solver import REDUCE_KEYS, _prec_of, _ptr, _stream


class Solver3:
    """One D3Q19 lattice of nx x ny x nz nodes; fields are (nz, ny, nx).
    bc: per axis (x, y, z) "periodic" or "abb" (anti-bounce-back walls with the
    values phi_wall = (x-, x+, y-, y+, z-, z+))."""

    def __init__(self, nx: int, ny: int, nz: int, prec: str = "f32", block_rows: int = 0, device=None,
                 bc=("periodic", "periodic", "periodic"), phi_wall=(0.0,) * 6):
        from .solver import BC
        self.lib = C.lib()
        self.nx, self.ny, self.nz, self.prec = int(nx), int(ny), int(nz), prec
        self.device = torch.device(device if device is not None else "cuda")
        d = C.Desc3()
        d.nx, d.ny, d.nz, d.prec, d.block_rows = self.nx, self.ny, self.nz, C.PREC[prec], int(block_rows)
        d.bc[:] = [BC[b] for b in bc]
        d.phi_wall[:] = [float(v) for v in phi_wall]
        size = ctypes.c_size_t()
        C.check(self.lib.lbm3_workspace_size(ctypes.byref(d), ctypes.byref(size)))
        self.workspace = torch.empty(size.value, dtype=torch.uint8, device=self.device)
        self.h = ctypes.c_void_p()
        C.check(self.lib.lbm3_create(ctypes.byref(self.h), ctypes.byref(d), _ptr(self.workspace), size.value))
        self._out = torch.zeros(8, dtype=torch.float64, device=self.device)

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            try:
                self.lib.lbm3_destroy(h)
            except Exception:
                pass
            self.h = None

    def set_coeffs(self, conv: int = 0, u=(0.0, 0.0, 0.0), diff: int = 0, K=(0.0,) * 6, s0: float = 1.0,
                   se: float = 1.0, r0: float = 0.0, r1: float = 0.0):
        """K = (Kxx, Kxy, Kxz, Kyy, Kyz, Kzz); se: rate of every moment other than rho and j."""
        c = C.Coeffs3()
        c.conv, c.diff = int(conv), int(diff)
        c.u[:] = [float(v) for v in u]
        c.K[:] = [float(v) for v in K]
        c.s0, c.se, c.r0, c.r1 = float(s0), float(se), float(r0), float(r1)
        C.check(self.lib.lbm3_set_coeffs(self.h, ctypes.byref(c)))
        return self

    def set_phi(self, phi0: torch.Tensor, stream=None):
        assert phi0.shape == (self.nz, self.ny, self.nx) and phi0.is_cuda and phi0.is_contiguous()
        C.check(self.lib.lbm3_set_phi(self.h, _ptr(phi0), _prec_of(phi0), _stream(stream)))
        return self

    def step(self, n: int = 1, stream=None):
        C.check(self.lib.lbm3_step(self.h, int(n), _stream(stream)))
        return self

    # -- checkpoint / resume -------------------------------------------------------
    def state_bytes(self) -> int:
        n = ctypes.c_size_t()
        C.check(self.lib.lbm3_state_bytes(self.h, ctypes.byref(n)))
        return n.value

    def save(self, dst: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if dst is None:
            dst = torch.empty(self.state_bytes(), dtype=torch.uint8, device=self.device)
        assert dst.is_cuda and dst.numel() * dst.element_size() >= self.state_bytes()
        C.check(self.lib.lbm3_save(self.h, _ptr(dst), _stream(stream)))
        return dst

    def load(self, src: torch.Tensor, stream=None):
        assert src.is_cuda and src.numel() * src.element_size() >= self.state_bytes()
        C.check(self.lib.lbm3_load(self.h, _ptr(src), _stream(stream)))
        return self

    # -- CUDA graphs -------------------------------------------------------------
    def capture(self, nsteps: int):
        """Record nsteps (even, so that every replay ends on the buffer it
        started from) time steps into a CUDA graph; replay() relaunches them."""
        if nsteps < 2 or nsteps % 2:
            raise ValueError("capture needs an even number of steps")
        torch.cuda.current_stream().synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            C.check(self.lib.lbm3_step(self.h, int(nsteps), _stream()))
        self._graph, self._graph_steps = g, int(nsteps)
        return self

    def replay(self):
        self._graph.replay()
        return self

    def phi(self, dtype=torch.float64, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.nz, self.ny, self.nx), dtype=dtype, device=self.device)
        C.check(self.lib.lbm3_get_phi(self.h, _ptr(out), _prec_of(out), _stream(stream)))
        return out

    def reduce_async(self, ref: torch.Tensor | None = None, out: torch.Tensor | None = None, stream=None):
        out = self._out if out is None else out
        if ref is not None:
            ref = ref.to(device=self.device, dtype=torch.float64).contiguous()
            self._ref = ref
        C.check(self.lib.lbm3_reduce(self.h, _ptr(ref) if ref is not None else None, _ptr(out), _stream(stream)))
        return out

    def reduce(self, ref: torch.Tensor | None = None) -> dict:
        return dict(zip(REDUCE_KEYS, self.reduce_async(ref).cpu().tolist()))
