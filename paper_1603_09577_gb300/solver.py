"""Python front end of one lattice: torch provides device memory and streams,
every computation runs in liblbm's CUDA kernels.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as C

BC = {"periodic": C.LBM_PERIODIC, "abb": C.LBM_ABB, "nee": C.LBM_NEE,
      0: C.LBM_PERIODIC, 1: C.LBM_ABB, 2: C.LBM_NEE}
SCHEME = {"B": C.LBM_SCHEME_B, "A": C.LBM_SCHEME_A}
REDUCE_KEYS = ("sum", "abs_err", "abs_ref", "sq_err", "sq_ref", "max_abs", "nonfinite", "sum_sq")


def _stream(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _prec_of(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return C.LBM_F64
    if t.dtype == torch.float32:
        return C.LBM_F32
    raise TypeError("phi must be float64 or float32")


class Solver:
    """One D2Q9 lattice of nx x ny nodes (see include/lbm.h for the contract).

    prec: "f64", "f32" or "bf16s"; bc: (x, y) boundary kinds "periodic", "abb"
    (anti-bounce-back walls with the constant phi_wall values: west, east, south,
    north) or "nee" (extrapolated Dirichlet nodes, values from set_dirichlet);
    scheme: "B" (Eq. 34) or "A" (Remark II).
    """

    def __init__(self, nx: int, ny: int, prec: str = "f32", bc=("periodic", "periodic"),
                 phi_wall=(0.0, 0.0, 0.0, 0.0), steps_per_pass: int = 1, per_cell_K: bool = False,
                 kernel_variant: int = 0, block_rows: int = 0, scheme: str = "B", device=None):
        self.lib = C.lib()
        self.nx, self.ny, self.prec = int(nx), int(ny), prec
        self.device = torch.device(device if device is not None else "cuda")
        d = C.Desc()
        d.nx, d.ny, d.prec = self.nx, self.ny, C.PREC[prec]
        d.bc_x, d.bc_y = BC[bc[0]], BC[bc[1]]
        d.phi_wall[:] = [float(v) for v in phi_wall]
        d.steps_per_pass = int(steps_per_pass)
        d.per_cell_K = int(bool(per_cell_K))
        d.kernel_variant, d.block_rows = int(kernel_variant), int(block_rows)
        d.scheme = SCHEME[scheme]
        self.desc = d
        size = ctypes.c_size_t()
        C.check(self.lib.lbm_workspace_size(ctypes.byref(d), ctypes.byref(size)))
        # torch's caching allocator returns 512-byte aligned blocks
        self.workspace = torch.empty(size.value, dtype=torch.uint8, device=self.device)
        self.h = ctypes.c_void_p()
        C.check(self.lib.lbm_create(ctypes.byref(self.h), ctypes.byref(d), _ptr(self.workspace), size.value))
        self._out = torch.zeros(8, dtype=torch.float64, device=self.device)

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            try:
                self.lib.lbm_destroy(h)
            except Exception:
                pass
            self.h = None

    # -- set-up ------------------------------------------------------------
    def set_coeffs(self, conv: int = 0, u=(0.0, 0.0), diff: int = 0, K=(0.0, 0.0, 0.0),
                   s=(1.0, 1.2, 1.2, 0.0, 1.0, 0.0, 1.0, 1.1, 1.1), r0: float = 0.0, r1: float = 0.0,
                   src_family: int = 0, power: int = 1, b: float = 0.0, cfree: int = 0, Dm=(1.0, 0.0, 1.0)):
        """conv 0 / 1 / 2 (power-law flux of degree `power`) / 3 (Buckley-Leverett,
        cfree only), diff 0 / 1 / 2; src_family 0: R = r0 + r1 phi, 1: R = b phi
        (1 - phi^power) (Scheme A); cfree 1: the C-free variant of Remark III;
        diff 3: D = Dm phi (Dm = (xx, xy, yy))."""
        c = C.Coeffs()
        c.conv, c.diff = int(conv), int(diff)
        c.u[:] = [float(v) for v in u]
        c.K[:] = [float(v) for v in K]
        c.s[:] = [float(v) for v in s]
        c.r0, c.r1 = float(r0), float(r1)
        c.src_family, c.power, c.b = int(src_family), int(power), float(b)
        c.cfree = int(cfree)
        c.Dm[:] = [float(v) for v in Dm]
        C.check(self.lib.lbm_set_coeffs(self.h, ctypes.byref(c)))
        self.coeffs = c
        return self

    def set_K_field(self, K: torch.Tensor, stream=None):
        K = K.to(device=self.device, dtype=torch.float64).contiguous()
        assert K.shape == (3, self.ny, self.nx)
        self._K = K
        C.check(self.lib.lbm_set_K_field(self.h, _ptr(K), _stream(stream)))
        return self

    def set_phi(self, phi0: torch.Tensor, stream=None):
        assert phi0.shape == (self.ny, self.nx) and phi0.is_cuda and phi0.is_contiguous()
        C.check(self.lib.lbm_set_phi(self.h, _ptr(phi0), _prec_of(phi0), _stream(stream)))
        return self

    def set_phi_host(self, phi0: torch.Tensor, stream=None):
        assert phi0.shape == (self.ny, self.nx) and not phi0.is_cuda and phi0.is_contiguous()
        C.check(self.lib.lbm_set_phi_host(self.h, _ptr(phi0), _prec_of(phi0), _stream(stream)))
        return self

    def set_dirichlet(self, values: torch.Tensor):
        """Dirichlet records of the extrapolated axes: (nrec, 2 (nx + ny)) float64
        on the device, each record west[ny], east[ny], south[nx], north[nx];
        record j serves the (j + 1)-th step from now (or from the next set_phi);
        the last one is reused after it. The step count is kept on the device,
        so graph replays advance through the records."""
        v = values.to(device=self.device, dtype=torch.float64).contiguous()
        if v.dim() == 1:
            v = v.view(1, -1)
        assert v.shape[1] == 2 * (self.nx + self.ny), v.shape
        self._dirichlet = v
        C.check(self.lib.lbm_set_dirichlet(self.h, _ptr(v), int(v.shape[0])))
        return self

    # -- time stepping -------------------------------------------------------
    def step(self, n: int = 1, stream=None):
        C.check(self.lib.lbm_step(self.h, int(n), _stream(stream)))
        return self

    # -- CUDA graphs -------------------------------------------------------------
    def capture(self, nsteps: int):
        """Record nsteps time steps into a CUDA graph; replay() relaunches them,
        advancing the state by nsteps each time. The recorded launches must be
        even in number (nsteps even with one step per pass, a multiple of 4 with
        two), so that every replay ends on the buffer it started from. One step
        is run first and undone (save / load) so that kernel attributes are set
        outside the capture (the Dirichlet record count is saved and restored
        with the state). With extrapolated walls each replay takes the next
        records, as direct steps would."""
        spp = int(self.desc.steps_per_pass)
        launches = nsteps // spp + nsteps % spp
        if nsteps < 1 or launches % 2:
            raise ValueError("capture needs an even number of launches")
        snap = self.save()
        self.step(spp)
        self.load(snap)
        torch.cuda.current_stream().synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            C.check(self.lib.lbm_step(self.h, int(nsteps), _stream()))
        self._graph, self._graph_steps = g, int(nsteps)
        return self

    def replay(self):
        self._graph.replay()
        return self

    # -- read-out ------------------------------------------------------------
    def phi(self, dtype=torch.float64, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.ny, self.nx), dtype=dtype, device=self.device)
        C.check(self.lib.lbm_get_phi(self.h, _ptr(out), _prec_of(out), _stream(stream)))
        return out

    def phi_host(self, out: torch.Tensor, stream=None) -> torch.Tensor:
        assert not out.is_cuda and out.shape == (self.ny, self.nx) and out.is_contiguous()
        C.check(self.lib.lbm_get_phi_host(self.h, _ptr(out), _prec_of(out), _stream(stream)))
        return out

    def reduce_async(self, ref: torch.Tensor | None = None, out: torch.Tensor | None = None, stream=None):
        out = self._out if out is None else out
        if ref is not None:
            ref = ref.to(device=self.device, dtype=torch.float64).contiguous()
            self._ref = ref
        C.check(self.lib.lbm_reduce(self.h, _ptr(ref) if ref is not None else None, _ptr(out), _stream(stream)))
        return out

    def reduce(self, ref: torch.Tensor | None = None) -> dict:
        v = self.reduce_async(ref).cpu().tolist()
        return dict(zip(REDUCE_KEYS, v))

    def check_finite(self, stream=None) -> None:
        """Raise LBMError (LBM_ENONFINITE) if any node's phi is not finite."""
        n = ctypes.c_longlong()
        C.check(self.lib.lbm_check_finite(self.h, ctypes.byref(n), _stream(stream)))

    # -- checkpoints -----------------------------------------------------------
    def state_bytes(self) -> int:
        n = ctypes.c_size_t()
        C.check(self.lib.lbm_state_bytes(self.h, ctypes.byref(n)))
        return n.value

    def save(self, dst: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if dst is None:
            dst = torch.empty(self.state_bytes(), dtype=torch.uint8, device=self.device)
        C.check(self.lib.lbm_save(self.h, _ptr(dst), _stream(stream)))
        return dst

    def load(self, src: torch.Tensor, stream=None):
        assert src.numel() * src.element_size() >= self.state_bytes()
        C.check(self.lib.lbm_load(self.h, _ptr(src), _stream(stream)))
        return self
