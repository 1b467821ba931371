"""Plain FP64 CPU oracle of the D2Q9 MRT lattice Boltzmann model for nonlinear
anisotropic convection-diffusion equations (arXiv:1603.09577, Sec. 2).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The arithmetic lives
in ``lbm_oracle.c`` (plain C, FP64, ``-ffp-contract=off``); this module only
compiles it with gcc and marshals numpy arrays through ctypes. It shares no
code with the CUDA library.

Array conventions: phi is (ny, nx) float64, C-contiguous; population states
are (9, ny, nx) float64; a per-cell tensor field is (3, ny, nx) = (Kxx, Kxy, Kyy).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_HDR = os.path.join(_HERE, "lbm_oracle.h")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, OpenMP over rows)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Problem(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("bc_x", ctypes.c_int), ("bc_y", ctypes.c_int),
        ("phi_wall", ctypes.c_double * 4),
        ("conv", ctypes.c_int), ("u", ctypes.c_double * 2),
        ("diff", ctypes.c_int), ("K", ctypes.c_double * 3),
        ("Kfield", ctypes.POINTER(ctypes.c_double)),
        ("s", ctypes.c_double * 9),
        ("r0", ctypes.c_double), ("r1", ctypes.c_double),
        ("src", ctypes.c_int), ("src_par", ctypes.c_double * 8),
        ("collision", ctypes.c_int),
        ("scheme", ctypes.c_int), ("power", ctypes.c_int),
        ("src_family", ctypes.c_int), ("b", ctypes.c_double),
        ("Dm", ctypes.c_double * 3), ("cfree", ctypes.c_int),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            P = ctypes.POINTER(Problem)
            L.oracle_num_threads.restype = ctypes.c_int
            L.oracle_feq.argtypes = [P, ctypes.c_double, dp]
            L.oracle_source_pop.argtypes = [P, ctypes.c_double, ctypes.c_double, dp]
            L.oracle_relax_block.argtypes = [dp, dp]
            L.oracle_collide_cell.argtypes = [P, dp, dp, ctypes.c_double, dp, dp]
            L.oracle_pform_matrices.argtypes = [P, dp, dp, dp]
            L.oracle_init.argtypes = [P, dp, dp]
            L.oracle_step.argtypes = [P, dp, dp, ctypes.c_int, dp]
            L.oracle_phi_from_post.argtypes = [P, dp, ctypes.c_int, dp]
            L.oracle_run.argtypes = [P, dp, ctypes.c_int, dp, dp]
            L.oracle_adjoint.argtypes = [P, dp, dp, ctypes.c_int, dp, dp, dp, dp]
            L.oracle_init_x.argtypes = [P, dp, dp, dp]
            L.oracle_step_x.argtypes = [P, dp, dp, dp, dp, dp]
            L.oracle_run_x.argtypes = [P, dp, ctypes.c_int, dp, dp]
            L.oracle_collide_cell_x.argtypes = [P, dp, dp, ctypes.c_double, dp, dp]
            _lib = L
    return _lib


def num_threads() -> int:
    return lib().oracle_num_threads()


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Spec:
    """Problem parameters in lattice units (c = dx/dt = 1)."""
    nx: int
    ny: int
    bc_x: int = 0                 # 0 periodic, 1 anti-bounce-back
    bc_y: int = 0
    phi_wall: tuple = (0.0, 0.0, 0.0, 0.0)   # west, east, south, north
    conv: int = 0                 # 0: B = u phi; 1: B = a phi^2 / 2
    u: tuple = (0.0, 0.0)
    diff: int = 0                 # g(phi): 0 phi, 1 phi + phi^2/2, 2 phi + phi^3/3
    K: tuple = (0.0, 0.0, 0.0)    # Kxx, Kxy, Kyy
    Kfield: np.ndarray | None = None
    s: tuple = (1.0, 1.2, 1.2, 1.0, 1.0, 1.0, 1.0, 1.1, 1.1)  # s0..s8 (s3, s5 unused)
    r0: float = 0.0
    r1: float = 0.0
    src: int = 0
    src_par: tuple = ()
    collision: int = 0            # 0 moment form, 1 P-form, 2 BGK loop
    scheme: int = 0               # 0 Scheme B, 1 Scheme A (general path only)
    power: int = 1                # delta of conv 2 and of the Fisher source
    src_family: int = 0           # 0 R = r0 + r1 phi, 1 R = b phi (1 - phi^delta)
    b: float = 0.0
    cfree: int = 0                # 1: Remark III variant (C = 0 plus G_k; Scheme A)
    Dm: tuple = (1.0, 0.0, 1.0)   # diff 3: D = Dm phi (Eq. 62's isotropic form)
    _keep: list = field(default_factory=list, repr=False)

    def c(self) -> Problem:
        p = Problem()
        p.nx, p.ny, p.bc_x, p.bc_y = self.nx, self.ny, self.bc_x, self.bc_y
        p.phi_wall[:] = list(self.phi_wall)
        p.conv = self.conv
        p.u[:] = list(self.u)
        p.diff = self.diff
        p.K[:] = list(self.K)
        if self.Kfield is not None:
            kf = _f64(self.Kfield)
            assert kf.shape == (3, self.ny, self.nx)
            self._keep = [kf]
            p.Kfield = _ptr(kf)
        else:
            p.Kfield = ctypes.POINTER(ctypes.c_double)()
        p.s[:] = list(self.s)
        p.r0, p.r1 = self.r0, self.r1
        p.src = self.src
        sp = list(self.src_par) + [0.0] * (8 - len(self.src_par))
        p.src_par[:] = sp
        p.collision = self.collision
        p.scheme, p.power, p.src_family, p.b = self.scheme, self.power, self.src_family, float(self.b)
        p.cfree = self.cfree
        p.Dm[:] = list(self.Dm)
        return p


def feq(spec: Spec, phi: float) -> np.ndarray:
    out = np.zeros(9)
    lib().oracle_feq(ctypes.byref(spec.c()), float(phi), _ptr(out))
    return out


def source_pop(spec: Spec, phi: float, R: float) -> np.ndarray:
    out = np.zeros(9)
    lib().oracle_source_pop(ctypes.byref(spec.c()), float(phi), float(R), _ptr(out))
    return out


def relax_block(K) -> np.ndarray:
    k = _f64(K)
    A = np.zeros(4)
    if lib().oracle_relax_block(_ptr(k), _ptr(A)):
        raise ValueError("K is not symmetric positive definite in the sense of Eq. 26")
    return A.reshape(2, 2)


def collide_cell(spec: Spec, f, K=None, Rexp: float = 0.0):
    k = _f64(spec.K if K is None else K)
    fi = _f64(f)
    out = np.zeros(9)
    phi = ctypes.c_double()
    if lib().oracle_collide_cell(ctypes.byref(spec.c()), _ptr(k), _ptr(fi), float(Rexp), _ptr(out),
                                 ctypes.byref(phi)):
        raise ValueError("invalid relaxation block")
    return out, phi.value


def pform_matrices(spec: Spec, K=None):
    k = _f64(spec.K if K is None else K)
    P = np.zeros(81)
    Qm = np.zeros(81)
    if lib().oracle_pform_matrices(ctypes.byref(spec.c()), _ptr(k), _ptr(P), _ptr(Qm)):
        raise ValueError("invalid relaxation block")
    return P.reshape(9, 9), Qm.reshape(9, 9)


def init(spec: Spec, phi0) -> np.ndarray:
    p = spec.c()
    ph = _f64(phi0)
    F = np.zeros((9, spec.ny, spec.nx))
    if lib().oracle_init(ctypes.byref(p), _ptr(ph), _ptr(F)):
        raise ValueError("oracle_init rejected the problem")
    return F


def step(spec: Spec, F, n: int):
    p = spec.c()
    Fi = _f64(F)
    Fo = np.zeros_like(Fi)
    phi = np.zeros((spec.ny, spec.nx))
    if lib().oracle_step(ctypes.byref(p), _ptr(Fi), _ptr(Fo), int(n), _ptr(phi)):
        raise ValueError("oracle_step rejected the problem")
    return Fo, phi


def phi_from_post(spec: Spec, F, n: int) -> np.ndarray:
    p = spec.c()
    Fi = _f64(F)
    phi = np.zeros((spec.ny, spec.nx))
    lib().oracle_phi_from_post(ctypes.byref(p), _ptr(Fi), int(n), _ptr(phi))
    return phi


def run(spec: Spec, phi0, nsteps: int, return_state: bool = False):
    p = spec.c()
    ph = _f64(phi0)
    assert ph.shape == (spec.ny, spec.nx)
    out = np.zeros_like(ph)
    F = np.zeros((9, spec.ny, spec.nx)) if return_state else None
    rc = lib().oracle_run(ctypes.byref(p), _ptr(ph), int(nsteps), _ptr(out),
                          _ptr(F) if F is not None else ctypes.POINTER(ctypes.c_double)())
    if rc:
        raise ValueError(f"oracle_run failed with status {rc}")
    return (out, F) if return_state else out


def adjoint(spec: Spec, phi0, target, nsteps: int):
    """Loss 1/2 |phi_N - target|^2 and its gradients (dphi0, dK planes, du)."""
    p = spec.c()
    ph, tg = _f64(phi0), _f64(target)
    loss = np.zeros(1)
    dphi0 = np.zeros_like(ph)
    dK = np.zeros((3, spec.ny, spec.nx))
    du = np.zeros(2)
    rc = lib().oracle_adjoint(ctypes.byref(p), _ptr(ph), _ptr(tg), int(nsteps), _ptr(loss),
                              _ptr(dphi0), _ptr(dK), _ptr(du))
    if rc:
        raise ValueError(f"oracle_adjoint failed with status {rc}")
    return float(loss[0]), dphi0, dK, du


# ---- general path: Scheme A, Fisher source, extrapolation boundary (bc 2) ----

def _null():
    return ctypes.POINTER(ctypes.c_double)()


def collide_cell_x(spec: Spec, f, phi_prev: float = 0.0, K=None):
    k = _f64(spec.K if K is None else K)
    fi = _f64(f)
    out = np.zeros(9)
    phi = ctypes.c_double()
    if lib().oracle_collide_cell_x(ctypes.byref(spec.c()), _ptr(k), _ptr(fi), float(phi_prev), _ptr(out),
                                   ctypes.byref(phi)):
        raise ValueError("invalid collision request")
    return out, phi.value


def init_x(spec: Spec, phi0):
    """State (F, Phi) after Eq. 40 and the first collision."""
    p = spec.c()
    ph = _f64(phi0)
    F = np.zeros((9, spec.ny, spec.nx))
    Phi = np.zeros((spec.ny, spec.nx))
    if lib().oracle_init_x(ctypes.byref(p), _ptr(ph), _ptr(F), _ptr(Phi)):
        raise ValueError("oracle_init_x rejected the problem")
    return F, Phi


def step_x(spec: Spec, F, Phi, bvals=None):
    """One step; bvals: 2 (nx + ny) Dirichlet values (west, east, south, north)."""
    p = spec.c()
    Fi, Pi = _f64(F), _f64(Phi)
    Fo, Po = np.zeros_like(Fi), np.zeros_like(Pi)
    bv = _f64(bvals) if bvals is not None else None
    if bv is not None:
        assert bv.size == 2 * (spec.nx + spec.ny)
    if lib().oracle_step_x(ctypes.byref(p), _ptr(Fi), _ptr(Pi), _ptr(bv) if bv is not None else _null(),
                           _ptr(Fo), _ptr(Po)):
        raise ValueError("oracle_step_x rejected the problem")
    return Fo, Po


def run_x(spec: Spec, phi0, nsteps: int, bvals=None) -> np.ndarray:
    """phi(t_N) from phi0; bvals: (nsteps, 2 (nx + ny)) Dirichlet records, record
    n for the step that produces t_{n+1}."""
    p = spec.c()
    ph = _f64(phi0)
    assert ph.shape == (spec.ny, spec.nx)
    out = np.zeros_like(ph)
    bv = None
    if bvals is not None:
        bv = _f64(bvals)
        assert bv.shape == (nsteps, 2 * (spec.nx + spec.ny)), bv.shape
    rc = lib().oracle_run_x(ctypes.byref(p), _ptr(ph), int(nsteps), _ptr(bv) if bv is not None else _null(),
                            _ptr(out))
    if rc:
        raise ValueError(f"oracle_run_x failed with status {rc}")
    return out
