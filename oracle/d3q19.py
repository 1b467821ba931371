"""Plain FP64 numpy oracle of the three-dimensional extension (D3Q19) of the
MRT model for nonlinear anisotropic convection-diffusion equations
(arXiv:1603.09577: lattice of Eq. 6, equilibrium of Eq. 3, source of Eq. 9,
Scheme B of Eq. 33-35).

TEST INFRASTRUCTURE. Only the test suite and the benchmark's CPU-baseline leg
load this module; it shares no code with the CUDA library.

The paper states the lattice but no D3Q19 moment matrix. Reading used here:
M is a moment basis whose rows are mutually orthogonal (plain dot product) and
contain rho = sum_k f_k and j = sum_k c_k f_k (as Eq. 15's M0 does in 2-D); S
relaxes rho with s0, j with the 3 x 3 block A = (K / (d c_s^2) + I/2)^-1
(Eq. 26 in 3-D), and every other moment with one rate s_e. With the other rates
equal, the choice of the remaining 15 rows does not matter; they are completed
here by a QR factorisation. The collision is Eq. 34 written with the matrices
P = M^-1 S M and Q = M^-1 (I - S/2) M, and the streaming is a pull with
periodic wrap, or, on an axis with anti-bounce-back walls, the anti-bounce-back
rule of the 2-D model (Sec. 3.6) applied to every link whose source lies beyond
a wall half-way between the boundary node and the missing node:
    fbar_k(x, t+1) = -fbar*_opp(k)(x, t) + feq_k(phi_w) + feq_opp(k)(phi_w),
phi_w the wall's value, the mean of the walls' values for a link that crosses
two or three walls. Arrays: populations (19, nz, ny, nx), phi (nz, ny, nx),
velocity index k in the order of Eq. 6.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# Eq. 6: D3Q19 velocities (columns) and weights
CX = np.array([0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1, 0, 0, 0, 0])
CY = np.array([0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1])
CZ = np.array([0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1])
C = np.stack([CX, CY, CZ], axis=1).astype(np.float64)          # (19, 3)
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
CS2 = 1.0 / 3.0
D = 1.0                                                         # d of Eq. 3 (Sec. 3 default)
Q19 = 19


@dataclass
class Spec3:
    nx: int
    ny: int
    nz: int
    conv: int = 0                     # 0: B = u phi, C = u u phi; 1: B = a phi^2/2, C = a a phi^3/3 (Eq. 7)
    u: tuple = (0.0, 0.0, 0.0)
    diff: int = 0                     # D = g(phi) I, g = phi, phi + phi^2/2, phi + phi^3/3
    K: tuple = (0.0, 0.0, 0.0, 0.0, 0.0, 0.0)   # Kxx, Kxy, Kxz, Kyy, Kyz, Kzz
    s0: float = 1.0
    se: float = 1.0                   # rate of every moment other than rho and j
    r0: float = 0.0
    r1: float = 0.0
    bc: tuple = (0, 0, 0)             # per axis x, y, z: 0 periodic, 1 anti-bounce-back walls
    phi_wall: tuple = (0.0, 0.0, 0.0, 0.0, 0.0, 0.0)   # x-, x+, y-, y+, z-, z+


def k_matrix(K) -> np.ndarray:
    kxx, kxy, kxz, kyy, kyz, kzz = K
    return np.array([[kxx, kxy, kxz], [kxy, kyy, kyz], [kxz, kyz, kzz]], dtype=np.float64)


def relax_block(K) -> np.ndarray:
    """Eq. 26 solved for A: A^-1 = K / (d c_s^2) + I/2 (dt = 1)."""
    Ainv = k_matrix(K) / (D * CS2) + 0.5 * np.eye(3)
    if np.any(np.linalg.eigvalsh(Ainv - 0.5 * np.eye(3)) <= 0):
        raise ValueError("K is not positive definite")
    return np.linalg.inv(Ainv)


def moment_basis() -> np.ndarray:
    """Rows 0..3: 1, c_x, c_y, c_z (mutually orthogonal); rows 4..18: an
    orthogonal completion (QR of those four columns padded with the unit
    vectors)."""
    first = np.stack([np.ones(Q19), CX, CY, CZ], axis=1).astype(np.float64)
    q, _ = np.linalg.qr(np.concatenate([first, np.eye(Q19)], axis=1), mode="reduced")
    rest = q[:, 4:Q19]
    M = np.concatenate([first.T, rest.T], axis=0)
    assert np.allclose(M @ M.T, np.diag(np.diag(M @ M.T)), atol=1e-12)
    return M


def pq_matrices(spec: Spec3):
    """P = M^-1 S M and Q = M^-1 (I - S/2) M."""
    M = moment_basis()
    S = np.eye(Q19) * spec.se
    S[0, 0] = spec.s0
    S[1:4, 1:4] = relax_block(spec.K)
    Minv = np.linalg.inv(M)
    return Minv @ S @ M, Minv @ (np.eye(Q19) - 0.5 * S) @ M


def coefficients(spec: Spec3, phi):
    """B, B' (3-vectors) and C (3 x 3) per node: Eq. 7 families; g(phi)."""
    a = np.asarray(spec.u, dtype=np.float64)
    if spec.conv == 0:
        B = a[:, None] * phi[None]
        Bp = np.broadcast_to(a[:, None], (3,) + phi.shape) * np.ones_like(phi)[None]
        Cm = np.einsum("a,b->ab", a, a)[:, :, None] * phi.reshape(-1)[None, None]
    else:
        B = 0.5 * a[:, None] * (phi * phi)[None]
        Bp = a[:, None] * phi[None]
        Cm = np.einsum("a,b->ab", a, a)[:, :, None] * (phi ** 3 / 3).reshape(-1)[None, None]
    g = [phi, phi + phi ** 2 / 2, phi + phi ** 3 / 3][spec.diff]
    return B.reshape(3, -1), Bp.reshape(3, -1), Cm.reshape(3, 3, -1), g.reshape(-1)


def feq(spec: Spec3, phi) -> np.ndarray:
    """Eq. 3 with D = g(phi) I, per node; returns (19, n)."""
    phi = np.asarray(phi, dtype=np.float64).reshape(-1)
    B, _, Cm, g = coefficients(spec, phi)
    Qt = Cm + (D * CS2 * g - CS2 * phi)[None, None] * np.eye(3)[:, :, None]
    cB = C @ B                                                   # (19, n)
    cc = np.einsum("ka,kb->kab", C, C) - CS2 * np.eye(3)[None]   # (19, 3, 3)
    qc = np.einsum("kab,abn->kn", cc, Qt)
    return W[:, None] * (phi[None] + cB / CS2 + qc / (2 * CS2 * CS2))


def source_pop(spec: Spec3, phi, R) -> np.ndarray:
    """Eq. 9 with Btilde = B' (Scheme B); (19, n)."""
    phi = np.asarray(phi, dtype=np.float64).reshape(-1)
    _, Bp, _, _ = coefficients(spec, phi)
    return W[:, None] * (1.0 + (C @ Bp) / CS2) * np.asarray(R).reshape(-1)[None]


def collide(spec: Spec3, f, P, Qm):
    """Eq. 34: fbar* = fbar - P (fbar - feq) + Q R_vec, phi from Eq. 35; f (19, n)."""
    phi = (f.sum(axis=0) + 0.5 * spec.r0) / (1.0 - 0.5 * spec.r1)
    R = spec.r0 + spec.r1 * phi
    fe = feq(spec, phi)
    Rk = source_pop(spec, phi, R)
    return f - P @ (f - fe) + Qm @ Rk, phi


def init(spec: Spec3, phi0) -> np.ndarray:
    """Eq. 40 in the shifted variable (Eq. 33), then one collision."""
    P, Qm = pq_matrices(spec)
    phi = np.asarray(phi0, dtype=np.float64).reshape(-1)
    R = spec.r0 + spec.r1 * phi
    f = feq(spec, phi) - 0.5 * source_pop(spec, phi, R)
    out, _ = collide(spec, f, P, Qm)
    return out.reshape(Q19, spec.nz, spec.ny, spec.nx)


def opposite(k: int) -> int:
    """The direction with c_opp = -c_k."""
    return int(np.flatnonzero((CX == -CX[k]) & (CY == -CY[k]) & (CZ == -CZ[k]))[0])


def wall_links(spec: Spec3, k: int):
    """For direction k: a mask (nz, ny, nx) of the nodes whose source x - c_k
    lies beyond a wall, and the wall value phi_w of each such link."""
    shape = (spec.nz, spec.ny, spec.nx)
    idx = np.indices(shape)                                      # z, y, x
    coords = (idx[2], idx[1], idx[0])
    c = (CX[k], CY[k], CZ[k])
    n = (spec.nx, spec.ny, spec.nz)
    total = np.zeros(shape)
    count = np.zeros(shape)
    for ax in range(3):
        if not spec.bc[ax] or c[ax] == 0:
            continue
        src = coords[ax] - c[ax]
        low, high = src < 0, src >= n[ax]
        total += low * spec.phi_wall[2 * ax] + high * spec.phi_wall[2 * ax + 1]
        count += low | high
    mask = count > 0
    return mask, np.where(mask, total / np.maximum(count, 1), 0.0)


_WALLS = {}


def _wall_terms(spec: Spec3):
    """(k, opp(k), mask, feq at the links' wall values) for every direction with
    links beyond a wall; computed once per problem."""
    key = (spec.nx, spec.ny, spec.nz, tuple(spec.bc), tuple(spec.phi_wall), spec.conv, tuple(spec.u), spec.diff)
    if key not in _WALLS:
        out = []
        for k in range(1, Q19):
            mask, phiw = wall_links(spec, k)
            if mask.any():
                out.append((k, opposite(k), mask, feq(spec, phiw[mask])))
        _WALLS[key] = out
    return _WALLS[key]


def step(spec: Spec3, F, P=None, Qm=None):
    """Pull streaming (periodic wrap, anti-bounce-back at walls), then the
    collision. Returns the new state and phi(t_{n+1})."""
    if P is None:
        P, Qm = pq_matrices(spec)
    pulled = np.empty_like(F)
    for k in range(Q19):
        # f_k(x) = f*_k(x - c_k): np.roll by +c_k along each axis
        pulled[k] = np.roll(F[k], shift=(CZ[k], CY[k], CX[k]), axis=(0, 1, 2))
    if any(spec.bc):
        for k, ko, mask, fe in _wall_terms(spec):
            pulled[k][mask] = -F[ko][mask] + fe[k] + fe[ko]
    out, phi = collide(spec, pulled.reshape(Q19, -1), P, Qm)
    shape = (spec.nz, spec.ny, spec.nx)
    return out.reshape((Q19,) + shape), phi.reshape(shape)


def run(spec: Spec3, phi0, nsteps: int) -> np.ndarray:
    F = init(spec, phi0)
    P, Qm = pq_matrices(spec)
    phi = np.asarray(phi0, dtype=np.float64).copy()
    for _ in range(nsteps):
        F, phi = step(spec, F, P, Qm)
    return phi
