"""Seeded synthetic inputs and problem parameters of the five workloads.

This module holds no arithmetic of the lattice Boltzmann method: it only states
each workload's physical parameters in lattice units (c = dx/dt = 1) and draws
its seeded initial fields, so that the CPU oracle and the CUDA path receive
bit-identical inputs. Each side derives its own relaxation rates from K.

Workloads (sizes, parameters and seeds):
  gaussian_iso_128     linear isotropic CDE, 128^2 periodic, u = (0.05, 0.02),
                       K = 0.01 I, Gaussian hill sigma = 8 at the centre, 1000 steps
  burgers_1024         Burgers flux B = a phi^2/2, a = (1,1)/sqrt2, 1024^2 periodic,
                       0.5 sin sin + 1e-3 uniform noise (seed 2), 5000 steps
  aniso_dirichlet_4096 D(phi) = (1 + phi^2) K, K = [[0.02,0.008],[0.008,0.01]],
                       R = -0.1 phi (t in [0,1]), 4096^2 with phi = 0 walls, U[0,1) smoothed by
                       three Jacobi passes (seed 3), 2000 steps
  adjoint_512          linear anisotropic CDE with a per-cell K(x), 512^2 periodic,
                       u = (0.03, 0), 500 steps, smooth seeded fields (seed 4)
  ensemble_256         256 nonlinear CDE instances, sides log-uniform in [64, 1024],
                       |u| <= 0.1, D(phi) = D0 (1 + phi), D0 in [0.001, 0.05] (seed 5)
  buckley_leverett_*   2-D Buckley-Leverett equation (Eq. 52-54) on [-1.5, 1.5]^2, the disc
                       of Eq. 53 as initial data, kappa = 0.1 or 0.01, C-free variant
                       (Remark III) with zero-valued extrapolated walls
  burgers_fisher_*     2-D Burgers-Fisher equation (Eq. 46-51) on [-1, 2]^2 with the
                       travelling-wave solution of Eq. 47-48 as initial and Dirichlet
                       data, a = 4, b = 1, delta = 1, kappa = 0.12 (Pe = La/kappa = 100,
                       L = 3), Scheme A with the extrapolation boundary

The Burgers workload reads the diffusivity D = 0.005 on the unit square with
dx = dt = 1/1024, i.e. K = 0.005 * 1024 = 5.12 in lattice units, while the
flux vector keeps |a| = 1 (c = 1).

The anisotropic Dirichlet workload keeps K in lattice units and reads the
source R = -0.1 phi per unit of physical time with the 2000 steps spanning
t in [0, 1] (dt = 1/2000), i.e. r1 = -0.1 / 2000 per step: taken per lattice
step the rate would shrink phi by e^-200 over the run, below FP32's range.
"""
from __future__ import annotations

import math

import numpy as np

# relaxation rates of the non-diffusive moments (s0, s1, s2, s4, s6, s7, s8),
# the values the 128^2 Gaussian-hill workload prescribes, used for every workload
S_OTHER = (1.0, 1.2, 1.2, 1.0, 1.0, 1.1, 1.1)


def s9(s_other=S_OTHER):
    """s0..s8 with placeholders at the diffusive indices 3 and 5."""
    s0, s1, s2, s4, s6, s7, s8 = s_other
    return (s0, s1, s2, 0.0, s4, 0.0, s6, s7, s8)


WORKLOADS = {
    "gaussian_iso_128": dict(
        nx=128, ny=128, bc=(0, 0), phi_wall=(0.0, 0.0, 0.0, 0.0), conv=0, u=(0.05, 0.02),
        diff=0, K=(0.01, 0.0, 0.01), r0=0.0, r1=0.0, steps=1000),
    "burgers_1024": dict(
        nx=1024, ny=1024, bc=(0, 0), phi_wall=(0.0, 0.0, 0.0, 0.0), conv=1,
        u=(1.0 / math.sqrt(2.0), 1.0 / math.sqrt(2.0)), diff=0, K=(5.12, 0.0, 5.12),
        r0=0.0, r1=0.0, steps=5000),
    "aniso_dirichlet_4096": dict(
        nx=4096, ny=4096, bc=(1, 1), phi_wall=(0.0, 0.0, 0.0, 0.0), conv=0, u=(0.0, 0.0),
        diff=2, K=(0.02, 0.008, 0.01), r0=0.0, r1=-0.1 / 2000, steps=2000),
    "adjoint_512": dict(
        nx=512, ny=512, bc=(0, 0), phi_wall=(0.0, 0.0, 0.0, 0.0), conv=0, u=(0.03, 0.0),
        diff=0, K=(0.01, 0.0, 0.01), r0=0.0, r1=0.0, steps=500, ckpt_every=50),
}


def params(name: str, **over) -> dict:
    d = dict(WORKLOADS[name])
    d.update(over)
    return d


# ---- initial fields ---------------------------------------------------------

def gaussian_hill(nx: int, ny: int, xc: float, yc: float, sigma: float, amp: float = 1.0):
    """Periodic Gaussian hill on integer nodes (nearest-image distance)."""
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    dx = (x - xc + nx / 2) % nx - nx / 2
    dy = (y - yc + ny / 2) % ny - ny / 2
    return amp * np.exp(-(dy[:, None] ** 2 + dx[None, :] ** 2) / (2.0 * sigma * sigma))


def phi0_gaussian(n: int = 128, sigma: float = 8.0):
    return gaussian_hill(n, n, n / 2, n / 2, sigma, 1.0)


def phi0_burgers(n: int = 1024, seed: int = 2):
    rng = np.random.default_rng(seed)
    x = np.arange(n, dtype=np.float64) / n
    base = 0.5 * np.sin(2 * np.pi * x)[None, :] * np.sin(2 * np.pi * x)[:, None]
    return base + rng.uniform(-1e-3, 1e-3, size=(n, n))


def jacobi_smooth(a, passes: int = 3):
    """phi <- mean of the 4 neighbours, zero outside the domain."""
    a = np.array(a, dtype=np.float64)
    for _ in range(passes):
        p = np.pad(a, 1)
        a = 0.25 * (p[:-2, 1:-1] + p[2:, 1:-1] + p[1:-1, :-2] + p[1:-1, 2:])
    return a


def phi0_aniso(n: int = 4096, seed: int = 3, ny: int | None = None):
    rng = np.random.default_rng(seed)
    return jacobi_smooth(rng.random((ny or n, n)), 3)


def smooth_field(nx: int, ny: int, rng, modes: int = 8, kmax: int = 4):
    """Sum of random periodic Fourier modes with |k| <= kmax, scaled to unit max."""
    x = np.arange(nx, dtype=np.float64) / nx
    y = np.arange(ny, dtype=np.float64) / ny
    f = np.zeros((ny, nx))
    for _ in range(modes):
        kx, ky = rng.integers(-kmax, kmax + 1, size=2)
        if kx == 0 and ky == 0:
            kx = 1
        ph = rng.uniform(0, 2 * np.pi)
        f += rng.normal() * np.cos(2 * np.pi * (kx * x[None, :] + ky * y[:, None]) + ph)
    return f / max(np.abs(f).max(), 1e-300)


def adjoint_inputs(n: int = 512, seed: int = 4, ny: int | None = None):
    """Per-cell tensor field (3, ny, nx), initial phi and target phi."""
    ny = ny or n
    rng = np.random.default_rng(seed)
    sig = lambda z: 1.0 / (1.0 + np.exp(-z))
    kxx = 0.005 + 0.045 * sig(2.0 * smooth_field(n, ny, rng))
    kyy = 0.005 + 0.045 * sig(2.0 * smooth_field(n, ny, rng))
    kxy = 0.5 * np.sqrt(kxx * kyy) * np.tanh(smooth_field(n, ny, rng))
    phi0 = 0.5 + 0.4 * smooth_field(n, ny, rng)
    target = 0.5 + 0.4 * smooth_field(n, ny, rng)
    return np.stack([kxx, kxy, kyy]), phi0, target


def ensemble(count: int = 256, seed: int = 5, side_min: int = 64, side_max: int = 1024, lam: float = 0.25):
    """Per-instance parameters of the batched ensemble.

    Free relaxation rates: the odd moments q_x, q_y relax at the diffusive rate
    s_j (1/s_j - 1/2 = 3 D0) and the even moments e, eps, p_xx, p_xy at s_plus
    with (1/s_j - 1/2)(1/s_plus - 1/2) = lam = 1/4. With the 128^2 workload's
    rates the low-D0, high-|u| instances (s_j near 1.99) are linearly unstable."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        side = int(round(math.exp(rng.uniform(math.log(side_min), math.log(side_max)))))
        r = 0.1 * math.sqrt(rng.uniform())
        th = rng.uniform(0, 2 * math.pi)
        D0 = rng.uniform(0.001, 0.05)
        xc, yc = rng.uniform(0, side, size=2)
        sigma = max(4.0, rng.uniform(side / 32, side / 8))
        amp = rng.uniform(0.5, 1.0)
        odd = 1.0 / (0.5 + 3.0 * D0)
        even = 1.0 / (0.5 + lam / (3.0 * D0))
        out.append(dict(nx=side, ny=side, u=(r * math.cos(th), r * math.sin(th)), D0=D0,
                        K=(D0, 0.0, D0), diff=1, conv=0, xc=xc, yc=yc, sigma=sigma, amp=amp,
                        s=(1.0, even, even, 0.0, odd, 0.0, odd, even, even)))
    return out


def ensemble_phi0(inst: dict):
    return gaussian_hill(inst["nx"], inst["ny"], inst["xc"], inst["yc"], inst["sigma"], inst["amp"])


# ---- Burgers-Fisher travelling wave (Eq. 46-51) ---------------------------------

def burgers_fisher_exact(x, y, t, a=4.0, b=1.0, kappa=0.12, delta=1):
    """Eq. 47 with A of Eq. 48 and the wave speed omega = (a^2 + 2 b kappa
    (delta + 1)^2) / (a (delta + 1)). As printed, Eq. 48 has (delta + 1) in place
    of (delta + 1)^2 in omega; only the squared form makes Eq. 47 an exact
    solution of Eq. 46 (substitution: the travelling-wave reduction with
    xi = x + y has diffusivity 2 kappa)."""
    A = -a * delta / (4.0 * kappa * (delta + 1))
    w = (a * a + 2.0 * b * kappa * (delta + 1) ** 2) / (a * (delta + 1))
    return (0.5 + 0.5 * np.tanh(A * (x + y - w * t))) ** (1.0 / delta)


def burgers_fisher(N: int, T: float, c: float = 40.0, a: float = 4.0, b: float = 1.0, kappa: float = 0.12,
                   delta: int = 1, x0: float = -1.0, L: float = 3.0) -> dict:
    """The Burgers-Fisher problem on [x0, x0 + L]^2 with N intervals per side
    (N + 1 nodes), lattice speed c = dx/dt, run to time T.

    Lattice units (dx = dt = 1 on the lattice): the flux direction becomes
    a dt / dx, the source rate b dt and the diffusivity kappa dt / dx^2 (reading
    of the paper, which leaves dt unstated). Returns the lattice parameters, the
    initial field, the Dirichlet records of every step (west, east, south,
    north; record n holds t_{n+1}) and the exact field at the final time."""
    dx = L / N
    dt = dx / c
    steps = int(round(T / dt))
    xs = x0 + dx * np.arange(N + 1)
    X, Y = np.meshgrid(xs, xs)               # (ny, nx): row y, column x
    ex = lambda xx, yy, t: burgers_fisher_exact(xx, yy, t, a, b, kappa, delta)
    n = N + 1
    bv = np.empty((steps, 4 * n))
    for s in range(steps):
        t = (s + 1) * dt
        bv[s, 0:n] = ex(xs[0], xs, t)              # west: x = x0, all y
        bv[s, n:2 * n] = ex(xs[-1], xs, t)         # east
        bv[s, 2 * n:3 * n] = ex(xs, xs[0], t)      # south: y = x0, all x
        bv[s, 3 * n:4 * n] = ex(xs, xs[-1], t)     # north
    return dict(nx=n, ny=n, dx=dx, dt=dt, steps=steps, u=(a * dt / dx, 0.0), K=kappa * dt / dx ** 2,
                b=b * dt, power=delta, phi0=ex(X, Y, 0.0), bvals=bv, exact=ex(X, Y, steps * dt))


# ---- Buckley-Leverett (Eq. 52-54) -------------------------------------------------

def buckley_leverett(N: int, kappa: float, T: float, c: float = 20.0, L: float = 3.0) -> dict:
    """The Buckley-Leverett problem on [-L/2, L/2]^2 with N intervals (N + 1
    nodes per side), lattice speed c = dx/dt, to time T. Lattice units: the flux
    is scaled by dt/dx per axis and kappa by dt/dx^2. Walls: zero Dirichlet
    values (the disc of Eq. 53 stays far from them up to T = 0.5)."""
    dx = L / N
    dt = dx / c
    xs = -L / 2 + dx * np.arange(N + 1)
    X, Y = np.meshgrid(xs, xs)
    n = N + 1
    return dict(nx=n, ny=n, dx=dx, dt=dt, steps=int(round(T / dt)), u=(dt / dx, dt / dx), K=kappa * dt / dx ** 2,
                phi0=np.where(X ** 2 + Y ** 2 < 0.5, 1.0, 0.0), bvals=np.zeros((1, 4 * n)))


# ---- Gaussian hill of Sec. 3.4 / 3.6 (Eq. 58-60) -------------------------------------

def gaussian_hill_square(K, u, T, n: int = 400, sigma0: float = 0.01, L: float = 2.0) -> dict:
    """The Gaussian hill of Eq. 60 on the periodic square [-L/2, L/2)^2 with n
    nodes per side (dx = L / n, c = 1 so dt = dx), physical K (Kxx, Kxy, Kyy)
    and u, run to time T. Returns lattice units (u dt/dx, K dt/dx^2), the
    initial field and Eq. 60 at the final time, each summed over the 3 x 3
    nearest periodic images. phi0 = 2 pi sigma0^2 makes the peak 1."""
    dx = L / n
    dt = dx
    steps = int(round(T / dt))
    xs = -L / 2 + dx * np.arange(n)
    X, Y = np.meshgrid(xs, xs)

    def hill(t):
        S = sigma0 ** 2 * np.eye(2) + 2 * np.array([[K[0], K[1]], [K[1], K[2]]]) * t
        Si = np.linalg.inv(S)
        out = np.zeros((n, n))
        for mx in (-1, 0, 1):
            for my in (-1, 0, 1):
                ddx = X - u[0] * t + mx * L
                ddy = Y - u[1] * t + my * L
                out += np.exp(-(Si[0, 0] * ddx * ddx + 2 * Si[0, 1] * ddx * ddy + Si[1, 1] * ddy * ddy) / 2)
        return sigma0 ** 2 / math.sqrt(np.linalg.det(S)) * out

    return dict(n=n, dx=dx, dt=dt, steps=steps, u=(u[0] * dt / dx, u[1] * dt / dx),
                K=tuple(k * dt / dx ** 2 for k in K), phi0=hill(0.0), exact=hill(steps * dt))


S_EQ41 = (0.0, 1.0, 1.0, 0.0, 1.0, 0.0, 1.0, 1.0, 1.0)   # Eq. 41 (s3, s5 come from K)


def read_golden(name: str) -> dict:
    """case -> printed value from a tests/golden table (comment lines start with #)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden", name)
    out = {}
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                key, val = line.split()[:2]
                out[key] = float(val)
    return out
