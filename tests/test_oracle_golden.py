"""The oracle against numbers the paper prints (tests/golden/gaussian_hill_gre.txt):
the GRE of the isotropic Gaussian hill of Sec. 3.4, the Sec. 3.6 stability
comparison (the MRT model's GRE at kappa = 1e-4, and the BGK model's blow-up
there), and the Sec. 3.5 variable-tensor problem at Pe = 100. The remaining printed Sec. 3.4 values are compared through the FP64 GPU
path (tests/test_gpu_general.py), whose parity with this oracle is tested."""
import math

import numpy as np

import oracle as O
import workloads as W

GOLD = W.read_golden("gaussian_hill_gre.txt")


def gre(a, e):
    return float(np.abs(a - e).sum() / np.abs(e).sum())


def test_sec34_isotropic_gaussian_gre():
    """Printed 1.199e-4 (four digits): 400^2 periodic nodes on [-1, 1)^2, c = 1,
    2000 steps, Eq. 41 rates."""
    g = W.gaussian_hill_square((1e-3, 0.0, 1e-3), (0.01, 0.01), 10.0)
    sp = O.Spec(nx=g["n"], ny=g["n"], conv=0, u=g["u"], diff=0, K=g["K"], s=W.S_EQ41)
    e = gre(O.run(sp, g["phi0"], g["steps"]), g["exact"])
    assert abs(e / GOLD["sec34_first_iso"] - 1) < 1e-3, e


def test_sec36_mrt_stable_where_bgk_blows_up():
    """Eq. 75-76 at kappa = 1e-4, u = (0.1, 0.1), T = 5 (1000 steps), second
    approach D = Dm phi with Dm = [[1, 1], [1, 2]] and K = kappa I: the MRT
    model (free rates 0.6) reproduces the printed GRE 4.438e-2; with every rate
    equal to s3 (BGK) the run diverges."""
    kap = 1e-4
    g = W.gaussian_hill_square((kap, kap, 2 * kap), (0.1, 0.1), 5.0)
    kl = g["K"][0]
    mrt = O.Spec(nx=g["n"], ny=g["n"], conv=0, u=g["u"], diff=3, Dm=(1.0, 1.0, 2.0), K=(kl, 0.0, kl),
                 s=(0.0, 0.6, 0.6, 0.0, 0.6, 0.0, 0.6, 0.6, 0.6))
    e = gre(O.run_x(mrt, g["phi0"], g["steps"]), g["exact"])
    assert abs(e / GOLD["sec36_mrt_kappa1e-4"] - 1) < 1e-3, e
    sj = O.relax_block((kl, 0.0, kl))[0, 0]
    bgk = O.Spec(nx=g["n"], ny=g["n"], conv=0, u=g["u"], diff=3, Dm=(1.0, 1.0, 2.0), K=(kl, 0.0, kl), s=(sj,) * 9)
    with np.errstate(all="ignore"):
        phi = O.run_x(bgk, g["phi0"], g["steps"])
    assert not np.all(np.isfinite(phi)) or np.abs(phi).max() > 1e3


def test_tensor_diffusion_function_reduces_to_identity():
    """diff 3 with Dm = I is D = phi I (diff 0)."""
    nx, ny = 21, 17
    phi0 = W.phi0_aniso(nx, seed=5, ny=ny)
    common = dict(nx=nx, ny=ny, conv=1, u=(0.06, 0.03), K=(0.02, 0.005, 0.015), s=W.s9())
    a = O.run_x(O.Spec(diff=0, **common), phi0, 30)
    b = O.run_x(O.Spec(diff=3, Dm=(1.0, 0.0, 1.0), **common), phi0, 30)
    assert np.abs(a - b).max() < 1e-14


def test_sec35_variable_tensor_gre():
    """Eq. 64-68 at Pe = 100 (kappa = 1e-3, u = (0.1, 0.1)), 400^2 periodic nodes on
    [0, 1)^2, c = 1, T = 3 (1200 steps), Eq. 41 rates, the source of Eq. 66 taken
    at each step's new time level: the oracle's GRE is 5.73e-4 against the printed
    6.207e-4. The paper does not say at which time level it evaluates the
    explicit source; the match is to 10 %."""
    n, kap, u, T = 400, 1e-3, (0.1, 0.1), 3.0
    dx = 1.0 / n
    dt = dx
    steps = int(round(T / dt))
    x = np.arange(n) * dx
    X, Y = np.meshgrid(x, x)
    scale = dt / dx ** 2
    Kf = np.stack([kap * (2 - np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)) * scale,
                   np.zeros_like(X), kap * np.ones_like(X) * scale])          # Eq. 65
    sp = O.Spec(nx=n, ny=n, conv=0, u=(u[0] * dt / dx, u[1] * dt / dx), Kfield=Kf, s=W.S_EQ41,
                src=2, src_par=(0.0, 0.0, dx, dt, kap, u[0], u[1]))
    phi0 = np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)                     # Eq. 67
    e = gre(O.run(sp, phi0, steps), math.exp((1 - 12 * np.pi ** 2 * kap) * steps * dt) * phi0)   # Eq. 68
    assert abs(e / GOLD["sec35_pe100"] - 1) < 0.1, e
