"""Parity of the D3Q19 CUDA path (include/lbm3.h) with the numpy FP64 oracle
(oracle/d3q19.py): FP64 <= 1e-12, FP32 <= 1e-5 relative L2, on ragged grids
spanning several blocks, both flux families, the three diffusion functions and
sources; the 3-D Gaussian hill of Eq. 60 at 96^3 for the full run."""
import math

import numpy as np
import pytest
import torch

import workloads as W
from oracle import d3q19 as D
from paper_1603_09577_gb300 import Solver3

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "bf16s": 2e-3}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [
    (37, 21, 9, dict(conv=0, u=(0.05, -0.03, 0.02), diff=0, K=(0.02, 0.004, -0.003, 0.015, 0.002, 0.012), se=1.2)),
    (33, 17, 12, dict(conv=1, u=(0.06, 0.02, -0.04), diff=2, K=(0.03, 0.0, 0.01, 0.02, -0.005, 0.025), se=0.9,
                      r0=0.001, r1=-0.02)),
    (64, 8, 5, dict(conv=1, u=(-0.04, 0.05, 0.03), diff=1, K=(0.01, 0.002, 0.0, 0.01, 0.0, 0.01), se=1.5, s0=0.5)),
    (5, 40, 7, dict(conv=0, u=(0.0, 0.08, 0.0), diff=2, K=(0.05, 0.0, 0.0, 0.04, 0.01, 0.03), se=1.0, r1=0.03)),
]


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16s"])
@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}x{c[2]}" for c in CASES])
@pytest.mark.parametrize("block_rows", [0, 2])
def test_d3q19_parity(prec, case, block_rows):
    nx, ny, nz, coef = case
    rng = np.random.default_rng(nx * ny + nz)
    phi0 = rng.uniform(0.2, 0.8, (nz, ny, nx))
    ref = D.run(D.Spec3(nx=nx, ny=ny, nz=nz, **coef), phi0, 25)
    s = Solver3(nx, ny, nz, prec=prec, block_rows=block_rows).set_coeffs(**coef)
    s.set_phi(torch.from_numpy(phi0).cuda())
    s.step(25)
    got = s.phi().cpu().numpy()
    assert rel(got, ref) <= TOL[prec], rel(got, ref)
    r = s.reduce(torch.from_numpy(ref).cuda())
    assert abs(r["sum"] - got.sum()) <= 1e-9 * abs(got.sum())
    if prec == "bf16s" and coef.get("r0", 0.0) == 0.0 and coef.get("r1", 0.0) == 0.0:
        # the shift plane keeps each node's stored mass: the total is conserved to FP32 rounding
        assert abs(got.sum() - phi0.sum()) <= 1e-5 * phi0.sum()


def test_d3q19_gaussian_hill_96():
    """The 3-D Gaussian hill with a full tensor K at 96^3, 200 steps: FP64 and
    FP32 against the oracle, and both within 4e-3 (GRE) of Eq. 60."""
    from test_oracle_d3q19 import gaussian3
    n, K, u = 96, (0.02, 0.006, 0.004, 0.015, 0.003, 0.01), (0.02, 0.01, -0.015)
    phi0 = gaussian3(n, n / 2, 8.0, u, K, 0.0)
    sp = D.Spec3(nx=n, ny=n, nz=n, conv=0, u=u, K=K, se=1.1)
    ref = D.run(sp, phi0, 200)
    exact = gaussian3(n, n / 2, 8.0, u, K, 200)
    for prec in ("f64", "f32", "bf16s"):
        s = Solver3(n, n, n, prec=prec).set_coeffs(conv=0, u=u, K=K, se=1.1)
        s.set_phi(torch.from_numpy(phi0).cuda())
        s.step(200)
        got = s.phi().cpu().numpy()
        assert rel(got, ref) <= TOL[prec], (prec, rel(got, ref))
        assert np.abs(got - exact).sum() / np.abs(exact).sum() < 4e-3      # oracle: 2.25e-3


@pytest.mark.parametrize("prec", ["f32", "bf16s"])
def test_d3q19_replays_from_a_cuda_graph(prec):
    """Solver3.capture / replay: four replays of 6 recorded steps equal 24 direct
    steps bit for bit, and match the oracle."""
    nx, ny, nz, coef = CASES[1]
    rng = np.random.default_rng(44)
    phi0 = rng.uniform(0.2, 0.8, (nz, ny, nx))
    dev = torch.from_numpy(phi0).cuda()
    s = Solver3(nx, ny, nz, prec=prec).set_coeffs(**coef).set_phi(dev).capture(6)
    for _ in range(4):
        s.replay()
    torch.cuda.synchronize()
    d = Solver3(nx, ny, nz, prec=prec).set_coeffs(**coef).set_phi(dev).step(24)
    assert torch.equal(s.phi().cpu(), d.phi().cpu())
    ref = D.run(D.Spec3(nx=nx, ny=ny, nz=nz, **coef), phi0, 24)
    assert rel(s.phi().cpu().numpy(), ref) <= TOL[prec]
    with pytest.raises(ValueError):
        s.capture(5)


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16s"])
def test_d3q19_checkpoint_resume(prec):
    """lbm3_save / lbm3_load: resuming from the state saved at step 10 repeats
    steps 11..20 bit for bit (the BF16S shift plane travels with the state), and
    a fresh solver loaded from the checkpoint continues identically."""
    nx, ny, nz, coef = CASES[2]
    rng = np.random.default_rng(9)
    phi0 = torch.from_numpy(rng.uniform(0.2, 0.8, (nz, ny, nx))).cuda()
    s = Solver3(nx, ny, nz, prec=prec).set_coeffs(**coef).set_phi(phi0).step(10)
    ck = s.save()
    s.step(10)
    first = s.phi().cpu()
    s.load(ck).step(10)
    assert torch.equal(first, s.phi().cpu())
    t = Solver3(nx, ny, nz, prec=prec).set_coeffs(**coef).load(ck).step(10)
    assert torch.equal(first, t.phi().cpu())
    ref = D.run(D.Spec3(nx=nx, ny=ny, nz=nz, **coef), phi0.cpu().numpy(), 20)
    assert rel(first.numpy(), ref) <= TOL[prec]


WALLS = [((1, 0, 0), (0.2, 0.7, 0, 0, 0, 0)), ((0, 1, 1), (0, 0, 0.1, 0.9, 0.5, 0.3)),
         ((1, 1, 1), (0.3, 0.6, 0.2, 0.8, 0.4, 0.5)), ((0, 0, 1), (0, 0, 0, 0, 0.0, 1.0))]


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16s"])
@pytest.mark.parametrize("walls", WALLS, ids=["x", "yz", "xyz", "z"])
@pytest.mark.parametrize("case", CASES[:3], ids=[f"{c[0]}x{c[1]}x{c[2]}" for c in CASES[:3]])
def test_d3q19_walls_parity(prec, walls, case):
    """Anti-bounce-back walls on one, two or all three axes (edge and corner
    links included) against the oracle, on ragged grids with every flux family
    and sources, all elements."""
    nx, ny, nz, coef = case
    bc, pw = walls
    rng = np.random.default_rng(nx + 7 * ny + 31 * nz)
    phi0 = rng.uniform(0.2, 0.8, (nz, ny, nx))
    ref = D.run(D.Spec3(nx=nx, ny=ny, nz=nz, bc=bc, phi_wall=pw, **coef), phi0, 25)
    names = ["abb" if b else "periodic" for b in bc]
    s = Solver3(nx, ny, nz, prec=prec, bc=names, phi_wall=pw).set_coeffs(**coef)
    s.set_phi(torch.from_numpy(phi0).cuda())
    s.step(25)
    got = s.phi().cpu().numpy()
    assert rel(got, ref) <= TOL[prec], rel(got, ref)
    band = np.zeros_like(got, dtype=bool)
    for ax, b in zip((2, 1, 0), bc):
        if b:
            idx = [slice(None)] * 3
            idx[ax] = [0, got.shape[ax] - 1]
            band[tuple(idx)] = True
    assert float(np.linalg.norm((got - ref)[band]) / np.linalg.norm(ref[band])) <= TOL[prec]


def test_d3q19_channel_slip_on_the_gpu():
    """The Sec. 3.6 channel embedded in 3-D (walls along y, periodic x and z,
    flow along x): the FP64 GPU state reaches Eq. 71 with the slip of Eq. 72b
    (s1 -> s_e) to 1e-12, as the oracle does."""
    N, se, s3 = 6, 0.8, 0.3
    kap = D.CS2 * (1.0 / s3 - 0.5)
    s = Solver3(4, N, 3, prec="f64", bc=("periodic", "abb", "periodic"), phi_wall=(0, 0, 0, 1, 0, 0))
    s.set_coeffs(conv=0, u=(0.04, 0.0, -0.03), K=(kap, 0, 0, kap, 0, kap), se=se, r0=2 * kap / N ** 2)
    s.set_phi(torch.zeros((3, N, 4), dtype=torch.float64, device="cuda"))
    s.step(int(60 * N * N / kap) + 200)
    phi = s.phi().cpu().numpy()
    yb = (np.arange(N) + 0.5) / N
    exact = yb * (2 - yb) + (se * s3 - 8 * (se + s3) + 16) / (12 * N ** 2 * se * s3)
    assert np.abs(phi - exact[None, :, None]).max() < 1e-12



@pytest.mark.parametrize("prec", ["f64", "f32", "bf16s"])
@pytest.mark.parametrize("walls", [False, True], ids=["periodic", "y-walls"])
def test_d3q19_large_plane_addressing(prec, walls):
    """A lattice whose 19 planes hold more than 2^32 elements (2 x 54 x 65472 with
    rows padded to 64 elements: 19 x 226,271,232) is addressed through 64-bit
    plane pointers, a small one through 32-bit offsets from the buffer. A field of
    period 64 along z stays periodic, so the large lattice must repeat the
    64-layer lattice's result bit for bit in every period."""
    nx, ny, nz, per = 2, 54, 65472, 64
    coef = dict(conv=1, u=(0.03, -0.05, 0.04), diff=2, K=(0.02, 0.003, -0.002, 0.03, 0.004, 0.025), se=1.1,
                r0=0.001, r1=-0.02)
    bc = ("periodic", "abb", "periodic") if walls else ("periodic",) * 3
    extra = dict(bc=bc, phi_wall=(0.0, 0.0, 0.3, 0.7, 0.0, 0.0)) if walls else {}
    rng = np.random.default_rng(64)
    small0 = torch.from_numpy(rng.uniform(0.2, 0.8, (per, ny, nx))).cuda()
    s = Solver3(nx, ny, per, prec=prec, **extra).set_coeffs(**coef).set_phi(small0).step(7)
    want = s.phi()
    del s
    big = Solver3(nx, ny, nz, prec=prec, **extra).set_coeffs(**coef).set_phi(small0.repeat(nz // per, 1, 1)).step(7)
    got = big.phi().view(nz // per, per, ny, nx)
    del big
    torch.cuda.empty_cache()
    assert torch.equal(got, want.expand_as(got))
