"""The CUDA adjoint (through the C ABI and the autograd Function) against the
FP64 oracle's discrete adjoint, central finite differences on the FP64 CUDA
path at the full 512^2 x 500-step workload, and the dot-product identity."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from paper_1603_09577_gb300 import Solver, adjoint

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def gpu_grads(phi0, Kf, tgt, u, steps, ckpt, prec):
    p0 = torch.from_numpy(phi0).cuda().requires_grad_(True)
    K = torch.from_numpy(Kf).cuda().requires_grad_(True)
    uu = torch.tensor(u, dtype=torch.float64, device="cuda", requires_grad=True)
    out = adjoint.run(p0, K, uu, steps, ckpt_every=ckpt, prec=prec, s_rates=W.s9())
    loss = 0.5 * ((out - torch.from_numpy(tgt).cuda()) ** 2).sum()
    loss.backward()
    return float(loss.detach()), p0.grad.cpu().numpy(), K.grad.cpu().numpy(), uu.grad.cpu().numpy()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-4)])
def test_adjoint_matches_oracle(prec, tol):
    nx, ny, steps, ckpt = 40, 24, 30, 7
    Kf, phi0, tgt = W.adjoint_inputs(nx, seed=21, ny=ny)
    u = (0.03, -0.01)
    L_o, dphi_o, dK_o, du_o = O.adjoint(O.Spec(nx=nx, ny=ny, conv=0, u=u, Kfield=Kf, s=W.s9()), phi0, tgt, steps)
    L_g, dphi_g, dK_g, du_g = gpu_grads(phi0, Kf, tgt, u, steps, ckpt, prec)
    assert abs(L_g - L_o) <= tol * abs(L_o)
    assert rel(dphi_g, dphi_o) <= tol
    assert rel(dK_g, dK_o) <= tol
    assert rel(du_g, du_o) <= tol


def test_adjoint_dot_product_f64():
    nx, ny, steps = 36, 20, 25
    Kf, _, _ = W.adjoint_inputs(nx, seed=22, ny=ny)
    rng = np.random.default_rng(23)
    r, d = rng.normal(size=(ny, nx)), rng.normal(size=(ny, nx))
    s = Solver(nx, ny, prec="f64", per_cell_K=True)
    s.set_coeffs(conv=0, u=(0.02, 0.01), diff=0, s=W.s9())
    s.set_K_field(torch.from_numpy(Kf).cuda())
    s.set_phi(torch.from_numpy(d).cuda())
    s.step(steps)
    Td = s.phi().cpu().numpy()
    # T^T r = gradient of 1/2 |T phi0 - (-r)|^2 at phi0 = 0
    _, g, _, _ = gpu_grads(np.zeros((ny, nx)), Kf, -r, (0.02, 0.01), steps, 6, "f64")
    lhs, rhs = float((r * Td).sum()), float((g * d).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.fixture(scope="module")
def full_case():
    p = W.params("adjoint_512")
    Kf, phi0, tgt = W.adjoint_inputs(512, seed=4)
    return p, Kf, phi0, tgt


def phi_f64(p, Kf, phi0):
    s = Solver(512, 512, prec="f64", per_cell_K=True)
    s.set_coeffs(conv=0, u=p["u"], diff=0, s=W.s9())
    s.set_K_field(torch.from_numpy(Kf).cuda())
    s.set_phi(torch.from_numpy(phi0).cuda())
    s.step(p["steps"])
    return s.phi()


def loss_diff(pp, pm, tgt):
    """L(+) - L(-) for L = 1/2 |phi - tgt|^2, summed from the field difference so
    that the cancellation happens node by node, not in two large sums."""
    t = torch.from_numpy(tgt).cuda()
    return float(((pp - pm) * (0.5 * (pp + pm) - t)).sum())


def test_adjoint_full_size_finite_differences_f64(full_case):
    """512^2, 500 steps, checkpoints every 50: central differences (h = 1e-6) on
    32 random entries of K(x) and phi0 against the FP64 adjoint.

    Bar: 1e-4 relative plus 1e-6 of the largest gradient entry. A central
    difference with h = 1e-6 over 262,144 nodes and 500 FP64 steps carries
    rounding noise of order eps sqrt(steps) sqrt(nodes) |phi - target| / (2h),
    up to ~5e-7 absolute here, so a tighter bar would test the noise; the
    adjoint's exactness is pinned against the FP64 oracle (1e-10) above."""
    p, Kf, phi0, tgt = full_case
    L, dphi, dK, du = gpu_grads(phi0, Kf, tgt, p["u"], p["steps"], p["ckpt_every"], "f64")
    L0 = 0.5 * float(((phi_f64(p, Kf, phi0) - torch.from_numpy(tgt).cuda()) ** 2).sum())
    assert abs(L - L0) <= 1e-12 * L
    rng = np.random.default_rng(24)
    h = 1e-6
    scale_K, scale_phi = np.abs(dK).max(), np.abs(dphi).max()
    for n in range(32):
        c, y, x = rng.integers(3), rng.integers(512), rng.integers(512)
        if n % 2 == 0:
            Kp, Km = Kf.copy(), Kf.copy()
            Kp[c, y, x] += h
            Km[c, y, x] -= h
            fd = loss_diff(phi_f64(p, Kp, phi0), phi_f64(p, Km, phi0), tgt) / (2 * h)
            assert abs(fd - dK[c, y, x]) <= 1e-4 * abs(fd) + 1e-6 * scale_K, (n, fd, dK[c, y, x])
        else:
            pp, pm = phi0.copy(), phi0.copy()
            pp[y, x] += h
            pm[y, x] -= h
            fd = loss_diff(phi_f64(p, Kf, pp), phi_f64(p, Kf, pm), tgt) / (2 * h)
            assert abs(fd - dphi[y, x]) <= 1e-4 * abs(fd) + 1e-6 * scale_phi, (n, fd, dphi[y, x])


def test_adjoint_full_size_f32_forward_vs_f64(full_case):
    """FP32 forward with FP64 gradient accumulation against the FP64 adjoint."""
    p, Kf, phi0, tgt = full_case
    _, d64, K64, u64 = gpu_grads(phi0, Kf, tgt, p["u"], p["steps"], p["ckpt_every"], "f64")
    _, d32, K32, u32 = gpu_grads(phi0, Kf, tgt, p["u"], p["steps"], p["ckpt_every"], "f32")
    assert rel(d32, d64) <= 1e-4
    assert rel(K32, K64) <= 1e-4
    assert rel(u32, u64) <= 1e-4


def test_adjoint_rejects_unsupported_solvers():
    from paper_1603_09577_gb300 import LBMError
    import ctypes
    from paper_1603_09577_gb300 import _lib as C
    s = Solver(16, 16, prec="bf16s")
    s.set_coeffs(conv=0, u=(0.01, 0.0), diff=0, K=(0.01, 0.0, 0.01), s=W.s9())
    n = ctypes.c_size_t()
    assert s.lib.lbm_adjoint_workspace_size(s.h, ctypes.byref(n)) == C.LBM_EUNSUPPORTED
    s = Solver(16, 16, prec="f32", bc=("abb", "periodic"))
    s.set_coeffs(conv=0, u=(0.01, 0.0), diff=0, K=(0.01, 0.0, 0.01), s=W.s9())
    assert s.lib.lbm_adjoint_workspace_size(s.h, ctypes.byref(n)) == C.LBM_EUNSUPPORTED
    s = Solver(16, 16, prec="f32")
    s.set_coeffs(conv=1, u=(0.01, 0.0), diff=0, K=(0.01, 0.0, 0.01), s=W.s9())
    with pytest.raises(LBMError):
        C.check(s.lib.lbm_adjoint_workspace_size(s.h, ctypes.byref(n)))
