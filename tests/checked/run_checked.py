"""Runs every kernel family of liblbm_checked.so on small grids (ragged sizes,
all wall combinations) and prints one JSON line: the index-fault words and the
largest relative error against the FP64 oracle. Started by test_gpu_checked.py
with LBM_LIBRARY=checked in a fresh process."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import ctypes  # noqa: E402

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402
from paper_1603_09577_gb300 import Ensemble, Solver, adjoint  # noqa: E402
from paper_1603_09577_gb300 import _lib as C  # noqa: E402

BCN = {0: "periodic", 1: "abb", 2: "nee"}


def flags(s):
    f = ctypes.c_int()
    C.check(s.lib.lbm_debug_flags(s.h, ctypes.byref(f), None))
    return f.value


def main():
    out = {"checked": C.lib().lbm_build_checked(), "faults": [], "max_rel": 0.0}
    cases = [(37, 29, (1, 1)), (64, 40, (0, 0)), (100, 66, (0, 1)), (132, 35, (1, 0)), (8, 5, (1, 1)),
             (201, 90, (0, 0)), (190, 77, (1, 1))]
    configs = [("f64", 1, 1, 0), ("f32", 1, 1, 0), ("f32", 2, 1, 0), ("bf16s", 2, 1, 0),
               ("f32", 0, 2, 0), ("f32", 0, 2, 4), ("bf16s", 0, 2, 4), ("f32", 3, 2, 1),
               ("f32", 4, 2, 0), ("f32", 5, 2, 0), ("f32", 5, 2, 4), ("bf16s", 5, 2, 0), ("bf16s", 5, 2, 4),
               ("bf16s", 5, 2, 2)]
    coef = dict(conv=1, u=(0.06, -0.03), diff=2, K=(0.02, 0.008, 0.01), r1=-0.05)
    for nx, ny, bc in cases:
        phi0 = W.phi0_aniso(nx, seed=nx + ny, ny=ny)
        walls = (0.1, 0.2, 0.3, 0.4)
        ref = O.run(O.Spec(nx=nx, ny=ny, bc_x=bc[0], bc_y=bc[1], phi_wall=walls, s=W.s9(), **coef), phi0, 10)
        for prec, var, spp, br in configs:
            if var == 2 and nx % 4:
                continue
            s = Solver(nx, ny, prec=prec, bc=(BCN[bc[0]], BCN[bc[1]]), phi_wall=walls, steps_per_pass=spp,
                       kernel_variant=var, block_rows=br)
            s.set_coeffs(s=W.s9(), **coef)
            s.set_phi(torch.from_numpy(phi0).cuda())
            s.step(10)
            got = s.phi().cpu().numpy()
            out["faults"].append(flags(s))
            out["max_rel"] = max(out["max_rel"], float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
                                 if prec != "bf16s" else 0.0)
    # general path: Scheme A, power-law flux, Fisher source, extrapolated walls
    for nx, ny, bc in [(37, 29, (2, 2)), (40, 26, (2, 0)), (33, 41, (0, 2)), (3, 5, (2, 2)), (35, 22, (1, 0)),
                       (61, 31, (2, 2))]:
        phi0 = W.phi0_aniso(nx, seed=nx * ny, ny=ny)
        rng = np.random.default_rng(nx)
        bv = rng.uniform(0.3, 0.7, (10, 2 * (nx + ny))) if 2 in bc else None
        gcoef = dict(conv=2, power=1, u=(0.06, -0.03), diff=1, K=(0.02, 0.008, 0.01), src_family=1, b=0.02)
        ref = O.run_x(O.Spec(nx=nx, ny=ny, bc_x=bc[0], bc_y=bc[1], phi_wall=(0.1, 0.2, 0.3, 0.4), s=W.s9(),
                             scheme=1, **gcoef), phi0, 10, bv)
        for prec, spp in (("f64", 1), ("f32", 1), ("f32", 2)):
            s = Solver(nx, ny, prec=prec, bc=(BCN[bc[0]], BCN[bc[1]]), phi_wall=(0.1, 0.2, 0.3, 0.4), scheme="A",
                       steps_per_pass=spp)
            s.set_coeffs(s=W.s9(), **gcoef)
            if bv is not None:
                s.set_dirichlet(torch.from_numpy(bv).cuda())
            s.set_phi(torch.from_numpy(phi0).cuda())
            s.step(10)
            got = s.phi().cpu().numpy()
            out["faults"].append(flags(s))
            out["max_rel"] = max(out["max_rel"], float(np.linalg.norm(got - ref) / np.linalg.norm(ref)))
    # D3Q19
    from oracle import d3q19 as D3
    from paper_1603_09577_gb300 import Solver3
    for nx, ny, nz, bc in [(21, 9, 6, (0, 0, 0)), (5, 33, 3, (0, 0, 0)), (40, 2, 4, (0, 0, 0)), (21, 9, 6, (1, 1, 1)),
                           (33, 4, 5, (1, 0, 1))]:
        c3 = dict(conv=1, u=(0.05, -0.03, 0.02), diff=1, K=(0.02, 0.004, -0.003, 0.015, 0.002, 0.012), se=1.2)
        pw = (0.1, 0.2, 0.3, 0.4, 0.5, 0.6)
        phi3 = np.random.default_rng(nx).uniform(0.2, 0.8, (nz, ny, nx))
        ref3 = D3.run(D3.Spec3(nx=nx, ny=ny, nz=nz, bc=bc, phi_wall=pw, **c3), phi3, 6)
        for prec in ("f64", "f32", "bf16s"):
            s3 = Solver3(nx, ny, nz, prec=prec, bc=["abb" if b else "periodic" for b in bc], phi_wall=pw).set_coeffs(**c3)
            s3.set_phi(torch.from_numpy(phi3).cuda())
            s3.step(6)
            got = s3.phi().cpu().numpy()
            f = ctypes.c_int()
            C.check(s3.lib.lbm3_debug_flags(s3.h, ctypes.byref(f), None))
            out["faults"].append(f.value)
            if prec != "bf16s":
                out["max_rel"] = max(out["max_rel"], float(np.linalg.norm(got - ref3) / np.linalg.norm(ref3)))
    # adjoint and ensemble
    Kf, phi0, tgt = W.adjoint_inputs(36, seed=3, ny=20)
    p0 = torch.from_numpy(phi0).cuda().requires_grad_(True)
    K = torch.from_numpy(Kf).cuda().requires_grad_(True)
    u = torch.tensor((0.02, 0.01), dtype=torch.float64, device="cuda", requires_grad=True)
    o = adjoint.run(p0, K, u, 12, ckpt_every=5, prec="f32", s_rates=W.s9())
    (0.5 * ((o - torch.from_numpy(tgt).cuda()) ** 2).sum()).backward()
    inst = W.ensemble(count=5, seed=9)
    inst = [dict(d, nx=n, ny=m, xc=n / 2, yc=m / 2, sigma=4.0) for d, (n, m) in
            zip(inst, [(33, 40), (64, 64), (70, 31), (8, 9), (129, 65)])]
    e = Ensemble(inst)
    e.set_phi(e.pack([W.ensemble_phi0(d) for d in inst]))
    e.step(7)
    f = ctypes.c_int()
    C.check(e.lib.lbm_ensemble_debug_flags(e.h, ctypes.byref(f), None))
    out["faults"].append(f.value)
    torch.cuda.synchronize()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
