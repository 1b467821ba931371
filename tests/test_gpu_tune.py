"""The autotuner: picks a valid configuration, persists it, reuses the cache,
and the tuned solver still matches the oracle."""
import json

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from paper_1603_09577_gb300 import Solver, tune

pytestmark = pytest.mark.gpu


def test_tune_persists_and_tuned_solver_is_correct(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("LBM_TUNE_CACHE", str(path))
    nx, ny = 256, 192
    cfg = tune.tune(nx, ny, "f32", bc=("abb", "periodic"), conv=1, diff=2, steps=5, reps=1)
    assert cfg in tune.candidates(nx, "f32")
    data = json.loads(path.read_text())
    (entry,) = data.values()
    assert entry["config"] == cfg and len(entry["all"]) == len(tune.candidates(nx, "f32"))
    assert tune.tune(nx, ny, "f32", bc=("abb", "periodic"), conv=1, diff=2) == cfg     # cached
    phi0 = W.phi0_aniso(nx, seed=5, ny=ny)
    coef = dict(conv=1, u=(0.05, 0.03), diff=2, K=(0.02, 0.008, 0.01), r1=-0.1)
    s = Solver(nx, ny, prec="f32", bc=("abb", "periodic"), phi_wall=(0.1, 0.2, 0, 0), **cfg)
    s.set_coeffs(s=W.s9(), **coef)
    s.set_phi(torch.from_numpy(phi0).cuda())
    s.step(31)
    ref = O.run(O.Spec(nx=nx, ny=ny, bc_x=1, bc_y=0, phi_wall=(0.1, 0.2, 0, 0), s=W.s9(), **coef), phi0, 31)
    got = s.phi().cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5


def test_tune_general_path(tmp_path, monkeypatch):
    """A Scheme A problem with extrapolated walls tunes among the general kernels,
    and the tuned solver matches the oracle."""
    monkeypatch.setenv("LBM_TUNE_CACHE", str(tmp_path / "tune.json"))
    nx, ny = 200, 150
    cfg = tune.tune(nx, ny, "f32", bc=("nee", "nee"), conv=2, diff=0, scheme="A", steps=6, reps=1)
    assert cfg in tune.general_candidates("f32", False)
    rng = np.random.default_rng(3)
    phi0 = W.jacobi_smooth(rng.uniform(0.2, 0.8, (ny, nx)), 2)
    bv = rng.uniform(0.3, 0.7, (1, 2 * (nx + ny)))
    coef = dict(conv=2, power=1, u=(0.06, 0.0), diff=0, K=(0.05, 0.0, 0.05), src_family=1, b=0.01)
    s = Solver(nx, ny, prec="f32", bc=("nee", "nee"), scheme="A", **cfg).set_coeffs(s=W.s9(), **coef)
    s.set_dirichlet(torch.from_numpy(bv).cuda())
    s.set_phi(torch.from_numpy(phi0).cuda())
    s.step(31)
    sp = O.Spec(nx=nx, ny=ny, bc_x=2, bc_y=2, s=W.s9(), scheme=1, **coef)
    ref = O.run_x(sp, phi0, 31, np.repeat(bv, 31, axis=0))
    got = s.phi().cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
