"""Host logic of the autotuner, on the CPU: every candidate it may time is a
description the library accepts, it keeps the fastest, caches it per device
and problem in JSON (atomically, surviving a corrupt file), reuses the cache,
and routes general-path problems to the general kernels. The timing itself
(CUDA events) is replaced by a fake here; the GPU test times real kernels."""
import ctypes
import json

import pytest

from paper_1603_09577_gb300 import _lib as C
from paper_1603_09577_gb300 import tune
from paper_1603_09577_gb300.solver import BC, SCHEME


def desc_rc(nx, ny, prec, bc, cfg, per_cell_K=False, scheme="B"):
    d = C.Desc()
    d.nx, d.ny, d.prec = nx, ny, C.PREC[prec]
    d.bc_x, d.bc_y = BC[bc[0]], BC[bc[1]]
    d.steps_per_pass = cfg["steps_per_pass"]
    d.per_cell_K = int(per_cell_K)
    d.kernel_variant, d.block_rows = cfg["kernel_variant"], cfg["block_rows"]
    d.scheme = SCHEME[scheme]
    n = ctypes.c_size_t()
    return C.lib().lbm_workspace_size(ctypes.byref(d), ctypes.byref(n))


@pytest.mark.parametrize("nx,ny,prec", [(4096, 4096, "f32"), (4096, 4096, "bf16s"), (4096, 4096, "f64"),
                                        (1002, 517, "f32"), (64, 48, "bf16s")])
@pytest.mark.parametrize("bc", [("abb", "abb"), ("periodic", "periodic")])
def test_every_candidate_is_a_valid_description(nx, ny, prec, bc):
    cands = tune.candidates(nx, prec)
    assert len(cands) == len({json.dumps(c, sort_keys=True) for c in cands})      # no duplicates
    for cfg in cands:
        assert desc_rc(nx, ny, prec, bc, cfg) == C.LBM_OK, cfg
    if prec == "f64":
        assert all(c["steps_per_pass"] == 1 for c in cands)                     # no FP64 two-step kernel
    if nx % 4:
        assert all(c["kernel_variant"] != 2 for c in cands)                      # four-node kernel needs nx % 4 == 0


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("per_cell_K", [False, True])
def test_general_candidates_are_valid(prec, per_cell_K):
    cands = tune.general_candidates(prec, per_cell_K)
    for cfg in cands:
        assert desc_rc(200, 150, prec, ("nee", "nee"), cfg, per_cell_K, scheme="A") == C.LBM_OK, cfg
    two_step = [c for c in cands if c["steps_per_pass"] == 2]
    assert bool(two_step) == (prec == "f32" and not per_cell_K)


@pytest.fixture
def fake_device(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "tune.json"
    monkeypatch.setenv("LBM_TUNE_CACHE", str(path))
    name = {"value": "FakeGPU-A"}
    monkeypatch.setattr(tune.torch.cuda, "get_device_name", lambda *a, **k: name["value"])
    calls = []

    def fake_time(cfg, nx, ny, prec, bc, conv, diff, per_cell_K, steps, reps, scheme="B"):
        calls.append((dict(cfg), scheme))
        # a fixed cost per configuration; the TMA-staged variant (4) is the fastest
        return 0.5 if cfg["kernel_variant"] == 4 else 1.0 + 0.01 * cfg["block_rows"] + 0.1 * cfg["kernel_variant"]

    monkeypatch.setattr(tune, "_time", fake_time)
    return path, name, calls


def test_tune_keeps_the_fastest_and_reuses_the_cache(fake_device):
    path, name, calls = fake_device
    cfg = tune.tune(512, 256, "f32", bc=("abb", "periodic"), conv=1, diff=2)
    assert cfg == dict(kernel_variant=4, block_rows=0, steps_per_pass=2)
    n_cands = len(tune.candidates(512, "f32"))
    assert len(calls) == n_cands
    data = json.loads(path.read_text())
    (key, entry), = data.items()
    assert key.startswith("FakeGPU-A|512x256|f32|abb,periodic|c1d2|K0|sB")
    assert entry["config"] == cfg and entry["ms_per_step"] == 0.5 and len(entry["all"]) == n_cands
    assert not list(path.parent.glob("*.tmp*"))                               # written atomically
    # cached: no more timing
    assert tune.tune(512, 256, "f32", bc=("abb", "periodic"), conv=1, diff=2) == cfg
    assert len(calls) == n_cands
    # use_cache=False times again; another problem and another device get their own entries
    tune.tune(512, 256, "f32", bc=("abb", "periodic"), conv=1, diff=2, use_cache=False)
    assert len(calls) == 2 * n_cands
    tune.tune(512, 256, "bf16s", bc=("abb", "periodic"), conv=1, diff=2)
    name["value"] = "FakeGPU-B"
    tune.tune(512, 256, "f32", bc=("abb", "periodic"), conv=1, diff=2)
    assert len(json.loads(path.read_text())) == 3


def test_tune_survives_a_corrupt_cache(fake_device):
    path, _, calls = fake_device
    path.parent.mkdir(parents=True)
    path.write_text("{not json")
    cfg = tune.tune(256, 256, "f64", bc=("periodic", "periodic"))
    assert cfg["steps_per_pass"] == 1 and calls
    assert list(json.loads(path.read_text()).values())[0]["config"] == cfg


@pytest.mark.parametrize("kw", [dict(scheme="A"), dict(bc=("nee", "periodic")), dict(conv=2), dict(diff=3)])
def test_general_problems_time_the_general_kernels(fake_device, kw):
    _, _, calls = fake_device
    args = dict(bc=("periodic", "periodic"), conv=0, diff=0, scheme="B")
    args.update(kw)
    cfg = tune.tune(300, 200, "f32", **args)
    cands = tune.general_candidates("f32", False)
    assert [c for c, _ in calls] == cands
    assert cfg in cands
    assert all(s == args["scheme"] for _, s in calls)
