"""The batched ensemble (one persistent launch per step over all instances)
against the FP64 oracle per instance, against one launch per instance and a
replayed CUDA graph (bit for bit), and on the full 256-instance workload."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from paper_1603_09577_gb300.ensemble import Ensemble

pytestmark = pytest.mark.gpu


_ORACLE = {}


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def small_instances():
    base = W.ensemble(count=7, seed=17)
    sizes = [(33, 40), (40, 33), (64, 64), (70, 96), (96, 70), (100, 100), (130, 65)]
    out = []
    for d, (nx, ny) in zip(base, sizes):
        d = dict(d, nx=nx, ny=ny, xc=nx / 2, yc=ny / 3, sigma=max(4.0, nx / 8))
        out.append(d)
    return out


def oracle_phi(d, phi0, steps, conv=0, diff=1):
    sp = O.Spec(nx=d["nx"], ny=d["ny"], conv=conv, u=d["u"], diff=diff, K=d["K"], s=d["s"])
    return O.run(sp, phi0, steps)


@pytest.mark.parametrize("conv,diff", [(0, 1), (1, 2)])
def test_ensemble_matches_oracle(conv, diff):
    inst = small_instances()
    phis = [W.ensemble_phi0(d) for d in inst]
    e = Ensemble(inst, conv=conv, diff=diff)
    e.set_phi(e.pack(phis))
    e.step(150)
    got = e.unpack(e.phi().cpu())
    for d, p0, g in zip(inst, phis, got):
        ref = oracle_phi(d, p0, 150, conv, diff)
        assert rel(g.numpy(), ref) <= 1e-5, (d["nx"], d["ny"], rel(g.numpy(), ref))


@pytest.mark.parametrize("steps", [150, 151])
def test_ensemble_two_steps_per_pass_matches_oracle(steps):
    inst = small_instances()
    phis = [W.ensemble_phi0(d) for d in inst]
    e = Ensemble(inst, steps_per_pass=2)
    e.set_phi(e.pack(phis))
    e.step(steps)
    got = e.unpack(e.phi().cpu())
    for d, p0, g in zip(inst, phis, got):
        ref = oracle_phi(d, p0, steps)
        assert rel(g.numpy(), ref) <= 1e-5, (d["nx"], d["ny"], rel(g.numpy(), ref))
    # a replayed graph of two-step launches gives the same state as direct launches
    e2 = Ensemble(inst, steps_per_pass=2)
    e2.set_phi(e2.pack(phis))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        e2.capture(20)
        for _ in range(3):
            e2.replay()
    torch.cuda.current_stream().wait_stream(side)
    e.set_phi(e.pack(phis))
    e.step(60)
    assert torch.equal(e2.phi().cpu(), e.phi().cpu())
    # the persistent grid walking the tile list computes the same state bit for bit
    e3 = Ensemble(inst, steps_per_pass=2, persistent=True)
    e3.set_phi(e3.pack(phis))
    e3.step(60)
    assert torch.equal(e3.phi().cpu(), e.phi().cpu())


def test_ensemble_modes_agree_bitwise():
    inst = small_instances()
    packed = None
    outs = []
    for mode in ("one_launch", "per_instance", "graph", "persistent_grid"):
        e = Ensemble(inst, persistent=mode == "persistent_grid")
        if packed is None:
            packed = e.pack([W.ensemble_phi0(d) for d in inst])
        e.set_phi(packed)
        if mode in ("one_launch", "persistent_grid"):
            e.step(40)
        elif mode == "per_instance":
            e.step(40, mode=1)
        else:
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                e.capture(10)
                for _ in range(4):
                    e.replay()
            torch.cuda.current_stream().wait_stream(s)
        outs.append(e.phi().cpu())
    assert all(torch.equal(outs[0], o) for o in outs[1:])


@pytest.mark.parametrize("spp", [1, 2])
def test_ensemble_full_workload(spp):
    """256 instances (sides 64..1024, 48.6 M nodes), 1000 steps through a
    replayed graph: finite, mass conserved per instance, and the six smallest
    instances and the largest one (1022^2 nodes) within the FP32 bar of the
    oracle, as relative L2 and node by node."""
    inst = W.ensemble()
    e = Ensemble(inst, steps_per_pass=spp)
    phis = [W.ensemble_phi0(d) for d in inst]
    e.set_phi(e.pack(phis))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        e.capture(100)
        for _ in range(10):
            e.replay()
    torch.cuda.current_stream().wait_stream(s)
    out = e.unpack(e.phi().cpu())
    assert all(torch.isfinite(o).all() for o in out)
    for p0, o in zip(phis, out):
        assert abs(float(o.sum()) - p0.sum()) <= 1e-5 * p0.sum()
    sizes = [d["nx"] * d["ny"] for d in inst]
    order = list(np.argsort(sizes)[:6]) + [int(np.argmax(sizes))]
    for i in order:
        key = (i, 1000)
        if key not in _ORACLE:
            _ORACLE[key] = oracle_phi(inst[i], phis[i], 1000)
        ref = _ORACLE[key]
        g = out[i].numpy()
        mx = float(np.abs(g - ref).max() / np.abs(ref).max())
        print(f"[parity] ensemble instance {i} ({inst[i]['nx']}^2) spp {spp}: rel_l2={rel(g, ref):.3e} max_node={mx:.3e}")
        assert rel(g, ref) <= 1e-5, (i, rel(g, ref))
        assert mx <= 2e-5, (i, mx)


def test_ensemble_per_instance_reductions():
    """lbm_ensemble_reduce: every instance's eight statistics equal their
    definitions evaluated with numpy on the returned phi (sums to 1e-12, the
    maximum and the non-finite count exactly), the GRE against the oracle stays at
    the parity level, repeated calls agree bit for bit, and a NaN placed in one
    instance is counted there alone."""
    inst = small_instances()
    phis = [W.ensemble_phi0(d) for d in inst]
    e = Ensemble(inst, steps_per_pass=2)
    e.set_phi(e.pack(phis))
    e.step(60)
    refs = [oracle_phi(d, p0, 60) for d, p0 in zip(inst, phis)]
    packed_ref = e.pack(refs)
    out = e.reduce_async(packed_ref)
    again = e.reduce_async(packed_ref, out=torch.empty_like(out))
    assert torch.equal(out, again)
    stats = e.reduce(packed_ref)
    got = e.unpack(e.phi().cpu())
    for st, g, r in zip(stats, got, refs):
        g = g.numpy()
        d = g - r
        assert st["nonfinite"] == 0.0
        assert st["max_abs"] == np.abs(g).max()
        for key, val in (("sum", g.sum()), ("sum_sq", (g * g).sum()), ("abs_err", np.abs(d).sum()),
                         ("abs_ref", np.abs(r).sum()), ("sq_err", (d * d).sum()), ("sq_ref", (r * r).sum())):
            assert abs(st[key] - val) <= 1e-12 * abs(val) + 1e-300, (key, st[key], val)
        assert st["abs_err"] / st["abs_ref"] <= 1e-5
    plain = e.reduce()
    for st in plain:
        assert st["abs_err"] == st["abs_ref"] == st["sq_err"] == st["sq_ref"] == 0.0
    # a NaN in instance 3's initial field is counted in instance 3 only
    bad = [p.copy() for p in phis]
    bad[3][5, 7] = np.nan
    e.set_phi(e.pack(bad))
    counts = [st["nonfinite"] for st in e.reduce()]
    assert counts == [0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0]


def mixed_instances():
    """Small instances plus two with interior tiles of both two-step shapes."""
    out = small_instances()
    extra = W.ensemble(count=2, seed=23)
    for d, (nx, ny) in zip(extra, [(260, 150), (199, 131)]):
        out.append(dict(d, nx=nx, ny=ny, xc=nx / 3, yc=ny / 2, sigma=nx / 10))
    return out


@pytest.mark.parametrize("pair_tiles", [False, True])
@pytest.mark.parametrize("persistent", [0, 1, 2])
def test_ensemble_two_step_launches_agree_bitwise(pair_tiles, persistent):
    """Every two-step launch of the ensemble (30 x 30 or 62 x 14 pair tiles; one
    block per tile, a strided persistent grid, or a persistent grid claiming
    tiles from a counter) gives the same state bit for bit, directly and when
    replayed from a CUDA graph (the claim counter starts from zero in every
    replay), and the state matches the oracle."""
    inst = mixed_instances()
    phis = [W.ensemble_phi0(d) for d in inst]
    base = Ensemble(inst, steps_per_pass=2)
    base.set_phi(base.pack(phis))
    base.step(61)
    want = base.phi().cpu()
    e = Ensemble(inst, steps_per_pass=2, persistent=persistent, pair_tiles=pair_tiles)
    e.set_phi(e.pack(phis))
    e.step(61)
    assert torch.equal(e.phi().cpu(), want)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        e.set_phi(e.pack(phis))
        e.capture(20)
        for _ in range(3):
            e.replay()
        e.step(1)
    torch.cuda.current_stream().wait_stream(side)
    assert torch.equal(e.phi().cpu(), want)
    got = e.unpack(want)
    for i in (len(inst) - 2, len(inst) - 1, 0):
        key = (repr(sorted(inst[i].items())), 61)
        if key not in _ORACLE:
            _ORACLE[key] = oracle_phi(inst[i], phis[i], 61)
        assert rel(got[i].numpy(), _ORACLE[key]) <= 1e-5


def test_ensemble_autotuner_picks_a_candidate_and_caches(tmp_path, monkeypatch):
    from paper_1603_09577_gb300 import tune
    monkeypatch.setenv("LBM_TUNE_CACHE", str(tmp_path / "tune.json"))
    inst = mixed_instances()
    cfg = tune.tune_ensemble(inst, conv=0, diff=1, steps=4, reps=1)
    assert cfg in tune.ensemble_candidates()
    import json
    cache = json.loads((tmp_path / "tune.json").read_text())
    (key, entry), = cache.items()
    assert "ensemble" in key and len(entry["all"]) == len(tune.ensemble_candidates())
    assert tune.tune_ensemble(inst, conv=0, diff=1) == cfg           # from the cache
