"""Throughput benchmark of the fused D2Q9 MRT stream-collide path.

Workload: the anisotropic nonlinear diffusion problem with a source on a
4096 x 4096 grid with phi = 0 anti-bounce-back walls (D(phi) = (1 + phi^2) K,
K = [[0.02, 0.008], [0.008, 0.01]], R = -0.1 phi), 2000 time steps. One bench
step is that whole job: initialisation from the resident initial field, 2000
fused stream-collide steps and the FP64 mass reduction. The metric is MLUPS
(million lattice-node updates per second) over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec f32|bf16s|f64]
                  [--impl reference]

--impl reference times the FP64 CPU oracle on the host cores instead (each
step: one time step of the same 4096^2 workload).
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import math
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

WORKLOAD = "aniso_dirichlet_4096"
BYTES_PER_UPDATE = {"f32": 72, "bf16s": 44, "f64": 144}
# FP64 path: FP64 thread instructions per node update of k_step<F64> on this workload (ncu counts per launch of
# 16.8 M nodes: 906.0 M DADD + 335.8 M DFMA + 201.5 M DMUL = 86.0 per update); its roof is the FP64 pipe's rate,
# measured in the same run by the DFMA probe
FP64_INST_PER_UPDATE = 86
KERNEL_SRC = [os.path.join(ROOT, "paper_1603_09577_gb300", "csrc", f)
              for f in ("kernels_step.cu", "kernels_step_vec.cu", "kernels_step2.cuh", "kernels_step2_f32.cu",
                        "kernels_step2_bf16.cu", "lbm_device.cuh")]
PAIR_SRC = [os.path.join(ROOT, "paper_1603_09577_gb300", "csrc", f)
            for f in ("kernels_step2p.cuh", "kernels_step2p_f32.cu", "kernels_step2p_bf16.cu", "kernels_step2.cuh",
                      "lbm_device.cuh")]
GENERAL_SRC = [os.path.join(ROOT, "paper_1603_09577_gb300", "csrc", f)
               for f in ("kernels_general.cuh", "kernels_general_f32.cu", "kernels_general_f64.cu", "lbm_device.cuh")]
STEP2G_SRC = [os.path.join(ROOT, "paper_1603_09577_gb300", "csrc", f)
              for f in ("kernels_step2g.cu", "kernels_general.cuh", "lbm_device.cuh")]


def src_sha(files) -> str:
    return hashlib.sha256(b"".join(open(f, "rb").read() for f in files)).hexdigest()
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--prec", default="f32", choices=["f32", "bf16s", "f64"])
    ap.add_argument("--spp", type=int, default=1, help="time steps per sweep (1 or 2)")
    ap.add_argument("--lbm-steps", type=int, default=None, help="time steps per bench step")
    ap.add_argument("--variant", type=int, default=0, help="0 auto, 1 one node per thread, 2 four nodes per thread")
    ap.add_argument("--block-rows", type=int, default=0)
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="use --variant/--block-rows/--spp as given instead of the autotuner's choice")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--nx", type=int, default=None,
                    help="grid side (default: 4096 for the headline workload, 256 for gaussian3d; smaller sides serve profiler captures)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the sub-records (BF16S, FP64, adjoint, ensemble, 1024^2 Burgers) of the default run")
    ap.add_argument("--ens-count", type=int, default=256, help="instances of the ensemble workload")
    ap.add_argument("--ens-spp", type=int, default=2, help="time steps per persistent ensemble launch (1 or 2)")
    ap.add_argument("--ens-launch", default=None,
                    help="PERSISTENT,PAIR: the two-step ensemble launch to use instead of the autotuner's (with "
                         "--ens-only, time that launch alone, e.g. for a profiler capture)")
    ap.add_argument("--ens-only", action="store_true", help="ensemble workload: time the chosen launch only")
    ap.add_argument("--bf-spp", type=int, default=2, help="time steps per launch of the Burgers-Fisher workload")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "ensemble_256", "adjoint_512", "burgers_fisher_4096", "stability_sweep",
                             "gaussian3d_256"],
                    help="the default is the headline workload; the others print their own line")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (the slowest rank's time); identity on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world: int, cells: int, lbm_steps: int, ms_per_step: float) -> float:
    """Units all ranks processed (each rank runs the full workload: replicas) per second."""
    return world * cells * lbm_steps / (ms_per_step / 1e3) / 1e6


def config(args, lbm_steps):
    p = W.params(WORKLOAD)
    n = args.nx or p["nx"]
    return {"workload": f"{WORKLOAD}: D2Q9 MRT, D(phi)=(1+phi^2)K, K=[[0.02,0.008],[0.008,0.01]], "
                        f"R=-0.1 phi, {n}x{n}, phi=0 anti-bounce-back walls, {lbm_steps} steps per job",
            "nx": n, "ny": n, "lbm_steps_per_bench_step": lbm_steps,
            "storage": args.prec, "steps_per_pass": args.spp, "kernel_variant": args.variant,
            "block_rows": args.block_rows, "autotuned": bool(getattr(args, "autotuned", False)),
            "parallelism": f"replicas x{args.gpus}" if args.gpus > 1 else "single GPU",
            "l2": "inputs larger than L2 (two population buffers of 604 MB each, FP32)"}


def oracle_problem():
    import oracle as O
    p = W.params(WORKLOAD)
    return O, O.Spec(nx=p["nx"], ny=p["ny"], bc_x=p["bc"][0], bc_y=p["bc"][1], phi_wall=p["phi_wall"],
                     conv=p["conv"], u=p["u"], diff=p["diff"], K=p["K"], s=W.s9(), r0=p["r0"], r1=p["r1"])


def cpu_sample(target_s=15.0):
    """The oracle as it stands on the host cores: the full 4096^2 grid for as
    many time steps as fit about target_s seconds."""
    O, sp = oracle_problem()
    phi0 = W.phi0_aniso(4096, seed=3)
    t0 = time.perf_counter()
    F = O.init(sp, phi0)
    F, _ = O.step(sp, F, 0)
    one = time.perf_counter() - t0
    nsteps = int(max(1, min(40, target_s / max(one / 2, 1e-3))))
    t0 = time.perf_counter()
    for n in range(nsteps):
        F, _ = O.step(sp, F, n + 1)
    dt = time.perf_counter() - t0
    cells = 4096 * 4096
    return {"value": cells * nsteps / dt / 1e6, "unit": "MLUPS", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"4096x4096 grid of the same workload, {nsteps} time steps ({dt:.1f} s), FP64"}


def clocks_sampler():
    try:
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        gpu = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or "0"
        return subprocess.Popen(["nvidia-smi", "-i", gpu, f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except Exception:
        return None


def clocks_summary(proc):
    if proc is None:
        return None
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except Exception:
        return None
    mhz, maxm, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            mhz.append(float(f[1]))
            maxm = float(f[2])
        except ValueError:
            continue
        for n, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not mhz:
        return None
    return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": maxm, "reasons": sorted(reasons), "samples": len(mhz)}


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_per_launch(kernel_sha, key="k_step2"):
    """DRAM bytes per launch from the committed ncu capture of this kernel, or
    None when the kernel's sources changed since the capture."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)[key]
        if t.get("kernel_src_sha256") != kernel_sha:
            return None
        return t["dram_bytes_per_full_launch"]
    except Exception:
        return None


def step_kernel(prec, spp, variant):
    """Name of the step kernel a launch configuration runs, and its DRAM bytes per
    launch from the committed ncu capture (None when there is none or the
    kernel's sources changed since)."""
    if spp == 2 and variant == 5:
        return ("k_step2p (two fused pull-stream + collide steps per sweep, pair tiles)",
                traffic_per_launch(src_sha(PAIR_SRC), f"k_step2p_{prec}"))
    if spp == 2:
        return ("k_step2 (two fused pull-stream + collide steps per sweep)",
                traffic_per_launch(src_sha(KERNEL_SRC)) if prec == "f32" else None)
    if variant == 2 or (variant == 0 and prec == "bf16s"):
        return "k_step_v4 (fused pull-stream + collide, four nodes per thread)", None
    return "k_step (fused pull-stream + collide)", None


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    O, sp = oracle_problem()
    phi0 = W.phi0_aniso(4096, seed=3)
    F = O.init(sp, phi0)
    for n in range(args.warmup):
        F, _ = O.step(sp, F, n)
    times = []
    for n in range(args.steps):
        t0 = time.perf_counter()
        F, _ = O.step(sp, F, args.warmup + n)
        times.append(time.perf_counter() - t0)
    cells = 4096 * 4096
    ms = 1e3 * sum(times) / len(times)
    val = cells / (ms / 1e3) / 1e6
    out = {"metric": "MLUPS", "value": val, "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": config(args, args.lbm_steps or W.params(WORKLOAD)["steps"]),
           "cpu_baseline": {"value": val, "unit": "MLUPS", "cores": O.num_threads(), "kind": "oracle",
                            "sample": "one time step of the 4096x4096 workload per bench step"},
           "e2e": {"value": val, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def timed(fn, reps, stream):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def run_ensemble(args):
    """256 independent lattices (sides 64..1024), 1000 steps per job: one
    persistent launch per step replayed from a CUDA graph, against one launch
    per instance per step."""
    import torch
    import torch.distributed as dist

    from paper_1603_09577_gb300.ensemble import Ensemble, shard
    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    all_inst = W.ensemble(count=args.ens_count)
    # independent instances: each rank runs its share, no exchange on the data path
    inst = [all_inst[i] for i in shard(all_inst, rank, world)] if world > 1 else all_inst
    from paper_1603_09577_gb300 import tune
    if args.ens_launch:
        pers, pair = (int(v) for v in args.ens_launch.split(","))
        cfg = dict(persistent=pers, pair_tiles=bool(pair))
    else:
        cfg = tune.tune_ensemble(inst, conv=0, diff=1) if args.ens_spp == 2 else {}
    e = Ensemble(inst, steps_per_pass=args.ens_spp, **cfg)
    packed = e.pack([W.ensemble_phi0(d) for d in inst], dtype=torch.float32)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    steps = args.lbm_steps or 1000
    with torch.cuda.stream(side):
        e.set_phi(packed)
        e.capture(100)

        def job_graph():
            e.set_phi(packed)
            for _ in range(steps // 100):
                e.replay()

        def job_launches():
            e.set_phi(packed)
            e.step(steps, mode=1)

        def job_persistent():
            e.set_phi(packed)
            e.step(steps, mode=0)

        e1 = Ensemble(inst, steps_per_pass=1)
        e1.set_phi(packed)
        e1.capture(100)

        def job_graph_one_step():
            e1.set_phi(packed)
            for _ in range(steps // 100):
                e1.replay()

        for _ in range(args.warmup):
            job_graph()
        if world > 1:
            dist.barrier()
        clk = clocks_sampler()
        ms_graph = max_over_ranks(timed(job_graph, args.steps, side), device="cuda")
        clocks = clocks_summary(clk)
        if args.ens_only:
            nodes = sum(d["nx"] * d["ny"] for d in inst)
            print(json.dumps({"metric": "MLUPS", "value": nodes * steps / (ms_graph / 1e3) / 1e6, "unit": "MLUPS",
                              "ensemble_launch": cfg, "ms_per_step": ms_graph, "clocks": clocks}), flush=True)
            return
        ms_pers = timed(job_persistent, max(1, args.steps // 2), side)
        ep = Ensemble(inst, steps_per_pass=args.ens_spp, persistent=True)
        ep.set_phi(packed)
        ep.capture(100)

        def job_graph_persistent_grid():
            ep.set_phi(packed)
            for _ in range(steps // 100):
                ep.replay()

        ms_pgrid = timed(job_graph_persistent_grid, max(1, args.steps // 2), side)
        ms_sep = timed(job_launches, max(1, args.steps // 2), side)
        ms_g1 = timed(job_graph_one_step, max(1, args.steps // 2), side)

        # end to end through the public API: phi0 from pinned host memory, the
        # replayed steps, every instance's statistics back to the host
        host_in = packed.cpu().pin_memory()
        dev_in = torch.empty_like(packed)
        stats = torch.empty((len(inst), 8), dtype=torch.float64, device="cuda")
        host_stats = torch.empty((len(inst), 8), dtype=torch.float64).pin_memory()

        def job_e2e():
            dev_in.copy_(host_in, non_blocking=True)
            e.set_phi(dev_in)
            for _ in range(steps // 100):
                e.replay()
            e.reduce_async(out=stats)
            host_stats.copy_(stats, non_blocking=True)
            side.synchronize()

        job_e2e()
        w0 = time.perf_counter()
        for _ in range(args.steps):
            job_e2e()
        e2e_ms = 1e3 * (time.perf_counter() - w0) / args.steps
        mass0 = torch.tensor([float(t.double().sum()) for t in e.unpack(host_in)], dtype=torch.float64)
        mass_drift = float(((host_stats[:, 0] - mass0).abs() / mass0.abs()).max())
    nodes = sum(d["nx"] * d["ny"] for d in all_inst)         # every rank's instances
    val = nodes * steps / (ms_graph / 1e3) / 1e6
    if world > 1:
        dist.destroy_process_group()
        if rank != 0:
            return
        # the comparison timings below are the rank-0 share's
        nodes_r0 = e.nodes
    else:
        nodes_r0 = nodes
    peak, src = measured_peak()
    achieved = 72.0 * nodes_r0 * (steps // args.ens_spp) / (ms_graph / 1e3) / 1e9
    out = {"metric": "MLUPS", "value": val, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True,
           "scaling": "strong" if world > 1 else "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"ensemble_256: 256 D2Q9 MRT instances, sides 64..1024 ({nodes} nodes), "
                                  f"D(phi)=D0(1+phi), {steps} steps per job", "instances": len(all_inst),
                      "instances_rank0": len(inst), "tiles_rank0": e.tiles, "persistent_grid_blocks": e.grid,
                      "parallelism": f"instances sharded over {world} ranks" if world > 1 else "single GPU"},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak,
                        "kernel": (f"k_ens_step2 (two steps per launch, graph-replayed, autotuned launch {cfg})"
                                   if args.ens_spp == 2 else "k_ens_step (persistent, graph-replayed)"),
                        "peak_source": src},
           "steps_per_launch": args.ens_spp, "tuner_timings": ensemble_tuner_timings(inst),
           "one_step_graph_mlups": nodes_r0 * steps / (ms_g1 / 1e3) / 1e6,
           "persistent_grid_graph_mlups": nodes_r0 * steps / (ms_pgrid / 1e3) / 1e6,
           "persistent_no_graph_mlups": nodes_r0 * steps / (ms_pers / 1e3) / 1e6,
           "one_launch_per_instance_mlups": nodes_r0 * steps / (ms_sep / 1e3) / 1e6,
           "graph_speedup_vs_per_instance": ms_sep / ms_graph,
           "e2e": {"value": nodes_r0 * steps / (e2e_ms / 1e3) / 1e6, "unit": "MLUPS",
                   "h2d_bytes_per_step": int(host_in.numel() * host_in.element_size()),
                   "d2h_bytes_per_step": int(host_stats.numel() * host_stats.element_size()),
                   "read_back": "per-instance FP64 statistics (lbm_ensemble_reduce)",
                   "max_relative_mass_drift": mass_drift},
           "gpu_launches": args.steps * (1 + steps // args.ens_spp)}
    if clocks is not None:
        out["clocks"] = clocks
    print(json.dumps(out), flush=True)


def run_adjoint(args):
    """512^2 linear anisotropic CDE with per-node K(x), 500 steps, checkpoints
    every 50: time of one reverse (adjoint) step against one forward step, and
    of the whole backward pass against the forward pass."""
    import ctypes

    import torch

    from paper_1603_09577_gb300 import Solver, adjoint
    from paper_1603_09577_gb300 import _lib as C
    p = W.params("adjoint_512")
    Kf, phi0, tgt = W.adjoint_inputs(512, seed=4)
    prec = args.prec if args.prec in ("f32", "f64") else "f32"
    st = torch.cuda.current_stream()
    s = Solver(512, 512, prec=prec, per_cell_K=True)
    s.set_coeffs(conv=0, u=p["u"], diff=0, s=W.s9())
    s.set_K_field(torch.from_numpy(Kf).cuda())
    s.set_phi(torch.from_numpy(phi0).cuda())
    state = s.save()
    n = 200
    ms_fwd = timed(lambda: s.step(1), n, st)
    size = ctypes.c_size_t()
    C.check(s.lib.lbm_adjoint_workspace_size(s.h, ctypes.byref(size)))
    ws = torch.empty(size.value, dtype=torch.uint8, device="cuda")
    g = torch.from_numpy(tgt).cuda()
    C.check(s.lib.lbm_adjoint_begin(s.h, ctypes.c_void_p(ws.data_ptr()), size.value, ctypes.c_void_p(g.data_ptr()),
                                    C.LBM_F64, ctypes.c_void_p(st.cuda_stream)))
    ms_adj = timed(lambda: C.check(s.lib.lbm_adjoint_step(s.h, ctypes.c_void_p(state.data_ptr()),
                                                          ctypes.c_void_p(st.cuda_stream))), n, st)
    # whole passes through the autograd Function
    p0 = torch.from_numpy(phi0).cuda().requires_grad_(True)
    K = torch.from_numpy(Kf).cuda().requires_grad_(True)
    u = torch.tensor(p["u"], dtype=torch.float64, device="cuda", requires_grad=True)
    t = torch.from_numpy(tgt).cuda()
    for _ in range(args.warmup):
        out = adjoint.run(p0, K, u, p["steps"], p["ckpt_every"], prec, W.s9())
        (0.5 * ((out - t) ** 2).sum()).backward()
    torch.cuda.synchronize()
    a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    a.record(st)
    out = adjoint.run(p0, K, u, p["steps"], p["ckpt_every"], prec, W.s9())
    loss = 0.5 * ((out - t) ** 2).sum()
    b.record(st)
    loss.backward()
    c.record(st)
    torch.cuda.synchronize()
    fwd_ms, bwd_ms = a.elapsed_time(b), b.elapsed_time(c)
    cells = 512 * 512
    res = {"metric": "adjoint_step_over_forward_step", "value": ms_adj / ms_fwd, "unit": "ratio",
           "higher_is_better": False, "n_gpus": 1, "steps": n, "warmup": args.warmup, "dtype": prec,
           "data": "synthetic",
           "config": {"workload": "adjoint_512: linear anisotropic CDE, per-node K(x), u=(0.03,0), 512x512, "
                                  "500 steps, checkpoints every 50, FP64 gradient accumulation"},
           "forward_step_ms": ms_fwd, "adjoint_step_ms": ms_adj,
           "forward_mlups": cells / (ms_fwd / 1e3) / 1e6, "adjoint_mlups": cells / (ms_adj / 1e3) / 1e6,
           "forward_pass_ms": fwd_ms, "backward_pass_ms": bwd_ms,
           "backward_over_forward_pass": bwd_ms / fwd_ms}
    print(json.dumps(res), flush=True)


def run_burgers_fisher(args):
    """Scheme A with the extrapolation boundary on the Burgers-Fisher travelling
    wave (Eq. 46-51: a = 4, b = 1, kappa = 0.12, delta = 1, [-1, 2]^2, c = 40)
    at 4096^2 nodes, 2000 steps per job: set_phi, the steps with per-step
    Dirichlet records, and the error reduction against Eq. 47."""
    import torch

    from paper_1603_09577_gb300 import Solver
    prec = args.prec if args.prec in ("f32", "f64") else "f32"
    n = 4096
    lbm_steps = args.lbm_steps or 2000
    bf = W.burgers_fisher(n - 1, 0.0)
    T = lbm_steps * bf["dt"]
    bf = W.burgers_fisher(n - 1, T)
    assert bf["steps"] == lbm_steps
    tdt = torch.float64 if prec == "f64" else torch.float32
    phi0 = torch.from_numpy(bf["phi0"]).to(tdt).cuda()
    exact = torch.from_numpy(bf["exact"]).cuda()
    bv = torch.from_numpy(bf["bvals"]).cuda()
    spp = args.bf_spp if prec == "f32" else 1
    variant, rows = 0, 0
    if args.tune and prec == "f32" and args.bf_spp == 2:
        from paper_1603_09577_gb300 import tune
        cfg = tune.tune(n, n, prec, bc=("nee", "nee"), conv=2, diff=0, scheme="A")
        spp, variant, rows = cfg["steps_per_pass"], cfg["kernel_variant"], cfg["block_rows"]
    s = Solver(n, n, prec=prec, bc=("nee", "nee"), scheme="A", steps_per_pass=spp, kernel_variant=variant,
               block_rows=rows)
    s.set_coeffs(conv=2, power=1, u=bf["u"], diff=0, K=(bf["K"], 0.0, bf["K"]), s=W.s9(), src_family=1, b=bf["b"])
    red = torch.zeros(8, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def job():
        s.set_phi(phi0)
        s.set_dirichlet(bv)
        s.step(lbm_steps)
        s.reduce_async(exact, out=red)

    for _ in range(args.warmup):
        job()
    torch.cuda.synchronize()
    clk = clocks_sampler()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for a, b in ev:
        s.set_phi(phi0)
        s.set_dirichlet(bv)
        a.record(stream)
        s.step(lbm_steps)
        b.record(stream)
        s.reduce_async(exact, out=red)
    t1.record(stream)
    torch.cuda.synchronize()
    clocks = clocks_summary(clk)
    ms = t0.elapsed_time(t1) / args.steps
    launches = lbm_steps // spp + lbm_steps % spp
    launch_ms = statistics.mean(a.elapsed_time(b) for a, b in ev) / launches
    cells = n * n
    value = cells * lbm_steps / (ms / 1e3) / 1e6
    g = red.cpu().tolist()
    # end to end with host buffers
    host_in = torch.from_numpy(bf["phi0"]).to(tdt).pin_memory()
    host_out = torch.empty((n, n), dtype=tdt).pin_memory()
    s.set_phi_host(host_in)
    s.set_dirichlet(bv)
    s.step(lbm_steps)
    s.phi_host(host_out)
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(args.steps):
        s.set_phi_host(host_in)
        s.set_dirichlet(bv)
        s.step(lbm_steps)
        s.phi_host(host_out)
    e2e_ms = 1e3 * (time.perf_counter() - w0) / args.steps
    esz = 8 if prec == "f64" else 4
    bpu = 9 * 2 * esz + 2 * esz          # populations read + written, phi(t_n) plane read + written, per launch
    peak, src = measured_peak()
    achieved = bpu * cells / (launch_ms / 1e3) / 1e9
    out = {"metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": prec, "data": "synthetic",
           "config": {"workload": f"burgers_fisher_4096: Scheme A, B = a phi^2/2 (a = 4 along x), R = b phi (1 - phi), "
                                  f"kappa = 0.12, [-1,2]^2 at 4096x4096 (c = 40), extrapolated Dirichlet walls from "
                                  f"Eq. 47, {lbm_steps} steps per job",
                      "nx": n, "ny": n, "lattice": {"u": bf["u"], "K": bf["K"], "b": bf["b"]},
                      "l2": "inputs larger than L2 (two population buffers of 604 MB each, FP32)"},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "traffic": (None if prec != "f32" else
                                    traffic_per_launch(src_sha(GENERAL_SRC), "k_step_g") if spp == 1 else
                                    traffic_per_launch(src_sha(STEP2G_SRC), "k_step2g")),
                        "kernel": ("k_step2g (general two-step tile kernel, Scheme A)" if spp == 2
                                   else "k_step_g (general one-step kernel, Scheme A)"),
                        "steps_per_launch": spp,
                        "algorithmic_bytes_per_update": bpu, "avg_launch_ms": launch_ms,
                        "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else src},
           "e2e": {"value": cells * lbm_steps / (e2e_ms / 1e3) / 1e6, "unit": "MLUPS",
                   "h2d_bytes_per_step": int(host_in.numel() * esz), "d2h_bytes_per_step": int(host_out.numel() * esz)},
           "gre_vs_eq47": g[1] / g[2],
           # per job: the initialisation, the sweeps, the record-count advance, two reduction kernels
           "gpu_launches": args.steps * (1 + launches + 1 + 2)}
    if clocks is not None:
        out["clocks"] = clocks
    if not args.no_cpu_baseline:
        import oracle as O
        sp = O.Spec(nx=n, ny=n, bc_x=2, bc_y=2, conv=2, u=bf["u"], diff=0, K=(bf["K"], 0.0, bf["K"]), s=W.s9(),
                    scheme=1, power=1, src_family=1, b=bf["b"])
        F, P = O.init_x(sp, bf["phi0"])
        k = 8
        w0 = time.perf_counter()
        for j in range(k):
            F, P = O.step_x(sp, F, P, bf["bvals"][j])
        dt = time.perf_counter() - w0
        out["cpu_baseline"] = {"value": cells * k / dt / 1e6, "unit": "MLUPS", "cores": O.num_threads(),
                               "kind": "oracle", "sample": f"the same 4096x4096 problem, {k} time steps ({dt:.1f} s), FP64"}
    print(json.dumps(out), flush=True)


def run_stability_sweep(args):
    """Sec. 3.6's stability comparison as a sweep: the fully anisotropic
    Gaussian hill (Eq. 75, second approach D = Dm phi, u = (0.1, 0.1), 400^2,
    c = 1, T = 5: 1000 steps) for decreasing kappa, with the MRT rates of Eq. 76
    (s = 0.6) and with every rate s3 (BGK). Each run reports its GRE against
    Eq. 60, or "unstable" (a non-finite phi or max |phi| > 10)."""
    import torch

    from paper_1603_09577_gb300 import Solver
    import oracle as O
    prec = args.prec if args.prec in ("f32", "f64") else "f64"
    rows = []
    ms_all, updates = 0.0, 0
    for kap in (1e-3, 5e-4, 2e-4, 1e-4, 5e-5, 2e-5, 1e-5):
        g = W.gaussian_hill_square((kap, kap, 2 * kap), (0.1, 0.1), 5.0)
        kl = g["K"][0]
        sj = float(O.relax_block((kl, 0.0, kl))[0, 0])
        phi0 = torch.from_numpy(g["phi0"]).cuda()
        ex = torch.from_numpy(g["exact"]).cuda()
        row = {"kappa": kap, "kappa_lattice": kl, "s3": sj}
        for name, rates in (("mrt", (0.0, 0.6, 0.6, 0.0, 0.6, 0.0, 0.6, 0.6, 0.6)), ("bgk", (sj,) * 9)):
            s = Solver(g["n"], g["n"], prec=prec)
            s.set_coeffs(conv=0, u=g["u"], diff=3, Dm=(1.0, 1.0, 2.0), K=(kl, 0.0, kl), s=rates)
            s.set_phi(phi0)
            st = torch.cuda.current_stream()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            s.step(g["steps"])
            b.record(st)
            r = s.reduce(ex)
            ms_all += a.elapsed_time(b)
            updates += g["n"] ** 2 * g["steps"]
            ok = r["nonfinite"] == 0 and r["max_abs"] <= 10.0
            row[name] = r["abs_err"] / r["abs_ref"] if ok else "unstable"
            if name == "mrt" and kap == 1e-3:
                # the same 1000 steps replayed from a CUDA graph of 100 steps
                s.set_phi(phi0)
                s.capture(100)
                s.set_phi(phi0)
                a.record(st)
                for _ in range(g["steps"] // 100):
                    s.replay()
                b.record(st)
                torch.cuda.synchronize()
                graph_ms, graph_updates = a.elapsed_time(b), g["n"] ** 2 * g["steps"]
                direct_ms = ms_all
        rows.append(row)
    out = {"metric": "MLUPS", "value": updates / (ms_all / 1e3) / 1e6, "unit": "MLUPS", "n_gpus": 1,
           "higher_is_better": True, "dtype": prec, "data": "synthetic",
           "config": {"workload": "stability_sweep: Sec. 3.6 fully anisotropic Gaussian hill (Eq. 75), second "
                                  "approach D = [[1,1],[1,2]] phi, u = (0.1, 0.1), 400x400, c = 1, 1000 steps per run, "
                                  "MRT (Eq. 76, s = 0.6) against BGK (all rates s3)"},
           "sweep": rows, "gpu_launches": len(rows) * 2 * (1 + 1000 + 2),
           "graph_replay_mlups": graph_updates / (graph_ms / 1e3) / 1e6,
           "direct_launch_mlups_same_run": graph_updates / (direct_ms / 1e3) / 1e6}
    print(json.dumps(out), flush=True)


def run_gaussian3d(args):
    """The D3Q19 extension on a 256^3 periodic lattice: the 3-D Gaussian hill
    (Eq. 60) with a full tensor K, 500 steps per job (set_phi, the steps, the
    error reduction against Eq. 60)."""
    import torch

    from paper_1603_09577_gb300 import Solver3
    prec = args.prec
    n = args.nx or 256
    lbm_steps = args.lbm_steps or 500
    K, u, sig = (0.02, 0.006, 0.004, 0.015, 0.003, 0.01), (0.02, 0.01, -0.015), 16.0
    x = torch.arange(n, dtype=torch.float64, device="cuda")
    Z, Y, X = torch.meshgrid(x, x, x, indexing="ij")

    def hill(t):
        Km = torch.tensor([[K[0], K[1], K[2]], [K[1], K[3], K[4]], [K[2], K[4], K[5]]], dtype=torch.float64)
        Sig = sig ** 2 * torch.eye(3, dtype=torch.float64) + 2 * Km * t
        Si = torch.linalg.inv(Sig).cuda()
        dx, dy, dz = X - n / 2 - u[0] * t, Y - n / 2 - u[1] * t, Z - n / 2 - u[2] * t
        S = Si.cpu().tolist()
        q = (S[0][0] * dx * dx + S[1][1] * dy * dy + S[2][2] * dz * dz
             + 2 * (S[0][1] * dx * dy + S[0][2] * dx * dz + S[1][2] * dy * dz))
        return (sig ** 3 / math.sqrt(float(torch.linalg.det(Sig)))) * torch.exp(-0.5 * q)

    phi0 = hill(0.0).to(torch.float64 if prec == "f64" else torch.float32).contiguous()   # bf16s takes FP32 input
    exact = hill(float(lbm_steps)).contiguous()
    s = Solver3(n, n, n, prec=prec, block_rows=args.block_rows).set_coeffs(conv=0, u=u, K=K, se=1.1)
    red = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()

    def job():
        s.set_phi(phi0)
        s.step(lbm_steps)
        s.reduce_async(exact, out=red)

    for _ in range(args.warmup):
        job()
    torch.cuda.synchronize()
    clk = clocks_sampler()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(st)
    for a, b in ev:
        s.set_phi(phi0)
        a.record(st)
        s.step(lbm_steps)
        b.record(st)
        s.reduce_async(exact, out=red)
    t1.record(st)
    torch.cuda.synchronize()
    clocks = clocks_summary(clk)
    ms = t0.elapsed_time(t1) / args.steps
    launch_ms = statistics.mean(a.elapsed_time(b) for a, b in ev) / lbm_steps
    cells = n ** 3
    # populations read + written (BF16S: 2 B each plus the 4 B shift plane)
    bpu = {"f64": 19 * 2 * 8, "f32": 19 * 2 * 4, "bf16s": 19 * 2 * 2 + 2 * 4}[prec]
    peak, src = measured_peak()
    achieved = bpu * cells / (launch_ms / 1e3) / 1e9
    g = red.cpu().tolist()
    out = {"metric": "MLUPS", "value": cells * lbm_steps / (ms / 1e3) / 1e6, "unit": "MLUPS", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
           "config": {"workload": f"gaussian3d_{n}: D3Q19, linear anisotropic CDE with a full 3x3 K, {n}^3 periodic, "
                                  f"{lbm_steps} steps per job", "nx": n, "ny": n, "nz": n,
                      "l2": "inputs larger than L2 (two population buffers of 0.67 to 2.5 GB each)"},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "traffic": None, "kernel": "k_step3 (D3Q19 fused pull-stream + collide)",
                        "algorithmic_bytes_per_update": bpu, "avg_launch_ms": launch_ms,
                        "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else src},
           "gre_vs_eq60": g[1] / g[2], "gpu_launches": args.steps * (1 + lbm_steps + 2)}
    if clocks is not None:
        out["clocks"] = clocks
    print(json.dumps(out), flush=True)


def fp64_peak_probe():
    """The FP64 pipe's measured rate (G thread instructions/s): the DFMA probe of
    the library on every SM (8 resident blocks of 256 threads each), best of 5
    launches timed with CUDA events, with the SM clock sampled meanwhile."""
    import ctypes

    import torch

    from paper_1603_09577_gb300 import _lib as C
    L = C.lib()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks, threads, iters = sms * 8, 256, 4096
    sink = torch.zeros(blocks, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    n = ctypes.c_longlong()

    def launch():
        C.check(L.lbm_probe_fp64(blocks, threads, iters, ctypes.c_void_p(sink.data_ptr()), ctypes.byref(n),
                                 ctypes.c_void_p(st.cuda_stream)))

    launch()
    torch.cuda.synchronize()
    clk = clocks_sampler()
    best = min(timed(launch, 4, st) for _ in range(5))
    clocks = clocks_summary(clk)
    ginst = n.value / (best / 1e3) / 1e9
    mhz = clocks["sm_mhz"] if clocks else None
    out = {"value": ginst, "unit": "G FP64 thread instructions/s",
           "how": f"lbm_probe_fp64: {blocks} blocks x {threads} threads x {iters} iterations x 8 independent DFMA "
                  f"chains, best of 5 x 4 launches (CUDA events)", "sms": sms}
    if mhz:
        out["per_sm_per_clock"] = ginst * 1e3 / (sms * mhz)
    if clocks is not None:
        out["clocks"] = clocks
    return out


def c3_measure(prec, cfg, lbm_steps, steps, warmup, warm_lbm_steps=None):
    """The 4096^2 Dirichlet job (set_phi, lbm_steps steps, mass reduction) in one
    storage precision: MLUPS over `steps` timed jobs, the average launch time of
    the step kernel, clocks, and the final phi (FP64, host)."""
    import torch

    from paper_1603_09577_gb300 import Solver
    p = W.params(WORKLOAD)
    n = p["nx"]
    phi0 = torch.from_numpy(W.phi0_aniso(n, seed=3).astype(np.float64 if prec == "f64" else np.float32)).cuda()
    s = Solver(n, n, prec=prec, bc=("abb", "abb"), phi_wall=p["phi_wall"], **cfg)
    s.set_coeffs(conv=p["conv"], u=p["u"], diff=p["diff"], K=p["K"], s=W.s9(), r0=p["r0"], r1=p["r1"])
    red = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    for _ in range(warmup):
        s.set_phi(phi0)
        s.step(warm_lbm_steps or lbm_steps)
        s.reduce_async(out=red)
    torch.cuda.synchronize()
    clk = clocks_sampler()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(st)
    for a, b in ev:
        s.set_phi(phi0)
        a.record(st)
        s.step(lbm_steps)
        b.record(st)
        s.reduce_async(out=red)
    t1.record(st)
    torch.cuda.synchronize()
    clocks = clocks_summary(clk)
    ms = t0.elapsed_time(t1) / steps
    spp = cfg.get("steps_per_pass", 1)
    launches = lbm_steps // spp + lbm_steps % spp
    launch_ms = statistics.mean(a.elapsed_time(b) for a, b in ev) / launches
    phi = s.phi().cpu().numpy()
    del s
    torch.cuda.empty_cache()
    return {"mlups": n * n * lbm_steps / (ms / 1e3) / 1e6, "ms_per_job": ms, "avg_launch_ms": launch_ms,
            "launches_per_job": launches, "clocks": clocks, "phi": phi}


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def extra_c3(prec, lbm_steps, steps, warmup, fp64_phi, peak, src):
    """Sub-record of the 4096^2 workload in BF16S storage (autotuned launch)."""
    from paper_1603_09577_gb300 import tune
    p = W.params(WORKLOAD)
    cfg = tune.tune(p["nx"], p["ny"], prec, bc=("abb", "abb"), conv=p["conv"], diff=p["diff"])
    assert cfg in tune.candidates(p["nx"], prec), cfg
    r = c3_measure(prec, cfg, lbm_steps, steps, warmup)
    cells = p["nx"] * p["ny"]
    achieved = BYTES_PER_UPDATE[prec] * cells / (r["avg_launch_ms"] / 1e3) / 1e9
    kernel, traffic = step_kernel(prec, cfg["steps_per_pass"], cfg["kernel_variant"])
    out = {"workload": f"{WORKLOAD}, {lbm_steps} steps per job, storage {prec}", "value": r["mlups"],
           "unit": "MLUPS", "ms_per_job": r["ms_per_job"], "timed_jobs": steps, "config": cfg,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "kernel": kernel, "traffic": traffic,
                        "algorithmic_bytes_per_launch": BYTES_PER_UPDATE[prec] * cells,
                        "avg_launch_ms": r["avg_launch_ms"], "peak_source": src,
                        "one_step_roof_mlups": peak * 1e3 / BYTES_PER_UPDATE[prec]},
           "rel_l2_vs_fp64_path": rel_l2(r["phi"], fp64_phi) if fp64_phi is not None else None,
           "clocks": r["clocks"]}
    return out, r["phi"]


def extra_adjoint(warmup):
    """Sub-record of the differentiable 512^2 workload: adjoint step over forward
    step (one launch each), and whole backward pass (checkpoints every 50,
    recomputation included) over the forward pass, FP32 forward with FP64
    gradient accumulation."""
    import ctypes

    import torch

    from paper_1603_09577_gb300 import Solver, adjoint
    from paper_1603_09577_gb300 import _lib as C
    p = W.params("adjoint_512")
    Kf, phi0, tgt = W.adjoint_inputs(512, seed=4)
    st = torch.cuda.current_stream()
    clk = clocks_sampler()
    s = Solver(512, 512, prec="f32", per_cell_K=True)
    s.set_coeffs(conv=0, u=p["u"], diff=0, s=W.s9())
    s.set_K_field(torch.from_numpy(Kf).cuda())
    s.set_phi(torch.from_numpy(phi0).cuda())
    state = s.save()
    n = 200
    s.step(10)
    ms_fwd = timed(lambda: s.step(1), n, st)
    size = ctypes.c_size_t()
    C.check(s.lib.lbm_adjoint_workspace_size(s.h, ctypes.byref(size)))
    ws = torch.empty(size.value, dtype=torch.uint8, device="cuda")
    g = torch.from_numpy(tgt).cuda()
    C.check(s.lib.lbm_adjoint_begin(s.h, ctypes.c_void_p(ws.data_ptr()), size.value, ctypes.c_void_p(g.data_ptr()),
                                    C.LBM_F64, ctypes.c_void_p(st.cuda_stream)))
    adj = lambda: C.check(s.lib.lbm_adjoint_step(s.h, ctypes.c_void_p(state.data_ptr()),  # noqa: E731
                                                 ctypes.c_void_p(st.cuda_stream)))
    adj()
    ms_adj = timed(adj, n, st)
    p0 = torch.from_numpy(phi0).cuda().requires_grad_(True)
    K = torch.from_numpy(Kf).cuda().requires_grad_(True)
    u = torch.tensor(p["u"], dtype=torch.float64, device="cuda", requires_grad=True)
    t = torch.from_numpy(tgt).cuda()
    for _ in range(max(1, warmup)):
        out = adjoint.run(p0, K, u, p["steps"], p["ckpt_every"], "f32", W.s9())
        (0.5 * ((out - t) ** 2).sum()).backward()
    torch.cuda.synchronize()
    fw, bw = [], []
    for _ in range(3):
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(st)
        out = adjoint.run(p0, K, u, p["steps"], p["ckpt_every"], "f32", W.s9())
        loss = 0.5 * ((out - t) ** 2).sum()
        b.record(st)
        loss.backward()
        c.record(st)
        torch.cuda.synchronize()
        fw.append(a.elapsed_time(b))
        bw.append(b.elapsed_time(c))
    clocks = clocks_summary(clk)
    fwd_ms, bwd_ms = statistics.median(fw), statistics.median(bw)
    return {"workload": "adjoint_512: linear anisotropic CDE, per-node K(x), u=(0.03,0), 512x512, 500 steps, "
                        "checkpoints every 50, FP32 forward, FP64 gradient accumulation",
            "adjoint_step_over_forward_step": ms_adj / ms_fwd, "forward_step_ms": ms_fwd, "adjoint_step_ms": ms_adj,
            "forward_pass_ms": fwd_ms, "backward_pass_ms": bwd_ms, "backward_over_forward_pass": bwd_ms / fwd_ms,
            "target": "adjoint step <= 3 x forward step", "clocks": clocks}


def extra_ensemble(warmup, steps):
    """Sub-record of the 256-instance ensemble (1000 steps per job): two steps
    per launch replayed from a CUDA graph, against one launch per instance and
    step (256 launches per step)."""
    import torch

    from paper_1603_09577_gb300 import tune
    from paper_1603_09577_gb300.ensemble import Ensemble
    inst = W.ensemble(count=256)
    lbm_steps = 1000
    cfg = tune.tune_ensemble(inst, conv=0, diff=1)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        e = Ensemble(inst, steps_per_pass=2, **cfg)
        packed = e.pack([W.ensemble_phi0(d) for d in inst], dtype=torch.float32)
        e.set_phi(packed)
        e.capture(100)

        def job_graph():
            e.set_phi(packed)
            for _ in range(lbm_steps // 100):
                e.replay()

        e1 = Ensemble(inst, steps_per_pass=1)

        def job_launches():
            e1.set_phi(packed)
            e1.step(lbm_steps, mode=1)

        for _ in range(warmup):
            job_graph()
        job_launches()
        torch.cuda.synchronize()
        clk = clocks_sampler()
        ms_graph = timed(job_graph, steps, side)
        clocks = clocks_summary(clk)
        ms_sep = timed(job_launches, max(1, steps // 2), side)
        out_phi = e.phi()
        finite = bool(torch.isfinite(out_phi).all())
    nodes = e.nodes
    del e, e1
    torch.cuda.empty_cache()
    return {"workload": f"ensemble_256: 256 instances, sides 64..1024 ({nodes} nodes), D(phi)=D0(1+phi), "
                        f"{lbm_steps} steps per job, FP32",
            "value": nodes * lbm_steps / (ms_graph / 1e3) / 1e6, "unit": "MLUPS",
            "mode": "two steps per launch over the tiles of all instances, 100-step CUDA graph replayed",
            "autotuned_launch": cfg, "tuner_timings": ensemble_tuner_timings(inst),
            "per_instance_launches_mlups": nodes * lbm_steps / (ms_sep / 1e3) / 1e6,
            "speedup_vs_256_launches_per_step": ms_sep / ms_graph, "finite": finite, "clocks": clocks}


def ensemble_tuner_timings(inst):
    """The autotuner's per-candidate MLUPS for this ensemble (from its cache)."""
    import json as _json

    from paper_1603_09577_gb300 import tune
    try:
        with open(tune.cache_path()) as f:
            entry = _json.load(f)[tune._ensemble_key(inst, 0, 1)]
    except Exception:
        return None
    nodes = sum(d["nx"] * d["ny"] for d in inst)
    return [{**c["config"], "mlups": nodes / (c["ms_per_step"] / 1e3) / 1e6} for c in entry["all"]]


def extra_burgers(steps):
    """Sub-record of the 1024^2 Burgers workload (5000 steps per job): FP64, FP32
    and BF16S storage (the autotuned launch for the last two), MLUPS and the
    relative L2 difference of phi from the FP64 path."""
    import torch

    from paper_1603_09577_gb300 import Solver
    p = W.params("burgers_1024")
    n, lbm_steps = p["nx"], p["steps"]
    phi0_np = W.phi0_burgers()
    st = torch.cuda.current_stream()
    clk = clocks_sampler()
    res, phis = {}, {}
    from paper_1603_09577_gb300 import tune
    tuned = {pr: tune.tune(n, n, pr, conv=p["conv"], diff=p["diff"]) for pr in ("f32", "bf16s")}
    for prec, cfg in (("f64", {}), ("f32", tuned["f32"]), ("bf16s", tuned["bf16s"])):
        phi0 = torch.from_numpy(phi0_np.astype(np.float64 if prec == "f64" else np.float32)).cuda()
        s = Solver(n, n, prec=prec, **cfg)
        s.set_coeffs(conv=p["conv"], u=p["u"], diff=p["diff"], K=p["K"], s=W.s9())

        def job():
            s.set_phi(phi0)
            s.step(lbm_steps)

        job()
        reps = 1 if prec == "f64" else steps
        ms = timed(job, reps, st)
        phis[prec] = s.phi().cpu().numpy()
        res[prec] = {"value": n * n * lbm_steps / (ms / 1e3) / 1e6, "unit": "MLUPS", "ms_per_job": ms,
                     "timed_jobs": reps, "config": cfg or {"steps_per_pass": 1}}
        del s
    clocks = clocks_summary(clk)
    for prec in ("f32", "bf16s"):
        res[prec]["rel_l2_vs_fp64_path"] = rel_l2(phis[prec], phis["f64"])
    torch.cuda.empty_cache()
    return {"workload": "burgers_1024: D2Q9 MRT, B = a phi^2/2, a=(1,1)/sqrt2, K = 5.12 (D=0.005 on the unit "
                        "square), 1024x1024 periodic, 5000 steps per job", **res, "clocks": clocks}


def fp64_roofline(ginst, rate, kernel, hbm_frac, launch_ms):
    """Roofline of the FP64 step kernel against the FP64 pipe's measured rate."""
    return {"bound": "alu", "achieved": ginst, "peak": rate["value"], "unit": "G FP64 thread instructions/s",
            "frac": ginst / rate["value"], "traffic": None, "kernel": kernel,
            "fp64_inst_per_update": FP64_INST_PER_UPDATE, "hbm_frac": hbm_frac, "avg_launch_ms": launch_ms,
            "peak_source": "measured in this run: " + rate["how"]}


def extras(args, lbm_steps, headline_phi, peak, src, fp64_rate):
    """The rest of the metric in the default run, each with its own clocks: the
    FP64 and BF16S paths of the 4096^2 workload (with their relative L2 from the
    FP64 path), the FP64 pipe's rate, the adjoint / forward time, the batched
    ensemble against per-instance launches, and the 1024^2 Burgers workload in
    the three precisions."""
    p = W.params(WORKLOAD)
    cells = p["nx"] * p["ny"]
    ex = {"fp64_pipe": fp64_rate}
    # FP64: one full job (about 8 s), the reference field of the other precisions
    r = c3_measure("f64", {}, lbm_steps, 1, 1, warm_lbm_steps=20)
    ginst = FP64_INST_PER_UPDATE * cells / (r["avg_launch_ms"] / 1e3) / 1e9
    ex["fp64"] = {"workload": f"{WORKLOAD}, {lbm_steps} steps per job, storage f64", "value": r["mlups"],
                  "unit": "MLUPS", "ms_per_job": r["ms_per_job"], "timed_jobs": 1,
                  "roofline": fp64_roofline(ginst, fp64_rate, "k_step<F64> (fused pull-stream + collide)",
                                            BYTES_PER_UPDATE["f64"] * cells / (r["avg_launch_ms"] / 1e3) / 1e9 / peak,
                                            r["avg_launch_ms"]),
                  "clocks": r["clocks"]}
    fp64_phi = r["phi"]
    ex[f"{args.prec}_headline_rel_l2_vs_fp64_path"] = rel_l2(headline_phi, fp64_phi) if headline_phi is not None else None
    ex["bf16s"], _ = extra_c3("bf16s", lbm_steps, max(3, args.steps // 2), 2, fp64_phi, peak, src)
    ex["adjoint"] = extra_adjoint(1)
    ex["ensemble"] = extra_ensemble(2, 3)
    ex["burgers_1024"] = extra_burgers(3)
    return ex


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ensemble_256":
        return run_ensemble(args)
    if args.workload == "adjoint_512":
        return run_adjoint(args)
    if args.workload == "burgers_fisher_4096":
        return run_burgers_fisher(args)
    if args.workload == "stability_sweep":
        return run_stability_sweep(args)
    if args.workload == "gaussian3d_256":
        return run_gaussian3d(args)
    import torch
    import torch.distributed as dist

    from paper_1603_09577_gb300 import Solver

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    p = W.params(WORKLOAD)
    lbm_steps = args.lbm_steps or p["steps"]
    nx, ny = (args.nx, args.nx) if args.nx else (p["nx"], p["ny"])
    cells = nx * ny

    phi0_np = W.phi0_aniso(nx, seed=3).astype(np.float32)
    phi0 = torch.from_numpy(phi0_np).cuda()
    if args.tune and args.variant == 0 and args.block_rows == 0 and args.spp == 1:
        from paper_1603_09577_gb300 import tune
        cfg = tune.tune(nx, ny, args.prec, bc=("abb", "abb"), conv=p["conv"], diff=p["diff"])
        # the tuned launch is one of the candidates the full-grid parity test
        # compares with the oracle (tests/test_gpu_headline.py)
        assert cfg in tune.candidates(nx, args.prec), cfg
        args.spp, args.variant, args.block_rows = cfg["steps_per_pass"], cfg["kernel_variant"], cfg["block_rows"]
        args.autotuned = True
    s = Solver(nx, ny, prec=args.prec, bc=("abb", "abb"), phi_wall=p["phi_wall"], steps_per_pass=args.spp,
               kernel_variant=args.variant, block_rows=args.block_rows)
    s.set_coeffs(conv=p["conv"], u=p["u"], diff=p["diff"], K=p["K"], s=W.s9(), r0=p["r0"], r1=p["r1"])
    red = torch.zeros(8, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def job():
        s.set_phi(phi0)
        s.step(lbm_steps)
        s.reduce_async(out=red)

    for _ in range(args.warmup):
        job()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    clk = clocks_sampler()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for e0, e1, e2 in ev:
        s.set_phi(phi0)
        e0.record(stream)
        s.step(lbm_steps)
        e1.record(stream)
        s.reduce_async(out=red)
        e2.record(stream)
    t_end.record(stream)
    torch.cuda.synchronize()
    clocks = clocks_summary(clk)
    total_ms = t_start.elapsed_time(t_end)
    step_kernels_ms = [e0.elapsed_time(e1) for e0, e1, _ in ev]
    mass = float(red[0].item())
    total_ms = max_over_ranks(total_ms, device="cuda")
    if world > 1:
        dist.barrier()

    ms_per_step = total_ms / args.steps
    value = whole_job_mlups(world, cells, lbm_steps, ms_per_step)

    # end to end through the C ABI with host buffers (pinned), copies included
    host_in = torch.from_numpy(phi0_np).pin_memory()
    host_out = torch.empty((ny, nx), dtype=torch.float32).pin_memory()
    for _ in range(1):
        s.set_phi_host(host_in)
        s.step(lbm_steps)
        s.phi_host(host_out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.set_phi_host(host_in)
        s.step(lbm_steps)
        s.phi_host(host_out)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, device="cuda")
    e2e_val = whole_job_mlups(world, cells, lbm_steps, e2e_s * 1e3)

    headline_phi = s.phi().cpu().numpy() if (rank == 0 and world == 1 and not args.no_extras) else None
    del s
    torch.cuda.empty_cache()

    if rank == 0:
        launches_per_job = lbm_steps // args.spp + lbm_steps % args.spp
        launch_ms = statistics.mean(step_kernels_ms) / launches_per_job
        # one launch reads and writes every population once, whatever the
        # number of time steps it advances
        alg_bytes = BYTES_PER_UPDATE[args.prec] * cells
        achieved = alg_bytes / (launch_ms / 1e3) / 1e9
        peak, src = measured_peak()
        kernel, traffic = step_kernel(args.prec, args.spp, args.variant)
        out = {
            "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.prec, "data": "synthetic", "config": config(args, lbm_steps),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic if nx == 4096 else None,
                         "kernel": kernel,
                         "one_step_roof_mlups": peak * 1e3 / BYTES_PER_UPDATE[args.prec],
                         "value_over_one_step_roof": value / world / (peak * 1e3 / BYTES_PER_UPDATE[args.prec]),
                         "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": launch_ms,
                         "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else src},
            "e2e": {"value": e2e_val, "unit": "MLUPS", "h2d_bytes_per_step": int(host_in.numel() * 4),
                    "d2h_bytes_per_step": int(host_out.numel() * 4)},
            "gpu_launches": args.steps * (1 + launches_per_job + 2),
            "mass_after_job": mass,
        }
        out["config"]["parity_tested"] = ("the launch is one of the autotuner's candidates, each compared with "
                                          "the oracle on the full grid by tests/test_gpu_headline.py"
                                          if getattr(args, "autotuned", False) else None)
        fp64_rate = fp64_peak_probe() if (args.prec == "f64" or (world == 1 and not args.no_extras)) else None
        if args.prec == "f64":
            # the FP64 kernel is bound by the FP64 pipe, not HBM
            ginst = FP64_INST_PER_UPDATE * cells * lbm_steps / (statistics.mean(step_kernels_ms) / 1e3) / 1e9
            out["roofline"] = fp64_roofline(ginst, fp64_rate, kernel, achieved / peak, launch_ms)
        if clocks is not None:
            out["clocks"] = clocks
        if world == 1 and not args.no_extras:
            out["extras"] = extras(args, lbm_steps, headline_phi, peak, src, fp64_rate)
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_sample()
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
