"""Benchmark: ORCA agent-steps/s on one GB300 (or N replicas, one per GPU).

Workload: bidirectional flow, 524,288 agents (two crowds in opposite quarter-width bands of
a 1 km square, radius U[0.3, 0.5] m, speed U[1.2, 1.6] m/s, r_obs 10 m, k = 10,
tau 5 s, dt 1/60 s), seeded synthetic data.  A step is one full ORCA step (binning, sort,
neighbour search, half-planes, LP, integrate) through the C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Timing: W untimed steps, then K steps, each bracketed by CUDA events on the launching
stream with a 256 MiB buffer write (larger than the 129 MB L2) between steps; the sum of
the K step durations is the device time.  Barrier + synchronize on both sides, max over
ranks.  Prints one JSON line on rank 0.

--impl reference times the FP64 CPU oracle (the "reference arm") on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ORCA agent-steps/sec at 524,288 agents; ms/step; % of HBM roofline"
UNIT = "agent-steps/s"
WORKLOAD = ("bidirectional flow, 524,288 agents (two crowds in opposite 250 m bands of a 1 km "
            "square), radius U[0.3,0.5] m, speed U[1.2,1.6] m/s, r_obs 10 m, k 10, tau 5 s, dt 1/60 s")
# algorithmic HBM bytes per agent of the per-agent ORCA kernel: read pos, vel, goal (8 B
# each), radius, max speed, pref speed, tau, id, k-th-neighbour hint (4 B each); write pos,
# vel (8 B each) and the hint (4 B).  Neighbour reads (candidate records, the id -> slot
# map, neighbour velocities) are re-reads of cell-sorted data and are not counted.
ORCA_KERNEL_BYTES_PER_AGENT = 48 + 20

# Arithmetic model of one agent-step (FP32 operations of the formulas, an FMA counting as
# two): 6 per candidate examined (d^2 and its test), 45 per half-plane built, 25 per LP1
# call (disc interval, objective, point), 14 per LP1 bound, 6 per violation check, 24 per
# LP3 bisector.  The counts come from the operation-counting replay of the timed steps.
FLOPS = {"candidates": 6, "lines": 45, "lp1_calls": 25, "lp1_bounds": 14, "lp_checks": 6,
         "bisectors": 24}
FP32_LANES_PER_SM = 128

# Algorithmic HBM bytes of one whole step per agent (the minimal traffic model of a step):
# state read 40 (pos, vel, goal 8 each; radius, max speed, pref speed, tau 4 each), state
# write 16, cell key and index written and read once 16, one sort scatter (read + write)
# 16, the cell-ordered message record written and read once 2 x 20.  It counts no re-read
# and no permutation of the parameters, so it is the lower bound any implementation moves.
STEP_BYTES_PER_AGENT = 40 + 16 + 16 + 16 + 40


def host_cpu_model() -> str:
    """The host CPU's model name (lscpu), for the CPU baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def fma_peak(torch, abi, stream, repeats: int = 5) -> dict:
    """Measured FP32 FMA rate (TFLOP/s): the library's FMA microbenchmark, 8 CTAs of 256
    threads per SM, best of `repeats` launches timed with CUDA events on the launching
    stream, after one warm-up launch."""
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    blocks = 8 * props.multi_processor_count
    out = torch.empty(blocks, dtype=torch.float32, device="cuda")
    iters = 4096
    abi.orca_fma_bench(blocks, iters, out, stream=stream)
    torch.cuda.synchronize()
    best = None
    for _ in range(repeats):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        flops = abi.orca_fma_bench(blocks, iters, out, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        r = flops / (ms * 1e-3) / 1e12
        best = r if best is None else max(best, r)
    return {"tflops": best, "blocks": blocks, "iters": iters, "repeats": repeats}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_hash() -> str:
    src = os.path.join(ROOT, "paper_1908_10107_gb300", "csrc", "orca_main.cu")
    return hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the ORCA kernel from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "orca_main_bidirectional_524288.md")
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    t = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", txt)
    if h and t and h.group(1) == kernel_hash():
        return float(t.group(1))
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int, out_path: str | None = None):
        self.proc = None
        self.lines = []
        self.idx = device_index
        self.out_path = out_path

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", str(self.idx)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.12)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        self.lines = [l for l in out.splitlines() if l.strip()]
        if self.out_path:
            try:
                with open(self.out_path, "w") as f:
                    f.write(self.FIELDS + "\n" + "\n".join(self.lines) + "\n")
            except Exception:
                pass
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def device_smi_index(torch, dev: int) -> int:
    try:
        props = torch.cuda.get_device_properties(dev)
        bus = "%08x:%02x:%02x.0" % (getattr(props, "pci_domain_id", 0), props.pci_bus_id,
                                    props.pci_device_id)
        out = subprocess.run(["nvidia-smi", "--query-gpu=index,pci.bus_id",
                              "--format=csv,noheader"], capture_output=True, text=True,
                             timeout=20).stdout
        for line in out.splitlines():
            i, b = [x.strip() for x in line.split(",")]
            if b.lower().endswith(bus[-7:].lower()) and b.lower().split(":")[-2:] == bus.lower().split(":")[-2:]:
                return int(i)
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if vis and vis.split(",")[0].strip().isdigit():
        return int(vis.split(",")[dev].strip())
    return dev


def cpu_baseline(scene, budget_s: float = 12.0, max_steps: int = 30):
    """The FP64 oracle (grid neighbour search, OpenMP over agents) on the host cores:
    whole steps of the full crowd, repeated until the budget is used."""
    import oracle
    oracle.build()
    cores = oracle.max_threads()
    st = scene.copy()
    steps, t0 = 0, time.perf_counter()
    while steps < max_steps and (steps == 0 or time.perf_counter() - t0 < budget_s):
        r = oracle.step_scene(st, knn_mode=1)
        st.pos = r["pos"].astype(np.float32)
        st.vel = r["vel"].astype(np.float32)
        steps += 1
    dt = time.perf_counter() - t0
    return {"value": scene.n * steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu_model": host_cpu_model(),
            "sample": f"{steps} whole steps of the {scene.n:,}-agent crowd (FP64, grid search, "
                      f"OpenMP {cores} threads), {dt:.1f} s"}


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle timed on the host, same metric and workload."""
    if rank != 0:
        return
    import oracle
    from paper_1908_10107_gb300 import scenarios
    oracle.build()
    cores = oracle.max_threads()
    sc = scenarios.bidirectional()
    m = args.ref_sample
    subset = np.sort(np.random.default_rng(7).choice(sc.n, m, replace=False))
    for _ in range(args.warmup):
        oracle.step_scene(sc, knn_mode=1, subset=subset)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.step_scene(sc, knn_mode=1, subset=subset)
    dt = time.perf_counter() - t0
    value = m * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD, "n_agents": sc.n, "sample_agents_per_step": m},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "cpu_model": host_cpu_model(),
                         "sample": f"{m} sampled agents of the {sc.n:,}-agent crowd per step "
                                   f"(neighbours searched among all agents), FP64, {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def timed_steps(torch, step_fn, steps, warmup, flush, stream):
    """Device time (ms) of `steps` calls of step_fn, L2 flushed before each, CUDA events on
    the launching stream."""
    for _ in range(warmup):
        step_fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xff)
        ev[k][0].record(stream)
        step_fn()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return float(sum(a.elapsed_time(b) for a, b in ev))


def run_batched(args):
    """256 independent scenes (counts log-uniform in [500, 50,000], circle swaps and
    bidirectional flows) advanced by one persistent launch per step in a CUDA graph:
    untuned, autotuned (cell-edge factor and launch shape), and one context per scene."""
    import torch
    from paper_1908_10107_gb300 import abi, autotune, multigpu, scenarios
    local = int(os.environ.get("LOCAL_RANK", "0"))
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    full = scenarios.batched()
    # scenes split across ranks by agent count (no collective on the data path)
    lo, hi = multigpu.shard_scenes([s.n for s in full.scenes], world)[rank]
    batch = scenarios.Batch(full.scenes[lo:hi])
    n = batch.n
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    sim = abi.OrcaSim.for_batch(batch)
    sim.set_batch(batch)
    untuned = timed_steps(torch, lambda: sim.step(1), args.steps, args.warmup, flush, stream)
    tune = autotune.tune_batch(sim, batch, between=lambda: flush.fill_(0x5a))
    tuned = timed_steps(torch, lambda: sim.step(1), args.steps, args.warmup, flush, stream)
    launches = abi.orca_launches_per_step(sim.ctx)
    sim.close()
    per_scene = None
    if not args.no_per_scene:
        sims = []
        for sc, cs in zip(batch.scenes, tune["cell_sizes"]):
            s1 = abi.OrcaSim.for_scene(sc, cell_size=cs)
            s1.set_scene(sc)
            sims.append(s1)

        def step_all():
            for s1 in sims:
                s1.step(1)
        per_scene = timed_steps(torch, step_all, max(args.steps // 4, 3), args.warmup, flush, stream)
        per_scene_steps = max(args.steps // 4, 3)
        for s1 in sims:
            s1.close()
    value, tuned_max = multigpu.job_throughput(float(n * args.steps), tuned, dist, device="cuda")
    if rank != 0:
        dist.destroy_process_group()
        return
    line = {
        "metric": "batched ORCA agent-steps/sec (256 scenes, one persistent launch per step)",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tuned / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
        "config": {"workload": f"256 scenes, {full.n:,} agents, counts log-uniform in [500, 50000], "
                               "circle swaps and bidirectional flows", "n_agents": full.n,
                   "rank0_scenes": [lo, hi], "parallelism": f"scenes sharded over {world} GPU(s)",
                   "l2": "flushed between steps (256 MiB write)"},
        "untuned": {"value": n * args.steps / (untuned * 1e-3), "ms_per_step": untuned / args.steps,
                    "setting": "cell edge r_obs/4 per scene, 128 threads, default LP3 lanes"},
        "tuned": {"value": n * args.steps / (tuned * 1e-3), "ms_per_step": tuned / args.steps,
                  "scope": "rank 0's scenes",
                  "cell_factor": tune["factor"], "shape": list(tune["shape"]),
                  "factor_timings_ms": {str(k): round(v, 4) for k, v in tune["factor_timings_ms"].items()},
                  "shape_timings_ms": {k: round(v, 4) for k, v in tune["timings_ms"].items()}},
        "gpu_launches": launches * args.steps,
    }
    if per_scene is not None:
        line["one_context_per_scene"] = {"value": n * per_scene_steps / (per_scene * 1e-3),
                                         "ms_per_step": per_scene / per_scene_steps,
                                         "setting": "one context and graph launch per scene, tuned cells"}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def fd_check_patch(sc, T, C, rel=1e-3, m=64, seed=0):
    """Adjoint of the mean squared position error on an m-agent patch of the crowd (full
    horizon T) against FP64 central differences of the oracle: the FP32 rollout adjoint
    (checkpoints every C steps) and the FP64 validation instantiation of the same adjoint
    (orca_validate_rollout_fp64).  Entries whose stencil crosses a branch (one-sided slopes
    differ by > 1%) are excluded; the others must be within 1e-3 relative plus the finite
    difference's own error (twice its change from h to h/2), plus, for FP32 only, 1e-6 of
    the largest gradient (FP32 rounding).  Returns a summary."""
    import torch
    import oracle
    from paper_1908_10107_gb300 import abi, adjoint, scenarios
    oracle.build()
    pt = scenarios.patch(sc, m, seed)
    tp, tr, tt = scenarios.perturbed_parameters(pt, seed + 1)

    def oracle_traj(pref, rad, tau):
        pos, vel = pt.pos.astype(np.float64), pt.vel.astype(np.float64)
        out = []
        for _ in range(T):
            r = oracle.step(pos, vel, pt.goal, rad, pt.max_speed, pref, tau, pt.neighbor_dist,
                            pt.max_neighbors, pt.dt, knn_mode=0, fp64_knn=False, nthreads=1)
            pos, vel = r["pos"], r["vel"]
            out.append(pos)
        return np.stack(out)

    target_traj = oracle_traj(tp.astype(np.float64), tr.astype(np.float64), tt.astype(np.float64))
    base = dict(pref=pt.pref_speed.astype(np.float64), rad=pt.radius.astype(np.float64),
                tau=pt.time_horizon.astype(np.float64))

    def loss(**kw):
        a = dict(base)
        a.update(kw)
        tr_ = oracle_traj(a["pref"], a["rad"], a["tau"])
        return float(((tr_ - target_traj) ** 2).sum() / (T * m))

    # FP32 rollout adjoint
    sim = abi.OrcaSim.for_scene(pt)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in pt.arrays()]
    pos0, vel0, goal, radius, vmax, pref, tau = dev
    for t in (radius, pref, tau):
        t.requires_grad_(True)
    traj = adjoint.rollout(sim, pos0, vel0, goal, radius, vmax, pref, tau, T, C)
    ref_traj = oracle_traj(base["pref"], base["rad"], base["tau"])
    drift_by_step = np.abs(traj.detach().cpu().numpy().astype(np.float64) - ref_traj).max(axis=(1, 2))
    tgt = torch.from_numpy(target_traj.astype(np.float32)).cuda()
    adjoint.mse_trajectory_loss(traj, tgt).backward()
    g32 = {"pref": pref.grad.cpu().numpy(), "rad": radius.grad.cpu().numpy(), "tau": tau.grad.cpu().numpy()}
    sim.close()
    # FP64 validation adjoint
    d64 = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda() for a in pt.arrays()]
    args64 = (np.float32(pt.neighbor_dist), pt.max_neighbors, float(np.float32(pt.dt)), T)
    traj64 = abi.orca_validate_rollout_fp64(*d64, *args64)["traj"].cpu().numpy()
    dl = torch.from_numpy(2.0 * (traj64 - target_traj) / (T * m)).cuda()
    r64 = abi.orca_validate_rollout_fp64(*d64, *args64, dl)
    g64 = {"pref": r64["pref"].cpu().numpy(), "rad": r64["radius"].cpu().numpy(),
           "tau": r64["tau"].cpu().numpy()}
    res = {k: {"within_1e-3": 0, "outside": 0, "worst_relative_error": 0.0} for k in ("fp32", "fp64")}
    excluded = 0
    L0 = loss()
    for key in ("pref", "rad", "tau"):
        scale32 = np.abs(g32[key]).max()
        for a in range(m):
            x0 = base[key][a]
            h = 1e-6 * max(abs(x0), 1.0)
            vals = {}
            for dx in (h, -h, h / 2, -h / 2):
                arr = base[key].copy()
                arr[a] = x0 + dx
                vals[dx] = loss(**{key: arr})
            central = (vals[h] - vals[-h]) / (2 * h)
            fd_err = abs(central - (vals[h / 2] - vals[-h / 2]) / h)
            fwd, bwd = (vals[h] - L0) / h, (L0 - vals[-h]) / h
            if abs(fwd - bwd) > 1e-2 * max(abs(fwd), abs(bwd)) + 4 * fd_err:
                excluded += 1
                continue
            for name, g, extra in (("fp32", g32, 1e-6 * scale32), ("fp64", g64, 0.0)):
                err = abs(g[key][a] - central)
                r = res[name]
                r["worst_relative_error"] = max(r["worst_relative_error"],
                                                float(err / max(abs(central), 1e-300)))
                if err <= rel * abs(central) + 2 * fd_err + extra:
                    r["within_1e-3"] += 1
                else:
                    r["outside"] += 1
    return {"agents": m, "steps": T, "excluded_non_differentiable": excluded,
            "fp32_adjoint": res["fp32"], "fp64_adjoint": res["fp64"],
            "fp32_fp64_trajectory_drift_m": {"step_1": float(drift_by_step[0]),
                                             "final": float(drift_by_step[-1]),
                                             "max": float(drift_by_step.max())}}


def run_adjoint(args):
    """Forward + adjoint rollout of the differentiable workload (16,384-agent flow, 64 steps
    at dt 0.1 s, loss = mean squared position error against a rollout with perturbed
    parameters) against the plain step on the same crowd, in both rollout modes: every step
    recorded by the forward pass (ckpt_every = 0, the headline) and checkpoints every 8
    steps with the segments re-run by the backward pass."""
    import torch
    from paper_1908_10107_gb300 import abi, adjoint, scenarios
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    T, C = 64, 8
    sc = scenarios.differentiable()
    n = sc.n
    target = scenarios.perturbed_parameters(sc, 7)
    sim = abi.OrcaSim.for_scene(sc)
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in sc.arrays()]
    pos0, vel0, goal, radius, vmax, pref, tau = dev
    tp, tr, tt = [torch.from_numpy(a).cuda() for a in target]
    with torch.no_grad():
        tgt = adjoint.rollout(sim, pos0, vel0, goal, tr, vmax, tp, tt, T, C)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    modes = {}
    for mode in (0, C):
        fwd_ms, bwd_ms = [], []
        for rep in range(args.warmup + max(args.steps // 100, 5)):
            for t in (radius, pref, tau):
                t.grad = None
                t.requires_grad_(True)
            flush.fill_(rep & 0xff)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            traj = adjoint.rollout(sim, pos0, vel0, goal, radius, vmax, pref, tau, T, mode)
            loss = adjoint.mse_trajectory_loss(traj, tgt)
            e1.record(stream)
            loss.backward()
            e2.record(stream)
            torch.cuda.synchronize()
            if rep >= args.warmup:
                fwd_ms.append(e0.elapsed_time(e1))
                bwd_ms.append(e1.elapsed_time(e2))
        modes[mode] = (float(np.median(fwd_ms)), float(np.median(bwd_ms)),
                       abi.orca_rollout_workspace_size(sim.ctx, T, mode))
    # the plain step on the same crowd: T steps through the graph
    sim.set_scene(sc)
    plain = []
    for rep in range(args.warmup + 5):
        sim.set_scene(sc)
        flush.fill_(rep & 0xff)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(T)
        e1.record(stream)
        torch.cuda.synchronize()
        if rep >= args.warmup:
            plain.append(e0.elapsed_time(e1))
    sim.close()
    pl = float(np.median(plain))
    f, b, ws = modes[0]
    fc, bc, wsc = modes[C]
    check = None if args.no_fd_check else {f"T{h}": fd_check_patch(sc, h, C) for h in (8, 16, T)}
    line = {
        "metric": "forward+adjoint ORCA rollout agent-steps/sec (16,384 agents, 64 steps)",
        "value": n * T / ((f + b) * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": T,
        "warmup": args.warmup, "ms_per_step": (f + b) / T, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
        "config": {"workload": "bidirectional flow, 16,384 agents, dt 0.1 s, 64 steps, every step "
                               "recorded by the forward pass; loss = mean squared position error "
                               "against a rollout with perturbed pref speed / radius / tau",
                   "n_agents": n, "workspace_bytes": ws},
        "forward_ms": f, "backward_ms": b, "plain_ms_for_T_steps": pl,
        "plain_value": n * T / (pl * 1e-3),
        "forward_adjoint_over_plain": (f + b) / pl,
        "checkpointed_every_8": {"value": n * T / ((fc + bc) * 1e-3), "forward_ms": fc,
                                 "backward_ms": bc, "forward_adjoint_over_plain": (fc + bc) / pl,
                                 "workspace_bytes": wsc},
        "fd_check_64_agent_patch_by_horizon": check,
    }
    print(json.dumps(line), flush=True)


def run_crossing(args):
    """The paper's own protocol (Section 4): two-way crossings with equal and with varied
    agents (2,500 each) and the eight-way crossing (10,000), each run until every agent has
    reached its goal, arrived agents removed every ``--remove-every`` steps; then the
    frame time of the equal-agent two-way crossing against the number of agents (the
    paper's Fig. 6 experiment, which reports no values) on a steady stretch of steps."""
    import torch
    from paper_1908_10107_gb300 import abi, scenarios
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    every = args.remove_every
    runs = {}
    for name, sc in (("two_way_2500", scenarios.two_way_crossing(2500)),
                     ("two_way_varied_2500", scenarios.two_way_crossing(2500, heterogeneous=True)),
                     ("eight_way_10000", scenarios.eight_way_crossing(10000))):
        sim = abi.OrcaSim.for_scene(sc)
        for timed in (False, True):  # an untimed pass first (library load, first captures)
            sim.set_scene(sc)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            steps, agent_steps, n, removals = 0, 0, sc.n, 0
            while n > 0 and steps < args.crossing_max_steps:
                sim.step(every)
                steps += every
                agent_steps += n * every
                n = abi.orca_remove_arrived(sim.ctx)
                removals += 1
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        runs[name] = {"agents": sc.n, "steps_until_all_arrived": steps if n == 0 else None,
                      "agents_left": n, "simulated_s": steps * sc.dt, "wall_s": wall,
                      "agent_steps": agent_steps, "agent_steps_per_s": agent_steps / wall,
                      "ms_per_step": 1e3 * wall / max(steps, 1), "removals": removals}
        sim.close()
    # the same crossing with the people entering during the run (Section 4's spawning):
    # every `every` steps each waiting person gets a random spot in its start region and is
    # admitted unless it could touch someone within the next `every` steps
    empty, _ = scenarios.two_way_stream(2500)
    for timed in (False, True):
        _, source = scenarios.two_way_stream(2500)
        sim = abi.OrcaSim(max_agents=2500, max_neighbors=empty.max_neighbors,
                          neighbor_dist=empty.neighbor_dist, dt=empty.dt)
        sim.set_scene(empty)
        rng = np.random.default_rng(1917)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        steps, agent_steps, n, waves, last_entry = 0, 0, 0, 0, 0
        while (source.n > 0 or n > 0) and steps < args.crossing_max_steps:
            if source.n > 0:
                admitted = sim.spawn(*source.candidates(rng), window=every * float(empty.dt))
                source.admit(admitted)
                waves += 1
                n = sim.n
                if admitted.any():
                    last_entry = steps
            sim.step(every)
            steps += every
            agent_steps += n * every
            n = abi.orca_remove_arrived(sim.ctx)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        sim.close()
    runs["two_way_2500_spawned_during_the_run"] = {
        "agents": 2500, "steps_until_all_arrived": steps if n == 0 and source.n == 0 else None,
        "agents_left": n + source.n, "simulated_s": steps * float(empty.dt), "wall_s": wall,
        "agent_steps": agent_steps, "agent_steps_per_s": agent_steps / wall,
        "ms_per_step": 1e3 * wall / max(steps, 1), "spawn_waves": waves,
        "last_entry_step": last_entry}
    sweep = []
    for n in (2500, 10000, 50000, 100000, 500000):
        sc = scenarios.two_way_crossing(n)
        sim = abi.OrcaSim.for_scene(sc)
        sim.set_scene(sc)
        sim.step(50)
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(200)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 200
        sweep.append({"agents": n, "ms_per_step": ms, "agent_steps_per_s": n / (ms * 1e-3),
                      "fps": 1e3 / ms})
        sim.close()
    total_as = sum(r["agent_steps"] for r in runs.values())
    total_wall = sum(r["wall_s"] for r in runs.values())
    total_steps = sum(round(r["simulated_s"] / 0.1) for r in runs.values())
    line = {
        "metric": "paper-protocol crossings: agent-steps/sec until every agent has arrived",
        "value": total_as / total_wall, "unit": UNIT, "n_gpus": 1,
        "steps": total_steps, "warmup": 1,
        "ms_per_step": 1e3 * total_wall / max(total_steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
        "config": {"workload": "two-way crossings (2,500 equal / varied agents) and eight-way "
                               "crossing (10,000), Section 4 protocol, dt 0.1 s, r_obs 10 m, k 10, "
                               "tau 5 s", "remove_every_steps": every,
                   "timing": "host wall clock over whole runs (removals synchronise)"},
        "runs": runs,
        "frame_time_vs_agents": sweep,
        "paper": "more than 100,000 agents at 60 fps and about 30 fps at 5e5 agents on a "
                 "GTX 970 (context, other hardware)",
    }
    print(json.dumps(line), flush=True)


def run_lp_ab(args):
    """A/B of the LP modes -- one lane per solve, the agent split (four lanes per agent), and
    warp work units (the paper's load-balanced LP) -- on LP3-heavy and lighter crowds.  Each mode
    replays the same steps from the same saved state (the modes give bitwise-equal
    trajectories); the ORCA kernel's mean time comes from the library's phase events."""
    import torch
    from paper_1908_10107_gb300 import abi, scenarios
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    modes = ((64, 1), (64, 4), (64, 32), (128, 32))
    cases = []
    flow = scenarios.bidirectional()
    cases.append(("flow_524288_steps_1_30", flow, 1, {}))
    cases.append(("flow_524288_steps_300_330", flow, 300, {}))
    dense = scenarios.dense()
    cases.append(("dense_2097152_k20_steps_10_40", dense, 10, {}))
    eight = scenarios.eight_way_crossing(10000)
    cases.append(("eight_way_10000_steps_1500_1530", eight, 1500, {}))
    out = {}
    for name, sc, skip, _ in cases:
        sim = abi.OrcaSim.for_scene(sc)
        sim.set_scene(sc)
        if skip > 1:
            sim.step(skip - 1)
        pos, vel = sim.get_state()
        start = sc.copy()
        start.pos, start.vel = pos, vel
        row = {}
        for tpb, lanes in modes:
            abi.orca_set_launch(sim.ctx, tpb, lanes)
            abi.orca_profile(sim.ctx, False)
            sim.set_scene(start)
            sim.step(1)  # graph capture; the first step from a loaded state has no radius hint
            abi.orca_profile(sim.ctx, True)
            ts = []
            for _ in range(args.ab_steps):
                sim.step(1)
                ts.append(float(abi.orca_profile_read(sim.ctx)[2]))
            c = sim.counters()
            row[f"{tpb}x{lanes}"] = {"orca_kernel_ms": float(np.mean(ts)),
                                     "lp3_fraction": c["lp3_agent_steps"] / max(c["agent_steps"], 1)}
        out[name] = row
        sim.close()
    line = {"metric": "ORCA kernel ms per LP mode (one lane / agent split / warp work units)",
            "value": None, "unit": "ms", "n_gpus": 1, "steps": args.ab_steps, "warmup": 1,
            "higher_is_better": False, "dtype": "f32", "data": "synthetic (seeded)",
            "config": {"workload": "LP-mode A/B on the 524,288-agent flow (early and later steps), "
                                   "the 2,097,152-agent dense crowd (k 20) and the eight-way crossing"},
            "cases": out}
    print(json.dumps(line), flush=True)


def run_table(args):
    """The five configurations side by side (GPU and, where it runs in seconds, the FP64
    oracle on the host cores): the 1,024-agent circle swap (100 steps both), the
    524,288-agent flow (20 steps both), the 2,097,152-agent dense crowd at k = 20 (GPU 100
    steps, oracle 3 steps); the batch and the forward + adjoint rollout come from their own
    workloads.  GPU: default cell edge r_obs / 4 autotuned, CUDA events, L2 flushed
    between steps."""
    import torch
    from paper_1908_10107_gb300 import abi, autotune, scenarios
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    rows = {}
    for name, sc, gpu_steps, cpu_steps in (("circle_swap_1024", scenarios.circle_swap(), 100, 100),
                                           ("bidirectional_524288", scenarios.bidirectional(), 20, 20),
                                           ("dense_2097152_k20", scenarios.dense(), 100, 3)):
        sim = abi.OrcaSim.for_scene(sc)
        sim.set_scene(sc)
        tune = autotune.tune_cell_size(sim, sc, use_cache=False, cache_path=None,
                                       between=lambda: flush.fill_(0x5a))
        shape = autotune.tune_launch(sim, lambda: sim.set_scene(sc), between=lambda: flush.fill_(0x5a))
        sim.set_scene(sc)
        ms = timed_steps(torch, lambda: sim.step(1), gpu_steps, args.warmup, flush, stream) / gpu_steps
        sim.close()
        cpu = cpu_baseline(sc, budget_s=1e9, max_steps=cpu_steps)
        rows[name] = {"agents": sc.n, "gpu_ms_per_step": ms, "gpu_agent_steps_per_s": sc.n / (ms * 1e-3),
                      "hbm_frac_128B": STEP_BYTES_PER_AGENT * sc.n / (ms * 1e-3) / 1e9 / peaks()[0],
                      "gpu_steps": gpu_steps, "cell_m": tune["cell_size"], "shape": list(shape["shape"]),
                      "cpu_ms_per_step": sc.n / cpu["value"] * 1e3, "cpu_agent_steps_per_s": cpu["value"],
                      "cpu_sample": cpu["sample"], "cpu_cores": cpu["cores"], "cpu_model": cpu["cpu_model"]}
    line = {"metric": "configurations table: GPU and FP64-oracle agent-steps/sec", "value":
            rows["bidirectional_524288"]["gpu_agent_steps_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": 20, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
            "config": {"workload": "circle swap 1,024; bidirectional flow 524,288; dense 2,097,152 "
                                   "(k 20)", "l2": "flushed between steps"}, "rows": rows}
    print(json.dumps(line), flush=True)


def run_dense(args):
    """The dense stress crowd (2,097,152 agents uniform in 2 km x 2 km, r 0.4 m, v_max 1.5
    m/s, r_obs 8 m, tau 4 s, dt 1/60 s): k = 10 and 20, each over the cell edges 1, 2, 4 and
    8 m and the autotuned edge, L2 flushed between steps, CUDA events on the stream."""
    import torch
    from paper_1908_10107_gb300 import abi, autotune, scenarios
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    base = scenarios.dense()
    n = base.n
    results = {}
    for k in (10, 20):
        sc = base.copy()
        sc.max_neighbors = k
        sim = abi.OrcaSim.for_scene(sc)
        sim.set_scene(sc)
        tune = autotune.tune_cell_size(sim, sc, use_cache=False, cache_path=None,
                                       between=lambda: flush.fill_(0x5a))
        shape = autotune.tune_launch(sim, lambda: sim.set_scene(sc),
                                     between=lambda: flush.fill_(0x5a))
        row = {"tuned_cell_m": tune["cell_size"], "tuned_shape": list(shape["shape"])}
        for cs in (1.0, 2.0, 4.0, 8.0, tune["cell_size"]):
            abi.orca_set_cell_size(sim.ctx, cs)
            sim.set_scene(sc)
            ms = timed_steps(torch, lambda: sim.step(1), args.dense_steps, args.warmup, flush, stream)
            key = "tuned" if cs == tune["cell_size"] else f"{cs:g}m"
            row[key] = {"ms_per_step": ms / args.dense_steps,
                        "agent_steps_per_s": n * args.dense_steps / (ms * 1e-3)}
        c = sim.counters()
        row["lp3_fraction"] = c["lp3_agent_steps"] / max(c["agent_steps"], 1)
        results[f"k{k}"] = row
        sim.close()
    best = max(r["tuned"]["agent_steps_per_s"] for r in results.values())
    line = {"metric": "dense-crowd ORCA agent-steps/sec (2,097,152 agents)", "value": best,
            "unit": UNIT, "n_gpus": 1, "steps": args.dense_steps, "warmup": args.warmup,
            "ms_per_step": n / best * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
            "config": {"workload": "dense stress: 2,097,152 agents uniform in 2 km x 2 km, goals "
                                   "uniform, r 0.4 m, v_max 1.5 m/s, r_obs 8 m, k 10 / 20, tau 4 s, "
                                   "dt 1/60 s; cell edge swept", "l2": "flushed between steps"},
            "results": results}
    print(json.dumps(line), flush=True)


def run_obstacles(args):
    """Static obstacles (the ORCA obstacle rule; not in the paper's experiments): a
    2,000-agent room emptying through a 2.4 m door until everyone has left, timed on the
    wall clock with removals every ``--remove-every`` steps; then the cost of the obstacle
    half-planes on two 524,288-agent crowds -- the bottleneck room and the bidirectional
    flow with 256 random segments -- each stepped from the same state with and without its
    obstacles (L2 flushed between steps, CUDA events on the stream; the ORCA kernel's time
    from the library's phase events)."""
    import torch
    from paper_1908_10107_gb300 import abi, scenarios
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    every = args.remove_every
    # 1. evacuation until the room is empty
    evac = None
    if args.evacuation:
        sc = scenarios.bottleneck(2000)
        sim = abi.OrcaSim.for_scene(sc)
        for timed in (False, True):  # an untimed pass first (library load, first captures)
            sim.set_scene(sc)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            steps, agent_steps, n = 0, 0, sc.n
            while n > 0 and steps < args.crossing_max_steps:
                sim.step(every)
                steps += every
                agent_steps += n * every
                n = abi.orca_remove_arrived(sim.ctx)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        evac = {"agents": sc.n, "steps_until_all_arrived": steps if n == 0 else None,
                "agents_left": n, "simulated_s": steps * sc.dt, "wall_s": wall,
                "agent_steps_per_s": agent_steps / wall, "ms_per_step": 1e3 * wall / max(steps, 1)}
        sim.close()
    # 2. obstacle cost on large crowds
    room = scenarios.bottleneck(524288)
    flow = scenarios.bidirectional()
    rng = np.random.default_rng(1917)
    lo, hi = flow.pos.min(0), flow.pos.max(0)
    a = rng.uniform(lo, hi, (256, 2))
    flow.obstacles = np.concatenate([a, a + rng.normal(0, 4, (256, 2))], 1).astype(np.float32)
    flow.obstacle_time_horizon = np.float32(3.0)
    flow.max_obstacle_neighbors = 4
    cases = {}
    for name, sc, skip in (("bottleneck_524288_steps_100_150", room, 100),
                           ("flow_524288_256_segments_steps_1_50", flow, 0)):
        sim = abi.OrcaSim.for_scene(sc)
        sim.set_scene(sc)
        if skip:
            sim.step(skip)
        pos, vel = sim.get_state()
        start = sc.copy()
        start.pos, start.vel = pos, vel
        bare = start.copy()
        bare.obstacles = None
        row = {"segments": int(len(sc.obstacles))}
        for key, s0 in (("obstacles", start), ("none", bare)):
            sim.set_scene(s0)
            ms = timed_steps(torch, lambda: sim.step(1), args.obst_steps, args.warmup, flush, stream)
            abi.orca_profile(sim.ctx, True)
            ks = []
            for _ in range(10):
                flush.fill_(0x5a)
                sim.step(1)
                ks.append(float(abi.orca_profile_read(sim.ctx)[2]))
            abi.orca_profile(sim.ctx, False)
            c = sim.counters()
            row[key] = {"ms_per_step": ms / args.obst_steps,
                        "agent_steps_per_s": sc.n * args.obst_steps / (ms * 1e-3),
                        "orca_kernel_ms": float(np.mean(ks)),
                        "lp3_fraction": c["lp3_agent_steps"] / max(c["agent_steps"], 1)}
        row["agents_within_reach_of_a_segment"] = agents_within_reach(start)
        cases[name] = row
        sim.close()
    head = cases["bottleneck_524288_steps_100_150"]["obstacles"]
    line = {"metric": "agent-steps/sec with static obstacles (524,288-agent bottleneck room)",
            "value": head["agent_steps_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.obst_steps, "warmup": args.warmup,
            "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
            "config": {"workload": "bottleneck rooms (2,000 agents until empty; 524,288 agents "
                                   "steady) and the 524,288-agent flow with 256 random segments; "
                                   "obstacle time horizon 2 s / 3 s, 4 obstacle lines per agent",
                       "remove_every_steps": every, "l2": "flushed between steps"},
            "evacuation_2000": evac, "cases": cases}
    print(json.dumps(line), flush=True)


def agents_within_reach(scene) -> int:
    """How many agents have a segment within their reach V tau_o + r (host geometry, FP64)."""
    seg = scene.obstacles.astype(np.float64)
    p = scene.pos.astype(np.float64)
    reach = scene.max_speed.astype(np.float64) * float(scene.obstacle_time_horizon) + scene.radius
    a, e = seg[:, :2], seg[:, 2:] - seg[:, :2]
    l2 = np.maximum((e * e).sum(1), 1e-300)
    best = np.full(len(p), np.inf)
    for lo in range(0, len(p), 1 << 14):
        w = p[lo:lo + (1 << 14), None, :] - a[None]
        t = np.clip((w * e[None]).sum(2) / l2[None], 0.0, 1.0)
        q = w - t[..., None] * e[None]
        best[lo:lo + (1 << 14)] = np.sqrt((q * q).sum(2)).min(1)
    return int((best < reach).sum())


def post_load_step(torch, abi, sim, sc, stream, flush, warmup, reps=5) -> dict:
    """Device time of one step right after the crowd is loaded with orca_set_agents (no
    search-radius predictions: the start radius comes from the local density) against one
    right after orca_update_state (predictions kept), both from the same evolved state of
    the crowd, L2 flushed before each; medians of `reps`."""
    sim.set_scene(sc)
    sim.step(warmup)
    pos, vel = sim.get_state()
    params = list(sc.arrays()[2:])
    times = {"after_set_agents": [], "after_update_state": []}
    phases = {k: [] for k in times}
    cands = {k: [] for k in times}
    abi.orca_profile(sim.ctx, True)
    for _ in range(reps):
        for kind in times:
            if kind == "after_set_agents":
                abi.orca_set_agents(sim.ctx, sc.n, pos, vel, *params, stream=stream)
            else:
                abi.orca_update_state(sim.ctx, pos, vel, stream=stream)
            c0 = sim.counters()
            s0 = sim.search_counters()
            flush.fill_(0x5a)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim.step(1)
            b.record(stream)
            torch.cuda.synchronize()
            times[kind].append(a.elapsed_time(b))
            phases[kind].append(abi.orca_profile_read(sim.ctx))
            c1 = sim.counters()
            s1 = sim.search_counters()
            na = max(c1["agent_steps"] - c0["agent_steps"], 1)
            cands[kind].append(((c1["candidates"] - c0["candidates"]) / na,
                                (s1["rows"] - s0["rows"]) / na,
                                (s1["extra_passes"] - s0["extra_passes"]) / na))
    abi.orca_profile(sim.ctx, False)
    out = {k: float(np.median(v)) for k, v in times.items()}
    out["search_per_agent"] = {k: dict(zip(("candidates", "rows", "extra_passes"),
                                           [round(float(x), 3) for x in np.median(np.array(v), axis=0)]))
                               for k, v in cands.items()}
    out["ratio"] = out["after_set_agents"] / out["after_update_state"]
    out["phases_ms"] = {k: [round(float(x), 4) for x in np.median(np.array(v), axis=0)]
                        for k, v in phases.items()}
    out["note"] = ("timed with event-record nodes between the phases (binning, reorder, ORCA "
                   "kernel); after orca_set_agents the agents arrive in agent order, so the "
                   "first binning sorts a random order")
    return out


def alu_roofline(sim, sc, abi, warmup, steps, main_ms, peak):
    """Arithmetic roofline of the ORCA kernel: the timed steps replayed (untimed, from the
    same loaded state, so the trajectory is identical) with operation counting on, the
    counts turned into FP32 operations by FLOPS, over the kernel's mean duration, against
    the measured FP32 FMA rate `peak` (fma_peak)."""
    abi.orca_profile(sim.ctx, False)
    abi.orca_count_ops(sim.ctx, True)
    sim.set_scene(sc)
    sim.step(warmup)
    c0, o0 = sim.counters(), sim.op_counters()
    sim.step(steps)
    c1, o1 = sim.counters(), sim.op_counters()
    abi.orca_count_ops(sim.ctx, False)
    agents = max(c1["agent_steps"] - c0["agent_steps"], 1)
    per = {"candidates": (c1["candidates"] - c0["candidates"]) / agents,
           "lines": (c1["lines"] - c0["lines"]) / agents}
    for k in ("lp1_calls", "lp1_bounds", "lp_checks", "bisectors"):
        per[k] = (o1[k] - o0[k]) / agents
    flops = sum(FLOPS[k] * v for k, v in per.items())
    achieved = flops * sc.n / (main_ms * 1e-3) / 1e12
    return {"kernel": "orca_main (neighbours + half-planes + LP + integrate)", "bound": "alu",
            "achieved": achieved, "peak": peak["tflops"], "unit": "TFLOP/s",
            "frac": achieved / peak["tflops"],
            "flops_per_agent": flops, "ops_per_agent": {k: round(v, 3) for k, v in per.items()},
            "launch_ms": main_ms,
            "peak_source": f"measured: FP32 FMA microbenchmark (orca_fma_bench, {peak['blocks']} "
                           f"CTAs x 256 threads x {peak['iters']} x 32 FMAs, best of "
                           f"{peak['repeats']}, CUDA events)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--agents", type=int, default=524288)
    ap.add_argument("--cell-size", type=float, default=0.0)
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-sample", type=int, default=4096)
    ap.add_argument("--clocks-out", default=None)
    ap.add_argument("--workload", choices=["plain", "batched", "adjoint", "crossing", "lp_ab", "obstacles",
                                           "dense", "table"], default="plain")
    ap.add_argument("--dense-steps", type=int, default=100, help="dense workload: timed steps")
    ap.add_argument("--obst-steps", type=int, default=50, help="obstacles workload: timed steps")
    ap.add_argument("--no-evacuation", dest="evacuation", action="store_false",
                    help="obstacles workload: only the two large crowds")
    ap.add_argument("--ab-steps", type=int, default=30, help="lp_ab workload: timed steps per mode")
    ap.add_argument("--remove-every", type=int, default=20,
                    help="crossing workload: steps between removals of arrived agents")
    ap.add_argument("--crossing-max-steps", type=int, default=30000)
    ap.add_argument("--no-per-scene", action="store_true")
    ap.add_argument("--no-fd-check", action="store_true",
                    help="adjoint workload: skip the finite-difference check (timing only)")
    ap.add_argument("--tpb", type=int, default=0, help="fix threads per CTA (skips shape tuning)")
    ap.add_argument("--lanes", type=int, default=0, help="fix LP3 lanes per agent (with --tpb)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.workload == "batched" and args.impl == "ours":
        run_batched(args)
        return
    if args.workload == "adjoint" and args.impl == "ours":
        run_adjoint(args)
        return
    if args.workload == "crossing" and args.impl == "ours":
        run_crossing(args)
        return
    if args.workload == "lp_ab" and args.impl == "ours":
        run_lp_ab(args)
        return
    if args.workload == "dense" and args.impl == "ours":
        run_dense(args)
        return
    if args.workload == "table" and args.impl == "ours":
        run_table(args)
        return
    if args.workload == "obstacles" and args.impl == "ours":
        run_obstacles(args)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1908_10107_gb300 import abi, build, scenarios
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()

    sc = scenarios.bidirectional(args.agents)
    sim = abi.OrcaSim.for_scene(sc, cell_size=args.cell_size)
    sim.set_scene(sc)
    tune = shape = None
    from paper_1908_10107_gb300 import autotune
    # the tuner flushes L2 between its timed steps, as the timed region below does
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    flush_l2 = lambda: flush.fill_(0x5a)  # noqa: E731
    if args.cell_size <= 0:
        tune = autotune.tune_cell_size(sim, sc, use_cache=False, cache_path=None,
                                       between=flush_l2)
        args.cell_size = tune["cell_size"]
    if args.tpb:
        abi.orca_set_launch(sim.ctx, args.tpb, args.lanes)
        shape = {"shape": (args.tpb, args.lanes), "timings_ms": None}
    else:
        shape = autotune.tune_launch(sim, lambda: sim.set_scene(sc), between=flush_l2)
    # the timed region runs the product step graph (no profiling events inside it)
    abi.orca_profile(sim.ctx, False)
    stream = torch.cuda.current_stream()
    sim.set_scene(sc)
    for _ in range(args.warmup):
        sim.step(1)
    torch.cuda.synchronize()
    ev_s = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev_e = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    sampler = ClockSampler(device_smi_index(torch, local), args.clocks_out)

    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.15)
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        ev_s[k].record(stream)
        sim.step(1)
        ev_e[k].record(stream)
    torch.cuda.synchronize()
    wall1 = time.perf_counter()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = np.array([ev_s[k].elapsed_time(ev_e[k]) for k in range(args.steps)])
    n = sc.n
    from paper_1908_10107_gb300 import multigpu
    # replicas: every rank advances its own copy of the crowd; whole-job agent-steps over
    # the slowest rank's device time
    value, total_ms = multigpu.job_throughput(float(n * args.steps), float(step_ms.sum()),
                                              dist, device="cuda")
    sim.sync()
    ms_per_step = total_ms / args.steps

    # the phase split: the same steps replayed from the same loaded state (identical
    # trajectory) with event-record nodes between the phases, L2 flushed as above
    abi.orca_profile(sim.ctx, True)
    sim.set_scene(sc)
    for _ in range(args.warmup):
        sim.step(1)
    torch.cuda.synchronize()
    phases = np.zeros((args.steps, 3))
    pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(k & 0xff)
        pev[k][0].record(stream)
        sim.step(1)
        pev[k][1].record(stream)
        phases[k] = abi.orca_profile_read(sim.ctx)
    torch.cuda.synchronize()
    prof_step_ms = float(np.mean([a.elapsed_time(b) for a, b in pev]))
    abi.orca_profile(sim.ctx, False)
    main_ms = float(phases[:, 2].mean())
    hbm_peak, peak_kind = peaks()
    gf, gi = None, None
    sim_cap = int(sim.params.max_cells) or min(max(4 * n, 65536), 1 << 30)
    achieved = ORCA_KERNEL_BYTES_PER_AGENT * n / (main_ms * 1e-3) / 1e9
    traffic = profiled_traffic()
    counters = sim.counters()
    launches = abi.orca_launches_per_step(sim.ctx) * args.steps

    try:
        sim_rec = abi.OrcaSim.for_scene(sc, cell_size=args.cell_size, flags=abi.ORCA_FLAG_RECORD)
        sim_rec.set_scene(sc)
        sim_rec.step(1)
        _, gf, gi = sim_rec.get_cells()
        sim_rec.close()
    except Exception:
        pass

    # the ORCA kernel is bound by FP32 issue, not HBM: its arithmetic roofline from an
    # operation-counting replay of exactly the timed steps, against the measured FMA rate
    fma = fma_peak(torch, abi, stream)
    alu = alu_roofline(sim, sc, abi, args.warmup, args.steps, main_ms, fma)
    alu["traffic"] = traffic
    first_step = post_load_step(torch, abi, sim, sc, stream, flush, args.warmup)

    # end to end through the C ABI, a host-driven loop over the same crowd: each step
    # writes the state from pinned host memory into the simulation (parameters and
    # search-radius predictions stay on the device), steps, and reads the new state back
    # into the buffers the next step writes
    abi.orca_profile(sim.ctx, False)
    sim.set_scene(sc)
    sim.step(args.warmup)
    pos_h, vel_h = sim.get_state()
    pinned = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
              for a in [pos_h, vel_h] + list(sc.arrays()[2:])]
    out_pos, out_vel = pinned[0], pinned[1]

    def host_loop(one_step):
        # every variant runs the same stretch of the crowd: reload, warm up, one untimed step
        sim.set_scene(sc)
        sim.step(args.warmup)
        abi.orca_get_state(sim.ctx, out_pos, out_vel, stream=stream)
        one_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            one_step()
        return time.perf_counter() - t0

    def three_calls_step(upload):
        upload()
        sim.step(1)
        abi.orca_get_state(sim.ctx, out_pos, out_vel, stream=stream)

    # one call per step: state in, step, state out (orca_step_host, one synchronisation)
    e2e_dt = host_loop(lambda: abi.orca_step_host(sim.ctx, out_pos, out_vel, 1, out_pos, out_vel,
                                                  stream=stream))
    # the same as three calls (orca_update_state, orca_step, orca_get_state)
    three_dt = host_loop(lambda: three_calls_step(
        lambda: abi.orca_update_state(sim.ctx, out_pos, out_vel, stream=stream)))
    e2e_val = n * args.e2e_steps / e2e_dt
    if dist:
        t = torch.tensor([e2e_dt], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_val = world * n * args.e2e_steps / float(t.item())
    h2d = out_pos.nbytes + out_vel.nbytes
    d2h = out_pos.nbytes + out_vel.nbytes
    # the same loop re-loading the whole crowd every step (orca_set_agents: parameters
    # uploaded too, predictions reset), for comparison
    full_dt = host_loop(lambda: three_calls_step(
        lambda: abi.orca_set_agents(sim.ctx, n, *pinned, stream=stream)))
    full_upload = {"value": n * args.e2e_steps / full_dt, "unit": UNIT,
                   "h2d_bytes_per_step": sum(a.nbytes for a in pinned), "d2h_bytes_per_step": d2h}
    three_calls = {"value": n * args.e2e_steps / three_dt, "unit": UNIT,
                   "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
    sim.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(sc)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
        "config": {"workload": WORKLOAD, "n_agents": n, "replicas": world,
                   "cell_size_m": float(gf[2]) if gf is not None else None,
                   "grid": [int(gi[0]), int(gi[1])] if gi is not None else None,
                   "cell_table_capacity": int(sim_cap),
                   "timed_graph": "product step graph (no profiling nodes)",
                   "l2": "flushed between steps (256 MiB write); per-step CUDA events summed",
                   "graph": "one CUDA graph replay per step",
                   "cell_size_tuning_ms": ({f"{k:.4g}": round(v, 4) for k, v in tune["timings_ms"].items()}
                                           if tune else "fixed by --cell-size"),
                   "launch_shape": list(shape["shape"]) if shape else [128, 1],
                   "launch_shape_tuning_ms": ({k: round(v, 4) for k, v in shape["timings_ms"].items()}
                                              if shape and shape["timings_ms"] else "fixed by --tpb")},
        "roofline": alu,
        "hbm_roofline": {"kernel": "orca_main (neighbours + half-planes + LP + integrate)",
                         "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": traffic,
                         "alg_bytes_per_agent": ORCA_KERNEL_BYTES_PER_AGENT,
                         "launch_ms": main_ms,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                         if peak_kind == "measured" else "fallback 6800 GB/s"},
        "step_roofline": {"bound": "hbm", "alg_bytes_per_agent": STEP_BYTES_PER_AGENT,
                          "bytes_model": "minimal step: state read 40, write 16, key+index 16, "
                                         "sort scatter 16, message record 2 x 20",
                          "achieved": STEP_BYTES_PER_AGENT * n / (ms_per_step * 1e-3) / 1e9,
                          "peak": hbm_peak, "unit": "GB/s",
                          "frac": STEP_BYTES_PER_AGENT * n / (ms_per_step * 1e-3) / 1e9 / hbm_peak},
        "phases_ms": {"binning": float(phases[:, 0].mean()), "reorder": float(phases[:, 1].mean()),
                      "orca_kernel": main_ms, "profiled_step": prof_step_ms,
                      "source": "a second run of the timed steps from the same state with "
                                "event-record nodes between the phases"},
        "post_load_step_ms": first_step,
        "lp3_fraction": counters["lp3_agent_steps"] / max(counters["agent_steps"], 1),
        "candidates_per_agent": counters["candidates"] / max(counters["agent_steps"], 1),
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
                "api": "orca_step_host (state in, step, state out), pinned host buffers",
                "three_calls_per_step": three_calls,
                "full_reload_per_step": full_upload},
        "gpu_launches": launches,
        "clocks": clocks,
        "wall_s_timed_region": wall1 - wall0,
        "kernel_source_sha256_16": kernel_hash(),
    }
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
