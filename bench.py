#!/usr/bin/env python3
"""Benchmark of the B300 PSDF hot path; prints ONE JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl b300|reference]

One step = one pass of the value+gradient path over the dense-clutter
workload (rectangle footprint 0.6 x 0.4 m; 25,000 random-yaw rectangles =
100,000 edges in a 200 x 200 m field; 4,096 pose queries; synthetic, seeded):
the exact cull (one fused kernel: each pose takes an upper bound from the 32
obstacle circles its cell of the scene's candidate grid keeps; when that
bound lies within the cell's completeness radius -- every pose of this
workload -- the candidates whose circle bound does not exceed it are
evaluated exactly, else every obstacle of every tile of the pose's cull-grid
cell whose bounds do not exceed it; then the epilogue with the pose
gradient) followed by PSDF_Backward (pose and edge-endpoint gradients of
sum(phi)) from the forward's saved rows.  The metric counts pose x edge
pairs of the whole scene per second (the cull's results equal the full
scan's bit for bit, checked in the run); the full scan, the bound-ordered
cull (upper bound from the tile of smallest AABB bound) and the learned
cull (the tile-proposal network re-ranking each pose's 8 nearest tiles) are
timed on the same GPU.

Under torchrun (N > 1) every rank evaluates its own 4,096 poses on the same
scene (weak scaling, no data-path collective); the value is the total pair
count over the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PSDF pose×edge pair-evals/s (value+grad), learned-cull vs full scan, ≤1e-5 m err"
UNIT = "pair-evals/s"
WORKLOAD = "dense-clutter: 4096 poses x 100000 edges (25000 rectangles, 200x200 m), 0.6x0.4 m footprint"
L2_FLUSH_BYTES = 256 << 20


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched uneven-instances measurement")
    ap.add_argument("--only-batched", action="store_true",
                    help="run only the batched uneven-instances measurement (profiling runs)")
    return ap.parse_args()


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _workload(rank: int):
    from paper_2607_04310_b300 import scenegen as sg
    w = sg.dense_clutter(4)
    if rank > 0:  # weak scaling: every rank gets its own queries on the same scene
        g = sg.rng(4000 + rank)
        w.poses = sg.poses_uniform(g, w.P, 0.0, 200.0)
    return w


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self._reader = None

    def _read(self):
        for line in self.proc.stdout:
            if line.strip():
                self.lines.append(line)

    def __enter__(self):
        self.lines = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        if self.proc is not None:
            self._reader = threading.Thread(target=self._read, daemon=True)
            self._reader.start()
            # the timed region starts once nvidia-smi has started up and
            # taken its first sample (its start-up can take a second on a
            # fresh box): only the periodic queries overlap the timing
            t0 = time.time()
            while not self.lines and time.time() - t0 < 10.0 and self.proc.poll() is None:
                time.sleep(0.01)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.proc.wait()
            if self._reader is not None:
                self._reader.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def _sources_digest() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2607_04310_b300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(csrc, fn), "rb") as f:
                h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


def _traffic(kernel: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken
    on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        rec = d.get(kernel, {})
        if rec.get("sources") == _sources_digest() and rec.get("workload") == workload:
            return rec.get("bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# --------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# --------------------------------------------------------------------------
def _oracle_rate(w, seconds: float, seed: int = 0, nthreads: int = 0):
    import oracle
    g = np.random.default_rng(seed)
    n = 4
    while True:
        idx = g.choice(w.P, size=min(n, w.P), replace=False)
        t0 = time.perf_counter()
        oracle.psdf_eval(w.footprint, w.edges, w.offsets, w.poses[idx], nthreads=nthreads)
        dt = time.perf_counter() - t0
        if dt >= seconds or n >= w.P:
            break
        n = min(w.P, max(n * 2, int(n * seconds / max(dt, 1e-3) * 1.05)))
    return len(idx) * w.E / dt, len(idx), dt


def run_reference(a, rank, world):
    if rank != 0:
        return 0
    import oracle
    w = _workload(0)
    cores = oracle.max_threads()
    per_step = max(0.3, 60.0 / max(a.steps + a.warmup, 1))
    rate, n, dt = _oracle_rate(w, min(per_step, 10.0))
    # each step: the oracle on a bounded sample of the same workload
    times = []
    g = np.random.default_rng(1)
    for i in range(a.warmup + a.steps):
        idx = g.choice(w.P, size=n, replace=False)
        t0 = time.perf_counter()
        oracle.psdf_eval(w.footprint, w.edges, w.offsets, w.poses[idx])
        t = time.perf_counter() - t0
        if i >= a.warmup:
            times.append(t)
    tot = sum(times)
    value = a.steps * n * w.E / tot
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1000.0 * tot / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample_poses_per_step": int(n),
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d of 4096 poses x 100000 edges per step" % n},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------------
# B300 arm
# --------------------------------------------------------------------------
CULL_K = 1
# Where the headline step's upper bound comes from: "circles" (the scene's
# candidate grid: the 32 obstacle circles nearest each cell, no proposal;
# with its completeness radius the candidates stand for the whole scene),
# "bound" (the circles of the tile of smallest AABB bound) or "mlp" (of the
# trained network's best tile).  On the sort-tile-recursive tiles of this
# workload the network picks the bound's tile 93 % of the time and adds its
# ranking to every pose's chain, and the grid needs neither a ranking nor
# tiles, so the grid is the fastest exact path; the other two are measured
# beside it.
HEADLINE_MODE = "circles"


def _time_steps(step, steps, flush, stream, clocks=None):
    """Device time of each step (CUDA events on the launching stream), L2
    flushed before every step outside the timed interval.  The steps queue
    up behind a short device-side wait, so that the host has launched many
    of them before the device reaches the first (a pause of the host thread
    then does not leave the device idle inside a timed interval)."""
    import torch
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    torch.cuda._sleep(2_000_000)  # about 1 ms of device time
    for i in range(steps):
        flush.zero_()
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)]


def _graph(step):
    """Capture one step (every launch of the library goes to the current
    stream) into a CUDA graph; returns its replay function."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        step()
    torch.cuda.synchronize()
    return g.replay, g


def _bench_batched(a, dev, flush, stream, peak):
    """Batched uneven instances (1,024 instances, horizons 10..100, 16..65,536
    edges, 4..12-vertex footprints): the plan's autotuned persistent launch as
    one CUDA graph, against one psdf_eval_grad call per instance (also one
    graph)."""
    import torch
    from paper_2607_04310_b300 import psdf, roofline
    from paper_2607_04310_b300 import scenegen as sg
    insts = sg.uneven_instances(2)
    plan = psdf.Plan([(w.footprint, w.edges, w.offsets, w.poses.shape[0]) for w in insts])
    poses = torch.as_tensor(np.concatenate([w.poses for w in insts]), device=dev).contiguous()
    P = plan.n_poses
    pairs = float(sum(w.poses.shape[0] * w.edges.shape[0] for w in insts))
    flops_instr = float(sum(w.poses.shape[0] *
                            roofline.flops_per_pose(w.footprint.shape[0], w.offsets)
                            for w in insts))
    flops = float(sum(roofline.flops_fixed(w.footprint.shape[0],
                                           float(w.poses.shape[0]) * w.edges.shape[0])
                      for w in insts))
    cfg, _ = psdf.psdf_plan_autotune(plan, poses, reps=3)
    phi = torch.empty(P, device=dev)
    dphi = torch.empty((P, 3), device=dev)
    act = torch.empty(P, dtype=torch.int32, device=dev)

    def step_plan():
        psdf.psdf_eval_batched(plan, poses, phi, dphi, act)

    # per-kernel device time of the eager launch
    for _ in range(3):
        step_plan()
    torch.cuda.synchronize()
    psdf.psdf_profile_reset()
    psdf.psdf_profile_enable(True)
    for _ in range(a.steps):
        flush.zero_()
        step_plan()
    torch.cuda.synchronize()
    psdf.psdf_profile_enable(False)
    n_k, k_ms = psdf.psdf_profile_read("batched")
    n_e, e_ms = psdf.psdf_profile_read("batched_epilogue")
    psdf.psdf_profile_reset()
    replay, g = _graph(step_plan)
    for _ in range(max(a.warmup, 3)):
        replay()
    ms = sum(_time_steps(replay, a.steps, flush, stream)) / a.steps
    ref = (phi.clone(), dphi.clone(), act.clone())

    # one psdf_eval_grad per instance
    scenes = [psdf.Scene.from_csr(w.edges, w.offsets) for w in insts]
    nmax = max(w.poses.shape[0] for w in insts)
    ws = psdf.workspace(nmax, dev)
    prm = psdf.make_params()
    offs = np.concatenate([[0], np.cumsum([w.poses.shape[0] for w in insts])])

    def step_each():
        for i, w in enumerate(insts):
            s0, s1 = int(offs[i]), int(offs[i + 1])
            psdf.psdf_eval_grad(w.footprint, scenes[i], poses[s0:s1], prm, phi[s0:s1],
                                dphi[s0:s1], act[s0:s1], ws)

    replay_each, g_each = _graph(step_each)
    for _ in range(3):
        replay_each()
    each_ms = sum(_time_steps(replay_each, a.steps, flush, stream)) / a.steps
    same = bool(torch.equal(ref[0].view(torch.int32), phi.view(torch.int32)) and
                torch.equal(ref[1].view(torch.int32), dphi.view(torch.int32)) and
                torch.equal(ref[2], act))
    kern_ms = k_ms / max(n_k, 1)
    achieved = flops / (kern_ms / 1000.0) / 1e12
    info = plan.info()
    return {
        "workload": "uneven instances: 1024 instances, horizons 10..100, 16..65536 edges "
                    "(log-uniform, random-yaw rectangles), 4..12-vertex footprints",
        "poses": int(P), "edges": int(plan.edges.shape[0]), "pair_evals": pairs,
        "value": pairs / (ms / 1000.0), "unit": "pair-evals/s", "ms_per_step": ms,
        "launch": "one CUDA graph: 2 memsets + persistent work-queue kernel + epilogue kernel",
        "gpu_launches_per_step": 2,
        "autotuned": {"threads": int(cfg.threads), "tiles_per_item": int(cfg.tiles_per_item),
                      "items": int(info.n_items), "grid": int(info.grid)},
        "per_instance_calls": {"ms_per_step": each_ms, "value": pairs / (each_ms / 1000.0),
                               "launches": 3 * len(insts)},
        "speedup_vs_per_instance_calls": each_ms / ms,
        "bitwise_equal_to_per_instance_calls": same,
        "kernels_ms_per_step": {"persistent": kern_ms, "epilogue": e_ms / max(n_e, 1)},
        "roofline": {"bound": "alu", "kernel": "batched persistent kernel",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "flops_per_step": flops,
                     "flop_model": "F(m) = 40 m + 26 per (pose, edge) pair",
                     "frac_instruction_count": flops_instr / (kern_ms / 1000.0) / 1e12 / peak},
    }


def _bench_scan_configs(dev, flush, stream, peak, steps: int = 20):
    """Full-scan throughput on the two other single-scene workloads: the
    octagon footprint over rectangles and LiDAR segments (3,200 poses x
    20,000 edges, value + gradient) and the backward workload (10,240 poses x
    10,000 edges, value + gradient + backward).  One CUDA graph per step, L2
    flushed before each; FP32 roofline of the step from the algorithmic flops
    of every (pose, edge) pair."""
    import torch
    from paper_2607_04310_b300 import psdf, roofline
    from paper_2607_04310_b300 import scenegen as sg
    out = {}
    for name, w, with_bwd in (("octagon_lidar", sg.octagon_lidar(1), False),
                              ("backward_rects", sg.backward_rects(3), True)):
        scene = psdf.Scene.from_csr(w.edges, w.offsets)
        prm = scene.params
        P = w.P
        poses = torch.as_tensor(w.poses, device=dev).contiguous()
        phi = torch.empty(P, device=dev)
        dphi = torch.empty((P, 3), device=dev)
        act = torch.empty(P, dtype=torch.int32, device=dev)
        ws = psdf.workspace(P, dev)
        gphi = torch.ones(P, device=dev)
        gpose = torch.empty((P, 3), device=dev)
        gedges = torch.zeros((w.E, 4), device=dev)

        def step():
            psdf.psdf_eval_grad(w.footprint, scene, poses, prm, phi, dphi, act, ws)
            if with_bwd:
                psdf.psdf_backward(w.footprint, scene, poses, prm, act, gphi, gpose, gedges)

        replay, _g = _graph(step)
        for _ in range(3):
            replay()
        ms = float(np.median(_time_steps(replay, steps, flush, stream)))
        m = w.footprint.shape[0]
        flops = roofline.flops_fixed(m, float(P) * w.E)
        flops_instr = roofline.flops_per_pose(m, w.offsets) * P
        pairs = float(P) * w.E
        out[name] = {"workload": w.name, "poses": P, "edges": w.E, "footprint_vertices": m,
                     "path": "full scan + pose gradient" + (" + backward" if with_bwd else ""),
                     "ms_per_step": ms, "value": pairs / (ms / 1000.0),
                     "unit": "pair-evals/s",
                     "roofline": {"bound": "alu", "achieved": flops / (ms / 1000.0) / 1e12,
                                  "peak": peak, "unit": "TFLOP/s",
                                  "frac": flops / (ms / 1000.0) / 1e12 / peak,
                                  "flops_per_step": flops,
                                  "flop_model": "F(m) = 40 m + 26 per (pose, edge) pair",
                                  "frac_instruction_count":
                                      flops_instr / (ms / 1000.0) / 1e12 / peak,
                                  "note": "whole step (scan, epilogue%s)"
                                          % (", backward" if with_bwd else "")}}
    return out


def _bench_table1(dev, reps: int = 200):
    """Latency grid of the paper's Table I: M in {1, 10, 100} random-yaw
    rectangles x B in {1, 10, 100} poses, rectangle footprint.  Three views:
    the autograd forward and backward as a PyTorch user calls them (host
    wall clock, synchronized, mean and std -- the paper's measurement; the
    backward includes PyTorch's autograd engine), the C ABI called directly
    (psdf_eval_grad, psdf_backward; median host wall clock, synchronized),
    and the device time of value + gradient + backward replayed as one CUDA
    graph."""
    import torch
    from paper_2607_04310_b300 import psdf
    from paper_2607_04310_b300 import scenegen as sg
    from paper_2607_04310_b300.autograd import PSDF
    g = np.random.default_rng(6)
    fp = sg.footprint_rect(0.6, 0.4)
    keys = ("autograd_forward_ms", "autograd_forward_std_ms", "autograd_backward_ms",
            "autograd_backward_std_ms", "cabi_forward_ms", "cabi_backward_ms", "graph_step_ms")
    res = {"M": [1, 10, 100], "B": [1, 10, 100]}
    for k in keys:
        res[k] = []
    for M in res["M"]:
        edges, offs = sg.rects(g, M, 0.2, 2.0, 0.0, 20.0)
        mod = PSDF(edges, offs, fp)
        prm = mod.scene.params
        rows = {k: [] for k in keys}
        for B in res["B"]:
            poses = torch.as_tensor(sg.poses_uniform(g, B, 0.0, 20.0), device=dev)
            pr = poses.clone().requires_grad_(True)
            for _ in range(10):
                mod(pr).sum().backward()
            torch.cuda.synchronize()
            tf, tb = [], []
            for _ in range(reps):
                t0 = time.perf_counter()
                phi = mod(pr)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                loss = phi.sum()
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                loss.backward()
                torch.cuda.synchronize()
                t3 = time.perf_counter()
                tf.append(1e3 * (t1 - t0))
                tb.append(1e3 * (t3 - t2))
            rows["autograd_forward_ms"].append(float(np.mean(tf)))
            rows["autograd_forward_std_ms"].append(float(np.std(tf)))
            rows["autograd_backward_ms"].append(float(np.mean(tb)))
            rows["autograd_backward_std_ms"].append(float(np.std(tb)))
            # the C ABI directly, preallocated buffers
            phi_o = torch.empty(B, device=dev)
            dphi_o = torch.empty((B, 3), device=dev)
            act_o = torch.empty(B, dtype=torch.int32, device=dev)
            gphi = torch.ones(B, device=dev)
            gpose = torch.empty((B, 3), device=dev)
            ws = psdf.workspace(B, dev)

            def fwd():
                psdf.psdf_eval_grad(fp, mod.scene, poses, prm, phi_o, dphi_o, act_o, ws)

            def bwd():
                psdf.psdf_backward(fp, mod.scene, poses, prm, act_o, gphi, gpose, None)

            for name, fn in (("cabi_forward_ms", fwd), ("cabi_backward_ms", bwd)):
                for _ in range(10):
                    fn()
                torch.cuda.synchronize()
                ts = []
                for _ in range(reps):
                    t0 = time.perf_counter()
                    fn()
                    torch.cuda.synchronize()
                    ts.append(1e3 * (time.perf_counter() - t0))
                rows[name].append(float(np.median(ts)))

            def step():
                fwd()
                bwd()

            replay, _g = _graph(step)
            for _ in range(5):
                replay()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                replay()
            e1.record()
            torch.cuda.synchronize()
            rows["graph_step_ms"].append(e0.elapsed_time(e1) / reps)
        for k in keys:
            res[k].append(rows[k])
    res["note"] = ("rows M, columns B; paper (RTX 4090, PyTorch autograd): forward 0.580-0.614 "
                   "ms, backward 2.021-2.238 ms (context, other hardware)")
    return res


def _fp32_peak(local: int):
    """The FP32 roofline's denominator measured on this GPU: the library's
    FMA microbenchmark (every SM full, 8 independent chains a thread), scalar
    and paired FFMA (the faster counts), with the SM clock sampled meanwhile."""
    from paper_2607_04310_b300 import psdf
    with ClockSampler(local) as clk:
        t_s, ms_s = psdf.psdf_measure_fp32_peak(False, iters=200000, reps=5)
        t_p, ms_p = psdf.psdf_measure_fp32_peak(True, iters=200000, reps=5)
    c = clk.summary()
    kind = "paired" if t_p >= t_s else "scalar"
    peak = max(t_s, t_p)
    return {"peak": peak, "unit": "TFLOP/s", "scalar_ffma": t_s, "paired_ffma": t_p,
            "clocks": c,
            "source": "measured: the library's FP32 FMA microbenchmark (%s FFMA, best of 5 "
                      "launches of about %.0f ms), median SM clock %s MHz"
                      % (kind, ms_p if kind == "paired" else ms_s, c.get("sm_mhz"))}


def run_b300(a, rank, world, local):
    import torch
    from paper_2607_04310_b300 import psdf, roofline
    from paper_2607_04310_b300 import train_cull

    if a.only_batched:
        torch.cuda.set_device(local)
        dev = torch.device("cuda", local)
        flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        peak = _fp32_peak(local)["peak"]
        print(json.dumps(_bench_batched(a, dev, flush, torch.cuda.current_stream(dev), peak)))
        return 0

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    fp32 = _fp32_peak(local)
    peak = fp32["peak"]
    w = _workload(rank)
    m = w.footprint.shape[0]
    scene = psdf.Scene.from_csr(w.edges, w.offsets)
    info = scene.info()
    T = int(info.n_tiles)
    W1, w2, b2, wmeta = train_cull.load_weights()
    mlp = psdf.Mlp(W1, w2, b2)
    prm = psdf.make_params()
    P = w.P
    poses = torch.as_tensor(w.poses, device=dev).contiguous()
    # phi, dphi and the active pair as views of one buffer, so that the
    # end-to-end leg reads the step's result back with one copy
    out = torch.empty(5 * P, device=dev)
    phi = out[:P]
    dphi = out[P:4 * P].view(P, 3)
    act = out[4 * P:].view(torch.int32)
    ws = psdf.workspace(P, dev)
    cws = torch.empty(psdf.psdf_cull_workspace_bytes(P, scene), dtype=torch.uint8, device=dev)
    gphi = torch.ones(P, device=dev)
    gpose = torch.empty((P, 3), device=dev)
    gedges = torch.zeros((w.E, 4), device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    learned = psdf.CullOpts(psdf.PROPOSE_MLP, CULL_K)
    bound = psdf.CullOpts(psdf.PROPOSE_BOUND, CULL_K)
    circles = psdf.CullOpts(psdf.PROPOSE_CIRCLES, CULL_K)

    # every library call launches on the current stream (None), so the same
    # step functions run eagerly or under CUDA-graph capture
    # every step saves its backward records in the forward (the active pair's
    # gradient rows, which the epilogue computes anyway) and scatters them
    saved = torch.empty((P, psdf.SAVED_FLOATS), dtype=torch.float32, device=dev)

    # the headline step's upper bound (HEADLINE_MODE); the bound-ordered and
    # the learned proposal are timed beside it on the same GPU
    head = {"circles": circles, "bound": bound, "mlp": learned}[HEADLINE_MODE]
    head_net = mlp if HEADLINE_MODE == "mlp" else None

    def step_head(ps=poses):
        psdf.psdf_eval_culled_save(w.footprint, scene, head_net, head, ps, prm, phi, dphi, act,
                                   saved, cws)
        psdf.psdf_backward_saved(scene, saved, gphi, gpose, gedges)

    def step_head_recompute():
        psdf.psdf_eval_culled(w.footprint, scene, head_net, head, poses, prm, phi, dphi, act,
                              cws)
        psdf.psdf_backward(w.footprint, scene, poses, prm, act, gphi, gpose, gedges)

    def step_learned():
        psdf.psdf_eval_culled_save(w.footprint, scene, mlp, learned, poses, prm, phi, dphi, act,
                                   saved, cws)
        psdf.psdf_backward_saved(scene, saved, gphi, gpose, gedges)

    def step_bound():
        psdf.psdf_eval_culled_save(w.footprint, scene, None, bound, poses, prm, phi, dphi, act,
                                   saved, cws)
        psdf.psdf_backward_saved(scene, saved, gphi, gpose, gedges)

    def step_full():
        psdf.psdf_eval_grad_save(w.footprint, scene, poses, prm, phi, dphi, act, saved, ws)
        psdf.psdf_backward_saved(scene, saved, gphi, gpose, gedges)

    # exactness in this run: both culls vs the full scan, every output bit
    step_full()
    ref = (phi.clone(), dphi.clone(), act.clone(), gpose.clone())

    def same_as_full():
        torch.cuda.synchronize()
        return bool(torch.equal(ref[0].view(torch.int32), phi.view(torch.int32)) and
                    torch.equal(ref[1].view(torch.int32), dphi.view(torch.int32)) and
                    torch.equal(ref[2], act) and
                    torch.equal(ref[3].view(torch.int32), gpose.view(torch.int32)))

    step_learned()
    exact_learned = same_as_full()
    step_bound()
    exact_bound = same_as_full()
    step_head()
    exact = same_as_full() and exact_learned and exact_bound
    for _ in range(max(a.warmup, 3)):
        step_head()
    torch.cuda.synchronize()
    # per-kernel device time of the eager step (CUDA events around each of the
    # library's launches, on its stream): the roofline of the dominant kernel
    psdf.psdf_profile_reset()
    psdf.psdf_profile_enable(True)
    for _ in range(a.steps):
        flush.zero_()
        step_head()
    torch.cuda.synchronize()
    psdf.psdf_profile_enable(False)
    prof = {k: psdf.psdf_profile_read(k) for k in ("cull", "backward")}
    psdf.psdf_profile_reset()
    st = psdf.psdf_cull_stats_read(cws, stream)

    # ---- headline: the cull step as one CUDA-graph launch ---------------------
    replay_head, g_head = _graph(step_head)
    for _ in range(max(a.warmup, 3)):
        replay_head()
    if pg:
        pg.barrier()
    with ClockSampler(local) as clk:
        ms = _time_steps(replay_head, a.steps, flush, stream)
    if pg:
        pg.barrier()
    ms_step = sum(ms) / len(ms)

    # ---- comparison paths on the same GPU, also graph-launched -----------------
    replay_full, g_full = _graph(step_full)
    for _ in range(3):
        replay_full()
    full_ms = sum(_time_steps(replay_full, a.steps, flush, stream)) / a.steps
    replay_learned, g_learned = _graph(step_learned)
    for _ in range(3):
        replay_learned()
    learned_ms = sum(_time_steps(replay_learned, a.steps, flush, stream)) / a.steps
    st_learned = psdf.psdf_cull_stats_read(cws, stream)
    replay_bound, g_bound = _graph(step_bound)
    for _ in range(3):
        replay_bound()
    bound_ms = sum(_time_steps(replay_bound, a.steps, flush, stream)) / a.steps
    st_bound = psdf.psdf_cull_stats_read(cws, stream)
    replay_rec, g_rec = _graph(step_head_recompute)
    for _ in range(3):
        replay_rec()
    recompute_ms = sum(_time_steps(replay_rec, a.steps, flush, stream)) / a.steps
    eager_ms = sum(_time_steps(step_head, a.steps, flush, stream)) / a.steps

    # ---- end to end through the C ABI with host buffers ----------------------
    e2e_step_ms = e2e_copy_ms = float("nan")
    e2e_exact = None
    if not a.no_e2e:
        h_poses = torch.as_tensor(w.poses).pin_memory()
        h_out = torch.empty(5 * P).pin_memory()
        d_poses = torch.empty_like(poses)
        side = torch.cuda.Stream(dev)

        def e2e_step():
            # poses in, the cull step, the result (phi, dphi, active) read
            # back on a side stream while the backward runs
            d_poses.copy_(h_poses, non_blocking=True)
            psdf.psdf_eval_culled_save(w.footprint, scene, head_net, head, d_poses, prm, phi, dphi,
                                       act, saved, cws)
            fwd_done = torch.cuda.Event()
            fwd_done.record()
            side.wait_event(fwd_done)
            with torch.cuda.stream(side):
                h_out.copy_(out, non_blocking=True)
            psdf.psdf_backward_saved(scene, saved, gphi, gpose, gedges)
            torch.cuda.current_stream().wait_stream(side)

        replay_e2e, g_e2e = _graph(e2e_step)
        for _ in range(3):
            replay_e2e()
        e2e_copy_ms = sum(_time_steps(replay_e2e, a.steps, flush, stream)) / a.steps

        # zero-copy: the kernels read the pinned, device-mapped host poses and
        # write phi / dphi / active into pinned host memory themselves (the
        # backward needs neither: it reads the saved rows)
        h_phi = h_out[:P]
        h_dphi = h_out[P:4 * P].view(P, 3)
        h_act = h_out[4 * P:].view(torch.int32)

        def e2e_zero_copy_step():
            psdf.psdf_eval_culled_save(w.footprint, scene, head_net, head, h_poses, prm, h_phi,
                                       h_dphi, h_act, saved, cws)
            psdf.psdf_backward_saved(scene, saved, gphi, gpose, gedges)

        replay_zc, g_zc = _graph(e2e_zero_copy_step)
        for _ in range(3):
            replay_zc()
        e2e_step_ms = sum(_time_steps(replay_zc, a.steps, flush, stream)) / a.steps
        torch.cuda.synchronize()
        e2e_exact = bool(np.array_equal(h_out.numpy().view(np.int32),
                                        out.cpu().numpy().view(np.int32)))

    # ---- aggregate over ranks ----------------------------------------------
    pairs = float(P) * w.E
    t_max = ms_step
    if pg:
        t = torch.tensor([ms_step, e2e_step_ms, full_ms, e2e_copy_ms], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        t_max, e2e_step_ms, full_ms = float(t[0]), float(t[1]), float(t[2])
        e2e_copy_ms = float(t[3])
    value = world * pairs / (t_max / 1000.0)
    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return 0

    # ---- roofline of the step's dominant kernel (the fused cull) ----------
    peaks = _measured_peaks()
    evaluated_pairs = float(st.evaluated_edges)  # pose x edge pairs evaluated exactly
    items = int(st.proposed_items + st.fallback_items)
    n_k, k_ms = prof["cull"]
    cull_ms = k_ms / max(n_k, 1)
    # FP32 work: the evaluated pairs by the fixed per-pair count, plus the
    # tile bounds and obstacle circles of the proposals
    f_fixed = roofline.flops_fixed(m, evaluated_pairs) + roofline.flops_propose(
        st.bound_evaluations, st.circle_evaluations)
    f_instr = roofline.flops_evaluated(m, st.evaluated_edges, st.evaluated_obstacles) + \
        roofline.flops_propose(st.bound_evaluations, st.circle_evaluations)
    # the network's tensor-core flops, when the headline step runs it
    f_net = roofline.flops_network(8 * P) if HEADLINE_MODE == "mlp" else 0.0
    ach = f_fixed / (cull_ms / 1000.0) / 1e12
    ach_instr = f_instr / (cull_ms / 1000.0) / 1e12
    bf16 = float(peaks.get("bf16_tflops", 0.0)) or None
    net_ach = f_net / (cull_ms / 1000.0) / 1e12
    launches_per_step = 2  # cull_kernel, backward_saved_kernel
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "impl": "b300",
        "config": {"workload": WORKLOAD, "poses_per_gpu": P, "edges": w.E,
                   "obstacles": w.M, "tiles": T, "footprint_vertices": m,
                   "path": ("%s + pose gradient + backward (from the forward's saved "
                            "rows); %s" % (
                                {"circles": "exact cull by the scene's candidate grid (each "
                                            "cell's 32 nearest obstacle circles and a "
                                            "completeness radius: a pose whose upper bound "
                                            "lies within it evaluates only those candidates, "
                                            "any other the tiles of its cull-grid cell)",
                                 "bound": "bound-ordered tile cull (k=%d)" % CULL_K,
                                 "mlp": "learned tile cull (k=%d)" % CULL_K}[HEADLINE_MODE],
                                "the bound-ordered cull (bound_cull) and the learned proposal "
                                "(learned_cull) are timed beside it; the network costs more "
                                "than it saves on these sort-tile-recursive tiles")),
                   "pair_count": "effective: poses x edges of the whole scene",
                   "l2": "flushed between timed steps (256 MiB write)"},
        "speedup_vs_full_scan": full_ms / ms_step,
        "launch": "one CUDA graph per step (eager launches: %.4f ms/step)" % eager_ms,
        "exact_vs_full_scan": exact,
        "full_scan": {"value": pairs / (full_ms / 1000.0), "ms_per_step": full_ms,
                      "roofline_frac": roofline.flops_fixed(m, float(P) * w.E)
                      / (full_ms / 1000.0) / 1e12 / fp32["peak"],
                      "roofline_frac_instruction_count": roofline.flops_per_pose(m, w.offsets) * P
                      / (full_ms / 1000.0) / 1e12 / fp32["peak"],
                      "note": "scan + epilogue + backward; FP32 flops of every pair (fixed "
                              "count F(m) = 40 m + 26; instruction-level count beside it)"},
        "backward_recompute": {"value": pairs / (recompute_ms / 1000.0),
                               "ms_per_step": recompute_ms,
                               "note": "the same step through psdf_eval_culled + psdf_backward "
                                       "(the backward recomputes the active pair's geometry "
                                       "instead of reading the forward's saved rows)"},
        "bound_cull": {"value": pairs / (bound_ms / 1000.0), "ms_per_step": bound_ms,
                       "exact_vs_full_scan": exact_bound,
                       "evaluated_obstacles": int(st_bound.evaluated_obstacles),
                       "listed_pairs": int(st_bound.proposed_items + st_bound.fallback_items),
                       "fallback_rate": st_bound.fallback_poses / P,
                       "note": "upper bound from the circles of each pose's tile of smallest "
                               "AABB bound (k = %d)" % CULL_K},
        "learned_cull": {"value": pairs / (learned_ms / 1000.0), "ms_per_step": learned_ms,
                         "exact_vs_full_scan": exact_learned,
                         "evaluated_fraction": (st_learned.proposed_items
                                                + st_learned.fallback_items) / (P * T),
                         "fallback_rate": st_learned.fallback_poses / P,
                         "evaluated_obstacles": int(st_learned.evaluated_obstacles),
                         "listed_pairs": int(st_learned.proposed_items
                                             + st_learned.fallback_items),
                         "network_heldout_top1": wmeta.get("heldout", {}).get("top1_mlp"),
                         "network_flops_per_step": roofline.flops_network(8 * P),
                         "gain_vs_bound": {
                             "ms_per_step": learned_ms - bound_ms,
                             "listed_pairs": int(st_learned.proposed_items
                                                 + st_learned.fallback_items)
                             - int(st_bound.proposed_items + st_bound.fallback_items),
                             "evaluated_obstacles": int(st_learned.evaluated_obstacles)
                             - int(st_bound.evaluated_obstacles),
                             "note": "positive = the learned proposal costs more than the "
                                     "bound order"}},
        "cull": {"candidates_per_pose": st.circle_evaluations / P
                 if HEADLINE_MODE == "circles" else None,
                 "tile_path_poses": int(st.fallback_poses) if HEADLINE_MODE == "circles"
                 else None,
                 "candidate_fraction": st.proposed_items / (P * T),
                 "evaluated_fraction": items / (P * T),
                 "evaluated_obstacles": int(st.evaluated_obstacles),
                 "evaluated_edges": int(st.evaluated_edges),
                 "fallback_rate": st.fallback_poses / P,
                 "proposed_pairs": int(st.proposed_items),
                 "fallback_pairs": int(st.fallback_items),
                 "bound_evaluations": int(st.bound_evaluations),
                 "circle_evaluations": int(st.circle_evaluations),
                 "evaluated_pair_evals_per_s": evaluated_pairs / (ms_step / 1000.0)},
        "roofline": {"bound": "alu", "kernel": "cull_kernel",
                     "achieved": ach, "peak": fp32["peak"], "unit": "TFLOP/s",
                     "frac": ach / fp32["peak"],
                     "note": "latency-bound: a few thousand dependent chains of loads per step",
                     "flop_model": "F(m) = 40 m + 26 per evaluated (pose, edge) pair, plus 7 "
                                   "per tile bound and 10 per obstacle circle",
                     "flops_per_step": f_fixed,
                     "instruction_count": {"flops_per_step": f_instr, "achieved": ach_instr,
                                           "frac": ach_instr / fp32["peak"],
                                           "model": "14 + 30 m per edge + 2 m per obstacle"},
                     "network_tensor": ({"flops_per_step": f_net, "achieved": net_ach,
                                         "peak": bf16, "frac": net_ach / bf16 if bf16 else None,
                                         "note": "FP16 mma.sync 16x64x1 over 8 candidates per "
                                                 "pose, against the measured dense bf16 rate "
                                                 "(FP16 dense has the same nominal rate)"}
                                        if HEADLINE_MODE == "mlp" else None),
                     "peak_source": fp32["source"],
                     "avg_launch_ms": cull_ms,
                     "traffic": _traffic("cull_kernel", WORKLOAD)},
        "kernels_ms_per_step": {k: v[1] / a.steps for k, v in prof.items()},
        "fp32_peak": fp32,
        "e2e": {"value": world * pairs / (e2e_step_ms / 1000.0), "unit": UNIT,
                "h2d_bytes_per_step": 12 * P, "d2h_bytes_per_step": (4 + 12 + 4) * P,
                "ms_per_step": e2e_step_ms,
                "note": "zero-copy, one CUDA graph: the cull kernel reads the poses from "
                        "pinned, device-mapped host memory (12 B per pose) and writes phi / "
                        "dphi / active into pinned host memory; no copy calls",
                "equal_to_device_outputs": e2e_exact,
                "copies": {"value": world * pairs / (e2e_copy_ms / 1000.0),
                           "ms_per_step": e2e_copy_ms, "h2d_bytes_per_step": 12 * P,
                           "d2h_bytes_per_step": (4 + 12 + 4) * P,
                           "note": "copy-engine leg: poses copied in, phi / dphi / active "
                                   "copied out on a side stream while the backward runs"}},
        "gpu_launches": launches_per_step * a.steps,
        "clocks": clk.summary(),
    }
    if not a.no_batched and world == 1:
        line["batched_uneven"] = _bench_batched(a, dev, flush, stream, peak)
        line["table1_latency"] = _bench_table1(dev)
        line["full_scan_configs"] = _bench_scan_configs(dev, flush, stream, peak)
    if not a.no_cpu_baseline and world == 1:
        import oracle
        rate, n, dt = _oracle_rate(w, a.cpu_seconds)
        rate1, n1, dt1 = _oracle_rate(w, min(4.0, a.cpu_seconds / 3), seed=1, nthreads=1)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": oracle.max_threads(),
                                "kind": "oracle",
                                "sample": "%d of 4096 poses x 100000 edges, %.1f s" % (n, dt),
                                "one_core": {"value": rate1, "cores": 1,
                                             "sample": "%d poses, %.1f s" % (n1, dt1)}}
    print(json.dumps(line))
    if pg:
        pg.destroy_process_group()
    return 0


def main():
    a = _args()
    rank, world, local = _dist()
    if a.impl == "reference":
        return run_reference(a, rank, world)
    return run_b300(a, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
