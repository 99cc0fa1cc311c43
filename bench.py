"""Benchmark of the whole-body evaluation (forward + backward) on GB300.

A step is one forward evaluation (FK, sphere placement, self-collision
map-reduce, RNEA) plus one backward pass (the VJP of all four with upstream
gradients on poses, spheres, d_min and torques) over one batch of synthetic
configurations of the 48-DoF humanoid-shaped tree (1024 seeds x 32 timesteps
= 32768 configurations).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--kernel tree|fused|plain] [--batch B] [--skip-cpu] [--skip-plain]
                  [--skip-uneven]
                  [--workload humanoid48|arm7|trajopt48|uneven|kinematics]
                  [--collision worst|hinge] [--sweep-shape FS,FC,BS,BC]
                  [--ref-total-s T] [--ref-step-s S] [--split]

--impl reference times the FP64 CPU oracle on the host cores instead, in
bounded samples that keep the whole run within about --ref-total-s seconds.
--sweep-shape pins the sweeps' launch shapes (segments and threads per block
of the forward and the backward) instead of autotuning, for profiler runs.
Under torchrun (N > 1) the humanoid48 workload is one seeded global batch
partitioned into contiguous column ranges, one per rank: N x --batch
configurations (weak scaling, the default) or --batch split over the ranks
(--split, strong scaling).  The step time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synthetic import configs as CF  # noqa: E402
from synthetic import inputs as I  # noqa: E402
from synthetic import robots as R  # noqa: E402

METRIC = "whole-body evals/s (FK+self-coll+RNEA, fwd+bwd) at 48 DoF"
L2_FLUSH_BYTES = 512 << 20


# ---------------------------------------------------------------------------
# algorithmic work per evaluation (flops; FMA = 2) and bytes
# ---------------------------------------------------------------------------
def work_per_eval(desc):
    """Algorithmic flops (FMA = 2) and HBM bytes per evaluation for each kernel
    of the step: the forward tree sweep (FK + RNEA), the sphere/pair kernel
    and the backward tree sweep."""
    n = desc.n
    nm = int((desc.jtype != R.FIXED).sum())
    S, P, d = desc.S, desc.P, desc.dof
    return {
        "tree_fwd": {"flops": 150 * nm + 330 * n, "bytes": 4 * (3 * d + 12 * n + d)},
        "pair": {"flops": 18 * S + 11 * P, "bytes": 4 * (12 * n + 3 * S + 2)},
        "tree_bwd": {"flops": 150 * nm + 330 * n + 660 * n + 60 * n + 15 * S,
                     "bytes": 4 * (3 * d + 12 * n + 3 * S + 2 + d + 3 * d)},
    }


# DRAM bytes (read + write) per evaluation from one ncu capture of each
# kernel at the bench's launch configuration (humanoid48 and trajopt48, both
# on their 32768 configurations), tied to the kernel launched and to the
# hash of the sources it is built from, including the host code that picks
# its launch shape (wbe_api.cu): a changed source, another launch-shape
# default or another kernel makes the figure stale, and it is reported as
# null until captured again.
API_SRC = ["paper_2603_05493_gb300/csrc/wbe_api.cu"]
TREE_SRC = ["paper_2603_05493_gb300/csrc/k_tree.cu", "paper_2603_05493_gb300/csrc/tree_sweep.cuh",
            "paper_2603_05493_gb300/csrc/spatial.cuh",
            "paper_2603_05493_gb300/csrc/spline_basis.cuh"] + API_SRC
PAIR_SRC = ["paper_2603_05493_gb300/csrc/k_pair.cu", "paper_2603_05493_gb300/csrc/pair_body.cuh",
            "paper_2603_05493_gb300/csrc/spatial.cuh"] + API_SRC
SPLINE_SRC = ["paper_2603_05493_gb300/csrc/k_traj.cu",
              "paper_2603_05493_gb300/csrc/spline_basis.cuh"] + API_SRC
TREE_SHA = "07a09d1949da5479c370f929d6354a1a1d6eb27af843fdf8497217fff37dee14"
PAIR_SHA = "400b679eaab398c46eb74122c4f202b9724b238f380a50da02b7c1e8b9f19d8f"
SPLINE_SHA = "610be5112e547b9a8bcf82c0f8d7e914f09a59ad580bfa1685a3d0b32a3c09f4"
MEASURED_TRAFFIC = {  # kernel[@workload]: (sources, their hash, bytes / evaluation)
    "tree_fwd_seg_kernel": (TREE_SRC, TREE_SHA, (23.94e6 + 50.73e6) / 32768),
    "pair_kernel": (PAIR_SRC, PAIR_SHA, (77.29e6 + 32.66e6) / 32768),
    "tree_bwd_seg_kernel": (TREE_SRC, TREE_SHA, (239.01e6 + 37.11e6) / 32768),
    "tree_fwd_spline_seg_kernel": (TREE_SRC, TREE_SHA, (5.66e6 + 52.47e6) / 32768),
    "pair_kernel@trajopt48": (PAIR_SRC, PAIR_SHA, (77.26e6 + 0.70e6) / 32768),
    "tree_bwd_spline_cost_seg_kernel": (TREE_SRC, TREE_SHA, (8.72e6 + 2.22e6) / 32768),
    "bspline_bwd_kernel": (SPLINE_SRC, SPLINE_SHA, (18.89e6 + 0.00e6) / 32768),
}


def source_hash(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def traffic_per_eval(kernel, workload=""):
    """Measured DRAM bytes per evaluation of this kernel (in this workload,
    where it has its own figure), or None when stale or never captured."""
    t = MEASURED_TRAFFIC.get("%s@%s" % (kernel, workload)) or MEASURED_TRAFFIC.get(kernel)
    if not t or source_hash(t[0]) != t[1]:
        return None
    return t[2]


def sweep_shapes(rob, B, args, spline=None):
    """Forward and backward sweep launch shapes: the library's autotuner at
    batch B (the control-point path's own autotuner when spline = (n_traj, K,
    T, dt) is given, timed with the trajectory cost's weights), or the ones
    --sweep-shape pins (segments and configurations per block of each sweep),
    so that a profiler run, whose slowed launches would sway the autotuner,
    times the same launches as the plain run."""
    from paper_2603_05493_gb300 import wbe
    if not args.sweep_shape:
        if spline is not None:
            ft, bt, _, _ = rob.autotune_spline(*spline, w_coll=CF.COLLISION_WEIGHT,
                                               smooth=CF.SMOOTH_WEIGHT,
                                               length=CF.LENGTH_WEIGHT,
                                               energy=CF.ENERGY_WEIGHT,
                                               dt_cost=spline[3] * (spline[1] - 3) / (spline[2] - 1))
        else:
            ft, bt, _, _ = rob.autotune(B)
        return ft, bt
    fs, fc, bs, bc = (int(x) for x in args.sweep_shape.split(","))
    mk = lambda g, c: wbe.Tune(kernel=wbe.L.WB_KERNEL_TREE, lanes_per_config=g,  # noqa: E731
                               configs_per_block=c)
    return mk(fs, fc), mk(bs, bc)


# ---------------------------------------------------------------------------
# the humanoid48 step: its launch shapes and its launches (the GPU parity
# tests run the same two functions at the full batch)
# ---------------------------------------------------------------------------
def humanoid48_launch(rob, B, kernel="tree", sweep_shape=""):
    """Launch choices of the humanoid48 step at batch B: for the tree kernels
    the sweep shapes (segments, threads per block) and the pair stage's warps
    per block from the library's autotuner at this batch size (or the sweep
    shapes --sweep-shape pins); for fused / plain one kernel family.  Returns
    {"fwd", "pair", "bwd": Tune, "names": kernel names, "chosen": the
    autotuner's picks or None}."""
    from paper_2603_05493_gb300 import wbe
    if kernel != "tree":
        t = {"plain": wbe.PLAIN, "fused": wbe.FUSED}[kernel]
        pre = "fused" if kernel == "fused" else "plain"
        return {"fwd": t, "pair": None, "bwd": t, "chosen": None,
                "names": {"tree_fwd": pre + "_fwd_kernel", "pair": "-",
                          "tree_bwd": pre + "_bwd_kernel"}}

    class _Pin:  # the argparse namespace sweep_shapes reads
        pass
    pin = _Pin()
    pin.sweep_shape = sweep_shape
    ft, bt = sweep_shapes(rob, B, pin)
    is_tree = lambda t: t.kernel == wbe.L.WB_KERNEL_TREE  # noqa: E731
    seg = lambda t: t.lanes_per_config if is_tree(t) else 0  # noqa: E731
    tpb = lambda t: t.configs_per_block if is_tree(t) else 0  # noqa: E731
    fwd = wbe.Tune(kernel=wbe.L.WB_KERNEL_TREE, lanes_per_config=seg(ft),
                   configs_per_block=tpb(ft))
    bwd = wbe.Tune(kernel=wbe.L.WB_KERNEL_TREE, lanes_per_config=seg(bt),
                   configs_per_block=tpb(bt))
    # the pair stage's warps per block as the autotuner timed them with the
    # forward (0 when pinned: the library's default)
    pair = wbe.Tune(kernel=wbe.L.WB_KERNEL_TREE, blocks_per_sm=ft.blocks_per_sm if is_tree(ft) else 0)
    return {"fwd": fwd, "pair": pair, "bwd": bwd,
            "chosen": {"fwd": dict(ft.__dict__), "bwd": dict(bt.__dict__)},
            "names": {"tree_fwd": "tree_fwd_seg_kernel" if seg(ft) > 1 else "tree_fwd_kernel",
                      "pair": "pair_kernel",
                      "tree_bwd": "tree_bwd_seg_kernel" if seg(bt) > 1 else "tree_bwd_kernel"}}


def humanoid48_step(rob, shapes, states, grads, out, gout, events=None, stream=None):
    """One humanoid48 step with the launch choices of humanoid48_launch:
    forward (FK + RNEA sweep, then spheres + self-collision; one launch for
    fused / plain) and backward with the upstream gradients grads = (g_pose,
    g_sphere, g_dmin, g_tau).  out: rob.empty_outputs(B), with a "diff" (B, 3)
    buffer for the worst pair's centre difference; gout: (gq, gqd, gqdd).  events[1], events[2] are recorded after the forward sweep and
    after the pair stage."""
    tq, tqd, tqdd = states
    tgp, tgs, tgm, tgt = grads
    if shapes["pair"] is None:  # one forward launch
        rob.eval(tq, tqd, tqdd, tune=shapes["fwd"], out=out, stream=stream)
        if events:
            events[1].record(stream)
            events[2].record(stream)
    else:
        rob.eval(tq, tqd, tqdd, tune=shapes["fwd"], dmin=False, sphere=False, stream=stream,
                 out={"pose": out["pose"], "sphere": None, "dmin": None, "worst": None,
                      "tau": out["tau"], "bits": None})
        if events:
            events[1].record(stream)
        rob.self_collision(out["pose"], tune=shapes["pair"], stream=stream,
                           out={"sphere": out["sphere"], "dmin": out["dmin"],
                                "worst": out["worst"], "diff": out.get("diff"), "bits": None})
        if events:
            events[2].record(stream)
    # the pair stage's worst-pair centre difference spares the backward the
    # forward kinematics of the pair's two links
    rob.eval_backward(tq, tqd, tqdd, out["worst"], tgp, tgs, tgm, tgt, tune=shapes["bwd"],
                      out=gout, stream=stream,
                      worst_diff=out.get("diff") if shapes["pair"] is not None else None)


# ---------------------------------------------------------------------------
# multi-rank host logic: one process per GPU, each evaluating its own batch
# (weak scaling); no collective touches the data path, only the timing
# ---------------------------------------------------------------------------
def rank_seed(base, rank):
    """Each rank draws its own inputs (the trajopt48, kinematics and uneven
    workloads)."""
    return base + 101 * rank


def rank_columns(world, rank, B, split=False):
    """The columns of one global batch that rank `rank` of `world` evaluates,
    a contiguous partition: weak scaling (default) makes the global batch
    world x B and gives rank r columns [r B, (r + 1) B); split keeps the
    global batch at B and gives rank r columns [r B / world, (r + 1) B /
    world).  Returns (lo, hi, global batch size)."""
    total = B if split else world * B
    return rank * total // world, (rank + 1) * total // world, total


def humanoid48_inputs(desc, lo, hi):
    """Columns [lo, hi) of the humanoid48 workload's one seeded batch:
    (q, qd, qdd, g_pose, g_sphere, g_dmin, g_tau)."""
    return I.batch_columns(desc, lo, hi, CF.HUMANOID48.seed)


def reduce_max(values, world, device):
    """Element-wise maximum over ranks (the slowest rank sets the time)."""
    if world <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_value(world, units_per_rank, ms):
    """Whole-job throughput: the units every rank processed / the slowest
    rank's time."""
    return world * units_per_rank / (ms * 1e-3)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def fp32_peak_tflops(num_sms, mhz):
    """FP32 FMA peak: SMs x 128 lanes x 2 flops x clock."""
    return num_sms * 128 * 2 * mhz * 1e6 / 1e12


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and --impl reference)
# ---------------------------------------------------------------------------
FD_PASS = ("forward + central-difference gradient (2*3d+1 forward evaluations per "
           "configuration: the oracle has no reverse mode; its dual-number gradient is for "
           "correctness only and is not timed)")


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or the machine type."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


class OracleTimer:
    """The FP64 oracle (g++ -O3, plain double, OpenMP over configurations) on
    the humanoid48 workload, timed on the host cores: the forward evaluation
    (FK, spheres, brute-force pairs, RNEA), and forward + backward as the
    forward plus a central-difference gradient of the same upstream loss as
    the GPU step."""

    def __init__(self, desc, seed=CF.HUMANOID48.seed):
        from oracle import oracle as O
        self.O = O
        self.desc = desc
        self.orob = O.OracleRobot(desc)
        self.seed = seed
        self.threads = O.max_threads()
        self._inputs = {}

    def inputs(self, n):
        if n not in self._inputs:
            q, qd, qdd = I.uniform_states(self.desc.dof, n, self.seed + 7)
            self._inputs = {n: (q, qd, qdd) + tuple(I.upstream_grads(self.desc, n,
                                                                      self.seed + 8))}
        return self._inputs[n]

    def run(self, n, threads, backward):
        """Wall seconds of one pass over n configurations."""
        q, qd, qdd, gp, gs, gm, gt = self.inputs(n)
        t0 = time.perf_counter()
        self.O.evaluate(self.orob, q, qd, qdd, nthreads=threads)
        if backward:
            self.O.gradient_fd(self.orob, q, qd, qdd, gp, gs, gm, gt, nthreads=threads)
        return time.perf_counter() - t0

    def size_for(self, target_s, threads, backward, cap):
        """Configurations that take about target_s (calibrated on a small run)."""
        n0 = max(threads, 4) if backward else max(16 * threads, 64)
        per = self.run(n0, threads, backward) / n0
        return int(max(n0, min(cap, target_s / max(per, 1e-9))))

    def rate(self, target_s, threads, backward, cap=200000):
        n = self.size_for(target_s, threads, backward, cap)
        dt = self.run(n, threads, backward)
        return n / dt, n, dt


def time_oracle(desc, target_s=15.0):
    """cpu_baseline: the oracle's forward + backward (forward + central
    differences) on all host cores over a sample sized to take about half of
    target_s, with the single-thread figure and the forward-only rates (all
    cores, and one thread on at most a 4096-configuration subset) beside it."""
    t = OracleTimer(desc)
    fb_n, n_fb, s_fb = t.rate(0.5 * target_s, t.threads, True)
    fb_1, n_fb1, s_fb1 = t.rate(0.2 * target_s, 1, True)
    f_n, n_f, s_f = t.rate(0.1 * target_s, t.threads, False)
    f_1, n_f1, s_f1 = t.rate(0.2 * target_s, 1, False, cap=4096)
    return {"value": fb_n, "unit": "evals/s", "cores": t.threads, "kind": "oracle",
            "pass": FD_PASS,
            "sample": "%d configurations of the %s workload on %d threads in %.1f s "
                      "(1 thread: %d in %.1f s)" % (n_fb, desc.name, t.threads, s_fb, n_fb1,
                                                     s_fb1),
            "threads_1": fb_1,
            "forward": {"threads_N": f_n, "threads_1": f_1, "unit": "evals/s",
                        "sample": "%d configurations on %d threads in %.2f s; %d on 1 thread "
                                  "in %.2f s" % (n_f, t.threads, s_f, n_f1, s_f1)},
            "nproc": os.cpu_count(), "cpu_model": cpu_model(),
            "build": "g++ -O3 -fopenmp, plain double"}


def reference_step_targets(steps, warmup, total_s, step_cap_s):
    """Seconds of oracle work for each warm-up and each timed step of the
    reference arm: the whole run stays within about total_s whatever the
    step counts (a timed step takes at most step_cap_s and at least 0.1 s;
    the warm-up gets a tenth of the budget)."""
    warm = min(2.0, max(0.05, 0.1 * total_s / max(1, warmup)))
    step = min(step_cap_s, max(0.1, 0.9 * total_s / max(1, steps)))
    return warm, step


HUMANOID48_WORKLOAD = ("humanoid48: 48-DoF tree, 200 spheres, 15392 pairs, 1024 x 32 "
                       "configurations, fwd + bwd (upstream grads on poses, spheres, d_min, tau)")


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle's forward + backward (forward +
    central differences) on all host cores.  Every timed step evaluates the
    same bounded sample of the humanoid48 workload, sized in the warm-up so
    that the run keeps to about --ref-total-s; ms_per_step is the measured
    wall time of a step."""
    if rank != 0:
        return
    desc = R.r48()
    t = OracleTimer(desc)
    warm_s, step_s = reference_step_targets(args.steps, args.warmup, args.ref_total_s,
                                            args.ref_step_s)
    n = t.size_for(step_s, t.threads, True, cap=CF.HUMANOID48.batch)
    for _ in range(args.warmup):
        t.run(max(t.threads, int(n * warm_s / step_s)), t.threads, True)
    secs = [t.run(n, t.threads, True) for _ in range(args.steps)]
    mean_s = float(np.mean(secs))
    value = n / mean_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * mean_s, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": HUMANOID48_WORKLOAD, "batch": CF.HUMANOID48.batch,
                   "sample_configs_per_step": n,
                   "step": "each timed step evaluates the same %d-configuration sample of "
                           "the batch (forward + backward); value = sample / measured step "
                           "time" % n},
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": t.threads, "kind": "oracle",
                         "pass": FD_PASS,
                         "sample": "%d configurations per step, %d timed steps of %.2f s "
                                   "mean" % (n, args.steps, mean_s),
                         "nproc": os.cpu_count(), "cpu_model": cpu_model(),
                         "build": "g++ -O3 -fopenmp, plain double"},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the GPU benchmark
# ---------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2603_05493_gb300 import build
    build()
    from paper_2603_05493_gb300 import wbe

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    desc = R.r48()
    B = args.batch or CF.HUMANOID48.batch
    rob = wbe.Robot(desc, device=local_rank)
    # this rank's contiguous slice of the one seeded global batch
    lo, hi, total = rank_columns(world, rank, B, args.split)
    B = hi - lo
    shapes = humanoid48_launch(rob, B, args.kernel, args.sweep_shape)
    tune, btune = shapes["fwd"], shapes["bwd"]
    names, chosen = shapes["names"], shapes["chosen"]
    q, qd, qdd, gp, gs, gm, gt = humanoid48_inputs(desc, lo, hi)
    h_in = [torch.from_numpy(x).pin_memory() for x in (q, qd, qdd, gp, gs, gm, gt)]
    d_in = [x.to(dev) for x in h_in]
    tq, tqd, tqdd, tgp, tgs, tgm, tgt = d_in
    out = rob.empty_outputs(B)
    out["diff"] = torch.empty((B, 3), device=dev)
    gout = tuple(torch.empty((desc.dof, B), device=dev) for _ in range(3))
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)
    stream = torch.cuda.current_stream()

    def step(events=None):
        humanoid48_step(rob, shapes, (tq, tqd, tqdd), (tgp, tgs, tgm, tgt), out, gout,
                        events=events, stream=stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select the timed steps
    for i in range(args.steps):
        flush.fill_(float(i))  # evict L2 between timed steps (outside the events)
        ev[i][0].record(stream)
        step(ev[i])
        ev[i][3].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    k_ms = {"tree_fwd": [e[0].elapsed_time(e[1]) for e in ev],
            "pair": [e[1].elapsed_time(e[2]) for e in ev],
            "tree_bwd": [e[2].elapsed_time(e[3]) for e in ev]}
    step_ms = float(np.mean([e[0].elapsed_time(e[3]) for e in ev]))
    fwd_ms = [a + b for a, b in zip(k_ms["tree_fwd"], k_ms["pair"])]
    bwd_ms = k_ms["tree_bwd"]

    # the pair stage's full map-reduce (every block screened, no culling) on
    # the same poses, for comparison with the default culled kernel
    brute_ms = None
    if args.kernel == "tree":
        bout = {"sphere": None, "dmin": torch.empty_like(out["dmin"]),
                "worst": torch.empty_like(out["worst"]), "bits": None}
        tb = []
        for i in range(max(5, min(args.steps, 20))):
            flush.fill_(float(i))
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            rob.self_collision(out["pose"], out=bout, tune=wbe.TREE_NOCULL)
            a1.record(stream)
            torch.cuda.synchronize()
            tb.append(a0.elapsed_time(a1))
        brute_ms = float(np.mean(tb[2:]))
        assert torch.equal(bout["dmin"], out["dmin"]) and torch.equal(bout["worst"], out["worst"])

    # end to end through the public API: every step copies the inputs in from
    # pinned host memory and every output back; wbe.StreamedStep cuts the
    # batch into chunks so that both copy directions and the kernels overlap
    e2e_chunks = 2 if args.kernel == "tree" else 1  # measured best on GB300 (4 and 8 slower)
    Bc = B // e2e_chunks
    pipe = wbe.StreamedStep(rob, Bc, e2e_chunks, fwd_tune=tune, bwd_tune=btune)
    h_in, h_out = pipe.host_buffers()
    src = {"q": q, "qd": qd, "qdd": qdd, "g_pose": gp, "g_sphere": gs, "g_dmin": gm,
           "g_tau": gt}
    for c in range(e2e_chunks):
        sl = slice(c * Bc, (c + 1) * Bc)
        for k, x in src.items():
            part = x[:, sl] if k in ("q", "qd", "qdd", "g_tau") else x[sl]
            h_in[c][k].copy_(torch.from_numpy(np.ascontiguousarray(part)))
    for _ in range(2):
        pipe.step(h_in, h_out)
    torch.cuda.synchronize()
    e2e_steps = max(3, min(args.steps, 20))
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(e2e_steps):
        pipe.step(h_in, h_out)
    t1.record(stream)
    torch.cuda.synchronize()
    clocks.stop()
    e2e_ms = t0.elapsed_time(t1) / e2e_steps
    h2d = int(sum(v.numel() * v.element_size() for c in h_in for v in c.values()))
    d2h = int(sum(v.numel() * v.element_size() for c in h_out for v in c.values()))
    # the chunked step computes what the whole-batch step computed
    ref_chunk = out["dmin"][:Bc].cpu()
    assert torch.equal(h_out[0]["dmin"], ref_chunk)

    kmean = {k: float(np.mean(v)) for k, v in k_ms.items()}
    keys = ("tree_fwd", "pair", "tree_bwd")
    vals = reduce_max([step_ms, e2e_ms] + [kmean[k] for k in keys], world, dev)
    step_ms, e2e_ms = vals[0], vals[1]
    kmean = dict(zip(keys, vals[2:]))
    fwd_mean, bwd_mean = kmean["tree_fwd"] + kmean["pair"], kmean["tree_bwd"]
    if rank != 0:
        return
    value = total / (step_ms * 1e-3)  # the whole global batch / the slowest rank's time
    e2e_value = total * (Bc * e2e_chunks / B) / (e2e_ms * 1e-3)  # the chunks cover Bc each
    work = work_per_eval(desc)
    peaks = measured_peaks()
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    alu_peak = fp32_peak_tflops(num_sms, sm_max)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    ridge = alu_peak * 1e12 / (hbm_peak * 1e9)
    kernels = {}
    for name, ms in kmean.items():
        w = work[name]
        if ms <= 0:
            continue
        if w["flops"] / w["bytes"] >= ridge:
            ach = w["flops"] * B / (ms * 1e-3) / 1e12
            kernels[name] = {"bound": "alu", "achieved": ach, "peak": alu_peak,
                             "unit": "TFLOP/s", "frac": ach / alu_peak}
        else:
            ach = w["bytes"] * B / (ms * 1e-3) / 1e9
            kernels[name] = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                             "frac": ach / hbm_peak}
        tr = traffic_per_eval(names[name])
        kernels[name].update({"kernel": names[name], "ms": ms, "flops_per_eval": w["flops"],
                              "bytes_per_eval": w["bytes"],
                              "traffic": None if tr is None else tr * B})
    kmean = {k: v for k, v in kmean.items() if v > 0}
    dom = max(kmean, key=kmean.get)
    cpu = None if args.skip_cpu else time_oracle(desc, target_s=args.cpu_s)
    line = {
        "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "strong" if args.split else "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": HUMANOID48_WORKLOAD,
                   "batch_per_gpu": B, "global_batch": total,
                   "partition": "contiguous columns of one seeded batch, rank 0 first",
                   "kernel": args.kernel, "autotuned": chosen,
                   "l2": "flushed between timed steps (512 MB write outside the events)"},
        "fwd_ms": fwd_mean, "bwd_ms": bwd_mean,
        "roofline": dict(kernel=names[dom], **{k: kernels[dom][k] for k in
                         ("bound", "achieved", "peak", "unit", "frac", "traffic")},
                         peak_basis=("FP32 FMA: %d SMs x 128 x 2 x %.0f MHz (max SM clock)"
                                     % (num_sms, sm_max)) if kernels[dom]["bound"] == "alu"
                         else "HBM copy bandwidth of measured"),
        "kernels": kernels,
        "pair_full_map_reduce_ms": brute_ms,
        "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "chunks": e2e_chunks,
                "note": "wbe.StreamedStep: copies in, kernels and copies out of different "
                        "chunks overlap on three streams"},
        "gpu_launches": (3 if args.kernel == "tree" else 2) * args.steps,
        "clocks": clocks.summary(),
        "cpu_baseline": cpu,
    }
    if args.kernel == "tree" and not args.skip_plain:
        # the plain one-thread-per-configuration kernels and the fused
        # (CTA-tiled, level-synchronous) kernels on the same inputs
        for key, kt, reps in (("plain", wbe.PLAIN, 3), ("fused", wbe.FUSED, 10)):
            for _ in range(2):
                rob.eval(tq, tqd, tqdd, tune=kt, out=out)
                rob.eval_backward(tq, tqd, tqdd, out["worst"], tgp, tgs, tgm, tgt, tune=kt,
                                  out=gout)
            torch.cuda.synchronize()
            a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            pf, pb = [], []
            for i in range(reps):
                flush.fill_(float(i))
                a.record(stream)
                rob.eval(tq, tqd, tqdd, tune=kt, out=out)
                b.record(stream)
                rob.eval_backward(tq, tqd, tqdd, out["worst"], tgp, tgs, tgm, tgt, tune=kt,
                                  out=gout)
                c.record(stream)
                torch.cuda.synchronize()
                pf.append(a.elapsed_time(b))
                pb.append(b.elapsed_time(c))
            line[key] = {"value": B / ((np.mean(pf) + np.mean(pb)) * 1e-3), "unit": "evals/s",
                         "fwd_ms": float(np.mean(pf)), "bwd_ms": float(np.mean(pb)),
                         "kernels": "%s_fwd_kernel, %s_bwd_kernel" % (key, key)}
    if args.kernel == "tree" and not args.skip_uneven:
        # the uneven-batch workload (one GPU, rank 0): graph-replayed forward +
        # backward with the batch's default and its autotuned launch choices
        u = uneven_measure(rank, dev, 50, 3)
        line["uneven"] = {
            "workload": "256 x R7 + 256 x R23 + 256 x R48, horizons U{16..64}, fwd + bwd, "
                        "one CUDA graph",
            "value": u["configurations"] / (u["ms"] * 1e-3), "unit": "evals/s",
            "ms_per_step": u["ms"], "configurations": u["configurations"],
            "default_launch_value": u["configurations"] / (u["default_ms"] * 1e-3),
            "default_launch_ms": u["default_ms"], "autotuned": u["autotuned"],
            "default_launch": u["default"]}
    print(json.dumps(line), flush=True)


def trajopt_work(desc, K, T):
    """Algorithmic flops and HBM bytes per configuration for the kernels of the
    trajectory-optimisation step (no pose or sphere gradients flow back; the
    pair kernel stores no sphere centres)."""
    n = desc.n
    nm = int((desc.jtype != R.FIXED).sum())
    S, P, d = desc.S, desc.P, desc.dof
    return {
        "bspline_fwd": {"flops": 84 * d, "bytes": 4 * 3 * d + 4 * d * K // T},
        # the states evaluated from the trajectory's control points in the sweep
        # (4 control points and 7 flops per state read; the K d control points of
        # a trajectory are read once for its T samples)
        "tree_fwd": {"flops": 150 * nm + 330 * n + 28 * d,
                     "bytes": 4 * (d * K // T + 12 * n + d)},
        "pair": {"flops": 18 * S + 11 * P, "bytes": 4 * (12 * n + 2)},
        # the whole adjoint with the cost in its prologue: the control points,
        # tau, d_min and worst in; gq, gqd, gqdd and the cost out (the hinges
        # and motion terms add ~22 flops per joint, the states ~56)
        "tree_bwd": {"flops": 150 * nm + 330 * n + 660 * n + 60 * n + 22 * d + 3 + 56 * d,
                     "bytes": 4 * (d * K // T + d + 2 + 3 * d + 1)},
        "bspline_bwd": {"flops": 24 * d, "bytes": 4 * 3 * d + 4 * d * K // T},
        # summed hinge: every pair screened from both spheres (sqrt-free, 8 flops)
        "hinge": {"flops": 18 * S + 16 * P, "bytes": 4 * (12 * n + 3 * S + 1)},
    }


def run_trajopt(args, rank=0, world=1, local_rank=0):
    """Trajectory-optimisation gradient step on the 48-DoF humanoid with 3 kg
    hand payloads: 512 seeds x 16 control points per joint -> 64 B-spline
    samples each (32768 configurations), the states evaluated from the
    control points inside the sweeps -> FK + RNEA sweep -> self-collision ->
    torque-limit + collision hinges and the smooth / length / energy terms,
    formed in the prologue of the adjoint sweep (which also adds the cost's
    direct qd / qdd gradients) -> B-spline adjoint -> dL/dU.  Value =
    configurations per second."""
    import torch
    from paper_2603_05493_gb300 import build
    build()
    from paper_2603_05493_gb300 import wbe
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    desc = I.hand_payload(R.r48())
    rob = wbe.Robot(desc, device=local_rank)
    n_traj, K, T, dt = CF.TRAJOPT_SEEDS, CF.TRAJOPT_KNOTS, CF.TRAJOPT_STEPS, CF.TRAJOPT_DT
    B, d = n_traj * T, desc.dof
    ft, bt = sweep_shapes(rob, B, args, spline=(n_traj, K, T, dt))
    seg = lambda t: t.lanes_per_config if t.kernel == wbe.L.WB_KERNEL_TREE else 0  # noqa
    tpb = lambda t: t.configs_per_block if t.kernel == wbe.L.WB_KERNEL_TREE else 0  # noqa
    ftune = wbe.Tune(kernel=wbe.L.WB_KERNEL_TREE, lanes_per_config=seg(ft),
                     configs_per_block=tpb(ft))
    btune = wbe.Tune(kernel=wbe.L.WB_KERNEL_TREE, lanes_per_config=seg(bt),
                     configs_per_block=tpb(bt))
    hU = torch.from_numpy(I.bspline_controls(d, n_traj, K, seed=rank_seed(CF.TRAJOPT48.seed, rank)))
    hU = hU.pin_memory()
    U = hU.to(dev)
    lo = torch.full((d,), -CF.TORQUE_LIMIT, device=dev)
    hi = torch.full((d,), CF.TORQUE_LIMIT, device=dev)
    out = rob.empty_outputs(B, sphere=False)
    fwd_out = {"pose": out["pose"], "sphere": None, "dmin": None, "worst": None,
               "tau": out["tau"], "bits": None}
    wdiff = torch.empty((B, 3), device=dev)  # the worst pair's centre difference
    pair_out = {"sphere": None, "dmin": out["dmin"], "worst": out["worst"], "diff": wdiff,
                "bits": None}
    cost = torch.empty((B,), device=dev)
    gout = tuple(torch.empty((d, B), device=dev) for _ in range(3))
    # the energy term's dt: the time between consecutive samples
    dt_sample = dt * (K - 3) / (T - 1)
    gU = torch.empty((n_traj, d, K), device=dev)
    stream = torch.cuda.current_stream()
    hinge = args.collision == "hinge"
    # the states come from the control points inside the sweeps
    # (wb_eval_spline, wb_eval_backward_spline_cost); the cost runs in the
    # backward sweep's prologue
    names = ["tree_fwd", "hinge" if hinge else "pair", "tree_bwd", "bspline_bwd"]
    hinge_cost = torch.empty((B,), device=dev)
    g_sph = torch.empty((B, desc.S, 3), device=dev) if hinge else None

    def step(ev=None):
        mark = (lambda i: ev[i].record(stream)) if ev else (lambda i: None)
        rob.eval_spline(U, T, dt, tune=ftune, out=fwd_out)
        mark(1)
        if hinge:  # every pair within the activation distance
            rob.self_collision_hinge(out["pose"], CF.ACTIVATION_DISTANCE, CF.COLLISION_WEIGHT,
                                     cost=hinge_cost, g_sphere=g_sph)
        else:  # the worst pair
            rob.self_collision(out["pose"], out=pair_out)
        mark(2)
        rob.eval_backward_spline_cost(U, T, dt, out["tau"], lo, hi, CF.COLLISION_WEIGHT,
                                      CF.SMOOTH_WEIGHT, CF.LENGTH_WEIGHT, CF.ENERGY_WEIGHT,
                                      dt_sample, d_min=None if hinge else out["dmin"],
                                      worst=None if hinge else out["worst"],
                                      worst_diff=None if hinge else wdiff,
                                      g_sphere=g_sph if hinge else None, cost=cost, tune=btune,
                                      out=gout)
        mark(3)
        wbe.bspline_backward(*gout, n_traj, K, T, dt, gU)

    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local_rank)
    clocks.start()
    nk = len(names)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(nk + 1)]
           for _ in range(args.steps)]
    torch.cuda.nvtx.range_push("timed")
    for i in range(args.steps):
        flush.fill_(float(i))
        evs[i][0].record(stream)
        step(evs[i])
        evs[i][nk].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier(world)
    step_ms = float(np.mean([e[0].elapsed_time(e[nk]) for e in evs]))
    k_ms = {nm: float(np.mean([e[i].elapsed_time(e[i + 1]) for e in evs]))
            for i, nm in enumerate(names)}
    # end to end: control points in from pinned host memory, dL/dU and the
    # per-configuration cost back, every step
    hgU = torch.empty(gU.shape, pin_memory=True)
    hcost = torch.empty(cost.shape, pin_memory=True)
    e2e_steps = max(3, min(args.steps, 20))
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(e2e_steps):
        U.copy_(hU, non_blocking=True)
        step()
        hgU.copy_(gU, non_blocking=True)
        hcost.copy_(cost, non_blocking=True)
    t1.record(stream)
    torch.cuda.synchronize()
    clocks.stop()
    e2e_ms = t0.elapsed_time(t1) / e2e_steps
    vals = reduce_max([step_ms, e2e_ms] + [k_ms[nm] for nm in names], world, dev)
    step_ms, e2e_ms = vals[0], vals[1]
    k_ms = dict(zip(names, vals[2:]))
    if rank != 0:
        return
    work = trajopt_work(desc, K, T)
    peaks = measured_peaks()
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = fp32_peak_tflops(num_sms, peaks.get("sm_max_mhz", 2070.0))
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    ridge = alu_peak * 1e12 / (hbm_peak * 1e9)
    kernels = {}
    kn = {"bspline_fwd": "bspline_fwd_kernel", "pair": "pair_kernel", "hinge": "hinge_kernel",
          "tree_fwd": "tree_fwd_spline_seg_kernel" if seg(ft) > 1 else "tree_fwd_spline_kernel",
          "tree_bwd": ("tree_bwd_spline_cost_seg_kernel" if seg(bt) > 1
                       else "tree_bwd_spline_cost_kernel"),
          "bspline_bwd": "bspline_bwd_kernel"}
    for nm, ms in k_ms.items():
        w = work[nm]
        if w["flops"] / w["bytes"] >= ridge:
            ach = w["flops"] * B / (ms * 1e-3) / 1e12
            kernels[nm] = {"bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s",
                           "frac": ach / alu_peak}
        else:
            ach = w["bytes"] * B / (ms * 1e-3) / 1e9
            kernels[nm] = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                           "frac": ach / hbm_peak}
        tr = traffic_per_eval(kn[nm], "trajopt48")
        kernels[nm].update({"kernel": kn[nm], "ms": ms, "flops_per_eval": w["flops"],
                            "bytes_per_eval": w["bytes"],
                            "traffic": None if tr is None else tr * B})
    dom = max(k_ms, key=k_ms.get)
    line = {
        "metric": "trajopt48 evals/s (B-spline -> FK+self-coll+RNEA -> hinge + motion cost "
                  "-> adjoint -> dL/dU)",
        "value": job_value(world, B, step_ms), "unit": "evals/s", "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "trajopt48: 48-DoF tree + 3 kg hand payloads, 512 seeds x 64 "
                               "B-spline samples (16 control points / joint, dt 0.25 s), "
                               "torque limits +-30 N m, collision weight 1, smooth / "
                               "length / energy weights %g / %g / %g, "
                               % (CF.SMOOTH_WEIGHT, CF.LENGTH_WEIGHT, CF.ENERGY_WEIGHT) +
                               ("summed hinge over all pairs, activation distance %.3g m"
                                % CF.ACTIVATION_DISTANCE if hinge else "worst-pair hinge"),
                   "configurations": B,
                   "autotuned": {"fwd": dict(ft.__dict__), "bwd": dict(bt.__dict__)},
                   "l2": "flushed between timed steps (512 MB write outside the events)"},
        "roofline": dict(kernel=kn[dom], **{k: kernels[dom][k] for k in
                         ("bound", "achieved", "peak", "unit", "frac", "traffic")}),
        "kernels": kernels,
        "active_torque_hinges": float((out["tau"].abs() > CF.TORQUE_LIMIT).float().mean()),
        "penetrating_configurations": None if hinge else float((out["dmin"] < 0).float().mean()),
        "e2e": {"value": job_value(world, B, e2e_ms), "unit": "evals/s",
                "h2d_bytes_per_step": world * int(hU.numel() * 4),
                "d2h_bytes_per_step": world * int(hgU.numel() * 4 + hcost.numel() * 4)},
        "gpu_launches": len(names) * args.steps * world,
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)


def run_kinematics(args, rank=0, world=1, local_rank=0):
    """Split forward kinematics on the 48-DoF humanoid with hand payloads,
    32768 configurations: the forward sweep writes the link poses, then one
    kernel computes the world Jacobians of the two hands and two feet, the
    centre of mass and its Jacobian.  Value = configurations per second."""
    import torch
    from paper_2603_05493_gb300 import build
    build()
    from paper_2603_05493_gb300 import wbe
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    desc = I.hand_payload(R.r48())
    rob = wbe.Robot(desc, device=local_rank)
    B, d, n = CF.HUMANOID48.batch, desc.dof, desc.n
    targets = list(R.hand_links(desc)) + [n - 1, n - 7]
    q, qd, qdd = (torch.from_numpy(x).to(dev) for x in
                  I.uniform_states(d, B, rank_seed(CF.HUMANOID48.seed, rank)))
    out = rob.empty_outputs(B, sphere=False, dmin=False, tau=False)
    jac = torch.empty((B, len(targets), 6, d), device=dev)
    com = torch.empty((B, 3), device=dev)
    jac_com = torch.empty((B, 3, d), device=dev)
    stream = torch.cuda.current_stream()

    def step(ev=None):
        rob.eval(q, tune=wbe.TREE, out=out, sphere=False, dmin=False, tau=False)
        if ev:
            ev[1].record(stream)
        rob.kinematics(out["pose"], targets, jac=jac, com=com, jac_com=jac_com)

    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local_rank)
    clocks.start()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    torch.cuda.nvtx.range_push("timed")
    for i in range(args.steps):
        flush.fill_(float(i))
        evs[i][0].record(stream)
        step(evs[i])
        evs[i][2].record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clocks.stop()
    barrier(world)
    step_ms = float(np.mean([e[0].elapsed_time(e[2]) for e in evs]))
    fk_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in evs]))
    kin_ms = float(np.mean([e[1].elapsed_time(e[2]) for e in evs]))
    step_ms, fk_ms, kin_ms = reduce_max([step_ms, fk_ms, kin_ms], world, dev)
    if rank != 0:
        return
    # kinematics kernel: reads the poses, writes the Jacobians, CoM and its
    # Jacobian (HBM-bound); per configuration ~(12 per driven link + 30 per
    # target-column) flops on the chain joints, ~60 per link for the moments
    nt = len(targets)
    kin_bytes = 4 * (12 * n + nt * 6 * d + 3 + 3 * d)
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    ach = kin_bytes * B / (kin_ms * 1e-3) / 1e9
    print(json.dumps({
        "metric": "split FK + link Jacobians + CoM evals/s (48-DoF humanoid + payloads)",
        "value": job_value(world, B, step_ms), "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "kinematics: 48-DoF tree + 3 kg hand payloads, 32768 "
                               "configurations, Jacobians of 4 links, CoM and its Jacobian",
                   "targets": targets, "l2": "flushed between timed steps"},
        "kernels": {"tree_fwd": {"kernel": "tree_fwd_seg_kernel or tree_fwd_kernel (poses only)",
                                 "ms": fk_ms},
                    "kinematics": {"kernel": "kin_kernel", "ms": kin_ms, "bound": "hbm",
                                   "bytes_per_eval": kin_bytes, "achieved": ach,
                                   "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak}},
        "roofline": {"kernel": "kin_kernel", "bound": "hbm", "achieved": ach, "peak": hbm_peak,
                     "unit": "GB/s", "frac": ach / hbm_peak, "traffic": None},
        "gpu_launches": 2 * args.steps * world, "clocks": clocks.summary()}), flush=True)


def run_arm7(args, rank=0, world=1, local_rank=0):
    """The 7-DoF chain at 4096 seeds x 32 timesteps (131072 configurations),
    forward only: FK, sphere placement, self-collision and RNEA with every
    output written (poses, sphere centres, d_min / worst pair, torques).  The
    HBM-bound workload.  Times the default path (the forward sweep with the
    autotuner's shape, then the pair kernel), the fused kernel and the plain
    single-robot kernel on the same inputs; value = configurations per second
    of the default path."""
    import torch
    from paper_2603_05493_gb300 import build
    build()
    from paper_2603_05493_gb300 import wbe
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    desc = R.r7()
    rob = wbe.Robot(desc, device=local_rank)
    lo, hi, total = rank_columns(world, rank, args.batch or CF.ARM7.batch, args.split)
    B = hi - lo
    q, qd, qdd = (torch.from_numpy(x).to(dev) for x in
                  I.batch_columns(desc, lo, hi, CF.ARM7.seed)[:3])
    out = rob.empty_outputs(B)
    ft, _, _, _ = rob.autotune(B)
    is_tree = ft.kernel == wbe.L.WB_KERNEL_TREE
    seg = ft.lanes_per_config if is_tree else 0
    sweep = wbe.Tune(kernel=wbe.L.WB_KERNEL_TREE, lanes_per_config=seg,
                     configs_per_block=ft.configs_per_block if is_tree else 0)
    pair = wbe.Tune(kernel=wbe.L.WB_KERNEL_TREE, blocks_per_sm=ft.blocks_per_sm if is_tree else 0)
    stream = torch.cuda.current_stream()
    fwd_out = {"pose": out["pose"], "sphere": None, "dmin": None, "worst": None,
               "tau": out["tau"], "bits": None}
    pair_out = {"sphere": out["sphere"], "dmin": out["dmin"], "worst": out["worst"],
                "bits": None}

    def tree_step(ev=None):
        rob.eval(q, qd, qdd, tune=sweep, out=fwd_out, sphere=False, dmin=False)
        if ev:
            ev.record(stream)
        rob.self_collision(out["pose"], tune=pair, out=pair_out)

    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)

    def timed(f, n, split_event=False, clk=None):
        for _ in range(max(args.warmup, 3)):
            f()
        torch.cuda.synchronize()
        barrier(world)
        if clk is not None:
            clk.start()
        tot, first = [], []
        for i in range(n):
            flush.fill_(float(i))
            a, m, b = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record(stream)
            f(m) if split_event else f()
            b.record(stream)
            torch.cuda.synchronize()
            tot.append(a.elapsed_time(b))
            if split_event:
                first.append(a.elapsed_time(m))
        if clk is not None:
            clk.stop()
        barrier(world)
        return float(np.mean(tot)), (float(np.mean(first)) if first else None)
    clocks = ClockSampler(local_rank)
    ms, sweep_ms = timed(tree_step, args.steps, split_event=True, clk=clocks)
    n_other = max(5, min(args.steps, 50))
    fused_ms, _ = timed(lambda: rob.eval(q, qd, qdd, tune=wbe.FUSED, out=out), n_other)
    plain_ms, _ = timed(lambda: rob.eval(q, qd, qdd, tune=wbe.PLAIN, out=out), n_other)
    ms, sweep_ms, fused_ms, plain_ms = reduce_max([ms, sweep_ms, fused_ms, plain_ms], world, dev)
    if rank != 0:
        return
    d, n, S = desc.dof, desc.n, desc.S
    w = work_per_eval(desc)
    bytes_fwd = 4 * (3 * d + 12 * n + 3 * S + 2 + d)  # states in; poses, spheres, d_min, worst, tau out
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)

    def hbm(bytes_per_eval, t_ms):
        ach = bytes_per_eval * B / (t_ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak}
    pair_ms = ms - sweep_ms
    kernels = {
        "tree_fwd": dict(hbm(w["tree_fwd"]["bytes"], sweep_ms), ms=sweep_ms,
                         kernel="tree_fwd_seg_kernel" if seg > 1 else "tree_fwd_kernel",
                         bytes_per_eval=w["tree_fwd"]["bytes"]),
        # robots of at most 32 spheres and 1024 pairs take the library's
        # one-thread-per-configuration pair kernel
        "pair": dict(hbm(w["pair"]["bytes"], pair_ms), ms=pair_ms,
                     kernel="pair_thread_kernel" if desc.S <= 32 and desc.P <= 1024
                     else "pair_kernel", bytes_per_eval=w["pair"]["bytes"]),
    }
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    print(json.dumps({
        "metric": "arm7 whole-body forward evals/s (FK+self-coll+RNEA, 7-DoF chain)",
        "value": total / (ms * 1e-3), "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if args.split else "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "arm7: 7-DoF chain, 28 spheres, 240 pairs, 4096 x 32 "
                               "configurations, forward with every output",
                   "batch_per_gpu": B, "global_batch": total,
                   "autotuned": dict(ft.__dict__), "l2": "flushed between timed steps"},
        "step_roofline": dict(hbm(bytes_fwd, ms), bytes_per_eval=bytes_fwd),
        "roofline": dict(kernel=kernels[dom]["kernel"], traffic=None,
                         **{k: kernels[dom][k] for k in ("bound", "achieved", "peak", "unit",
                                                         "frac")}),
        "kernels": kernels,
        "fused": dict(hbm(bytes_fwd, fused_ms), value=B / (fused_ms * 1e-3), ms=fused_ms,
                      kernel="fused_fwd_kernel"),
        "plain": dict(hbm(bytes_fwd, plain_ms), value=B / (plain_ms * 1e-3), ms=plain_ms,
                      kernel="plain_fwd_kernel"),
        "gpu_launches": 2 * args.steps * world, "clocks": clocks.summary()}), flush=True)


def uneven_measure(rank, dev, steps, warmup, clocks=None):
    """The uneven workload: 256 x R7 + 256 x R23 + 256 x R48 problems with
    horizons U{16..64}, forward (FK + RNEA, spheres + self-collision) and
    backward in one persistent launch per pass, captured in a CUDA graph and
    replayed; timed with the batch's default launch choices and again after
    wb_batch_autotune (a graph captured anew for each).  Returns the times
    and choices."""
    import torch
    from paper_2603_05493_gb300 import wbe
    mix = I.uneven_mix()  # the same problem mix on every rank; states differ
    robs = [wbe.Robot(d, device=dev.index) for d in mix.robots]
    problems = list(zip(mix.robot_of.tolist(), mix.horizon.tolist()))
    batch = wbe.Batch(robs, problems)
    total = int(mix.horizon.sum())

    def packed(kind, make, dtype=torch.float32):
        out = batch.empty(kind, dtype)
        for p, (ri, H) in enumerate(problems):
            x = make(mix.robots[ri], H, 7000 + p + 100000 * rank)
            o = int(batch.offsets[kind][p])
            t = torch.from_numpy(np.ascontiguousarray(x)).reshape(-1).to(dev)
            out[o:o + t.numel()] = t
        return out
    q = packed("joint", lambda d, H, s: I.uniform_states(d.dof, H, s)[0])
    qd = packed("joint", lambda d, H, s: I.uniform_states(d.dof, H, s)[1])
    qdd = packed("joint", lambda d, H, s: I.uniform_states(d.dof, H, s)[2])
    gp = packed("pose", lambda d, H, s: I.upstream_grads(d, H, s)[0])
    gs = packed("sphere", lambda d, H, s: I.upstream_grads(d, H, s)[1])
    gm = packed("config", lambda d, H, s: I.upstream_grads(d, H, s)[2])
    gt = packed("joint", lambda d, H, s: I.upstream_grads(d, H, s)[3])
    pose, sph, dmin, tau = batch.empty("pose"), batch.empty("sphere"), batch.empty("config"), \
        batch.empty("joint")
    worst = batch.empty("config", torch.int32)
    g = [batch.empty("joint") for _ in range(3)]

    def step():
        batch.eval(q, qd, qdd, pose, sph, dmin, worst, tau)
        batch.eval_backward(q, qd, qdd, worst, gp, gs, gm, gt, *g)
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)

    def timed(n, clk=None):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(3):
                step()
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        for _ in range(max(warmup, 3)):
            graph.replay()
        torch.cuda.synchronize()
        if clk is not None:
            clk.start()
        ts = []
        torch.cuda.nvtx.range_push("timed")
        for i in range(n):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            graph.replay()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        torch.cuda.nvtx.range_pop()
        if clk is not None:
            clk.stop()
        return float(np.mean(ts))
    default = batch.get_tune()
    ms_default = timed(max(3, steps // 2))
    tune, fseg, bseg, fms, bms = batch.autotune()
    ms = timed(steps, clocks)
    names = [d.name for d in mix.robots]
    return {"ms": ms, "configurations": total, "problems": len(problems),
            "default_ms": ms_default,
            "default": {"tune": default[0], "fwd_segments": dict(zip(names, default[1])),
                        "bwd_segments": dict(zip(names, default[2]))},
            "autotuned": {"tune": tune, "fwd_segments": dict(zip(names, fseg)),
                          "bwd_segments": dict(zip(names, bseg)),
                          "fwd_ms": fms, "bwd_ms": bms}}


def run_uneven(args, rank=0, world=1, local_rank=0):
    """Uneven batch: 256 x R7 + 256 x R23 + 256 x R48 problems with horizons
    U{16..64}, forward and backward in one persistent launch per pass with the
    launch choices of wb_batch_autotune, captured once in a CUDA graph and
    replayed.  Value = configurations per second (sum of horizons / step)."""
    import torch
    from paper_2603_05493_gb300 import build
    build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    barrier(world)
    clocks = ClockSampler(local_rank)
    u = uneven_measure(rank, dev, args.steps, args.warmup, clocks)
    barrier(world)
    ms, ms_default = reduce_max([u["ms"], u["default_ms"]], world, dev)
    if rank != 0:
        return
    total = u["configurations"]
    print(json.dumps({
        "metric": "uneven-batch evals/s (R7/R23/R48 problems, fwd+bwd, one graph)",
        "value": job_value(world, total, ms), "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "scaling": "weak",
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "uneven: 256 x R7 + 256 x R23 + 256 x R48, horizons U{16..64}",
                   "configurations": total, "problems": u["problems"],
                   "l2": "flushed between timed steps"},
        "autotuned": u["autotuned"],
        "default_launch": dict(u["default"], value=job_value(world, total, ms_default),
                               ms_per_step=ms_default),
        "gpu_launches": 3 * args.steps * world, "clocks": clocks.summary()}), flush=True)


def arg_parser():
    """bench.py's command line (the profile summaries' commands are checked
    against it)."""
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--kernel", choices=["tree", "fused", "plain"], default="tree")
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--split", action="store_true",
                    help="humanoid48 under torchrun: split the --batch configurations over "
                         "the ranks (strong scaling) instead of --batch per rank")
    ap.add_argument("--skip-uneven", action="store_true",
                    help="humanoid48: leave out the uneven-batch sub-result")
    ap.add_argument("--cpu-s", type=float, default=15.0)
    ap.add_argument("--ref-step-s", type=float, default=10.0,
                    help="reference arm: at most this many seconds of oracle work a step")
    ap.add_argument("--ref-total-s", type=float, default=120.0,
                    help="reference arm: about this many seconds for the whole run")
    ap.add_argument("--workload", choices=["humanoid48", "arm7", "uneven", "trajopt48",
                                           "kinematics"],
                    default="humanoid48")
    ap.add_argument("--collision", choices=["worst", "hinge"], default="worst",
                    help="trajopt48 collision cost: worst-pair hinge or summed hinge")
    ap.add_argument("--sweep-shape", default="",
                    help="pin the sweep launch shapes instead of autotuning: "
                         "fwd segments,fwd configs per block,bwd segments,bwd configs per block")
    return ap


def main():
    args = arg_parser().parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        run = {"humanoid48": run_ours, "arm7": run_arm7, "uneven": run_uneven,
               "trajopt48": run_trajopt, "kinematics": run_kinematics}
        run[args.workload](args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
