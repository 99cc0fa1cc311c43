"""The multi-rank host logic of bench.py on CPU: two gloo ranks on
127.0.0.1.  The humanoid48 workload is one seeded batch partitioned into
contiguous column ranges (weak or strong scaling); the other workloads draw
per-rank inputs.  The slowest rank's time sets the step and the whole-job
value counts every rank's configurations.  No GPU, no collective on the data
path."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from synthetic import configs as CF
        from synthetic import inputs as I
        from synthetic import robots as R
        seed = bench.rank_seed(CF.HUMANOID48.seed, rank)
        q, _, _ = I.uniform_states(R.r7().dof, 16, seed)
        # rank r takes (r + 1) ms per step and 2 (r + 1) ms end to end
        step, e2e = bench.reduce_max([1.0 + rank, 2.0 * (1 + rank)], world, "cpu")
        bench.barrier(world)
        out.put((rank, seed, q.sum(), step, e2e, bench.job_value(world, 32768, step)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, s0, q0, st0, e0, v0), (_, s1, q1, st1, e1, v1) = res
    assert s0 != s1 and q0 != q1             # each rank evaluates its own configurations
    assert st0 == st1 == 2.0                 # max over ranks
    assert e0 == e1 == 4.0
    assert v0 == v1 == pytest.approx(2 * 32768 / 2e-3)   # all ranks' work / slowest time


def _split_rank_main(rank, world, port, B, split, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from synthetic import robots as R
        lo, hi, total = bench.rank_columns(world, rank, B, split)
        mine = bench.humanoid48_inputs(R.r7(), lo, hi)
        got = [None] * world
        dist.all_gather_object(got, (rank, lo, hi, total, mine))
        if rank == 0:
            out.put(got)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("split", [False, True])
def test_two_gloo_ranks_partition_one_batch(split):
    """Each rank evaluates a contiguous slice of one seeded batch: the slices
    cover the global batch exactly once, in rank order, and each rank's
    inputs are the one-rank batch's columns, bit for bit (host arrays only)."""
    import bench
    from synthetic import robots as R
    world, port, B = 2, _free_port(), 70
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_split_rank_main, args=(r, world, port, B, split, out))
             for r in range(world)]
    for p in procs:
        p.start()
    got = out.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    total = got[0][3]
    assert total == (B if split else world * B)
    cols = sorted((lo, hi) for _, lo, hi, _, _ in got)
    assert cols[0][0] == 0 and cols[-1][1] == total
    assert all(a[1] == b[0] for a, b in zip(cols, cols[1:]))    # no gap, no overlap
    whole = bench.humanoid48_inputs(R.r7(), 0, total)
    for rank, lo, hi, _, mine in got:
        assert (lo, hi) == cols[rank]
        for part, ref in zip(mine, whole):
            want = ref[:, lo:hi] if ref.ndim == 2 and ref.shape[1] == total else ref[lo:hi]
            assert np.array_equal(part, want)


def test_rank_columns_partition_uneven_sizes():
    import bench
    for world in (1, 2, 3, 8):
        for B in (1, 7, 100, 32768):
            for split in (False, True):
                cols = [bench.rank_columns(world, r, B, split) for r in range(world)]
                total = cols[0][2]
                assert total == (B if split else world * B)
                assert cols[0][0] == 0 and cols[-1][1] == total
                assert all(a[1] == b[0] for a, b in zip(cols, cols[1:]))
                sizes = [hi - lo for lo, hi, _ in cols]
                assert max(sizes) - min(sizes) <= 1


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.reduce_max([3.0, 1.5], 1, "cpu") == [3.0, 1.5]
    assert bench.job_value(1, 1000, 2.0) == pytest.approx(5e5)
    assert bench.rank_seed(7, 0) == 7
    assert len({bench.rank_seed(7, r) for r in range(8)}) == 8
    assert np.isfinite(bench.job_value(8, 32768, 0.8))


@pytest.mark.parametrize("steps,warmup", [(1, 3), (20, 5), (300, 5), (1000, 10)])
def test_reference_arm_fits_its_time_budget(steps, warmup):
    """bench.py --impl reference times the oracle in bounded samples: however
    many steps it is asked for, the whole run stays within about its budget
    (120 s by default), and no step is longer than the per-step cap."""
    import bench
    total, cap = 120.0, 10.0
    warm, step = bench.reference_step_targets(steps, warmup, total, cap)
    assert 0.0 < warm <= 2.0 and 0.0 < step <= cap
    planned = warmup * warm + steps * step
    assert planned <= 1.05 * total or step == 0.1  # the floor: 0.1 s a step
    assert planned <= 240.0


def test_reference_arm_runs_end_to_end_quickly():
    """The reference arm's JSON line on a tiny budget (a few seconds of the
    FP64 oracle on the host cores)."""
    import json
    import subprocess
    import sys
    import time
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    t0 = time.perf_counter()
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "4",
                          "--warmup", "1", "--ref-total-s", "2"], cwd=root, capture_output=True,
                         text=True, timeout=300)
    wall = time.perf_counter() - t0
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["steps"] == 4
    # ms_per_step is the measured time of a step's sample, not an extrapolation
    n = line["config"]["sample_configs_per_step"]
    assert 0 < n <= line["config"]["batch"]
    assert line["steps"] * line["ms_per_step"] * 1e-3 < wall
    assert line["value"] == pytest.approx(n / (line["ms_per_step"] * 1e-3), rel=1e-9)
    assert line["e2e"]["value"] == line["value"]


def test_cpu_baseline_reports_forward_and_fd_rates():
    """cpu_baseline: forward + central-difference rate on all cores (value),
    on one thread, the forward-only rates, the thread count, nproc and the
    CPU model."""
    import bench
    from synthetic import robots as R
    cb = bench.time_oracle(R.r7(), target_s=1.0)
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["threads_1"] > 0
    assert cb["forward"]["threads_N"] > cb["value"] and cb["forward"]["threads_1"] > 0
    assert cb["cores"] >= 1 and cb["nproc"] >= 1 and cb["cpu_model"]
    assert "central-difference" in cb["pass"]


def test_work_model_matches_the_documented_figures():
    """bench.py's algorithmic flops and bytes per evaluation, on the bench's
    robots, are the closed forms of the work table (per kernel, in the link,
    joint, sphere and pair counts)."""
    import bench
    from synthetic import inputs as I
    from synthetic import robots as R
    r48 = R.r48()
    n, nm, S, P, d = r48.n, 48, r48.S, r48.P, r48.dof
    assert (n, S, P, d) == (49, 200, 15392, 48)
    w = bench.work_per_eval(r48)
    assert w["tree_fwd"] == {"flops": 150 * nm + 330 * n, "bytes": 4 * (3 * d + 12 * n + d)}
    assert w["pair"] == {"flops": 18 * S + 11 * P, "bytes": 4 * (12 * n + 3 * S + 2)}
    assert w["tree_bwd"] == {"flops": 150 * nm + 1050 * n + 15 * S,
                             "bytes": 4 * (7 * d + 12 * n + 3 * S + 2)}
    assert [w[k]["flops"] for k in ("tree_fwd", "pair", "tree_bwd")] == [23370, 172912, 61650]
    assert [w[k]["bytes"] for k in ("tree_fwd", "pair", "tree_bwd")] == [3120, 4760, 6104]
    t = bench.trajopt_work(I.hand_payload(r48), 16, 64)
    assert t["tree_fwd"] == {"flops": 24714, "bytes": 2592}
    assert t["pair"] == {"flops": 172912, "bytes": 2360}
    assert t["tree_bwd"] == {"flops": 62397, "bytes": 828}
    assert t["bspline_bwd"] == {"flops": 1152, "bytes": 624}
    assert t["hinge"] == {"flops": 249872, "bytes": 4756}
