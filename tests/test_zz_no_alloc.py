"""wb_batch_eval_noalloc (forward evaluation of an uneven batch with its work
tables in the library's static device scratch) against the allocating entry
point wb_batch_create + wb_batch_eval, called through the C ABI.

Collected last on purpose: it must also pass after every other GPU test has
run in the same process."""
import ctypes as C

import numpy as np
import pytest
import torch

from synthetic import inputs as I
from synthetic import robots as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    assert torch.cuda.is_available()
    from paper_2603_05493_gb300 import build
    build()
    from paper_2603_05493_gb300 import wbe
    return wbe


@pytest.fixture(scope="module")
def robots(W):
    descs = [R.r7(), R.r23(), R.r48(), R.mixed_joint_tree()]
    return descs, [W.Robot(d, device=0) for d in descs]


MIX_A = [(2, 37), (0, 64), (1, 0), (3, 5), (2, 1), (1, 70), (0, 33), (3, 0), (1, 12)]
MIX_B = [(1, 3), (3, 64), (0, 1), (2, 65), (0, 0), (2, 31), (1, 40)]


def case(W, descs, robs, problems, seed):
    """Inputs packed for `problems`, and the allocating entry point's outputs."""
    batch = W.Batch(robs, problems)
    dev = batch.device

    def packed(kind, parts):
        out = batch.empty(kind)
        for p, x in enumerate(parts):
            o = int(batch.offsets[kind][p])
            t = torch.from_numpy(np.ascontiguousarray(x)).reshape(-1).to(dev)
            out[o:o + t.numel()] = t
        return out
    st = [I.uniform_states(descs[ri].dof, H, seed + p) for p, (ri, H) in enumerate(problems)]
    x = {k: packed("joint", [s[i] for s in st]) for i, k in enumerate(("q", "qd", "qdd"))}
    ref = outputs(batch)
    batch.eval(x["q"], x["qd"], x["qdd"], ref["pose"], ref["sphere"], ref["dmin"], ref["worst"],
               ref["tau"])
    return batch, x, ref


def outputs(batch):
    o = {"pose": batch.empty("pose"), "sphere": batch.empty("sphere"),
         "dmin": batch.empty("config"), "tau": batch.empty("joint"),
         "worst": batch.empty("config", torch.int32)}
    for k, t in o.items():
        t.fill_(-7 if k == "worst" else float("nan"))
    return o


def call(W, robs, problems, x, o, n_robots=None):
    """wb_batch_eval_noalloc through the C ABI; returns its status."""
    lib = W.L.load()
    arr = (C.c_void_p * len(robs))(*[r.handle.value for r in robs])
    probs = (W.L.wb_problem * max(len(problems), 1))(*[W.L.wb_problem(a, h)
                                                       for a, h in problems])
    p = lambda t: None if t is None else t.data_ptr()  # noqa: E731
    return lib.wb_batch_eval_noalloc(arr, len(robs) if n_robots is None else n_robots, probs,
                                     len(problems), p(x["q"]), p(x["qd"]), p(x["qdd"]),
                                     p(o["pose"]), p(o["sphere"]), p(o["dmin"]), p(o["worst"]),
                                     p(o["tau"]), torch.cuda.current_stream().cuda_stream)


def same(o, ref):
    """Identical to the allocating entry point's outputs, bit for bit (the
    same kernels on the same work items)."""
    for k in ("pose", "sphere", "dmin", "tau", "worst"):
        assert torch.equal(o[k], ref[k]), k


def test_matches_allocating_entry_point_on_consecutive_calls(W, robots):
    descs, robs = robots
    ba, xa, ra = case(W, descs, robs, MIX_A, 900)
    bb, xb, rb = case(W, descs, robs, MIX_B, 950)
    oa, ob, oa2 = outputs(ba), outputs(bb), outputs(ba)
    # back to back on one stream: the second call rebuilds the tables of the first
    assert call(W, robs, MIX_A, xa, oa) == W.L.WB_OK
    assert call(W, robs, MIX_B, xb, ob) == W.L.WB_OK
    assert call(W, robs, MIX_A, xa, oa2) == W.L.WB_OK
    torch.cuda.synchronize()
    same(oa, ra)
    same(ob, rb)
    same(oa2, ra)


def test_allocates_nothing_after_setup(W, robots):
    descs, robs = robots
    ba, xa, ra = case(W, descs, robs, MIX_A, 910)
    oa = outputs(ba)
    assert call(W, robs, MIX_A, xa, oa) == W.L.WB_OK  # first call does the setup
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert call(W, robs, MIX_A, xa, oa) == W.L.WB_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    same(oa, ra)


def test_limits_rejected_without_side_effects(W, robots):
    descs, robs = robots
    ba, xa, ra = case(W, descs, robs, MIX_A, 920)
    o = outputs(ba)
    lim = W.L.load()
    too_many_problems = [(0, 0)] * 1025
    assert call(W, robs, too_many_problems, xa, o) == W.L.WB_ETOOBIG
    assert b"1025 problems" in lim.wb_last_error()
    too_many_configs = [(0, 40000), (1, 30000)]
    assert call(W, robs, too_many_configs, xa, o) == W.L.WB_ETOOBIG
    nine = robs + robs + robs[:1]
    assert call(W, nine, MIX_A, xa, o) == W.L.WB_ETOOBIG
    assert call(W, robs, [(4, 3)], xa, o) == W.L.WB_ERANGE
    assert call(W, robs, [(0, -1)], xa, o) == W.L.WB_EINVAL
    torch.cuda.synchronize()
    for k, t in o.items():  # nothing was launched
        assert (t == -7).all() if k == "worst" else torch.isnan(t).all()
    # an empty mix is a no-op
    assert call(W, robs, [(0, 0), (2, 0)], xa, o) == W.L.WB_OK
    torch.cuda.synchronize()
    assert torch.isnan(o["pose"]).all()


def test_python_binding_matches(W, robots):
    descs, robs = robots
    bb, xb, rb = case(W, descs, robs, MIX_B, 960)
    o = outputs(bb)
    W.batch_eval_noalloc(robs, MIX_B, xb["q"], xb["qd"], xb["qdd"], o["pose"], o["sphere"],
                         o["dmin"], o["worst"], o["tau"])
    torch.cuda.synchronize()
    same(o, rb)


def limit_mix(total, seed):
    """1024 problems over the four robots, empty ones first, in the middle and
    last, horizons summing to `total` configurations."""
    rng = np.random.default_rng(seed)
    n = 1024
    H = rng.integers(1, 2 * total // n, size=n)
    H[[0, n // 2, n - 1]] = 0
    H = (H * (total / H.sum())).astype(np.int64)
    H[[0, n // 2, n - 1]] = 0
    i = 1
    while H.sum() < total:  # exact total, spread over the non-empty problems
        if i not in (n // 2,):
            H[i] += 1
        i = i % (n - 2) + 1
    robot = rng.integers(0, 4, size=n)
    return [(int(r), int(h)) for r, h in zip(robot, H)]


def test_matches_allocating_entry_point_at_the_limits(W, robots):
    """1024 problems (empty ones first, in the middle and last) and exactly
    65536 configurations: the setup kernel runs 64 blocks, each rescanning
    every problem's offsets and searching all of them; outputs identical to
    wb_batch_eval's.  One configuration more is refused."""
    descs, robs = robots
    mix = limit_mix(65536, 3)
    assert len(mix) == 1024 and sum(h for _, h in mix) == 65536
    assert mix[0][1] == mix[512][1] == mix[1023][1] == 0
    b, x, ref = case(W, descs, robs, mix, 1300)
    o = outputs(b)
    assert call(W, robs, mix, x, o) == W.L.WB_OK
    torch.cuda.synchronize()
    same(o, ref)
    over = list(mix)
    over[5] = (over[5][0], over[5][1] + 1)
    o2 = outputs(b)
    assert call(W, robs, over, x, o2) == W.L.WB_ETOOBIG
    torch.cuda.synchronize()
    assert torch.isnan(o2["pose"]).all()
