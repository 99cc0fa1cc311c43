"""Uneven batches: several robots, uneven horizons, one persistent launch per
pass; per-problem parity against the oracle and CUDA-graph capture."""
import numpy as np
import pytest
import torch

from synthetic import inputs as I
from synthetic import robots as R
from tests import parity as PY

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    assert torch.cuda.is_available()
    from paper_2603_05493_gb300 import build
    build()
    from paper_2603_05493_gb300 import wbe
    return wbe


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


def make_batch(W, horizons_seed=0):
    descs = [R.r7(), R.r23(), R.r48(), R.mixed_joint_tree()]
    robs = [W.Robot(d, device=0) for d in descs]
    rng = np.random.default_rng(horizons_seed)
    problems = [(int(rng.integers(0, 4)), int(rng.integers(0, 70))) for _ in range(14)]
    problems += [(0, 0), (2, 33), (1, 1), (3, 64)]
    batch = W.Batch(robs, problems)
    return descs, robs, batch, problems


def fill(batch, descs, problems, seed):
    qs, qds, qdds, gps, gss, gms, gts = [], [], [], [], [], [], []
    for p, (ri, H) in enumerate(problems):
        d = descs[ri]
        q, qd, qdd = I.uniform_states(d.dof, H, seed + p)
        gp, gs, gm, gt = I.upstream_grads(d, H, seed + 100 + p)
        qs.append(q); qds.append(qd); qdds.append(qdd)
        gps.append(gp); gss.append(gs); gms.append(gm); gts.append(gt)
    dev = batch.device

    def packed(kind, parts, dtype=torch.float32):
        out = batch.empty(kind, dtype)
        for p, x in enumerate(parts):
            o = int(batch.offsets[kind][p])
            t = torch.from_numpy(np.ascontiguousarray(x)).reshape(-1).to(dev)
            out[o:o + t.numel()] = t
        return out
    return dict(q=packed("joint", qs), qd=packed("joint", qds), qdd=packed("joint", qdds),
                g_pose=packed("pose", gps), g_sph=packed("sphere", gss),
                g_dmin=packed("config", gms), g_tau=packed("joint", gts),
                raw=(qs, qds, qdds, gps, gss, gms, gts))


def run(batch, x):
    o = {k: batch.empty(k2) for k, k2 in (("pose", "pose"), ("sphere", "sphere"),
                                            ("dmin", "config"), ("tau", "joint"))}
    o["worst"] = batch.empty("config", torch.int32)
    batch.eval(x["q"], x["qd"], x["qdd"], o["pose"], o["sphere"], o["dmin"], o["worst"], o["tau"])
    g = [batch.empty("joint") for _ in range(3)]
    batch.eval_backward(x["q"], x["qd"], x["qdd"], o["worst"], x["g_pose"], x["g_sph"],
                        x["g_dmin"], x["g_tau"], *g)
    return o, g


def test_uneven_batch_matches_oracle(W, O):
    descs, robs, batch, problems = make_batch(W)
    x = fill(batch, descs, problems, 500)
    o, g = run(batch, x)
    torch.cuda.synchronize()
    qs, qds, qdds, gps, gss, gms, gts = x["raw"]
    for p, (ri, H) in enumerate(problems):
        if H == 0:
            continue
        d = descs[ri]
        got = {"pose": batch.view(o["pose"], "pose", p, (H, d.n, 12)).cpu().numpy(),
               "sphere": batch.view(o["sphere"], "sphere", p, (H, d.S, 3)).cpu().numpy(),
               "dmin": batch.view(o["dmin"], "config", p, (H,)).cpu().numpy(),
               "worst": batch.view(o["worst"], "config", p, (H,)).cpu().numpy(),
               "tau": batch.view(o["tau"], "joint", p, (d.dof, H)).cpu().numpy()}
        ref = O.evaluate(d, qs[p], qds[p], qdds[p])
        PY.check_forward(d, got, ref)
        gref = O.gradient(d, qs[p], qds[p], qdds[p], gps[p], gss[p], gms[p], gts[p])
        same = got["worst"] == ref["worst"]
        PY.check_gradient([batch.view(t, "joint", p, (d.dof, H)).cpu().numpy() for t in g],
                          gref, mask=same)


def test_batch_graph_capture_and_replay(W):
    descs, robs, batch, problems = make_batch(W, horizons_seed=3)
    x = fill(batch, descs, problems, 900)
    ref_o, ref_g = run(batch, x)
    torch.cuda.synchronize()
    # static buffers, captured once, replayed with new inputs
    static = {k: v.clone() for k, v in x.items() if k != "raw"}
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        run(batch, static)  # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        go, gg = run(batch, static)
    x2 = fill(batch, descs, problems, 1234)
    for k in static:
        static[k].copy_(x2[k])
    graph.replay()
    want_o, want_g = run(batch, x2)
    torch.cuda.synchronize()
    for k in ("pose", "sphere", "dmin", "tau", "worst"):
        assert torch.equal(go[k], want_o[k]), k
    for a, b in zip(gg, want_g):
        assert torch.equal(a, b)
    # and the earlier (pre-capture) results differ from the replayed ones
    assert not torch.equal(ref_o["dmin"], go["dmin"])


def test_streamed_step_matches_direct_calls(W):
    """wbe.StreamedStep (chunks, three streams, pinned host buffers) gives
    the same outputs as the direct calls on the whole batch, twice in a row."""
    desc = R.r23()
    rob = W.Robot(desc, device=0)
    K, Bc = 3, 40
    B = K * Bc
    q, qd, qdd = I.uniform_states(desc.dof, B, seed=31)
    gp, gs, gm, gt = I.upstream_grads(desc, B, seed=32)
    tune = W.Tune(kernel=3, lanes_per_config=1)
    cuda = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    o = rob.eval(cuda(q), cuda(qd), cuda(qdd), tune=tune)
    g = rob.eval_backward(cuda(q), cuda(qd), cuda(qdd), o["worst"], cuda(gp), cuda(gs),
                          cuda(gm), cuda(gt), tune=tune)
    pipe = W.StreamedStep(rob, Bc, K, fwd_tune=tune, bwd_tune=tune, run_streams=2)
    hin, hout = pipe.host_buffers()
    src = {"q": q, "qd": qd, "qdd": qdd, "g_pose": gp, "g_sphere": gs, "g_dmin": gm, "g_tau": gt}
    for c in range(K):
        sl = slice(c * Bc, (c + 1) * Bc)
        for k, x in src.items():
            part = x[:, sl] if k in ("q", "qd", "qdd", "g_tau") else x[sl]
            hin[c][k].copy_(torch.from_numpy(np.ascontiguousarray(part)))
    for _ in range(2):
        pipe.step(hin, hout)
        torch.cuda.synchronize()
        for c in range(K):
            sl = slice(c * Bc, (c + 1) * Bc)
            ref = {"pose": o["pose"][sl], "sphere": o["sphere"][sl], "dmin": o["dmin"][sl],
                   "worst": o["worst"][sl], "tau": o["tau"][:, sl], "gq": g[0][:, sl],
                   "gqd": g[1][:, sl], "gqdd": g[2][:, sl]}
            for k, v in ref.items():
                assert torch.equal(hout[c][k], v.cpu()), (c, k)


def test_uneven_full_size_sampled(W, O):
    """The bench's uneven workload (256 x R7 + 256 x R23 + 256 x R48, horizons
    U{16..64}, 30,398 configurations) in one batch, with the bench's input
    seeds; five problems of each robot checked against the oracle."""
    mix = I.uneven_mix()
    robs = [W.Robot(d, device=0) for d in mix.robots]
    problems = list(zip(mix.robot_of.tolist(), mix.horizon.tolist()))
    batch = W.Batch(robs, problems)
    raw = {}

    def packed(kind, k, make):
        out = batch.empty(kind)
        for p, (ri, H) in enumerate(problems):
            x = make(mix.robots[ri], H, 7000 + p)
            raw.setdefault(p, {})[k] = x
            o = int(batch.offsets[kind][p])
            t = torch.from_numpy(np.ascontiguousarray(x)).reshape(-1).cuda()
            out[o:o + t.numel()] = t
        return out
    q = packed("joint", "q", lambda d, H, s: I.uniform_states(d.dof, H, s)[0])
    qd = packed("joint", "qd", lambda d, H, s: I.uniform_states(d.dof, H, s)[1])
    qdd = packed("joint", "qdd", lambda d, H, s: I.uniform_states(d.dof, H, s)[2])
    gp = packed("pose", "gp", lambda d, H, s: I.upstream_grads(d, H, s)[0])
    gs = packed("sphere", "gs", lambda d, H, s: I.upstream_grads(d, H, s)[1])
    gm = packed("config", "gm", lambda d, H, s: I.upstream_grads(d, H, s)[2])
    gt = packed("joint", "gt", lambda d, H, s: I.upstream_grads(d, H, s)[3])
    x = dict(q=q, qd=qd, qdd=qdd, g_pose=gp, g_sph=gs, g_dmin=gm, g_tau=gt)
    o, g = run(batch, x)
    torch.cuda.synchronize()
    assert int(mix.horizon.sum()) == 30398
    for ri in range(len(mix.robots)):
        ps = [p for p, (r, _) in enumerate(problems) if r == ri][:5]
        for p in ps:
            d, H, rp = mix.robots[ri], problems[p][1], raw[p]
            got = {"pose": batch.view(o["pose"], "pose", p, (H, d.n, 12)).cpu().numpy(),
                   "sphere": batch.view(o["sphere"], "sphere", p, (H, d.S, 3)).cpu().numpy(),
                   "dmin": batch.view(o["dmin"], "config", p, (H,)).cpu().numpy(),
                   "worst": batch.view(o["worst"], "config", p, (H,)).cpu().numpy(),
                   "tau": batch.view(o["tau"], "joint", p, (d.dof, H)).cpu().numpy()}
            ref = O.evaluate(d, rp["q"], rp["qd"], rp["qdd"])
            PY.check_forward(d, got, ref)
            gref = O.gradient(d, rp["q"], rp["qd"], rp["qdd"], rp["gp"], rp["gs"], rp["gm"],
                              rp["gt"])
            same = got["worst"] == ref["worst"]
            PY.check_gradient([batch.view(t, "joint", p, (d.dof, H)).cpu().numpy() for t in g],
                              gref, mask=same)


def _per_problem(batch, o, g, p, d, H):
    return {"pose": batch.view(o["pose"], "pose", p, (H, d.n, 12)),
            "sphere": batch.view(o["sphere"], "sphere", p, (H, d.S, 3)),
            "dmin": batch.view(o["dmin"], "config", p, (H,)),
            "worst": batch.view(o["worst"], "config", p, (H,)),
            "tau": batch.view(o["tau"], "joint", p, (d.dof, H)),
            "g": [batch.view(t, "joint", p, (d.dof, H)) for t in g]}


def _check_against_single_robot(W, batch, robs, descs, problems, x, o, g, fseg, bseg, base):
    """Sweep outputs bit for bit those of the single-robot depth-first kernels
    with the same segment count on the same inputs (and the batch's worst
    pair); pair outputs bit for bit those of `base` (another tune of the same
    batch: the pair warps change the schedule, not the arithmetic)."""
    qs, qds, qdds, gps, gss, gms, gts = x["raw"]
    cuda = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    bo, bg = base
    for p, (ri, H) in enumerate(problems):
        if H == 0:
            continue
        d, rob = descs[ri], robs[ri]
        got = _per_problem(batch, o, g, p, d, H)
        ref = _per_problem(batch, bo, bg, p, d, H)
        for k in ("sphere", "dmin", "worst"):
            assert torch.equal(got[k], ref[k]), (p, k)
        f = rob.eval(cuda(qs[p]), cuda(qds[p]), cuda(qdds[p]), sphere=False, dmin=False,
                     tune=W.Tune(kernel=3, lanes_per_config=fseg[ri]))
        assert torch.equal(got["pose"], f["pose"]) and torch.equal(got["tau"], f["tau"]), p
        gr = rob.eval_backward(cuda(qs[p]), cuda(qds[p]), cuda(qdds[p]), got["worst"].clone(),
                               cuda(gps[p]), cuda(gss[p]), cuda(gms[p]), cuda(gts[p]),
                               tune=W.Tune(kernel=3, lanes_per_config=bseg[ri]))
        for a, b in zip(got["g"], gr):
            assert torch.equal(a, b), p


@pytest.mark.parametrize("threads,pair_warps", [(64, 2), (128, 4), (256, 8)])
def test_batch_tunes_match_single_robot_sweeps(W, threads, pair_warps):
    """Every launch choice of an uneven batch -- sweep blocks of 64 / 128 /
    256 threads, 2 / 4 / 8 pair warps, and per robot and pass 1 or 2 sweep
    segments (the mimic robot has no 2-segment plan) -- gives the
    single-robot kernels' results bit for bit."""
    descs, robs, batch, problems = make_batch(W, horizons_seed=5)
    x = fill(batch, descs, problems, 700)
    base = run(batch, x)
    for fseg, bseg in (([1, 1, 1, 1], [2, 2, 2, 1]), ([2, 2, 2, 1], [1, 1, 1, 1]),
                       ([2, 1, 2, 1], [1, 2, 1, 1])):
        batch.set_tune(threads, threads, pair_warps, fseg, bseg)
        t, f, b = batch.get_tune()
        assert (t["fwd_threads"], t["bwd_threads"], t["pair_warps"]) == (threads, threads,
                                                                          pair_warps)
        assert (f, b) == (fseg, bseg)
        o, g = run(batch, x)
        torch.cuda.synchronize()
        _check_against_single_robot(W, batch, robs, descs, problems, x, o, g, fseg, bseg, base)


def test_batch_autotune_choice_is_applied_and_exact(W, O):
    """wb_batch_autotune: valid choices, kept by the batch, results equal to
    the single-robot kernels with the chosen segments and to the oracle."""
    descs, robs, batch, problems = make_batch(W, horizons_seed=9)
    x = fill(batch, descs, problems, 800)
    base = run(batch, x)
    t, f, b, fm, bm = batch.autotune()
    assert fm > 0 and bm > 0
    assert t["fwd_threads"] in (64, 128, 256) and t["bwd_threads"] in (64, 128, 256)
    assert t["pair_warps"] in (2, 4, 8)
    assert all(s in (1, 2) for s in f + b) and f[3] == 1 and b[3] == 1
    assert batch.get_tune() == (t, f, b)
    o, g = run(batch, x)
    torch.cuda.synchronize()
    _check_against_single_robot(W, batch, robs, descs, problems, x, o, g, f, b, base)
    qs, qds, qdds, gps, gss, gms, gts = x["raw"]
    for p, (ri, H) in enumerate(problems[:6]):
        if H == 0:
            continue
        d = descs[ri]
        got = {k: v.cpu().numpy() for k, v in _per_problem(batch, o, g, p, d, H).items()
               if k != "g"}
        ref = O.evaluate(d, qs[p], qds[p], qdds[p])
        PY.check_forward(d, got, ref)
        gref = O.gradient(d, qs[p], qds[p], qdds[p], gps[p], gss[p], gms[p], gts[p])
        gg = [t_.cpu().numpy() for t_ in _per_problem(batch, o, g, p, d, H)["g"]]
        PY.check_gradient(gg, gref, mask=got["worst"] == ref["worst"])


def test_batch_set_tune_refusals(W):
    descs, robs, batch, problems = make_batch(W)
    for bad in (dict(fwd_threads=96), dict(bwd_threads=512), dict(pair_warps=9),
                dict(pair_warps=-1)):
        with pytest.raises(W.L.WbError) as ei:
            batch.set_tune(**bad)
        assert ei.value.code == W.L.WB_EINVAL
    with pytest.raises(W.L.WbError) as ei:  # the mimic robot has no 2-segment plan
        batch.set_tune(fwd_segments=[2, 2, 2, 2])
    assert ei.value.code == W.L.WB_EINVAL
    with pytest.raises(W.L.WbError):
        batch.set_tune(bwd_segments=[3, 1, 1, 1])
    # the defaults: 2 segments where a plan exists, 128 threads, the most pair warps
    batch.set_tune()
    t, f, b = batch.get_tune()
    assert (t["fwd_threads"], t["bwd_threads"], t["pair_warps"]) == (128, 128, 0)
    assert f == b == [2, 2, 2, 1]
