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
