"""GPU parity: the CUDA kernels against the FP64 oracle, element by element,
through the C ABI.  Sizes span several CTA tiles with a ragged tail; the
full-size workloads are checked on sampled configurations."""
import numpy as np
import pytest
import torch

from synthetic import configs as CF
from synthetic import inputs as I
from synthetic import robots as R
from tests import parity as PY

pytestmark = pytest.mark.gpu

ROBOTS = {"R7": R.r7, "R23": R.r23, "R48": R.r48, "mixed": R.mixed_joint_tree}


@pytest.fixture(scope="module")
def W():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2603_05493_gb300 import build
    build()
    from paper_2603_05493_gb300 import wbe
    return wbe


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


def kernels(W):
    return {"plain": W.PLAIN,
            "tree": W.TREE,
            "tree_nocull": W.TREE_NOCULL,
            "fused4": W.Tune(kernel=2, lanes_per_config=4),
            "fused8": W.Tune(kernel=2, lanes_per_config=8),
            "fused16": W.Tune(kernel=2, lanes_per_config=16),
            "fused32": W.Tune(kernel=2, lanes_per_config=32)}


KERNEL_NAMES = ["plain", "tree", "tree_nocull", "fused4", "fused8", "fused16", "fused32"]

_robots = {}


def robot(W, name):
    if name not in _robots:
        _robots[name] = (ROBOTS[name](), W.Robot(ROBOTS[name](), device=0))
    return _robots[name]


def cuda(x):
    return None if x is None else torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(o):
    return {k: (None if v is None else v.cpu().numpy()) for k, v in o.items()}


def run_fwd(rob, q, qd, qdd, tune, bits=False):
    o = rob.eval(cuda(q), cuda(qd), cuda(qdd), tune=tune, bits=bits)
    torch.cuda.synchronize()
    return host(o)


@pytest.mark.parametrize("rname", list(ROBOTS))
@pytest.mark.parametrize("kname", KERNEL_NAMES)
def test_forward_parity(W, O, rname, kname):
    desc, rob = robot(W, rname)
    B = 203 if rname != "R48" else 77  # several tiles and a ragged tail
    q, qd, qdd = I.uniform_states(desc.dof, B, seed=PY.stable_seed(rname, 1))
    got = run_fwd(rob, q, qd, qdd, kernels(W)[kname], bits=True)
    ref = O.evaluate(desc, q, qd, qdd)
    PY.check_forward(desc, got, ref)


@pytest.mark.parametrize("rname", list(ROBOTS))
@pytest.mark.parametrize("kname", KERNEL_NAMES)
def test_backward_parity(W, O, rname, kname):
    desc, rob = robot(W, rname)
    B = 19 if rname == "R48" else 45
    q, qd, qdd = I.uniform_states(desc.dof, B, seed=PY.stable_seed(rname, 2))
    gp, gs, gm, gt = I.upstream_grads(desc, B, seed=3)
    tune = kernels(W)[kname]
    o = rob.eval(cuda(q), cuda(qd), cuda(qdd), tune=tune)
    g = rob.eval_backward(cuda(q), cuda(qd), cuda(qdd), o["worst"], cuda(gp), cuda(gs),
                          cuda(gm), cuda(gt), tune=tune)
    torch.cuda.synchronize()
    ref = O.evaluate(desc, q, want=("dmin",))
    gref = O.gradient(desc, q, qd, qdd, gp, gs, gm, gt)
    same = o["worst"].cpu().numpy() == ref["worst"]
    assert same.mean() >= 0.9
    PY.check_gradient([x.cpu().numpy() for x in g], gref, mask=same)


@pytest.mark.parametrize("kname", KERNEL_NAMES)
@pytest.mark.parametrize("which", ["pose", "sph", "dmin", "tau"])
def test_backward_each_output_alone(W, O, kname, which):
    """Each upstream gradient on its own (the others NULL)."""
    desc, rob = robot(W, "mixed")
    B = 33
    q, qd, qdd = I.uniform_states(desc.dof, B, seed=9)
    gp, gs, gm, gt = I.upstream_grads(desc, B, seed=10, pose=which == "pose",
                                      sph=which == "sph", dmin=which == "dmin",
                                      tau=which == "tau")
    tune = kernels(W)[kname]
    o = rob.eval(cuda(q), cuda(qd), cuda(qdd), tune=tune)
    g = rob.eval_backward(cuda(q), cuda(qd), cuda(qdd), o["worst"], cuda(gp), cuda(gs),
                          cuda(gm), cuda(gt), tune=tune)
    torch.cuda.synchronize()
    gref = O.gradient(desc, q, qd, qdd, gp, gs, gm, gt)
    ref = O.evaluate(desc, q, want=("dmin",))
    same = o["worst"].cpu().numpy() == ref["worst"]
    PY.check_gradient([x.cpu().numpy() for x in g], gref, mask=same)


def test_small7_workload(W, O):
    """7-DoF chain, batch 64, forward FK + self-collision + RNEA."""
    desc, rob = robot(W, "R7")
    q, qd, qdd = I.uniform_states(desc.dof, CF.SMALL7.batch, CF.SMALL7.seed)
    for tune in kernels(W).values():
        got = run_fwd(rob, q, qd, qdd, tune, bits=True)
        PY.check_forward(desc, got, O.evaluate(desc, q, qd, qdd))


def _sample(B, k, seed):
    rng = np.random.default_rng(seed)
    s = np.unique(np.concatenate([[0, B - 1], rng.choice(B, k, replace=False)]))
    return s


def test_arm7_full_size_sampled(W, O):
    """7-DoF chain, 4096 x 32 configurations, default launch; sampled parity."""
    desc, rob = robot(W, "R7")
    B = CF.ARM7.batch
    q, qd, qdd = I.uniform_states(desc.dof, B, CF.ARM7.seed)
    got = run_fwd(rob, q, qd, qdd, None)
    s = _sample(B, 256, 1)
    ref = O.evaluate(desc, q[:, s], qd[:, s], qdd[:, s])
    PY.check_forward(desc, got, ref, sample=s)
    assert np.isfinite(got["tau"]).all() and np.isfinite(got["dmin"]).all()


def test_humanoid48_full_size_sampled(W, O):
    """48-DoF tree, 1024 x 32 configurations, forward + backward with the
    default launch; sampled parity."""
    desc, rob = robot(W, "R48")
    B = CF.HUMANOID48.batch
    q, qd, qdd = I.uniform_states(desc.dof, B, CF.HUMANOID48.seed)
    gp, gs, gm, gt = I.upstream_grads(desc, B, seed=CF.HUMANOID48.seed + 1)
    tq, tqd, tqdd = cuda(q), cuda(qd), cuda(qdd)
    o = rob.eval(tq, tqd, tqdd)
    g = rob.eval_backward(tq, tqd, tqdd, o["worst"], cuda(gp), cuda(gs), cuda(gm), cuda(gt))
    torch.cuda.synchronize()
    got = host(o)
    s = _sample(B, 40, 2)
    ref = O.evaluate(desc, q[:, s], qd[:, s], qdd[:, s])
    PY.check_forward(desc, got, ref, sample=s)
    gref = O.gradient(desc, q[:, s], qd[:, s], qdd[:, s], gp[s], gs[s], gm[s], gt[:, s])
    same = got["worst"][s] == ref["worst"]
    PY.check_gradient([x.cpu().numpy()[:, s] for x in g], gref, mask=same)
    for x in g:
        assert torch.isfinite(x).all()


def _bench_step_sample(B, block_configs, k, seed):
    """Sampled configurations of a full-size launch: the first and last 32
    (the first and last warp groups), the last sweep block's tail, the
    configurations on both sides of the first few block boundaries and k
    random ones."""
    rng = np.random.default_rng(seed)
    last_block = (B - 1) // block_configs * block_configs
    edges = [i * block_configs + o for i in range(1, 4) for o in (-1, 0)]
    s = np.concatenate([np.arange(32), np.arange(B - 32, B), np.arange(last_block, B), edges,
                        rng.choice(B, k, replace=False)])
    return np.unique(s[(s >= 0) & (s < B)])


@pytest.mark.parametrize("shape", ["autotuned", "fwd2x256_bwd2x448_pair4"])
def test_humanoid48_bench_step_parity(W, O, shape):
    """The humanoid48 step exactly as bench.py times it: 32768
    configurations, forward sweep, pair stage and backward sweep with the
    launch shapes bench.py takes (the library's autotuner at this batch, or
    the shapes it picked on GB300: forward 2 segments x 256 threads, backward
    2 segments x 448 threads = 147 blocks of 7 groups, 4 pair warps a block),
    through bench.py's own launch functions and on its inputs; >= 256 sampled
    configurations against the oracle (forward outputs and the three
    gradients)."""
    import bench
    desc, rob = robot(W, "R48")
    B = CF.HUMANOID48.batch
    if shape == "autotuned":
        shapes = bench.humanoid48_launch(rob, B)
    else:
        shapes = bench.humanoid48_launch(rob, B, sweep_shape="2,256,2,448")
        shapes["pair"] = W.Tune(kernel=3, blocks_per_sm=4)
    q, qd, qdd, gp, gs, gm, gt = bench.humanoid48_inputs(desc, 0, B)  # the bench's inputs
    out = rob.empty_outputs(B)
    out["diff"] = torch.empty((B, 3), device="cuda")  # as bench.py allocates it
    gout = tuple(torch.empty((desc.dof, B), device="cuda") for _ in range(3))
    bwd = shapes["bwd"]
    groups_per_block = max(1, bwd.configs_per_block // 32 // max(1, bwd.lanes_per_config))
    bench.humanoid48_step(rob, shapes, (cuda(q), cuda(qd), cuda(qdd)),
                          (cuda(gp), cuda(gs), cuda(gm), cuda(gt)), out, gout)
    torch.cuda.synchronize()
    got = host(out)
    s = _bench_step_sample(B, 32 * groups_per_block, 200, 12)
    assert len(s) >= 256
    ref = O.evaluate(desc, q[:, s], qd[:, s], qdd[:, s])
    PY.check_forward(desc, got, ref, sample=s)
    gref = O.gradient(desc, q[:, s], qd[:, s], qdd[:, s], gp[s], gs[s], gm[s], gt[:, s])
    same = got["worst"][s] == ref["worst"]
    assert same.mean() >= 0.95
    PY.check_gradient([x.cpu().numpy()[:, s] for x in gout], gref, mask=same)
    for x in gout:
        assert torch.isfinite(x).all()


def test_payload_via_set_inertials(W, O):
    """Runtime payload: 3 kg on each hand through wb_set_inertials."""
    desc = R.r48()
    loaded = I.hand_payload(desc)
    rob = W.Robot(desc, device=0)
    rob.set_inertials(loaded.mass, loaded.com, loaded.Icom, loaded.pm_link, loaded.pm_mass,
                      loaded.pm_pos)
    q, qd, qdd = I.uniform_states(desc.dof, 40, 77)
    got = run_fwd(rob, q, qd, qdd, None)
    PY.check_forward(loaded, got, O.evaluate(loaded, q, qd, qdd))
    base = O.evaluate(desc, q, qd, qdd, want=("tau",))
    assert np.abs(base["tau"] - got["tau"]).max() > 1.0  # the payload mattered


def test_edge_cases(W, O):
    desc, rob = robot(W, "R7")
    # B = 0 is a no-op
    z = torch.zeros((desc.dof, 0), device="cuda")
    o = rob.eval(z, z, z)
    assert o["dmin"].numel() == 0
    # B = 1
    q, qd, qdd = I.uniform_states(desc.dof, 1, 4)
    for tune in kernels(W).values():
        PY.check_forward(desc, run_fwd(rob, q, qd, qdd, tune, bits=True),
                         O.evaluate(desc, q, qd, qdd))
    # no pairs: d_min = +inf, worst = -1; forward without dynamics
    nop = desc.with_pairs(np.zeros((0, 2), np.int32))
    r0 = W.Robot(nop, device=0)
    q, qd, qdd = I.uniform_states(desc.dof, 50, 5)
    for tune in kernels(W).values():
        o = host(r0.eval(cuda(q), tau=False, tune=tune))
        assert np.isinf(o["dmin"]).all() and (o["worst"] == -1).all()
        PY.check_forward(nop, o, O.evaluate(nop, q, want=("pose", "sph")))


def test_joint_angles_far_from_zero(W, O):
    """The joint sine and cosine (a Cody-Waite reduction to [-pi, pi], then
    the fast intrinsic) stay within 1e-6 of the FP64 values of the same float
    angles up to |q| = 1e4 rad, multiples of pi / 2 included; link poses of
    the planar arm match the oracle there at the usual 1e-5."""
    desc = R.planar_2link()
    rob = W.Robot(desc, device=0)
    rng = np.random.default_rng(2024)
    half_pi = np.arange(-6366, 6367, 97) * (np.pi / 2)  # up to +-1e4 rad
    q1 = np.concatenate([np.linspace(-1e4, 1e4, 2001), half_pi, rng.uniform(-50, 50, 500),
                         [0.0, np.pi, -np.pi, 2 * np.pi, 4e4, -4e4]]).astype(np.float32)
    B = q1.size
    q = np.stack([q1, rng.uniform(-np.pi, np.pi, B).astype(np.float32)])
    ref = O.evaluate(desc, q.astype(np.float64), want=("pose",))
    c, s = np.cos(q1.astype(np.float64)), np.sin(q1.astype(np.float64))
    for tune in (W.TREE, W.PLAIN):
        o = host(rob.eval(cuda(q), tau=False, tune=tune))
        R0 = o["pose"][:, 0, :9]  # link 1: R_z(q1), row-major
        assert np.abs(R0[:, 0] - c).max() <= 1e-6 and np.abs(R0[:, 4] - c).max() <= 1e-6
        assert np.abs(R0[:, 3] - s).max() <= 1e-6 and np.abs(R0[:, 1] + s).max() <= 1e-6
        assert np.abs(o["pose"] - ref["pose"]).max() <= 1e-5


def test_exact_touching_and_ties(W, O):
    """Sliders with exact dyadic positions: touching spheres are not
    colliding, exact ties pick the smallest pair index."""
    n = 3
    desc = R._plain("sliders", [-1] * n, [R.PRISMATIC] * n, [[1, 0, 0]] * n,
                    [R._Tp(0, 0, 0)] * n, mass=[1.0] * n, com=np.zeros((n, 3)),
                    Icom=[[0.1, 0.1, 0.1, 0, 0, 0]] * n, sph_link=list(range(n)),
                    sph_c=np.zeros((n, 3)), sph_r=[0.25, 0.125, 0.5],
                    pairs=[[0, 1], [0, 2], [1, 2]])
    rob = W.Robot(desc, device=0)
    q = np.array([[0.0, 0.0, 0.0], [0.375, 0.375, 0.375], [2.0, 0.5, 1.0]], np.float32)
    for tune in kernels(W).values():
        o = host(rob.eval(cuda(q), cuda(np.zeros_like(q)), cuda(np.zeros_like(q)), tune=tune,
                          bits=True))
        assert list(o["dmin"]) == [0.0, -0.5, 0.0]
        assert list(o["worst"]) == [0, 2, 0]
        assert list(o["bits"][:, 0]) == [0, 0b110, 0]


def test_errors_are_reported(W):
    from paper_2603_05493_gb300 import _lib as L
    desc, rob = robot(W, "R7")
    q = torch.zeros((desc.dof, 8), device="cuda")
    with pytest.raises(L.WbError) as e:
        rob.eval(q.cpu(), tau=False)
    assert e.value.code == L.WB_EDEVICE
    big = torch.zeros(desc.dof * 8 + 1, device="cuda")
    with pytest.raises(L.WbError) as e:
        rob.eval(big[1:].view(desc.dof, 8), tau=False)
    assert e.value.code == L.WB_EINVAL
    with pytest.raises(L.WbError) as e:
        rob.eval(q, None, None, tau=True)
    assert e.value.code == L.WB_EINVAL
    with pytest.raises(L.WbError) as e:
        rob.eval(q, q, q, tune=W.Tune(kernel=2, lanes_per_config=5))
    assert e.value.code == L.WB_EINVAL
    # the tree path needs link_pose when spheres or pairs are wanted
    with pytest.raises(L.WbError) as e:
        rob.eval(q, q, q, pose=False, tune=W.TREE)
    assert e.value.code == L.WB_EINVAL
    # automatic choice falls back to the fused kernels then
    o = host(rob.eval(q, q, q, pose=False))
    assert np.isfinite(o["dmin"]).all()


@pytest.mark.parametrize("kname", ["default", "fused", "plain"])
def test_autograd_function(W, O, kname):
    """The torch.autograd.Function: the default path (sweep, then the pair
    stage handing the backward its worst-pair difference) and the fused and
    plain kernels, against the oracle's gradient."""
    desc, rob = robot(W, "R23")
    B = 24
    q, qd, qdd = I.uniform_states(desc.dof, B, 31)
    gp, gs, gm, gt = I.upstream_grads(desc, B, 32)
    tq, tqd, tqdd = (cuda(x).requires_grad_(True) for x in (q, qd, qdd))
    tune = {"default": None, "fused": W.FUSED, "plain": W.PLAIN}[kname]
    pose, sph, dmin, tau, worst = W.whole_body_eval(rob, tq, tqd, tqdd, tune=tune)
    loss = (pose * cuda(gp)).sum() + (sph * cuda(gs)).sum() + (dmin * cuda(gm)).sum() + \
        (tau * cuda(gt)).sum()
    loss.backward()
    gref = O.gradient(desc, q, qd, qdd, gp, gs, gm, gt)
    same = worst.cpu().numpy() == O.evaluate(desc, q, want=("dmin",))["worst"]
    PY.check_gradient([tq.grad.cpu().numpy(), tqd.grad.cpu().numpy(), tqdd.grad.cpu().numpy()],
                      gref, mask=same)


def test_deterministic(W):
    desc, rob = robot(W, "R48")
    q, qd, qdd = I.uniform_states(desc.dof, 300, 8)
    a = run_fwd(rob, q, qd, qdd, None)
    b = run_fwd(rob, q, qd, qdd, None)
    for k in a:
        if a[k] is not None:
            assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("rname", ["R48", "mixed"])
def test_self_collision_from_poses(W, O, rname):
    """Spheres and the pair map-reduce from given link poses (the split
    forward): same results as the oracle, bits included."""
    desc, rob = robot(W, rname)
    B = 131
    q, qd, qdd = I.uniform_states(desc.dof, B, seed=21)
    o = rob.eval(cuda(q), cuda(qd), cuda(qdd), sphere=False, dmin=False, tau=False,
                 tune=W.TREE)
    sc = host(rob.self_collision(o["pose"], bits=True))
    torch.cuda.synchronize()
    sc["pose"] = o["pose"].cpu().numpy()
    PY.check_forward(desc, sc, O.evaluate(desc, q, want=("pose", "sph", "dmin")))


def test_pair_stage_over_several_pass2_chunks(W, O):
    """The humanoid with every pair of links at least one joint apart masked
    in: 1224 pair blocks, 39 rounds of 32, so the culled kernel's pass 2 marks
    its survivors in two chunks of rounds (32 + 7) with the bounds kept as
    halves.  Against the oracle (pair bits included) and, d_min and the worst
    pair, bit for bit against the full map-reduce."""
    desc = R.r48(min_tree_dist=1)
    info, rounds = W.plan_info(desc)
    assert rounds[3] == 39  # lanes of 32: more than one chunk of 32 rounds
    rob = W.Robot(desc, device=0)
    B = 157
    q, qd, qdd = I.uniform_states(desc.dof, B, seed=44)
    o = rob.eval(cuda(q), cuda(qd), cuda(qdd), sphere=False, dmin=False, tau=False,
                 tune=W.TREE)
    ref = O.evaluate(desc, q, want=("pose", "sph", "dmin"))
    for bits in (True, False):
        sc = host(rob.self_collision(o["pose"], bits=bits, tune=W.TREE))
        full = host(rob.self_collision(o["pose"], bits=bits, tune=W.TREE_NOCULL))
        assert np.array_equal(sc["dmin"], full["dmin"]) and np.array_equal(sc["worst"], full["worst"])
        sc["pose"] = o["pose"].cpu().numpy()
        PY.check_forward(desc, sc, ref)


@pytest.mark.parametrize("rname", ["R7", "R48"])
def test_autotune_choice_is_valid_and_exact(W, O, rname, tmp_path):
    desc, rob = robot(W, rname)
    f, b, fm, bm = W.autotune_cached(rob, desc, 2048, path=str(tmp_path / "tune.json"))
    assert fm > 0 and bm > 0
    # cached on the second call
    f2, b2, _, _ = W.autotune_cached(rob, desc, 2048, path=str(tmp_path / "tune.json"))
    assert (f2, b2) == (f, b)
    B = 97
    q, qd, qdd = I.uniform_states(desc.dof, B, seed=61)
    gp, gs, gm, gt = I.upstream_grads(desc, B, seed=62)
    got = run_fwd(rob, q, qd, qdd, f)
    PY.check_forward(desc, got, O.evaluate(desc, q, qd, qdd))
    o = rob.eval(cuda(q), cuda(qd), cuda(qdd), tune=f)
    g = rob.eval_backward(cuda(q), cuda(qd), cuda(qdd), o["worst"], cuda(gp), cuda(gs), cuda(gm),
                          cuda(gt), tune=b)
    torch.cuda.synchronize()
    gref = O.gradient(desc, q, qd, qdd, gp, gs, gm, gt)
    same = o["worst"].cpu().numpy() == O.evaluate(desc, q, want=("dmin",))["worst"]
    PY.check_gradient([x.cpu().numpy() for x in g], gref, mask=same)


def _segments_available(desc, G):
    """The sweep kernels cut the depth-first order into G segments unless the
    robot has fewer links or a joint driving several links."""
    ji = [j for j in np.asarray(desc.jidx).tolist() if j >= 0]
    return G == 1 or (len(desc.parent) >= G and len(ji) == len(set(ji)))


@pytest.mark.parametrize("rname", list(ROBOTS))
@pytest.mark.parametrize("G,tpb", [(1, 0), (2, 0), (4, 0), (8, 0), (2, 512), (4, 512)])
def test_tree_segments_parity(W, O, rname, G, tpb):
    """Segmented depth-first sweeps (G warps per 32 configurations, shared
    ancestors' outputs summed across segments) against the oracle, forward
    and backward, on a ragged batch; also in 512-thread blocks (several
    groups of G warps sharing one block's staged link parameters)."""
    desc, rob = robot(W, rname)
    tune = W.Tune(kernel=3, lanes_per_config=G, configs_per_block=tpb)
    B = 77 if rname == "R48" else 203
    q, qd, qdd = I.uniform_states(desc.dof, B, seed=PY.stable_seed(rname, 5, G))
    if not _segments_available(desc, G):
        with pytest.raises(W.L.WbError) as ei:
            rob.eval(cuda(q), cuda(qd), cuda(qdd), tune=tune)
        assert ei.value.code == W.L.WB_EINVAL
        return
    got = run_fwd(rob, q, qd, qdd, tune)
    PY.check_forward(desc, got, O.evaluate(desc, q, qd, qdd))
    Bb = 45
    q, qd, qdd = q[:, :Bb].copy(), qd[:, :Bb].copy(), qdd[:, :Bb].copy()
    gp, gs, gm, gt = I.upstream_grads(desc, Bb, seed=G + 11)
    o = rob.eval(cuda(q), cuda(qd), cuda(qdd), tune=tune)
    g = rob.eval_backward(cuda(q), cuda(qd), cuda(qdd), o["worst"], cuda(gp), cuda(gs),
                          cuda(gm), cuda(gt), tune=tune)
    torch.cuda.synchronize()
    ref = O.evaluate(desc, q, want=("dmin",))
    gref = O.gradient(desc, q, qd, qdd, gp, gs, gm, gt)
    same = o["worst"].cpu().numpy() == ref["worst"]
    assert same.mean() >= 0.9
    PY.check_gradient([x.cpu().numpy() for x in g], gref, mask=same)
    # the same configurations through one thread per configuration: the
    # segments only change the order of the shared ancestors' sums
    g1 = rob.eval_backward(cuda(q), cuda(qd), cuda(qdd), o["worst"], cuda(gp), cuda(gs),
                           cuda(gm), cuda(gt), tune=W.Tune(kernel=3, lanes_per_config=1))
    torch.cuda.synchronize()
    for a, b in zip(g, g1):
        torch.testing.assert_close(a, b, rtol=1e-4, atol=1e-4 * float(b.abs().max()))


def test_one_segment_sweeps_refuse_512_threads(W):
    desc, rob = robot(W, "R7")
    q = cuda(np.zeros((desc.dof, 40)))
    with pytest.raises(W.L.WbError) as ei:
        rob.eval(q, q, q, tune=W.Tune(kernel=3, lanes_per_config=1, configs_per_block=512))
    assert ei.value.code == W.L.WB_EINVAL
    with pytest.raises(W.L.WbError) as ei:
        rob.eval(q, q, q, tune=W.Tune(kernel=3, lanes_per_config=2, configs_per_block=544))
    assert ei.value.code == W.L.WB_EINVAL


def test_maximum_size_robot(W, O):
    """The largest robot the library takes: 255 links, 1020 spheres, 32 tree
    levels (the sweep kernels' limit) and 330,624 masked pairs.  Forward
    (culled and full pair stage, with pair bits) and backward against the
    oracle on a ragged batch; the plain kernel refuses it; the pair kernel
    takes the 6 warps per block that fit in shared memory."""
    from paper_2603_05493_gb300 import _lib as L
    desc = R.max_size()
    assert (desc.n, desc.S, int(desc.depth().max()) + 1) == (255, 1020, 32)
    rob = W.Robot(desc, device=0)
    B = 45
    q, qd, qdd = I.uniform_states(desc.dof, B, seed=255)
    ref = O.evaluate(desc, q, qd, qdd)
    for tune in (W.TREE, W.TREE_NOCULL, None):
        PY.check_forward(desc, run_fwd(rob, q, qd, qdd, tune, bits=True), ref)
    with pytest.raises(L.WbError) as e:
        rob.eval(cuda(q), cuda(qd), cuda(qdd), tune=W.PLAIN)
    assert e.value.code == L.WB_ETOOBIG
    with pytest.raises(L.WbError) as e:  # 8 pair warps do not fit at this size
        rob.eval(cuda(q), cuda(qd), cuda(qdd), tune=W.Tune(kernel=3, blocks_per_sm=8))
    assert e.value.code == L.WB_ETOOBIG
    Bb = 7
    gp, gs, gm, gt = I.upstream_grads(desc, Bb, seed=256)
    o = rob.eval(cuda(q[:, :Bb]), cuda(qd[:, :Bb]), cuda(qdd[:, :Bb]))
    g = rob.eval_backward(cuda(q[:, :Bb]), cuda(qd[:, :Bb]), cuda(qdd[:, :Bb]), o["worst"],
                          cuda(gp), cuda(gs), cuda(gm), cuda(gt))
    torch.cuda.synchronize()
    gref = O.gradient(desc, q[:, :Bb], qd[:, :Bb], qdd[:, :Bb], gp, gs, gm, gt)
    same = o["worst"].cpu().numpy() == ref["worst"][:Bb]
    assert same.mean() >= 0.7
    PY.check_gradient([x.cpu().numpy() for x in g], gref, mask=same)
    # the summed hinge and the kinematics outputs at this size
    pose = o["pose"]
    cost, gsph = rob.self_collision_hinge(pose, 0.02, 1.0)
    rc, rg = O.pair_hinge(desc, q[:, :Bb], 0.02, 1.0)
    torch.cuda.synchronize()
    assert np.allclose(cost.cpu().numpy(), rc, rtol=1e-4, atol=1e-3)
    jac, com, jcom = rob.kinematics(pose, [desc.n - 1, 31])
    rJ, rcom, rJc = O.kinematics(desc, q[:, :Bb], [desc.n - 1, 31])
    torch.cuda.synchronize()
    assert np.abs(com.cpu().numpy() - rcom).max() <= 1e-4
    assert np.abs(jac.cpu().numpy() - rJ).max() <= 1e-4 * max(1.0, np.abs(rJ).max())
    assert np.abs(jcom.cpu().numpy() - rJc).max() <= 1e-4 * max(1.0, np.abs(rJc).max())


def test_too_large_robots_are_refused(W):
    """One link, one sphere or one tree level past the limits: the first two
    fail to load with WB_ETOOBIG; the 33-level chain loads, the tree kernels
    refuse it and the automatic choice runs the fused kernels."""
    from paper_2603_05493_gb300 import _lib as L
    big = R.max_size()
    from dataclasses import replace
    more_links = replace(big, parent=np.append(big.parent, 0), jtype=np.append(big.jtype, 1),
                         axis=np.vstack([big.axis, [[0, 0, 1]]]),
                         T_fixed=np.vstack([big.T_fixed, big.T_fixed[1:2]]),
                         jidx=np.append(big.jidx, big.dof), mimic_mult=np.append(big.mimic_mult, 1),
                         mimic_off=np.append(big.mimic_off, 0), mass=np.append(big.mass, 1),
                         com=np.vstack([big.com, [[0, 0, 0]]]),
                         Icom=np.vstack([big.Icom, big.Icom[1:2]]))
    with pytest.raises(L.WbError) as e:
        W.Robot(more_links, device=0)
    assert e.value.code == L.WB_ETOOBIG
    more_sph = replace(big, sph_link=np.append(big.sph_link, 1),
                       sph_c=np.vstack([big.sph_c, [[0, 0, 0]]]), sph_r=np.append(big.sph_r, 0.01))
    with pytest.raises(L.WbError) as e:
        W.Robot(more_sph, device=0)
    assert e.value.code == L.WB_ETOOBIG
    deep = R.deep_chain(33)
    rob = W.Robot(deep, device=0)
    q = torch.zeros((deep.dof, 40), device="cuda")
    with pytest.raises(L.WbError) as e:
        rob.eval(q, q, q, tune=W.TREE)
    assert e.value.code == L.WB_ETOOBIG
    o = rob.eval(q, q, q)
    torch.cuda.synchronize()
    assert torch.isfinite(o["tau"]).all()


@pytest.mark.parametrize("rname", ["R7", "R48", "mixed"])
def test_worst_diff_spares_the_backward_its_pair_kinematics(W, O, rname):
    """wb_self_collision_dir's worst-pair centre difference: c_i - c_j of the
    oracle's spheres for the reported pair, and wb_eval_backward_dir with it
    gives the tree kernels' gradients bit for bit as without it, for every
    segment count the robot takes."""
    desc, rob = robot(W, rname)
    B = 203
    q, qd, qdd = I.uniform_states(desc.dof, B, seed=PY.stable_seed(rname, 71))
    gp, gs, gm, gt = I.upstream_grads(desc, B, seed=72)
    tq, tqd, tqdd = cuda(q), cuda(qd), cuda(qdd)
    o = rob.eval(tq, tqd, tqdd, tune=W.TREE, sphere=False, dmin=False)
    c = rob.self_collision(o["pose"], diff=True)
    torch.cuda.synchronize()
    ref = O.evaluate(desc, q, qd, qdd, want=("sph", "dmin"))
    worst = c["worst"].cpu().numpy()
    i, j = desc.pairs[worst, 0], desc.pairs[worst, 1]
    want = ref["sph"][np.arange(B), i] - ref["sph"][np.arange(B), j]
    assert np.abs(c["diff"].cpu().numpy() - want).max() <= 2 * PY.POS_TOL
    for G in (1, 2, 4):
        if not _segments_available(desc, G):
            continue
        tune = W.Tune(kernel=3, lanes_per_config=G)
        args = (tq, tqd, tqdd, c["worst"], cuda(gp), cuda(gs), cuda(gm), cuda(gt))
        a = rob.eval_backward(*args, tune=tune)
        b = rob.eval_backward(*args, tune=tune, worst_diff=c["diff"])
        torch.cuda.synchronize()
        for x, y in zip(a, b):
            assert torch.equal(x, y), G
    # no pairs: a zero difference
    nop = desc.with_pairs(np.zeros((0, 2), np.int32))
    r0 = W.Robot(nop, device=0)
    c0 = r0.self_collision(o["pose"], diff=True)
    torch.cuda.synchronize()
    assert (c0["diff"] == 0).all() and (c0["worst"] == -1).all()
