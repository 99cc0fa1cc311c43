"""Seeded synthetic robots shaped like the paper's test robots.

The paper benchmarks a 7-DoF arm and a 48-DoF humanoid (Sec. 7.2, Sec. 7.3); their
robot description files are not available here, so these generators build
kinematic trees of the same shape from a seed.  This module only *creates input
data* (tree, joint axes, fixed transforms, collision spheres, the self-collision
pair mask, inertials).  It holds none of the evaluation arithmetic: no forward
kinematics, no distances, no dynamics.  Both the CUDA library and the CPU oracle
consume the arrays it returns.

Every floating-point parameter is rounded to a float32-representable value and
stored as float64, so the fp32 device copy and the fp64 oracle copy hold the
same numbers.

Conventions (shared with the C-ABI descriptor):
  parent[k]      index of the parent link, -1 for the world; parent[k] < k
  jtype[k]       0 fixed, 1 revolute, 2 prismatic
  axis[k]        unit joint axis in the link frame
  T_fixed[k]     12 numbers: rotation (row-major 3x3) then translation; the
                 pose of link k's joint frame in its parent's frame
  jidx[k]        actuated joint driving link k, -1 for fixed joints
  mimic_mult[k], mimic_off[k]
                 the joint variable of link k is mimic_mult*q[jidx] + mimic_off
  sph_link, sph_c, sph_r
                 collision spheres: link, centre in link frame, radius
  pairs          (P, 2) int32 sphere-index pairs, i < j, row-major sorted
  mass, com, Icom
                 per link inertials: mass, CoM in link frame, rotational
                 inertia about the CoM in link axes (xx, yy, zz, xy, xz, yz)
  pm_link, pm_mass, pm_pos
                 optional extra point masses (payloads) rigidly attached to a
                 link at a point given in that link's frame
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

FIXED, REVOLUTE, PRISMATIC = 0, 1, 2


def f32(x):
    """Round to float32-representable values, returned as float64."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


@dataclass
class Robot:
    name: str
    parent: np.ndarray
    jtype: np.ndarray
    axis: np.ndarray
    T_fixed: np.ndarray
    jidx: np.ndarray
    mimic_mult: np.ndarray
    mimic_off: np.ndarray
    gravity: np.ndarray
    sph_link: np.ndarray
    sph_c: np.ndarray
    sph_r: np.ndarray
    pairs: np.ndarray
    mass: np.ndarray
    com: np.ndarray
    Icom: np.ndarray
    pm_link: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int32))
    pm_mass: np.ndarray = field(default_factory=lambda: np.zeros(0))
    pm_pos: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))

    @property
    def n(self) -> int:
        return int(self.parent.shape[0])

    @property
    def dof(self) -> int:
        return int(self.jidx.max()) + 1 if (self.jidx >= 0).any() else 0

    @property
    def S(self) -> int:
        return int(self.sph_r.shape[0])

    @property
    def P(self) -> int:
        return int(self.pairs.shape[0])

    def with_pairs(self, pairs) -> "Robot":
        return replace(self, pairs=np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2))

    def with_point_masses(self, link, mass, pos) -> "Robot":
        return replace(self,
                       pm_link=np.asarray(link, np.int32).reshape(-1),
                       pm_mass=f32(np.asarray(mass).reshape(-1)),
                       pm_pos=f32(np.asarray(pos).reshape(-1, 3)))

    def depth(self) -> np.ndarray:
        d = np.zeros(self.n, np.int32)
        for k in range(self.n):
            d[k] = 0 if self.parent[k] < 0 else d[self.parent[k]] + 1
        return d


# --------------------------------------------------------------------------
# small helpers (input construction only)
# --------------------------------------------------------------------------

def _unit(rng) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def _rotation(rng) -> np.ndarray:
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _signed_permutation(rng) -> np.ndarray:
    """A random rotation from the 24 axis-aligned ones: exactly orthonormal in
    both float32 and float64."""
    while True:
        P = np.eye(3)[rng.permutation(3)] * rng.choice([-1.0, 1.0], size=3)
        if np.linalg.det(P) > 0:
            return P


def _box_inertia(rng, m) -> np.ndarray:
    """Inertia of a solid box of random dimensions, randomly rotated: SPD and
    satisfying the triangle inequality by construction."""
    a, b, c = rng.uniform(0.05, 0.3, size=3)
    lam = m / 12.0 * np.array([b * b + c * c, a * a + c * c, a * a + b * b])
    Q = _rotation(rng)
    I = Q @ np.diag(lam) @ Q.T
    return np.array([I[0, 0], I[1, 1], I[2, 2], I[0, 1], I[0, 2], I[1, 2]])


def tree_distance(parent: np.ndarray) -> np.ndarray:
    """Number of edges between every pair of links in the kinematic tree."""
    n = len(parent)
    depth = np.zeros(n, np.int64)
    for k in range(n):
        depth[k] = 0 if parent[k] < 0 else depth[parent[k]] + 1
    anc = [None] * n
    for k in range(n):
        anc[k] = ([k] + anc[parent[k]]) if parent[k] >= 0 else [k]
    D = np.zeros((n, n), np.int64)
    for a in range(n):
        sa = set(anc[a])
        for b in range(n):
            # lowest common ancestor = first ancestor of b that is also one of a
            lca = next((x for x in anc[b] if x in sa), None)
            if lca is None:       # different roots (a forest)
                D[a, b] = depth[a] + depth[b] + 2
            else:
                D[a, b] = depth[a] + depth[b] - 2 * depth[lca]
    return D


def mask_pairs(parent, sph_link, min_tree_dist) -> np.ndarray:
    """Sphere pairs (i < j, row-major sorted) whose links are at least
    `min_tree_dist` edges apart in the tree (the neighbour ignore rule)."""
    D = tree_distance(np.asarray(parent))
    L = np.asarray(sph_link)
    S = len(L)
    ii, jj = np.triu_indices(S, k=1)
    keep = D[L[ii], L[jj]] >= min_tree_dist
    return np.stack([ii[keep], jj[keep]], axis=1).astype(np.int32)


def _build(name, seed, parent, jtype, base_spheres, r_lo, r_hi, min_tree_dist,
           spheres_per_link=4, gravity=(0.0, 0.0, -9.81)):
    rng = np.random.default_rng(seed)
    parent = np.asarray(parent, np.int32)
    jtype = np.asarray(jtype, np.int32)
    n = len(parent)
    axis = np.zeros((n, 3))
    T = np.zeros((n, 12))
    jidx = -np.ones(n, np.int32)
    d = 0
    for k in range(n):
        T[k, 0:9] = np.eye(3).reshape(-1)
        if jtype[k] != FIXED:
            axis[k] = _unit(rng)
            jidx[k] = d
            d += 1
            T[k, 9:12] = rng.uniform(0.05, 0.4) * _unit(rng)
    # outgoing offset of each link: its first child's joint offset, or a fresh
    # random offset for leaves
    out = np.zeros((n, 3))
    for k in range(n):
        kids = [c for c in range(n) if parent[c] == k]
        out[k] = T[kids[0], 9:12] if kids else rng.uniform(0.05, 0.4) * _unit(rng)
    sl, sc, sr = [], [], []
    for k in range(n):
        if jtype[k] == FIXED:
            for _ in range(base_spheres):
                sl.append(k)
                sc.append(rng.uniform(-0.1, 0.1, size=3))
                sr.append(rng.uniform(r_lo, r_hi))
        else:
            for s in range(spheres_per_link):
                frac = (s + 0.5) / spheres_per_link
                sl.append(k)
                sc.append(frac * out[k] + rng.uniform(-0.01, 0.01, size=3))
                sr.append(rng.uniform(r_lo, r_hi))
    mass = rng.uniform(0.5, 3.0, size=n)
    com = np.zeros((n, 3))
    Icom = np.zeros((n, 6))
    for k in range(n):
        com[k] = rng.uniform(-0.05, 0.05, size=3) + 0.5 * out[k]
        Icom[k] = _box_inertia(rng, mass[k])
    sph_link = np.asarray(sl, np.int32)
    return Robot(
        name=name, parent=parent, jtype=jtype, axis=f32(axis), T_fixed=f32(T),
        jidx=jidx, mimic_mult=np.ones(n), mimic_off=np.zeros(n),
        gravity=f32(gravity), sph_link=sph_link, sph_c=f32(np.array(sc)),
        sph_r=f32(np.array(sr)),
        pairs=mask_pairs(parent, sph_link, min_tree_dist),
        mass=f32(mass), com=f32(com), Icom=f32(Icom))


def _chain(parent_of_first, length, start):
    """Parent indices for a serial chain of `length` links appended at index
    `start`, hanging from `parent_of_first`."""
    return [parent_of_first] + list(range(start, start + length - 1))


# --------------------------------------------------------------------------
# the robots
# --------------------------------------------------------------------------

def r7(seed: int = 7) -> Robot:
    """7-DoF serial revolute chain, fixed base, 4 spheres per link (S = 28),
    radii U(0.03, 0.08) m, pairs on links >= 2 apart (P = 240)."""
    parent = [-1] + list(range(6))
    return _build("R7", seed, parent, [REVOLUTE] * 7, 0, 0.03, 0.08, 2)


def humanoid_parents(arms: int, arm_len: int, legs: int, leg_len: int,
                     spine: int, neck: int, fingers: int, finger_len: int):
    """Parent list of a fixed-base humanoid-shaped tree.  Link 0 is the base
    (pelvis, fixed joint); spine hangs from the pelvis, neck and arms from the
    last spine link, legs from the pelvis, fingers from the last arm link."""
    parent = [-1]
    spine_ids = []
    p = 0
    for _ in range(spine):
        parent.append(p)
        p = len(parent) - 1
        spine_ids.append(p)
    top = spine_ids[-1] if spine_ids else 0
    p = top
    for _ in range(neck):
        parent.append(p)
        p = len(parent) - 1
    for _ in range(arms):
        p = top
        for _ in range(arm_len):
            parent.append(p)
            p = len(parent) - 1
        hand = p
        for _ in range(fingers):
            p = hand
            for _ in range(finger_len):
                parent.append(p)
                p = len(parent) - 1
    for _ in range(legs):
        p = 0
        for _ in range(leg_len):
            parent.append(p)
            p = len(parent) - 1
    return parent


def r48(seed: int = 48, min_tree_dist: int = 5) -> Robot:
    """48-DoF fixed-base humanoid-shaped tree: pelvis (8 spheres) -> spine 2 ->
    neck 2; two arms of 7 from the top of the spine; two legs of 6 from the
    pelvis; each hand has 3 fingers of 3 joints.  S = 200, radii
    U(0.02, 0.10) m, pairs on links >= 5 apart (P = 15,392)."""
    parent = humanoid_parents(arms=2, arm_len=7, legs=2, leg_len=6, spine=2, neck=2,
                              fingers=3, finger_len=3)
    jt = [FIXED] + [REVOLUTE] * (len(parent) - 1)
    return _build("R48", seed, parent, jt, 8, 0.02, 0.10, min_tree_dist)


def r23(seed: int = 23) -> Robot:
    """23-DoF tree: pelvis -> waist 1 -> two arms of 5; two legs of 6.  Same
    sphere rules as R48, pairs on links >= 2 apart."""
    parent = humanoid_parents(arms=2, arm_len=5, legs=2, leg_len=6, spine=1, neck=0,
                              fingers=0, finger_len=0)
    jt = [FIXED] + [REVOLUTE] * (len(parent) - 1)
    return _build("R23", seed, parent, jt, 8, 0.02, 0.10, 2)


def hand_links(robot: Robot) -> list:
    """Links that carry fingers: links with three or more children whose child
    subtrees are all serial chains (the two hands of R48)."""
    n = robot.n
    kids = [[c for c in range(n) if robot.parent[c] == k] for k in range(n)]

    def is_chain(k):
        while True:
            if len(kids[k]) > 1:
                return False
            if not kids[k]:
                return True
            k = kids[k][0]

    return [k for k in range(n) if len(kids[k]) >= 3 and all(is_chain(c) for c in kids[k])]


# --------------------------------------------------------------------------
# hand-built fixtures with closed forms
# --------------------------------------------------------------------------

def _plain(name, parent, jtype, axis, T, mass, com, Icom, sph_link, sph_c, sph_r,
           pairs=None, gravity=(0.0, 0.0, -9.81), mimic_mult=None, mimic_off=None):
    n = len(parent)
    jtype = np.asarray(jtype, np.int32)
    jidx = -np.ones(n, np.int32)
    d = 0
    for k in range(n):
        if jtype[k] != FIXED:
            jidx[k] = d
            d += 1
    sph_link = np.asarray(sph_link, np.int32)
    if pairs is None:
        pairs = np.zeros((0, 2), np.int32)
    return Robot(
        name=name, parent=np.asarray(parent, np.int32), jtype=jtype,
        axis=f32(np.asarray(axis, float).reshape(n, 3)),
        T_fixed=f32(np.asarray(T, float).reshape(n, 12)), jidx=jidx,
        mimic_mult=np.ones(n) if mimic_mult is None else f32(mimic_mult),
        mimic_off=np.zeros(n) if mimic_off is None else f32(mimic_off),
        gravity=f32(gravity), sph_link=sph_link,
        sph_c=f32(np.asarray(sph_c, float).reshape(-1, 3)),
        sph_r=f32(np.asarray(sph_r, float).reshape(-1)),
        pairs=np.asarray(pairs, np.int32).reshape(-1, 2),
        mass=f32(mass), com=f32(np.asarray(com, float).reshape(n, 3)),
        Icom=f32(np.asarray(Icom, float).reshape(n, 6)))


def _Tp(x, y, z):
    return [1, 0, 0, 0, 1, 0, 0, 0, 1, x, y, z]


def planar_2link(l1: float = 0.5, l2: float = 0.25) -> Robot:
    """Two revolute joints about z in the xy-plane.  Link 1 at the origin,
    link 2 offset by (l1, 0, 0); one sphere on link 2 at (l2, 0, 0) and one on
    link 1 at (l1/2, 0, 0)."""
    return _plain("planar2", [-1, 0], [REVOLUTE, REVOLUTE],
                  [[0, 0, 1], [0, 0, 1]], [_Tp(0, 0, 0), _Tp(l1, 0, 0)],
                  mass=[1.0, 1.0], com=[[l1 / 2, 0, 0], [l2 / 2, 0, 0]],
                  Icom=[[0.01, 0.01, 0.01, 0, 0, 0]] * 2,
                  sph_link=[0, 1], sph_c=[[l1 / 2, 0, 0], [l2, 0, 0]],
                  sph_r=[0.05, 0.05], pairs=[[0, 1]])


def pendulum(m: float = 2.0, l: float = 0.75, Ixx: float = 0.05) -> Robot:
    """Single revolute pendulum: axis x, CoM at (0, l, 0), gravity -z."""
    return _plain("pendulum", [-1], [REVOLUTE], [[1, 0, 0]], [_Tp(0, 0, 0)],
                  mass=[m], com=[[0, l, 0]], Icom=[[Ixx, 0.02, 0.03, 0, 0, 0]],
                  sph_link=[0], sph_c=[[0, l, 0]], sph_r=[0.05])


def chain_along_gravity(n: int = 4, seed: int = 3) -> Robot:
    """Serial revolute chain whose joint axes are all parallel to gravity (z):
    gravity does no work, so static torques vanish."""
    rng = np.random.default_rng(seed)
    T = [_Tp(*(rng.uniform(0.1, 0.3) * _unit(rng))) for _ in range(n)]
    Ic = [_box_inertia(rng, 1.0) for _ in range(n)]
    return _plain("zchain", [-1] + list(range(n - 1)), [REVOLUTE] * n,
                  [[0, 0, 1]] * n, T, mass=rng.uniform(0.5, 2, n),
                  com=rng.uniform(-0.1, 0.1, (n, 3)), Icom=Ic,
                  sph_link=list(range(n)), sph_c=np.zeros((n, 3)),
                  sph_r=[0.03] * n)


def mixed_joint_tree(seed: int = 11) -> Robot:
    """Small tree mixing revolute, prismatic and fixed joints with axis-aligned
    rotations in the fixed transforms and a mimic pair (link 5 follows joint of
    link 4 with multiplier -0.5 and an offset) - exercises every descriptor
    field."""
    rng = np.random.default_rng(seed)
    parent = [-1, 0, 1, 1, 3, 3, 2]
    jtype = [REVOLUTE, PRISMATIC, REVOLUTE, FIXED, REVOLUTE, REVOLUTE, REVOLUTE]
    n = len(parent)
    T = []
    for k in range(n):
        R = _signed_permutation(rng)
        p = rng.uniform(0.05, 0.3) * _unit(rng)
        T.append(list(R.reshape(-1)) + list(p))
    axis = [_unit(rng) for _ in range(n)]
    mass = rng.uniform(0.5, 2.0, n)
    Ic = [_box_inertia(rng, m) for m in mass]
    com = rng.uniform(-0.08, 0.08, (n, 3))
    sph_link = np.repeat(np.arange(n), 2)
    sph_c = rng.uniform(-0.1, 0.1, (2 * n, 3))
    sph_r = rng.uniform(0.02, 0.06, 2 * n)
    rob = _plain("mixed", parent, jtype, axis, T, mass, com, Ic, sph_link, sph_c, sph_r)
    # mimic: link 5 is driven by link 4's joint
    jidx = rob.jidx.copy()
    jidx[5] = jidx[4]
    jidx[6] = jidx[6] - 1
    mm = np.ones(n)
    mo = np.zeros(n)
    mm[5] = -0.5
    mo[5] = 0.1
    rob = replace(rob, jidx=jidx, mimic_mult=f32(mm), mimic_off=f32(mo))
    return rob.with_pairs(mask_pairs(parent, sph_link, 2))


def max_size(seed: int = 255, min_tree_dist: int = 24) -> Robot:
    """The largest robot the library accepts: 255 links (a fixed base with 4
    spheres and 254 revolute links: 8 chains of 31 and one of 6 hanging from
    the base), 1020 spheres (4 per link), 32 tree levels (the deepest tree the
    sweep kernels take); pairs on links >= `min_tree_dist` apart."""
    parent = [-1]
    for c in range(9):
        length = 31 if c < 8 else 6
        parent += _chain(0, length, len(parent))
    jtype = [FIXED] + [REVOLUTE] * (len(parent) - 1)
    return _build("max255", seed, parent, jtype, 4, 0.02, 0.06, min_tree_dist)


def deep_chain(n: int = 33, seed: int = 33) -> Robot:
    """A serial chain of n revolute links, 1 sphere each (one level deeper
    than the sweep kernels take when n = 33)."""
    parent = [-1] + list(range(n - 1))
    return _build("chain%d" % n, seed, parent, [REVOLUTE] * n, 0, 0.02, 0.05, 2,
                  spheres_per_link=1)


def get(name: str) -> Robot:
    return {"R7": r7, "R23": r23, "R48": r48}[name]()
