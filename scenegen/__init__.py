"""Seeded synthetic inputs for the particle-optimisation hot path.

This module only draws random numbers and packs them into the scene / skeleton /
particle layouts that the library's C ABI (``include/tamp.h``) documents.  It holds
none of the method's arithmetic: no kinematics, no signed distances, no costs, no
gradients, no optimiser.  Both the CUDA path (through its Python binding) and the
FP64 oracle consume what it returns; neither is imported here.

The paper's own scenes (Tetris blocks, bookshelf, stick button, Franka / UR5 /
Kinova sphere models) are not available, so every workload is synthetic, with the
shapes the paper's experiments use (7-DOF arms, box objects approximated by
spheres, oriented-cuboid obstacles, rectangular placement regions, pick-place
skeletons, batches of 256..65536 particles).

Conventions (metres, radians, z up):
  * the table top is the plane z = 0; the arm base frame is the world frame;
  * a box rests on a surface with its centre at z_top + h_z;
  * arm DH parameters follow the standard (distal) convention
    A_i = Rz(q_i + offset_i) Tz(d_i) Tx(a_i) Rx(alpha_i);
  * arm sphere k of link i sits on the segment between joint i's origin and joint
    i+1's origin, written in frame i (the frame at the distal end of link i);
    in frame i that segment runs from (-a_i, -d_i sin alpha_i, -d_i cos alpha_i)
    to the origin;
  * a box is modelled by 8 spheres of radius r = min(h) centred at
    (+-(h_x - r), +-(h_y - r), +-(h_z - r)) in the box frame;
  * an action is (kind, box, surface) with kind 0 = Pick, 1 = Place,
    2 = MinimizeObjDist (goal cost over every box moved so far).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PICK, PLACE, GOAL = 0, 1, 2


@dataclass
class Scene:
    """A synthetic scene; field names mirror ``tamp_scene_desc`` in include/tamp.h."""

    dh_a: np.ndarray
    dh_d: np.ndarray
    dh_alpha: np.ndarray
    dh_offset: np.ndarray
    q_lo: np.ndarray
    q_hi: np.ndarray
    base: np.ndarray          # [4,4]
    tool: np.ndarray          # [4,4]
    sphere_link: np.ndarray   # [S] int32, 1..n (frame index the sphere is fixed to)
    sphere_xyzr: np.ndarray   # [S,4] centre in that frame + radius
    box_half: np.ndarray      # [B,3]
    box_init: np.ndarray      # [B,4] x, y, z, yaw of the box centre
    box_spheres: np.ndarray   # [B,NBS,4] centre in the box frame + radius
    obs_center: np.ndarray    # [O,3]
    obs_rot: np.ndarray       # [O,3,3] columns = obstacle axes in world
    obs_half: np.ndarray      # [O,3]
    surf: np.ndarray          # [NS,6] cx, cy, yaw, hx, hy, z_top
    name: str = ""
    seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_joints(self) -> int:
        return int(self.dh_a.shape[0])

    @property
    def n_boxes(self) -> int:
        return int(self.box_half.shape[0])


def _rz3(yaw: float) -> np.ndarray:
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def random_arm(rng: np.random.Generator, n_joints: int = 7, spheres_per_link=5,
               r_range=(0.04, 0.08), q_limit: float = 2.8, min_twisted: int = 3):
    """Random serial revolute arm: a_i, d_i ~ U[0, 0.4] m, alpha_i in {0, +-pi/2}.

    Arms with fewer than ``min_twisted`` non-zero twists are redrawn: with almost
    all axes parallel the end effector cannot point down, and no top-down grasp
    could ever be reached.  ``spheres_per_link`` is an int or a per-link list.
    """
    while True:
        alpha = rng.choice(np.array([0.0, math.pi / 2, -math.pi / 2]), size=n_joints)
        if int(np.count_nonzero(alpha)) >= min_twisted:
            break
    a = rng.uniform(0.0, 0.4, n_joints)
    d = rng.uniform(0.0, 0.4, n_joints)
    if np.isscalar(spheres_per_link):
        spl = [int(spheres_per_link)] * n_joints
    else:
        spl = [int(v) for v in spheres_per_link]
    links, xyzr = [], []
    for i in range(n_joints):
        start = np.array([-a[i], -d[i] * math.sin(alpha[i]), -d[i] * math.cos(alpha[i])])
        n = spl[i]
        for k in range(n):
            t = (k + 0.5) / n
            links.append(i + 1)
            xyzr.append([*(start * (1.0 - t)), rng.uniform(*r_range)])
    return dict(
        dh_a=a, dh_d=d, dh_alpha=alpha, dh_offset=np.zeros(n_joints),
        q_lo=np.full(n_joints, -q_limit), q_hi=np.full(n_joints, q_limit),
        base=np.eye(4), tool=np.eye(4),
        sphere_link=np.array(links, dtype=np.int32), sphere_xyzr=np.array(xyzr),
    )


def box_sphere_model(half: np.ndarray) -> np.ndarray:
    """8 corner spheres of radius min(h) inside a box of half extents ``half``."""
    r = float(np.min(half))
    out = []
    for sx in (-1.0, 1.0):
        for sy in (-1.0, 1.0):
            for sz in (-1.0, 1.0):
                out.append([sx * (half[0] - r), sy * (half[1] - r), sz * (half[2] - r), r])
    return np.array(out)


def box_sphere_fill(half: np.ndarray, n_max: int = 8) -> np.ndarray:
    """Spheres of radius r = min(h) inside a box, centres on a grid over the box
    shrunk by r with spacing at most r per axis where the budget allows (axes
    of least extent give up spheres first); n_max slots, unused ones inert
    (radius -1 at the centre).  Unlike the 8-corner model this covers the long
    axis of an elongated box, so a thin strip actually blocks what sits on it."""
    half = np.asarray(half, dtype=float)
    r = float(half.min())
    ext = half - r
    counts = [1 if e <= 1e-9 else int(math.ceil(2.0 * e / r)) + 1 for e in ext]
    while int(np.prod(counts)) > n_max:
        cand = [a for a in range(3) if counts[a] > 1]
        a = min(cand, key=lambda a: ext[a])
        counts[a] -= 1
    axes = [np.linspace(-e, e, n) if n > 1 else np.zeros(1) for e, n in zip(ext, counts)]
    out = [[x, y, z, r] for x in axes[0] for y in axes[1] for z in axes[2]]
    out += [[0.0, 0.0, 0.0, -1.0]] * (n_max - len(out))
    return np.array(out)


def _polar(rng, r_lo, r_hi, ang_c=None, ang_w=math.pi):
    r = rng.uniform(r_lo, r_hi)
    ang = rng.uniform(-ang_w, ang_w) + (0.0 if ang_c is None else ang_c)
    return np.array([r * math.cos(ang), r * math.sin(ang)])


def _scatter(rng, n, radius_of, placed, sampler, tries=2000):
    """Rejection-sample n footprint centres whose bounding circles do not overlap."""
    out = []
    for i in range(n):
        rad = radius_of(i)
        for _ in range(tries):
            c = sampler()
            if all(np.hypot(*(c - pc)) > rad + pr for pc, pr in placed):
                break
        else:
            raise RuntimeError("scene generator: could not place item without overlap")
        placed.append((c, rad))
        out.append(c)
    return out


def make_scene(seed: int, n_boxes: int, n_obs: int, region_size, spheres_per_link=5,
               n_joints: int = 7, name: str = "", region_radius: float = 0.55,
               box_radius=(0.40, 0.85), obs_radius=(0.30, 1.15), obs_edges=(0.05, 0.30),
               arm_seed: int | None = None):
    """Pick-and-place scene: arm, ``n_boxes`` boxes on the table, ``n_obs`` cuboids,
    one rectangular target region (surface 0) on the table.  ``arm_seed`` fixes
    the arm independently of the rest of the scene (one robot, many scenes)."""
    rng = np.random.default_rng(seed)
    if arm_seed is None:
        arm = random_arm(rng, n_joints, spheres_per_link)
    else:
        arm = random_arm(np.random.default_rng(arm_seed), n_joints, spheres_per_link)
    half = rng.uniform(0.04, 0.10, size=(n_boxes, 3)) / 2.0
    reg_ang = rng.uniform(-math.pi, math.pi)
    reg_c = region_radius * np.array([math.cos(reg_ang), math.sin(reg_ang)])
    reg_yaw = rng.uniform(-math.pi, math.pi)
    reg_h = np.array(region_size, dtype=float) / 2.0
    placed = [(np.zeros(2), 0.22), (reg_c, float(np.hypot(*reg_h)) + 0.02)]
    box_xy = _scatter(rng, n_boxes, lambda i: float(np.hypot(*half[i, :2])) + 0.01, placed,
                      lambda: _polar(rng, *box_radius, ang_c=reg_ang + math.pi, ang_w=1.4))
    box_init = np.array([[c[0], c[1], half[i, 2], rng.uniform(-math.pi, math.pi)]
                         for i, c in enumerate(box_xy)]).reshape(n_boxes, 4)
    obs_half = rng.uniform(*obs_edges, size=(n_obs, 3)) / 2.0
    obs_xy = _scatter(rng, n_obs, lambda i: float(np.hypot(*obs_half[i, :2])) + 0.02, placed,
                      lambda: _polar(rng, *obs_radius))
    obs_center = np.array([[c[0], c[1], obs_half[i, 2]] for i, c in enumerate(obs_xy)]).reshape(n_obs, 3)
    obs_rot = np.stack([_rz3(rng.uniform(-math.pi, math.pi)) for _ in range(n_obs)]) if n_obs else np.zeros((0, 3, 3))
    surf = np.array([[reg_c[0], reg_c[1], reg_yaw, reg_h[0], reg_h[1], 0.0]])
    box_spheres = np.stack([box_sphere_model(h) for h in half])
    return Scene(**arm, box_half=half, box_init=box_init, box_spheres=box_spheres,
                 obs_center=obs_center, obs_rot=obs_rot, obs_half=obs_half, surf=surf,
                 name=name, seed=seed)


def pick_place_skeleton(box_order, surface: int = 0, goal: bool = False):
    """Pick(b) / Place(b, surface) for each box in order, optional goal action."""
    acts = []
    for b in box_order:
        acts.append((PICK, int(b), -1))
        acts.append((PLACE, int(b), int(surface)))
    if goal:
        acts.append((GOAL, -1, -1))
    return acts


# ---------------------------------------------------------------- named workloads

def plain_problem(seed: int = 1001):
    """One box, 4 cuboids, 0.6 x 0.4 m region, Pick-Place skeleton (D = 21)."""
    sc = make_scene(seed, n_boxes=1, n_obs=4, region_size=(0.6, 0.4), name="plain-1box")
    return sc, pick_place_skeleton([0])


def robot_plain_problem(seed: int, arm_seed: int = 4000):
    """The plain Pick-Place problem with one fixed arm across seeds: the scenes
    a learned proposal network for that robot trains and is tested on."""
    sc = make_scene(seed, n_boxes=1, n_obs=4, region_size=(0.6, 0.4), name="plain-1box-robot", arm_seed=arm_seed)
    return sc, pick_place_skeleton([0])


def robot_packing_problem(seed: int, arm_seed: int = 4000, n_boxes: int = 6):
    """The packing problem with the same fixed arm."""
    sc = make_scene(seed, n_boxes=n_boxes, n_obs=8, region_size=(0.3, 0.3), name="packing-robot",
                    arm_seed=arm_seed)
    return sc, pick_place_skeleton(range(n_boxes), goal=True)


def packing_problem(seed: int = 2001):
    """Six boxes packed into a 0.3 x 0.3 m region minimising the sum of pairwise
    centre distances, 8 cuboids, 6 Pick-Place pairs + goal (D = 126)."""
    sc = make_scene(seed, n_boxes=6, n_obs=8, region_size=(0.3, 0.3), name="packing-6box")
    return sc, pick_place_skeleton(range(6), goal=True)


def stress_problem(seed: int = 5001):
    """12 boxes, 64 cuboids, 100-sphere arm, 12 Pick-Place pairs (D = 252)."""
    spl = [15, 15, 14, 14, 14, 14, 14]
    sc = make_scene(seed, n_boxes=12, n_obs=64, region_size=(0.5, 0.5), spheres_per_link=spl,
                    name="stress-12box", box_radius=(0.45, 1.1), obs_radius=(0.3, 2.2),
                    obs_edges=(0.05, 0.20))
    return sc, pick_place_skeleton(range(12), goal=True)


def stacking_problem(seed: int = 3001, arm_seed: int | None = None):
    """Obstructed stacking: box A must go on box B, whose top face is fully
    covered by 2-4 blockers.  Surface 0 is B's top face, surface 1 a table
    region for the blockers; 16 static cuboids.  Returns (scene, skeletons,
    batch sizes): 16 candidate skeletons -- move 0, 1, 2 or 3 blockers (in
    every order, truncated to 16) to the table region, then Pick A / Place A on
    B -- of 2 to 8 actions, each with a batch size from {1024, 2048, 4096, 8192}."""
    import itertools
    rng = np.random.default_rng(seed)
    arm = random_arm(rng)
    if arm_seed is not None:
        arm = random_arm(np.random.default_rng(arm_seed))
    n_block = int(rng.integers(2, 5))
    hB = np.array([0.07, 0.07, 0.03])                      # B: 14 x 14 x 6 cm
    hA = rng.uniform(0.022, 0.03, 3)
    ang = rng.uniform(-math.pi, math.pi)
    Bxy = 0.6 * np.array([math.cos(ang), math.sin(ang)])
    Byaw = rng.uniform(-math.pi, math.pi)
    Axy = 0.6 * np.array([math.cos(ang + 0.8), math.sin(ang + 0.8)])
    reg_xy = 0.6 * np.array([math.cos(ang - 0.9), math.sin(ang - 0.9)])
    reg_h = np.array([0.15, 0.15])
    topB = 2 * hB[2]
    # blockers: strips across B's top (along B's x axis), each filling its strip
    halves = [hA, hB]
    init = [[Axy[0], Axy[1], hA[2], rng.uniform(-math.pi, math.pi)], [Bxy[0], Bxy[1], hB[2], Byaw]]
    c, s_ = math.cos(Byaw), math.sin(Byaw)
    w = 2 * hB[0] / n_block
    for i in range(n_block):
        hb = np.array([w / 2 - 0.001, hB[1] - 0.001, rng.uniform(0.02, 0.03)])
        lx = -hB[0] + w * (i + 0.5)
        halves.append(hb)
        init.append([Bxy[0] + c * lx, Bxy[1] + s_ * lx, topB + hb[2], Byaw])
    half = np.array(halves)
    box_init = np.array(init)
    placed = [(np.zeros(2), 0.22), (Bxy, 0.16), (Axy, 0.06), (reg_xy, float(np.hypot(*reg_h)) + 0.02)]
    n_obs = 16
    obs_half = rng.uniform(0.05, 0.25, size=(n_obs, 3)) / 2.0
    obs_xy = _scatter(rng, n_obs, lambda i: float(np.hypot(*obs_half[i, :2])) + 0.02, placed,
                      lambda: _polar(rng, 0.3, 1.4))
    obs_center = np.array([[q[0], q[1], obs_half[i, 2]] for i, q in enumerate(obs_xy)])
    obs_rot = np.stack([_rz3(rng.uniform(-math.pi, math.pi)) for _ in range(n_obs)])
    surf = np.array([[Bxy[0], Bxy[1], Byaw, hB[0], hB[1], topB],
                     [reg_xy[0], reg_xy[1], rng.uniform(-math.pi, math.pi), reg_h[0], reg_h[1], 0.0]])
    sc = Scene(**arm, box_half=half, box_init=box_init, box_spheres=np.stack([box_sphere_fill(h) for h in half]),
               obs_center=obs_center, obs_rot=obs_rot, obs_half=obs_half, surf=surf,
               name=f"stacking-{n_block}blockers", seed=seed, meta=dict(n_blockers=n_block))
    blockers = list(range(2, 2 + n_block))
    skels = []
    for k in range(0, min(3, n_block) + 1):
        for order in itertools.permutations(blockers, k):
            acts = []
            for b in order:
                acts += [(PICK, b, -1), (PLACE, b, 1)]
            acts += [(PICK, 0, -1), (PLACE, 0, 0)]
            skels.append(acts)
    skels = skels[:16]
    sizes = [int(v) for v in rng.choice([1024, 2048, 4096, 8192], size=len(skels))]
    return sc, skels, sizes


# ---------------------------------------------------------------- particle batches

def layout(actions, n_joints: int):
    """Variable blocks of one particle, in the order include/tamp.h documents:
    Pick -> grasp (x, y, z, yaw) then q; Place -> placement (x, y, yaw) then q;
    the goal action adds no variable.  Returns [(kind, box, offset, size)]."""
    out, off = [], 0
    for kind, box, _surf in actions:
        if kind == PICK:
            out.append(("grasp", box, off, 4)); off += 4
            out.append(("q", box, off, n_joints)); off += n_joints
        elif kind == PLACE:
            out.append(("place", box, off, 3)); off += 3
            out.append(("q", box, off, n_joints)); off += n_joints
    return out, off


def random_particles(scene: Scene, actions, n: int, seed: int, spread: float = 1.0):
    """[n, D] float64 particles drawn around the variables' natural bounds.

    Joint angles U[lo - 0.2, hi + 0.2]; grasp positions within the grasp box
    widened by 2 cm, yaw U[-pi, pi]; placements in the target region widened by
    5 cm (region frame, then rotated into the world), yaw U[-pi, pi].  ``spread``
    scales the widening margins.
    """
    rng = np.random.default_rng(seed)
    blocks, D = layout(actions, scene.n_joints)
    X = np.zeros((n, D))
    surf_of = {}
    for kind, box, s in actions:
        if kind == PLACE:
            surf_of[box] = s
    for kind, box, off, size in blocks:
        if kind == "q":
            m = 0.2 * spread
            X[:, off:off + size] = rng.uniform(scene.q_lo - m, scene.q_hi + m, size=(n, size))
        elif kind == "grasp":
            h = scene.box_half[box]
            m = 0.02 * spread
            lo = np.array([-h[0], -h[1], h[2] - 0.02]) - m
            hi = np.array([h[0], h[1], h[2]]) + m
            X[:, off:off + 3] = rng.uniform(lo, hi, size=(n, 3))
            X[:, off + 3] = rng.uniform(-math.pi, math.pi, n)
        elif kind == "place":
            cx, cy, yaw, hx, hy, _z = scene.surf[surf_of.get(box, 0)]
            m = 0.05 * spread
            u = rng.uniform(-hx - m, hx + m, n)
            v = rng.uniform(-hy - m, hy + m, n)
            c, s = math.cos(yaw), math.sin(yaw)
            X[:, off] = cx + c * u - s * v
            X[:, off + 1] = cy + s * u + c * v
            X[:, off + 2] = rng.uniform(-math.pi, math.pi, n)
    return X


def random_adam_state(n: int, D: int, seed: int):
    """First/second moment buffers and step counts for an Adam-step parity case."""
    rng = np.random.default_rng(seed)
    m = rng.normal(0.0, 1e-2, size=(n, D))
    v = rng.uniform(1e-8, 1e-3, size=(n, D))
    return m, v
