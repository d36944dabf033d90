"""FP32 work of the fused evaluation (cost + adjoint) and the Adam update.

Two figures:
  algorithmic_flops -- the method's work per particle-iteration, all sphere
      pairs evaluated forward (the paper's cost functions have no broad phase):
      forward kinematics 60 FLOP per joint, sphere transform 18 per sphere,
      sphere vs cuboid 32 per pair, sphere vs sphere 10 per pair, reverse sweep
      80 per joint, Adam 12 per component.  This is the roofline numerator.
  eval_flops / exact_flops -- what this kernel executes: the broad phase skips
      pairs that cannot touch, so it does a fraction of the algorithmic work.

FMA = 2 FLOP, add/mul/compare/max = 1; square roots, divisions and sines are
not counted, so the figures are lower bounds of the arithmetic done.

Fixed work per (particle, configuration) -- set by the scene and skeleton:
  forward kinematics            48 FLOP per joint (Rz, DH translation, Rx)
  reverse sweep                 69 FLOP per joint (inverse transforms 48, torque 21)
  sphere centres                18 FLOP per sphere (3x3 rotation + translation)
  wrench accumulation           15 FLOP per sphere
  held-box sphere into frame n  16 FLOP per sphere (G(g)^-1, tool)
  batch bounding sphere         18 FLOP per arm batch (table centre into the world),
                                80 FLOP per box batch (from its spheres)
  broad phase                   24 FLOP per (batch, cuboid)  (box-frame point 18, |u|-h 3, max 2, test 1)
                                10 FLOP per (batch, other box) (difference 3, norm^2 5, radius sum 1, test 1)
Data-dependent work (counted by the kernel, tamp_work_counters):
  exact cuboid test             40 FLOP per sphere of a candidate batch (point 18, q 3, clamp 3,
                                norm^2 5, test 1, gradient 10)
  exact sphere pair             11 FLOP per (batch sphere, box sphere) of a candidate
Per iteration and particle: 12 FLOP per sphere of every box on a placement
variable (its world centre), 12 FLOP per Adam component.

Trajectory knots (n_knots per motion between consecutive Pick/Place
configurations) are configurations without Kin: the arm, plus the held box on
a MoveHold, against the cuboids and every box not in the hand; each motion
adds TrajLength, 3n + 1 FLOP per polyline edge (difference, square sum, add)
and 2n per edge for its gradient.

SelfCollision (optional) per configuration: sphere vs sphere 10 FLOP per
tested pair (the arm's pairs on links i > j + 1 that do not touch at q = 0,
and the held box's spheres against links 0..n-2), plus one kinematic walk up
from every lower link (60 per joint step) and a reverse sweep (80 per joint).
"""
from __future__ import annotations

import math

FK_JOINT = 48
SWEEP_JOINT = 69
SPHERE_XFORM = 18
SPHERE_WRENCH = 15
HELD_SPHERE = 16
ARM_BOUND = 18
BOX_BOUND = 80
BROAD_OBB = 24
BROAD_BOX = 10
EXACT_OBB_SPHERE = 40
EXACT_PAIR = 11
ENV_SPHERE = 12
ADAM = 12
NB = 5


def _walk(scene, actions, n_knots: int = 0):
    """(kind, box, n_env, held) per configuration (kind 2: a knot; held: it
    carries a held box's spheres).  A Place's CFreePlace spheres are split with
    the Pick right before it."""
    B = scene.box_half.shape[0]
    out = []
    holding = False
    for kind, b, _s in actions:
        if kind not in (0, 1):
            continue
        if n_knots and out:
            out += [(2, -1, B - 1 if holding else B, holding)] * n_knots
        out.append((kind, b, B - 1, True))
        holding = kind == 0
    return out


def self_pairs(scene):
    """(arm sphere pairs, held-box sphere pairs) that SelfCollision tests:
    links i > j + 1 whose spheres do not overlap at q = 0 (standard DH at the
    joint offsets), and the box's spheres against the spheres of links 0..n-2."""
    import numpy as np
    n = scene.dh_a.shape[0]
    T = [np.asarray(scene.base, dtype=np.float64)]
    for j in range(n):
        th, al = scene.dh_offset[j], scene.dh_alpha[j]
        ct, st, ca, sa = math.cos(th), math.sin(th), math.cos(al), math.sin(al)
        A = np.array([[ct, -st * ca, st * sa, scene.dh_a[j] * ct], [st, ct * ca, -ct * sa, scene.dh_a[j] * st],
                      [0.0, sa, ca, scene.dh_d[j]], [0.0, 0.0, 0.0, 1.0]])
        T.append(T[-1] @ A)
    links = np.asarray(scene.sphere_link)
    xyz = np.asarray(scene.sphere_xyzr)[:, :3]
    r = np.asarray(scene.sphere_xyzr)[:, 3]
    c = np.stack([T[l][:3, :3] @ p + T[l][:3, 3] for l, p in zip(links, xyz)])
    touch = np.linalg.norm(c[:, None] - c[None], axis=-1) < r[:, None] + r[None]
    arm = 0
    for i in range(n + 1):
        for j in range(i - 1):
            a, b = links == i, links == j
            if a.any() and b.any() and not touch[np.ix_(a, b)].any():
                arm += int(a.sum()) * int(b.sum())
    held = int((links <= n - 2).sum()) * scene.box_spheres.shape[1]
    return arm, held


def self_collision_flops(scene, actions, n_knots: int = 0) -> int:
    """All-pairs FLOP of SelfCollision over one particle's configurations."""
    n = scene.dh_a.shape[0]
    arm, held = self_pairs(scene)
    total = 0
    for _kind, _b, _env, is_held in _walk(scene, actions, n_knots):
        total += (arm + (held if is_held else 0)) * 10 + (n * (n + 1) // 2) * 60 + n * 80
    return total


def _motions(actions, n_knots: int) -> int:
    return max(0, sum(1 for a in actions if a[0] in (0, 1)) - 1) if n_knots else 0


def eval_flops(scene, actions, n_knots: int = 0) -> int:
    """Fixed FLOP of one evaluation (cost + gradient) of one particle."""
    n = scene.dh_a.shape[0]
    links = list(scene.sphere_link)
    S = len(links)
    arm_batches = sum(int(math.ceil(links.count(l) / NB)) for l in range(n + 1))
    nbs = scene.box_spheres.shape[1]
    O = scene.obs_center.shape[0]
    cfgs = _walk(scene, actions, n_knots)
    total = 0
    n_place = 0
    for i, (kind, b, n_env, held) in enumerate(cfgs):
        held_batches = int(math.ceil(nbs / NB)) if held else 0
        if kind == 2:
            cp = 0
        elif kind == 1:
            half = nbs // 2 if i > 0 and cfgs[i - 1][0] == 0 and cfgs[i - 1][1] == b else 0
            cp = nbs - half
            n_place += 1
        else:
            nxt = cfgs[i + 1] if i + 1 < len(cfgs) else None
            cp = nbs // 2 if nxt is not None and nxt[0] == 1 and nxt[1] == b else 0
        place_batches = int(math.ceil(cp / NB))
        batches = arm_batches + held_batches + place_batches
        sph = S + (nbs if held else 0) + cp
        total += n * (FK_JOINT + SWEEP_JOINT)
        total += sph * (SPHERE_XFORM + SPHERE_WRENCH) + (nbs * HELD_SPHERE if held else 0)
        total += arm_batches * ARM_BOUND + (held_batches + place_batches) * BOX_BOUND
        total += batches * (O * BROAD_OBB + n_env * BROAD_BOX)
    total += n_place * nbs * ENV_SPHERE
    total += _motions(actions, n_knots) * (n_knots + 1) * 5 * n
    return total


def exact_flops(n_obb: int, n_box: int, nbs: int) -> int:
    """Data-dependent FLOP from the kernel's candidate counters."""
    return n_obb * NB * EXACT_OBB_SPHERE + n_box * NB * nbs * EXACT_PAIR


def algorithmic_flops(scene, actions, n_knots: int = 0) -> int:
    """All-pairs FLOP of one particle-iteration (evaluation, adjoint sweep, Adam)."""
    n = scene.dh_a.shape[0]
    S = len(scene.sphere_link)
    nbs = scene.box_spheres.shape[1]
    O = scene.obs_center.shape[0]
    total, D = 0, 0
    for kind, _b, n_env, held in _walk(scene, actions, n_knots):
        D += (4 if kind == 0 else (3 if kind == 1 else 0)) + n
        own = S + (nbs if held else 0)                 # arm (+ held box)
        total += n * 60 + own * 18 + own * O * 32 + own * nbs * n_env * 10 + n * 80
        if kind == 1:                                  # CFreePlace: the placed box
            total += nbs * 18 + nbs * O * 32 + nbs * nbs * n_env * 10
    total += _motions(actions, n_knots) * (n_knots + 1) * 5 * n
    return total + 12 * D


def adam_flops(D: int) -> int:
    return ADAM * D


def fp32_peak_tflops(sm_count: int = 148, sm_mhz: float = 2032.0) -> float:
    """FP32 CUDA-core peak: SMs x 128 FP32 lanes x 2 FLOP (FMA) x clock."""
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12
