"""Algorithmic FP32 work of one particle evaluation (cost + adjoint) and of one
Adam update, counted from a scene and a skeleton.

The counts are the arithmetic the definitions need per unit, with an FMA
counted as 2 FLOP and a compare/max as 1; square roots, divisions, sines and
the backward work of active (penetrating) pairs are data-dependent and not
counted, so the figure is a lower bound of the work done.

Per configuration (arm with n joints, S arm spheres, the held box's NBS spheres):
  forward kinematics           48 FLOP per joint (Rz, DH translation, Rx)
  reverse sweep                48 FLOP per joint (inverse transforms) + 21 (torque)
  sphere centres               18 FLOP per sphere (3x3 rotation + translation)
  wrench accumulation          15 FLOP per sphere
  sphere vs cuboid, forward    30 FLOP per pair (rotate 18, |u|-h 3, clamp 3, norm^2 5, test 1)
  sphere vs sphere, forward    11 FLOP per pair (difference 3, norm^2 5, radius sum/square 2, test 1)
  moving-box sphere centres     9 FLOP per environment sphere per register batch
Adam: 12 FLOP per component.
"""
from __future__ import annotations

import math

FK_JOINT = 48
SWEEP_JOINT = 48 + 21
SPHERE_XFORM = 18
SPHERE_WRENCH = 15
PAIR_OBB = 30
PAIR_SS = 11
ENV_SPHERE = 9
ADAM = 12
SB, HB = 5, 4


def _walk(scene, actions):
    """(kind, box, env boxes with 'moving' flags) per configuration, following the
    skeleton's effects (boxes placed earlier sit at placement variables)."""
    B = scene.box_half.shape[0]
    placed = [False] * B
    out = []
    for kind, b, _s in actions:
        if kind in (0, 1):
            env = [(j, placed[j]) for j in range(B) if j != b]
            out.append((kind, b, env))
            if kind == 1:
                placed[b] = True
    return out


def eval_flops(scene, actions) -> int:
    n = scene.dh_a.shape[0]
    links = list(scene.sphere_link)
    S_pad = sum(int(math.ceil(links.count(l) / SB)) * SB for l in range(n + 1))
    nbs = scene.box_spheres.shape[1]
    nbs_pad = int(math.ceil(nbs / HB)) * HB
    O = scene.obs_center.shape[0]
    total = 0
    for kind, b, env in _walk(scene, actions):
        sph = S_pad + nbs_pad + (nbs_pad if kind == 1 else 0)
        batches = S_pad // SB + nbs_pad // HB * (2 if kind == 1 else 1)
        env_sph = len(env) * nbs
        moving = sum(nbs for _j, mv in env if mv)
        total += n * (FK_JOINT + SWEEP_JOINT)
        total += sph * (SPHERE_XFORM + SPHERE_WRENCH)
        total += sph * O * PAIR_OBB + sph * env_sph * PAIR_SS
        total += batches * moving * ENV_SPHERE
    return total


def adam_flops(D: int) -> int:
    return ADAM * D


def fp32_peak_tflops(sm_count: int = 148, sm_mhz: float = 2032.0) -> float:
    """FP32 CUDA-core peak: SMs x 128 FP32 lanes x 2 FLOP (FMA) x clock."""
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12
