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
  contact-test preparation      8 FLOP per sphere ((|c|^2 - r^2) / 2)
  wrench accumulation          15 FLOP per sphere
  held-box sphere into frame n 16 FLOP per sphere (G(g)^-1, tool)
  sphere vs cuboid test        24 FLOP per pair (box-frame point 18, |u| - h 3, max 2, compare 1)
  sphere vs sphere test         9 FLOP per pair (c_a.c_b + r_a r_b - hb: 4 FMA, compare 1)
Per iteration and particle: 17 FLOP per sphere of every box standing on a
placement variable (world centre and (|c|^2 - r^2) / 2).
Adam: 12 FLOP per component.
"""
from __future__ import annotations

import math

FK_JOINT = 48
SWEEP_JOINT = 48 + 21
SPHERE_XFORM = 18
SPHERE_PREP = 8
SPHERE_WRENCH = 15
HELD_SPHERE = 16
PAIR_OBB = 24
PAIR_SS = 9
ENV_SPHERE = 17
ADAM = 12


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
    S = len(scene.sphere_link)              # real spheres only: padding slots are overhead
    nbs = scene.box_spheres.shape[1]
    O = scene.obs_center.shape[0]
    total = 0
    n_place = 0
    for kind, b, env in _walk(scene, actions):
        sph = S + nbs + (nbs if kind == 1 else 0)
        env_sph = len(env) * nbs
        total += n * (FK_JOINT + SWEEP_JOINT)
        total += sph * (SPHERE_XFORM + SPHERE_PREP + SPHERE_WRENCH) + nbs * HELD_SPHERE
        total += sph * O * PAIR_OBB + sph * env_sph * PAIR_SS
        n_place += kind == 1
    total += n_place * nbs * ENV_SPHERE
    return total


def adam_flops(D: int) -> int:
    return ADAM * D


def fp32_peak_tflops(sm_count: int = 148, sm_mhz: float = 2032.0) -> float:
    """FP32 CUDA-core peak: SMs x 128 FP32 lanes x 2 FLOP (FMA) x clock."""
    return sm_count * 128 * 2 * sm_mhz * 1e6 / 1e12
