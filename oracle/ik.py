"""Conditional configuration sampler by parallel inverse kinematics, FP64
(oracle; test infrastructure only).

Sec. VI initialises particles by composing samplers: grasps (and placements)
are drawn first, then a configuration sampler solves inverse kinematics for the
joint positions that put the end effector at the target pose those draws
imply (the paper calls cuRobo's batched IK there).  This is the library's
reading of that step, written out plainly:

* Configurations are visited in skeleton order.  Each has one free yaw: a
  Pick's grasp yaw (the gripper may turn about its vertical approach axis) or a
  Place's placement yaw (the box may turn about the vertical on the surface).
  The target is T*(y) = P_box G(g) (the Kin constraint's target), with the
  free yaw y substituted.
* Damped least squares on r = [t* - t_EE ; log(R* R_EE^T)] (position error
  and rotation vector of the orientation error, world frame) over the unknowns
  (q, y): A = [J_q | -dr*/dy] with the geometric Jacobian columns
  J_i = [z_{i-1} x (t_EE - o_{i-1}) ; z_{i-1}] and
  dr*/dy = [z x (t* - c_box) ; z] for a Place (the box turns about its own
  vertical axis through its centre c_box) and [0 ; z] for a Pick;
  step = A^T (A A^T + lam^2 I)^-1 r, scaled down so its largest entry is at
  most dmax, then q is clamped to the joint limits.  ITERS steps.
* Everything else in the particle is left as sampled; later configurations
  see the yaws earlier ones chose.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import geometry as G
from .problem import DT, KNOT, PICK, Problem

ITERS, LAM, DMAX = 64, 0.05, 0.4


def log_rotation(R: torch.Tensor) -> torch.Tensor:
    """Rotation vector (axis * angle) of rotation matrices R [..., 3, 3].

    theta = atan2(|v|, (tr R - 1) / 2) with v = vee(R - R^T) / 2 (= sin theta *
    axis); at theta = pi, where v vanishes, the axis comes from the largest
    diagonal entry of (R + I) / 2 = axis axis^T."""
    v = 0.5 * torch.stack([R[..., 2, 1] - R[..., 1, 2], R[..., 0, 2] - R[..., 2, 0], R[..., 1, 0] - R[..., 0, 1]], -1)
    s = v.norm(dim=-1)
    c = 0.5 * (R[..., 0, 0] + R[..., 1, 1] + R[..., 2, 2] - 1.0)
    th = torch.atan2(s, c)
    out = torch.where((s > 1e-9)[..., None], v * (th / torch.clamp(s, min=1e-300))[..., None], v)
    B = 0.5 * (R + torch.eye(3, dtype=R.dtype))
    diag = torch.diagonal(B, dim1=-2, dim2=-1)
    k = diag.argmax(dim=-1)
    col = torch.gather(B, -1, k[..., None, None].expand(*k.shape, 3, 1))[..., 0]
    kk = torch.gather(diag, -1, k[..., None])[..., 0]
    axis = col / torch.sqrt(torch.clamp(kk, min=1e-300))[..., None]
    at_pi = (s <= 1e-9) & (c <= 0.0)
    return torch.where(at_pi[..., None], math.pi * axis, out)


def dls_step(arm: dict, q: torch.Tensor, y: torch.Tensor, target, lam: float = LAM, dmax: float = DMAX,
             q_lo=None, q_hi=None):
    """One damped-least-squares step for a batch: q [P, n], y [P];
    target(y) -> (T* [P, 4, 4], dt*/dy [P, 3]).  Returns (q, y, residual [P, 6])."""
    n = q.shape[1]
    frames = G.forward_kinematics(arm, q)
    ee = G.end_effector(arm, frames)
    p = ee[:, :3, 3]
    Tt, dt = target(y)
    r = torch.cat([Tt[:, :3, 3] - p, log_rotation(Tt[:, :3, :3] @ ee[:, :3, :3].transpose(-1, -2))], dim=1)
    A = torch.zeros(q.shape[0], 6, n + 1, dtype=DT)
    for i in range(n):
        z = frames[:, i, :3, 2]
        o = frames[:, i, :3, 3]
        A[:, :3, i] = torch.linalg.cross(z, p - o)
        A[:, 3:, i] = z
    A[:, :3, n] = -dt
    A[:, 5, n] = -1.0
    M = A @ A.transpose(1, 2) + lam * lam * torch.eye(6, dtype=DT)
    step = (A.transpose(1, 2) @ torch.linalg.solve(M, r[..., None]))[..., 0]
    m = step.abs().max(dim=1).values
    step = step * torch.where(m > dmax, dmax / m, torch.ones_like(m))[:, None]
    q = q + step[:, :n]
    if q_lo is not None:
        q = torch.maximum(torch.minimum(q, torch.as_tensor(q_hi, dtype=DT)), torch.as_tensor(q_lo, dtype=DT))
    return q, y + step[:, n], r


def _target_fn(pr: Problem, cfg, x: torch.Tensor):
    """T*(y) and dt*/dy of one configuration (see the module docstring)."""
    b = cfg["box"]
    go = cfg["g_off"]
    zvec = torch.tensor([0.0, 0.0, 1.0], dtype=DT)
    if cfg["kind"] == PICK:
        Pb = pr._box_pose(cfg["target"], b, x)

        def target(y):
            Gp = pr._grasp(x, go, yaw=y)
            return Pb @ Gp, torch.zeros(x.shape[0], 3, dtype=DT)
        return target, go + 3
    _, po, s = cfg["target"]
    Gp = pr._grasp(x, go)
    z = float(pr.sc.surf[s, 5] + pr.sc.box_half[b, 2])

    def target(y):
        Pb = G.box_pose(x[:, po], x[:, po + 1], torch.full_like(y, z), y)
        Tt = Pb @ Gp
        dt = torch.linalg.cross(zvec.expand(x.shape[0], 3), Tt[:, :3, 3] - Pb[:, :3, 3])
        return Tt, dt
    return target, po + 2


def ik_configurations(pr: Problem, X: np.ndarray, iters: int = ITERS, lam: float = LAM, dmax: float = DMAX,
                      keep: int = 0):
    """The configuration sampler on particles X [P, D]: returns a copy with
    every configuration's q and free yaw replaced by the IK result.

    ``keep``: components below it are a prefix reused from another skeleton's
    samples (Sec. VI, reusing samples across skeletons that share a constraint
    subgraph); configurations whose joints lie there keep their values and the
    later ones read them."""
    x = torch.as_tensor(np.array(X, dtype=np.float64))
    n = pr.n
    for cfg in pr.configs:
        qo = cfg["q_off"]
        if qo < keep or cfg["kind"] == KNOT:   # knots are interpolated, not solved
            continue
        target, yo = _target_fn(pr, cfg, x)
        q, y = x[:, qo:qo + n].clone(), x[:, yo].clone()
        for _ in range(iters):
            q, y, _ = dls_step(pr.arm, q, y, target, lam, dmax, pr.sc.q_lo, pr.sc.q_hi)
        x[:, qo:qo + n] = q
        x[:, yo] = y
    return x.numpy()
