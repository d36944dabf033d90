"""Geometry and elementary costs in FP64 (oracle; test infrastructure only).

Every function takes torch float64 tensors with arbitrary leading batch dims.
Norms use the subgradient 0 at the origin (an autodiff convention the paper's
PyTorch costs share; reading "norm at zero" in the design notes).
"""
from __future__ import annotations

import math

import torch

DT = torch.float64


def norm(v: torch.Tensor, dim: int = -1) -> torch.Tensor:
    """Euclidean norm with derivative 0 at exactly the zero vector."""
    s = (v * v).sum(dim)
    pos = s > 0
    s_safe = torch.where(pos, s, torch.ones_like(s))
    return torch.where(pos, torch.sqrt(s_safe), torch.zeros_like(s))


# ------------------------------------------------------------------ rigid poses

def eye4(shape=()) -> torch.Tensor:
    return torch.eye(4, dtype=DT).expand(*shape, 4, 4).clone()


def translation(x, y, z) -> torch.Tensor:
    x, y, z = torch.broadcast_tensors(torch.as_tensor(x, dtype=DT), torch.as_tensor(y, dtype=DT),
                                      torch.as_tensor(z, dtype=DT))
    T = eye4(x.shape)
    T[..., 0, 3] = x
    T[..., 1, 3] = y
    T[..., 2, 3] = z
    return T


def rot_z(th) -> torch.Tensor:
    th = torch.as_tensor(th, dtype=DT)
    c, s = torch.cos(th), torch.sin(th)
    T = eye4(th.shape)
    T[..., 0, 0] = c
    T[..., 0, 1] = -s
    T[..., 1, 0] = s
    T[..., 1, 1] = c
    return T


def rot_y(be) -> torch.Tensor:
    be = torch.as_tensor(be, dtype=DT)
    c, s = torch.cos(be), torch.sin(be)
    T = eye4(be.shape)
    T[..., 0, 0] = c
    T[..., 0, 2] = s
    T[..., 2, 0] = -s
    T[..., 2, 2] = c
    return T


def rot_x(al) -> torch.Tensor:
    al = torch.as_tensor(al, dtype=DT)
    c, s = torch.cos(al), torch.sin(al)
    T = eye4(al.shape)
    T[..., 1, 1] = c
    T[..., 1, 2] = -s
    T[..., 2, 1] = s
    T[..., 2, 2] = c
    return T


def rigid_inverse(T: torch.Tensor) -> torch.Tensor:
    R = T[..., :3, :3]
    t = T[..., :3, 3]
    Ri = R.transpose(-1, -2)
    out = eye4(T.shape[:-2])
    out[..., :3, :3] = Ri
    out[..., :3, 3] = -(Ri @ t.unsqueeze(-1)).squeeze(-1)
    return out


def apply(T: torch.Tensor, p: torch.Tensor) -> torch.Tensor:
    """Transform points p[..., 3] by poses T[..., 4, 4] (broadcasting)."""
    return (T[..., :3, :3] @ p.unsqueeze(-1)).squeeze(-1) + T[..., :3, 3]


# ------------------------------------------------------------------ kinematics

def dh_transform(theta, d, a, alpha) -> torch.Tensor:
    """Standard (distal) DH joint transform Rz(theta) Tz(d) Tx(a) Rx(alpha)."""
    theta = torch.as_tensor(theta, dtype=DT)
    z = torch.zeros_like(theta)
    return rot_z(theta) @ translation(z, z, z + d) @ translation(z + a, z, z) @ rot_x(z + alpha)


def forward_kinematics(arm: dict, q: torch.Tensor) -> torch.Tensor:
    """Frames T_0..T_n of a serial revolute arm, [..., n+1, 4, 4].

    T_0 is the base; T_i = T_{i-1} A_i(q_i + offset_i).  The end effector is
    T_n composed with the tool transform (see ``end_effector``).  The paper's
    kinematics constraint compares FK(q) with the grasped object's target pose
    (Sec. III, "Kin"; Sec. V-A).
    """
    n = q.shape[-1]
    frames = [torch.as_tensor(arm["base"], dtype=DT).expand(*q.shape[:-1], 4, 4)]
    for i in range(n):
        A = dh_transform(q[..., i] + float(arm["dh_offset"][i]), float(arm["dh_d"][i]),
                         float(arm["dh_a"][i]), float(arm["dh_alpha"][i]))
        frames.append(frames[-1] @ A)
    return torch.stack(frames, dim=-3)


def end_effector(arm: dict, frames: torch.Tensor) -> torch.Tensor:
    return frames[..., -1, :, :] @ torch.as_tensor(arm["tool"], dtype=DT)


# ------------------------------------------------------------------ object poses

def box_pose(x, y, z, yaw) -> torch.Tensor:
    """Upright box pose Trans(x, y, z) Rz(yaw) (placements are 4-DOF, Sec. VIII)."""
    return translation(x, y, z) @ rot_z(yaw)


def grasp_pose(gx, gy, gz, gyaw) -> torch.Tensor:
    """Top-down 4-DOF grasp: end-effector pose in the object frame,
    Trans(g) Rz(yaw) Rx(pi) (the gripper's z axis points down)."""
    return translation(gx, gy, gz) @ rot_z(gyaw) @ rot_x(torch.full_like(torch.as_tensor(gx, dtype=DT), math.pi))


def grasp_pose6(gx, gy, gz, gyaw, groll, gpitch) -> torch.Tensor:
    """6-DOF grasp: Trans(g) Rz(yaw) Ry(pitch) Rx(roll) Rx(pi); zero roll and
    pitch give the top-down grasp."""
    return (translation(gx, gy, gz) @ rot_z(gyaw) @ rot_y(gpitch) @ rot_x(groll)
            @ rot_x(torch.full_like(torch.as_tensor(gx, dtype=DT), math.pi)))


# ------------------------------------------------------------------ distances

def box_sdf(c: torch.Tensor, center: torch.Tensor, R: torch.Tensor, half: torch.Tensor) -> torch.Tensor:
    """Signed distance from points c[..., 3] to an oriented box.

    u = R^T (c - t) is the point in the box frame, q = |u| - h; outside the
    distance is ||max(q, 0)||, inside it is max_i q_i (<= 0).
    """
    u = ((c - center).unsqueeze(-2) @ R).squeeze(-2)
    qv = u.abs() - half
    outside = norm(qv.clamp(min=0.0))
    inside = qv.amax(dim=-1).clamp(max=0.0)
    return outside + inside


def sphere_box_penetration(c, r, center, R, half) -> torch.Tensor:
    """max(0, r - sdf): depth by which a sphere enters a cuboid (0 when free)."""
    return (r - box_sdf(c, center, R, half)).clamp(min=0.0)


def sphere_sphere_penetration(ca, ra, cb, rb) -> torch.Tensor:
    """max(0, r_a + r_b - ||c_a - c_b||)."""
    return (ra + rb - norm(ca - cb)).clamp(min=0.0)


def dist_from_bounds(v: torch.Tensor, lo: torch.Tensor, hi: torch.Tensor) -> torch.Tensor:
    """Euclidean distance from the point v[..., d] to the axis-aligned box [lo, hi].

    The nearest point of the box is v with each coordinate clamped into its
    interval, so the distance is the norm of v minus that point (0 inside).
    The appendix scores joint limits (Motion), placement containment
    (StablePlace) and, in the library's reading, grasp bounds (Grasp) by this
    distance.
    """
    nearest = torch.minimum(torch.maximum(v, lo), hi)
    return norm(v - nearest)


def obj_dist(pos: torch.Tensor) -> torch.Tensor:
    """Sum over unordered pairs i < j of ||pos_i - pos_j|| for pos[..., n, 3]
    (appendix listing: the goal cost that pulls objects together)."""
    n = pos.shape[-2]
    total = torch.zeros(pos.shape[:-2], dtype=DT)
    for i in range(n):
        for j in range(i + 1, n):
            total = total + norm(pos[..., i, :] - pos[..., j, :])
    return total


def rotation_angle(R: torch.Tensor) -> torch.Tensor:
    """Geodesic angle of a rotation matrix: atan2(||vee(R - R^T)|| / 2, (tr R - 1) / 2)."""
    w = torch.stack([R[..., 2, 1] - R[..., 1, 2], R[..., 0, 2] - R[..., 2, 0],
                     R[..., 1, 0] - R[..., 0, 1]], dim=-1)
    s = 0.5 * norm(w)
    c = 0.5 * (R[..., 0, 0] + R[..., 1, 1] + R[..., 2, 2] - 1.0)
    return torch.atan2(s, c)


def pose_error(Ta: torch.Tensor, Tb: torch.Tensor):
    """(translation error in m, rotation error in rad) between two poses; the
    paper delegates this to cuRobo, whose formula it does not print."""
    e_pos = norm(Ta[..., :3, 3] - Tb[..., :3, 3])
    R = Ta[..., :3, :3].transpose(-1, -2) @ Tb[..., :3, :3]
    return e_pos, rotation_angle(R)
