"""Pins of 6-DOF grasps in the FP64 oracle (Sec. VIII setup: grasps are
top-down 4-DOF or 6-DOF poses): the pose against scipy's Euler composition,
its top-down special case, a constructed particle with zero Kin terms, the
bound, and central finite differences (CPU)."""
import math

import numpy as np
import torch
from scipy.spatial.transform import Rotation

import scenegen as sg
from oracle import geometry as G
from oracle import philox
from oracle.problem import GRASP, KIN_POS, KIN_ROT, Options, Problem

from test_oracle_pins import _fd_error

DT = torch.float64


def test_pose_is_the_euler_composition_and_reduces_to_top_down():
    g = np.random.default_rng(0)
    x, y, z = (torch.tensor(g.normal(size=8)) for _ in range(3))
    yaw, roll, pitch = (torch.tensor(g.uniform(-3, 3, 8)) for _ in range(3))
    T = G.grasp_pose6(x, y, z, yaw, roll, pitch).numpy()
    R = (Rotation.from_euler("ZYX", np.stack([yaw, pitch, roll], 1)) * Rotation.from_euler("x", math.pi)).as_matrix()
    assert np.allclose(T[:, :3, :3], R, atol=1e-12)
    assert np.allclose(T[:, :3, 3], np.stack([x, y, z], 1), atol=1e-15)
    zero = torch.zeros(8, dtype=DT)
    assert torch.equal(G.grasp_pose6(x, y, z, yaw, zero, zero), G.grasp_pose(x, y, z, yaw))


def test_grasp_read_from_the_end_effector_satisfies_kin():
    # choose q, read G = P^-1 FK(q) and its angles with scipy: Kin is then zero
    sc, acts = sg.robot_plain_problem(20001)
    pr = Problem(sc, acts, Options(grasp_dof=6))
    X = philox.sample_uniform(pr, 16, 3)
    pick = pr.configs[0]
    q = torch.tensor(X[:, pick["q_off"]:pick["q_off"] + pr.n])
    ee = G.end_effector(pr.arm, G.forward_kinematics(pr.arm, q)).numpy()
    P = pr._box_pose(pick["target"], pick["box"], torch.tensor(X)).numpy()
    Gm = np.linalg.inv(P) @ ee
    Rg = Rotation.from_matrix(Gm[:, :3, :3]) * Rotation.from_euler("x", -math.pi)
    yaw, pitch, roll = Rg.as_euler("ZYX").T
    go = pick["g_off"]
    X[:, go:go + 3] = Gm[:, :3, 3]
    X[:, go + 3], X[:, go + 4], X[:, go + 5] = yaw, roll, pitch
    tv = pr.term_values(torch.tensor(X)).numpy()
    kin = [i for i, t in enumerate(pr.terms) if t.kind in (KIN_POS, KIN_ROT) and t.cfg == 0]
    assert np.abs(tv[:, kin]).max() < 1e-9


def test_six_dof_grasp_bound_is_the_whole_box():
    sc, acts = sg.robot_plain_problem(20001)
    pr = Problem(sc, acts, Options(grasp_dof=6))
    h = sc.box_half[0]
    X = philox.sample_uniform(pr, 3, 4)
    go = pr.configs[0]["g_off"]
    X[:, go:go + 3] = [[0.0, 0.0, -0.9 * h[2]], [h[0], -h[1], -h[2]], [h[0] + 0.03, 0.0, -h[2] - 0.04]]
    ti = next(i for i, t in enumerate(pr.terms) if t.kind == GRASP)
    v = pr.term_values(torch.tensor(X)).numpy()[:, ti]
    assert np.allclose(v, [0.0, 0.0, 0.05], atol=1e-12)
    # the uniform draws stay inside it, the angles in [-pi/2, pi/2)
    Y = philox.sample_uniform(pr, 256, 5)
    assert (np.abs(Y[:, go:go + 3]) <= h + 1e-12).all()
    assert (np.abs(Y[:, go + 4:go + 6]) <= math.pi / 2 + 1e-12).all()


def test_gradient_with_six_dof_grasps_matches_central_differences():
    sc, acts = sg.robot_packing_problem(21002, n_boxes=2)
    pr = Problem(sc, acts, Options(grasp_dof=6))
    x = torch.tensor(philox.sample_uniform(pr, 24, 6))
    x = x[pr.kink_margin(x) > 1e-4][:4]
    assert x.shape[0] >= 2
    assert _fd_error(pr, x) < 1e-6


def test_planted_mistakes_are_caught(monkeypatch):
    """Plausible slips in the 6-DOF grasp make one of the pins above fail."""
    import pytest
    orig = G.grasp_pose6

    # 1. Euler factors in the other order (roll before pitch)
    def swapped(gx, gy, gz, gyaw, groll, gpitch):
        return (G.translation(gx, gy, gz) @ G.rot_z(gyaw) @ G.rot_x(groll) @ G.rot_y(gpitch)
                @ G.rot_x(torch.full_like(torch.as_tensor(gx, dtype=DT), math.pi)))
    monkeypatch.setattr(G, "grasp_pose6", swapped)
    with pytest.raises(AssertionError):
        test_pose_is_the_euler_composition_and_reduces_to_top_down()
    with pytest.raises(AssertionError):
        test_grasp_read_from_the_end_effector_satisfies_kin()

    # 2. the gripper not flipped to point down
    def unflipped(gx, gy, gz, gyaw, groll, gpitch):
        return G.translation(gx, gy, gz) @ G.rot_z(gyaw) @ G.rot_y(gpitch) @ G.rot_x(groll)
    monkeypatch.setattr(G, "grasp_pose6", unflipped)
    with pytest.raises(AssertionError):
        test_grasp_read_from_the_end_effector_satisfies_kin()
    monkeypatch.setattr(G, "grasp_pose6", orig)
