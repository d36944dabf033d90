"""Pins of the IK configuration sampler (oracle/ik.py) against what the
mathematics fixes: the rotation log against scipy, the DLS matrix against
finite differences of the residual, convergence to targets reachable by
construction, and agreement of converged particles with the independent Kin
terms of oracle/problem.py (CPU only)."""
import math

import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import scenegen as sg
from oracle import geometry as G
from oracle import ik, philox
from oracle.problem import DT, KIN_POS, KIN_ROT, Problem


def test_log_rotation_matches_scipy_rotvec():
    g = np.random.default_rng(0)
    Rs = Rotation.random(200, random_state=1)
    mats = list(Rs.as_matrix())
    # near the identity and near / at a half turn
    for ang in (1e-12, 1e-6, math.pi - 1e-6, math.pi):
        ax = g.normal(size=3)
        ax /= np.linalg.norm(ax)
        mats.append(Rotation.from_rotvec(ang * ax).as_matrix())
    M = torch.tensor(np.array(mats), dtype=DT)
    w = ik.log_rotation(M).numpy()
    ref = Rotation.from_matrix(np.array(mats)).as_rotvec()
    for a, b in zip(w, ref):
        if np.linalg.norm(b) > math.pi - 1e-5:        # axis sign is free at a half turn
            assert min(np.abs(a - b).max(), np.abs(a + b).max()) < 1e-5
        else:
            assert np.abs(a - b).max() < 1e-9


def _residual(arm, q, y, target):
    frames = G.forward_kinematics(arm, q)
    ee = G.end_effector(arm, frames)
    Tt, _ = target(y)
    return torch.cat([Tt[:, :3, 3] - ee[:, :3, 3],
                      ik.log_rotation(Tt[:, :3, :3] @ ee[:, :3, :3].transpose(-1, -2))], dim=1)


@pytest.mark.parametrize("which", [0, 1])          # the Pick and the Place configuration
def test_dls_matrix_is_minus_the_residual_jacobian(which):
    # with lam -> 0 and a full-rank square-enough system, one step solves the
    # linearisation: r(q + dq, y + dy) ~ r - A step, so A = -dr/d(q, y).  Check A
    # column by column against central differences of the residual.
    sc, acts = sg.robot_plain_problem(20001)
    pr = Problem(sc, acts)
    X = torch.tensor(philox.sample_uniform(pr, 3, 8))
    if which == 1:                                   # place after an IK'd pick
        X = torch.tensor(ik.ik_configurations(pr, X.numpy()[:, :], iters=8))
    cfg = pr.configs[which]
    target, yo = ik._target_fn(pr, cfg, X)
    q0, y0 = X[:, cfg["q_off"]:cfg["q_off"] + pr.n], X[:, yo]
    # A written out from the definition, independently of dls_step
    n = pr.n
    frames = G.forward_kinematics(pr.arm, q0)
    p = G.end_effector(pr.arm, frames)[:, :3, 3]
    A = torch.zeros(3, 6, n + 1, dtype=DT)
    for i in range(n):
        z, o = frames[:, i, :3, 2], frames[:, i, :3, 3]
        A[:, :3, i] = torch.linalg.cross(z, p - o)
        A[:, 3:, i] = z
    _, dt = target(y0)
    A[:, :3, n] = -dt
    A[:, 5, n] = -1.0
    h = 1e-6
    for j in range(n + 1):
        dq = torch.zeros_like(q0)
        dy = torch.zeros_like(y0)
        if j < n:
            dq[:, j] = h
        else:
            dy[:] = h
        fd = (_residual(pr.arm, q0 + dq, y0 + dy, target) - _residual(pr.arm, q0 - dq, y0 - dy, target)) / (2 * h)
        # position rows; the rotation rows (the joint axes and z) equal the
        # derivative of the rotation log only at zero error, so they are pinned
        # by the exact convergence test below instead
        assert torch.allclose(-A[:, :3, j], fd[:, :3], atol=1e-6)
    # and the steps use exactly this A
    q1, y1, r = ik.dls_step(pr.arm, q0, y0, target, lam=ik.LAM, dmax=1e9)
    M = A @ A.transpose(1, 2) + ik.LAM ** 2 * torch.eye(6, dtype=DT)
    step = (A.transpose(1, 2) @ torch.linalg.solve(M, r[..., None]))[..., 0]
    assert torch.allclose(q1 - q0, step[:, :n], atol=1e-12) and torch.allclose(y1 - y0, step[:, n], atol=1e-12)


def test_converges_to_a_target_reachable_by_construction():
    # T*(y) = Rz(y) FK(q*): the whole target turns about the world z axis
    # (dt*/dy = z x t*, rotation derivative z); started near (q*, 0) the
    # iteration must reach it exactly
    sc, _ = sg.robot_plain_problem(20002)
    arm = dict(base=sc.base, tool=sc.tool, dh_a=sc.dh_a, dh_d=sc.dh_d, dh_alpha=sc.dh_alpha, dh_offset=sc.dh_offset)
    g = np.random.default_rng(3)
    qs = torch.tensor(g.uniform(-2.0, 2.0, (16, 7)))
    T0 = G.end_effector(arm, G.forward_kinematics(arm, qs))
    zvec = torch.tensor([0.0, 0.0, 1.0], dtype=DT)

    def target(y):
        Tt = G.rot_z(y) @ T0
        return Tt, torch.linalg.cross(zvec.expand(16, 3), Tt[:, :3, 3])
    q = qs + torch.tensor(g.normal(0, 0.15, (16, 7)))
    y = torch.tensor(g.normal(0, 0.2, 16))
    for _ in range(60):
        q, y, r = ik.dls_step(arm, q, y, target, lam=1e-3, dmax=0.4)
    _, _, r = ik.dls_step(arm, q, y, target, lam=1e-3, dmax=0.4)
    assert r.abs().max() < 1e-9
    # the independent FK agrees: FK(q) = Rz(y) FK(q*)
    T = G.end_effector(arm, G.forward_kinematics(arm, q))
    assert torch.allclose(T, G.rot_z(y) @ T0, atol=1e-8)


def test_converged_particles_satisfy_the_kin_terms():
    # the sampler's target is the Kin constraint's target: particles whose IK
    # residual vanished must have zero Kin terms in oracle/problem.py
    sc, acts = sg.robot_plain_problem(20003)
    pr = Problem(sc, acts)
    X0 = philox.sample_uniform(pr, 96, 4)
    X = ik.ik_configurations(pr, X0, iters=120, lam=0.02)
    tv = pr.term_values(torch.tensor(X)).numpy()
    kin = [j for j, t in enumerate(pr.terms) if t.kind in (KIN_POS, KIN_ROT)]
    ok = (tv[:, kin] < 1e-6).all(axis=1)
    assert ok.mean() > 0.3, ok.mean()
    # uniform seeds essentially never satisfy Kin
    tv0 = pr.term_values(torch.tensor(X0)).numpy()
    assert (tv0[:, kin] < 1e-3).all(axis=1).mean() == 0.0
    # only the configurations and the free yaws moved; joint limits hold
    kinds = np.array(pr.kinds)
    moved = np.abs(X - X0).max(axis=0) > 0
    assert set(kinds[moved]) <= {"q", "gyaw", "pyaw"}
    q = kinds == "q"
    assert (X[:, q] >= -2.8 - 1e-12).all() and (X[:, q] <= 2.8 + 1e-12).all()


def test_kept_prefix_stays_and_later_configurations_are_solved():
    # subgraph caching (Sec. VI): the components of a prefix reused from another
    # skeleton's samples stay as they are; the configurations after it are
    # solved against their own targets, reading the prefix's grasps and yaws
    sc, acts = sg.robot_packing_problem(21002, n_boxes=2)
    pr = Problem(sc, acts)
    k = pr.configs[1]["q_off"] + pr.n            # components of (Pick 0, Place 0)
    src = ik.ik_configurations(pr, philox.sample_uniform(pr, 64, 5), iters=120, lam=0.02)
    X0 = philox.sample_uniform(pr, 64, 6)
    X0[:, :k] = src[:, :k]
    X = ik.ik_configurations(pr, X0, iters=120, lam=0.02, keep=k)
    assert np.array_equal(X[:, :k], X0[:, :k])
    tv = pr.term_values(torch.tensor(X)).numpy()
    later = [j for j, t in enumerate(pr.terms) if t.kind in (KIN_POS, KIN_ROT) and t.action >= 2]
    earlier = [j for j, t in enumerate(pr.terms) if t.kind in (KIN_POS, KIN_ROT) and t.action < 2]
    rate = (tv[:, later] < 1e-6).all(axis=1).mean()
    # as often as when the whole particle is solved from the same draws
    plain = pr.term_values(torch.tensor(ik.ik_configurations(pr, X0, iters=120, lam=0.02))).numpy()
    assert rate > 0.15 and rate >= 0.8 * (plain[:, later] < 1e-6).all(axis=1).mean(), rate
    # the kept prefix still satisfies Kin where the source's IK did
    tv_src = pr.term_values(torch.tensor(src)).numpy()
    assert np.array_equal(tv[:, earlier] < 1e-6, tv_src[:, earlier] < 1e-6)
    # keep = 0 is the plain sampler, keep = D leaves everything
    assert np.array_equal(ik.ik_configurations(pr, X0, iters=3, keep=0), ik.ik_configurations(pr, X0, iters=3))
    assert np.array_equal(ik.ik_configurations(pr, X0, iters=3, keep=pr.D), X0)
