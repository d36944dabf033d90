"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Closed forms (planar/SCARA kinematics, the textbook DH matrix, the Adam first
step), hand values (tests/golden/), brute force (box distance from dense surface
samples, constraint counts by explicit loops), library routines (scipy rotation
angles, scipy convex-hull containment), invariances (rigid motion of the whole
scene), constructed satisfying particles, and central finite differences.  The
mutation tests at the end plant plausible mistakes in the oracle and check that
one of these pins catches each of them.
"""
import dataclasses
import json
import math
import os

import numpy as np
import pytest
import torch

import scenegen as sg
from oracle import geometry as G
from oracle import philox
from oracle.problem import (CFREE_HOLD, CFREE_PLACE, GRASP, JOINT_LIMIT, KIN_POS, KIN_ROT,
                            OBJ_DIST, STABLE_PLACE, Options, Problem)

GOLD = os.path.join(os.path.dirname(__file__), "golden")
DT = torch.float64


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ------------------------------------------------------------------ kinematics

def _planar_arm(a):
    n = len(a)
    return dict(base=np.eye(4), tool=np.eye(4), dh_a=np.array(a), dh_d=np.zeros(n),
                dh_alpha=np.zeros(n), dh_offset=np.zeros(n))


def _fk_planar_error():
    rng = np.random.default_rng(0)
    a1, a2 = 0.37, 0.21
    q = torch.tensor(rng.uniform(-3, 3, size=(64, 2)))
    ee = G.end_effector(_planar_arm([a1, a2]), G.forward_kinematics(_planar_arm([a1, a2]), q))
    t1, t2 = q[:, 0], q[:, 1]
    x = a1 * torch.cos(t1) + a2 * torch.cos(t1 + t2)
    y = a1 * torch.sin(t1) + a2 * torch.sin(t1 + t2)
    err = max(float((ee[:, 0, 3] - x).abs().max()), float((ee[:, 1, 3] - y).abs().max()),
              float(ee[:, 2, 3].abs().max()))
    yaw = torch.atan2(ee[:, 1, 0], ee[:, 0, 0])
    dyaw = torch.remainder(yaw - (t1 + t2) + math.pi, 2 * math.pi) - math.pi
    return max(err, float(dyaw.abs().max()))


def test_fk_planar_two_link_closed_form():
    assert _fk_planar_error() < 1e-13


def test_fk_scara_yaw_is_sum_of_angles():
    rng = np.random.default_rng(1)
    arm = _planar_arm(rng.uniform(0, 0.4, 7))
    arm["dh_d"] = rng.uniform(0, 0.4, 7)
    q = torch.tensor(rng.uniform(-2.8, 2.8, size=(32, 7)))
    ee = G.end_effector(arm, G.forward_kinematics(arm, q))
    phi = torch.cumsum(q, dim=1)
    x = (torch.tensor(arm["dh_a"]) * torch.cos(phi)).sum(1)
    y = (torch.tensor(arm["dh_a"]) * torch.sin(phi)).sum(1)
    assert torch.allclose(ee[:, 0, 3], x, atol=1e-13) and torch.allclose(ee[:, 1, 3], y, atol=1e-13)
    assert torch.allclose(ee[:, 2, 3], torch.full_like(x, arm["dh_d"].sum()), atol=1e-13)
    Rz = G.rot_z(phi[:, -1])[:, :3, :3]
    assert torch.allclose(ee[:, :3, :3], Rz, atol=1e-13)


def _textbook_dh(theta, d, a, alpha):
    ct, st, ca, sa = math.cos(theta), math.sin(theta), math.cos(alpha), math.sin(alpha)
    return np.array([[ct, -st * ca, st * sa, a * ct], [st, ct * ca, -ct * sa, a * st],
                     [0.0, sa, ca, d], [0.0, 0.0, 0.0, 1.0]])


def _fk_textbook_error():
    sc, _ = sg.packing_problem(2001)
    arm = dict(base=sc.base, tool=sc.tool, dh_a=sc.dh_a, dh_d=sc.dh_d, dh_alpha=sc.dh_alpha,
               dh_offset=sc.dh_offset)
    rng = np.random.default_rng(2)
    worst = 0.0
    for _ in range(8):
        q = rng.uniform(-2.8, 2.8, 7)
        T = np.eye(4)
        for i in range(7):
            T = T @ _textbook_dh(q[i], sc.dh_d[i], sc.dh_a[i], sc.dh_alpha[i])
        got = G.end_effector(arm, G.forward_kinematics(arm, torch.tensor(q)[None]))[0].numpy()
        worst = max(worst, float(np.abs(got - T).max()))
    return worst


def test_fk_matches_textbook_dh_matrix():
    assert _fk_textbook_error() < 1e-13


def test_dh_single_joint_hand_value():
    g = _gold("geometry_hand_values.json")["dh_single_joint"]
    T = G.dh_transform(torch.tensor(g["theta"], dtype=DT), g["d"], g["a"], g["alpha"])
    assert np.allclose(T[:3, 3].numpy(), g["position"], atol=1e-15)
    assert np.allclose(T[:3, :3].numpy(), g["rotation"], atol=1e-15)


# ------------------------------------------------------------------ distances

def test_box_sdf_hand_values():
    g = _gold("geometry_hand_values.json")["box_sdf_axis_aligned"]
    half = torch.tensor(g["half"], dtype=DT)
    for case in g["cases"]:
        v = G.box_sdf(torch.tensor(case["p"], dtype=DT), torch.zeros(3, dtype=DT), torch.eye(3, dtype=DT), half)
        assert abs(float(v) - case["sdf"]) < 1e-14, case


def _random_rotation(rng):
    from scipy.spatial.transform import Rotation
    return Rotation.random(random_state=int(rng.integers(1 << 30))).as_matrix()


def _sdf_bruteforce_error(seed=3, n_points=60, res=120):
    """Signed box distance vs the nearest of dense surface samples (world frame)
    with the sign from scipy's Delaunay containment of the 8 world corners."""
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(seed)
    half = np.array([0.11, 0.05, 0.2])
    R = _random_rotation(rng)
    t = np.array([0.3, -0.2, 0.5])
    faces = []
    g = np.linspace(-1.0, 1.0, res)
    A, Bm = np.meshgrid(g, g, indexing="ij")
    for ax in range(3):
        o1, o2 = [k for k in range(3) if k != ax]
        for sgn in (-1.0, 1.0):
            pts = np.zeros((res * res, 3))
            pts[:, ax] = sgn * half[ax]
            pts[:, o1] = A.ravel() * half[o1]
            pts[:, o2] = Bm.ravel() * half[o2]
            faces.append(pts)
    surf = np.concatenate(faces) @ R.T + t
    corners = np.array([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)]) * half @ R.T + t
    hull = Delaunay(corners)
    p = t + rng.normal(0, 0.2, size=(n_points, 3))
    dist = np.sqrt(((p[:, None, :] - surf[None]) ** 2).sum(-1)).min(1)
    inside = hull.find_simplex(p) >= 0
    ref = np.where(inside, -dist, dist)
    got = G.box_sdf(torch.tensor(p), torch.tensor(t), torch.tensor(R), torch.tensor(half)).numpy()
    step = 2.0 * half.max() / (res - 1)
    return float(np.abs(got - ref).max()), step


def test_box_sdf_against_brute_force_surface_sampling():
    err, step = _sdf_bruteforce_error()
    assert err <= step, (err, step)


def test_sphere_sphere_penetration_hand_values():
    ca = torch.tensor([0.0, 0.0, 0.0], dtype=DT)
    cb = torch.tensor([0.3, 0.4, 0.0], dtype=DT)
    assert float(G.sphere_sphere_penetration(ca, 0.2, cb, 0.4)) == pytest.approx(0.1, abs=1e-15)
    assert float(G.sphere_sphere_penetration(ca, 0.2, cb, 0.2)) == 0.0


def test_dist_from_bounds_hand_values():
    g = _gold("geometry_hand_values.json")["dist_from_bounds"]
    lo, hi = torch.tensor(g["lo"], dtype=DT), torch.tensor(g["hi"], dtype=DT)
    for case in g["cases"]:
        assert float(G.dist_from_bounds(torch.tensor(case["v"], dtype=DT), lo, hi)) == pytest.approx(case["d"], abs=1e-15)


def test_obj_dist_hand_value_and_gradient():
    g = _gold("geometry_hand_values.json")["obj_dist"]
    pts = torch.tensor(g["points"], dtype=DT)
    assert float(G.obj_dist(pts)) == pytest.approx(g["value"], abs=1e-14)
    two = torch.tensor([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]], dtype=DT, requires_grad=True)
    G.obj_dist(two).backward()
    assert torch.allclose(two.grad, torch.tensor([[-0.6, -0.8, 0.0], [0.6, 0.8, 0.0]], dtype=DT), atol=1e-15)


def test_rotation_angle_matches_scipy():
    from scipy.spatial.transform import Rotation
    rots = Rotation.random(200, random_state=4)
    got = G.rotation_angle(torch.tensor(rots.as_matrix())).numpy()
    assert np.allclose(got, rots.magnitude(), atol=1e-12)


def test_pose_error_pure_offsets():
    T = G.box_pose(0.1, 0.2, 0.3, 0.4)
    d = torch.tensor([0.03, -0.04, 0.12], dtype=DT)
    Tb = T.clone()
    Tb[:3, 3] += d
    e_pos, e_rot = G.pose_error(T, Tb)
    assert float(e_pos) == pytest.approx(0.13, abs=1e-15) and float(e_rot) < 1e-15
    e_pos, e_rot = G.pose_error(T, T @ G.rot_z(torch.tensor(-0.7, dtype=DT)))
    assert float(e_pos) < 1e-15 and float(e_rot) == pytest.approx(0.7, abs=1e-14)


# ------------------------------------------------------------------ containment and grasp bounds

def _bounds_case_errors():
    """Largest error of the StablePlace and Grasp terms against the hand-worked
    cases, each case evaluated through the problem's own term list (the
    witness skeleton Pick(0)-Place(0) with box 0 and surface 0 replaced)."""
    gold = _gold("bounds_hand_values.json")
    sc0, acts, x0 = _scara_witness_scene()
    worst_c = 0.0
    for case in gold["containment"]:
        sc = dataclasses.replace(sc0, box_half=sc0.box_half.copy(), surf=sc0.surf.copy())
        sc.box_half[0, :2] = case["box_half"]
        sc.surf[0, :5] = case["surface"]
        pr = Problem(sc, acts)
        x = x0.clone()
        p_off = pr.configs[1]["target"][1]
        x[0, p_off:p_off + 3] = torch.tensor(case["placement"], dtype=DT)
        ti = [t.kind for t in pr.terms].index(STABLE_PLACE)
        got = float(pr.term_values(x)[0, ti])
        worst_c = max(worst_c, abs(got - case["value"]))
    worst_g = 0.0
    for case in gold["grasp"]:
        sc = dataclasses.replace(sc0, box_half=sc0.box_half.copy())
        sc.box_half[0] = case["box_half"]
        pr = Problem(sc, acts, Options(grasp_dof=case["dof"]))
        x = torch.zeros(1, pr.D, dtype=DT)
        x[0, 0:3] = torch.tensor(case["g"], dtype=DT)
        ti = [t.kind for t in pr.terms].index(GRASP)
        got = float(pr.term_values(x)[0, ti])
        worst_g = max(worst_g, abs(got - case["value"]))
    return worst_c, worst_g


def test_containment_and_grasp_bounds_hand_values():
    worst_c, worst_g = _bounds_case_errors()
    assert worst_c < 1e-12
    assert worst_g < 1e-12


# ------------------------------------------------------------------ constructed witness

def _scara_witness_scene(seed=5):
    """A SCARA arm (all twists 0) with a flipped tool, whose end-effector pose has
    the closed form Trans(sum a cos phi, sum a sin phi, sum d) Rz(phi_n) Rx(pi).
    Box 0 is placed where a top-down grasp at q1 holds it and its target surface
    so that the same grasp at q2 sets it down; everything else is far away."""
    rng = np.random.default_rng(seed)
    n = 7
    a = rng.uniform(0.05, 0.3, n)
    d = rng.uniform(0.0, 0.1, n)
    tool = np.diag([1.0, -1.0, -1.0, 1.0])         # Rx(pi)
    spheres = []
    links = []
    for i in range(n):
        for k in range(3):
            links.append(i + 1)
            spheres.append([-a[i] * (k + 0.5) / 3, 0.0, -d[i] * (k + 0.5) / 3, 0.03])
    half = np.array([[0.04, 0.03, 0.05], [0.03, 0.03, 0.03]])

    def ee(q):
        phi = np.cumsum(q)
        return np.array([(a * np.cos(phi)).sum(), (a * np.sin(phi)).sum(), d.sum()]), phi[-1]

    q1 = rng.uniform(-1.5, 1.5, n)
    q2 = rng.uniform(-1.5, 1.5, n)
    g = np.array([0.01, -0.01, half[0, 2] - 0.005, 0.0])
    yaw1, yaw2 = 0.3, -1.1
    e1, phi1 = ee(q1)
    e2, phi2 = ee(q2)
    g[3] = phi1 - yaw1
    # target of Kin is P(p) G(g): position p + Rz(yaw) g_xyz, yaw + g_yaw
    p1 = e1 - G.rot_z(torch.tensor(yaw1, dtype=DT))[:3, :3].numpy() @ g[:3]
    yaw2 = phi2 - g[3]
    p2 = e2 - G.rot_z(torch.tensor(yaw2, dtype=DT))[:3, :3].numpy() @ g[:3]
    z_top = p2[2] - half[0, 2]
    surf = np.array([[p2[0] + 0.02, p2[1] - 0.01, 0.4, 0.3, 0.25, z_top]])
    sc = sg.Scene(dh_a=a, dh_d=d, dh_alpha=np.zeros(n), dh_offset=np.zeros(n),
                  q_lo=np.full(n, -2.8), q_hi=np.full(n, 2.8), base=np.eye(4), tool=tool,
                  sphere_link=np.array(links, dtype=np.int32), sphere_xyzr=np.array(spheres),
                  box_half=half, box_init=np.array([[p1[0], p1[1], p1[2], yaw1], [50.0, 50.0, 0.03, 0.0]]),
                  box_spheres=np.stack([sg.box_sphere_model(h) for h in half]),
                  obs_center=np.array([[-40.0, 0.0, 0.5]]), obs_rot=np.eye(3)[None],
                  obs_half=np.array([[0.5, 0.5, 0.5]]), surf=surf)
    acts = sg.pick_place_skeleton([0])
    x = np.concatenate([g, q1, [p2[0], p2[1], yaw2], q2])[None]
    return sc, acts, torch.tensor(x)


def _witness_max_hard_cost():
    sc, acts, x = _scara_witness_scene()
    pr = Problem(sc, acts)
    terms = pr.term_values(x)
    return float(terms[:, pr.constraint_mask()].abs().max()), pr, terms


def test_zero_cost_at_constructed_satisfying_particle():
    worst, pr, terms = _witness_max_hard_cost()
    assert worst < 1e-12, terms
    assert bool(pr.satisfied(terms).all())


def test_kin_errors_of_shifted_witness_are_the_shift():
    sc, acts, x = _scara_witness_scene()
    pr = Problem(sc, acts)
    x2 = x.clone()
    x2[0, 11] += 0.03          # placement x
    x2[0, 12] -= 0.04          # placement y
    t = pr.term_values(x2)[0]
    kp = [i for i, tt in enumerate(pr.terms) if tt.kind == KIN_POS][1]
    kr = [i for i, tt in enumerate(pr.terms) if tt.kind == KIN_ROT][1]
    assert float(t[kp]) == pytest.approx(0.05, abs=1e-12) and float(t[kr]) < 1e-12


# ------------------------------------------------------------------ invariance

def _rigid_scene(sc, phi, shift):
    R = G.rot_z(torch.tensor(phi, dtype=DT))[:3, :3].numpy()
    M = np.eye(4)
    M[:3, :3] = R
    M[:3, 3] = shift
    bi = sc.box_init.copy()
    bi[:, :3] = bi[:, :3] @ R.T + shift
    bi[:, 3] += phi
    sf = sc.surf.copy()
    sf[:, :2] = sf[:, :2] @ R[:2, :2].T + shift[:2]
    sf[:, 2] += phi
    sf[:, 5] += shift[2]
    return dataclasses.replace(sc, base=M @ sc.base, obs_center=sc.obs_center @ R.T + shift,
                               obs_rot=np.einsum("ij,ojk->oik", R, sc.obs_rot), box_init=bi, surf=sf)


def _rigid_particles(pr, x, phi, shift):
    x = x.clone()
    c, s = math.cos(phi), math.sin(phi)
    for cfg in pr.configs:
        if cfg["kind"] == 1:
            po = cfg["target"][1]
            px, py = x[:, po].clone(), x[:, po + 1].clone()
            x[:, po] = c * px - s * py + shift[0]
            x[:, po + 1] = s * px + c * py + shift[1]
            x[:, po + 2] += phi
    return x


def _invariance_error(seed=7):
    sc, acts = sg.packing_problem(2003)
    pr = Problem(sc, acts)
    x = torch.tensor(sg.random_particles(sc, acts, 48, seed))
    phi, shift = 0.83, np.array([0.4, -1.3, 0.25])
    pr2 = Problem(_rigid_scene(sc, phi, shift), acts)
    t1 = pr.term_values(x)
    t2 = pr2.term_values(_rigid_particles(pr, x, phi, shift))
    return float((t1 - t2).abs().max()), float(t1.abs().max())


def test_costs_invariant_under_rigid_motion_of_scene():
    err, scale = _invariance_error()
    assert scale > 0.1 and err < 1e-11, err


# ------------------------------------------------------------------ gradients

def _fd_error(problem, x, h=1e-6):
    """max |autodiff - central FD| / max(1, |g|) over all components."""
    _, g = problem.gradient(x)
    P, D = x.shape
    worst = 0.0
    for p in range(P):
        xp = x[p].repeat(2 * D, 1)
        idx = torch.arange(D)
        xp[2 * idx, idx] += h
        xp[2 * idx + 1, idx] -= h
        J = problem.total_cost(xp)
        fd = (J[0::2] - J[1::2]) / (2 * h)
        worst = max(worst, float(((fd - g[p]).abs() / g[p].abs().clamp(min=1.0)).max()))
    return worst


@pytest.mark.parametrize("make", [sg.plain_problem, sg.packing_problem])
def test_gradient_matches_central_differences(make):
    sc, acts = make()
    pr = Problem(sc, acts)
    x = torch.tensor(sg.random_particles(sc, acts, 24, 11))
    keep = pr.kink_margin(x) > 1e-4
    x = x[keep][:6]
    assert x.shape[0] >= 3
    assert _fd_error(pr, x) < 1e-6


# ------------------------------------------------------------------ Eq. 3 / Eq. 5

def test_flags_and_counts_by_explicit_loops():
    sc, acts = sg.packing_problem()
    pr = Problem(sc, acts)
    x = torch.tensor(sg.random_particles(sc, acts, 64, 13))
    terms = pr.term_values(x)
    tol = Options().tol
    counts = [0] * len(pr.terms)
    sat = []
    for p in range(x.shape[0]):
        ok = True
        for ci, t in enumerate(pr.terms):
            if t.kind == OBJ_DIST:
                continue
            good = float(terms[p, ci]) <= tol[t.kind]
            counts[ci] += int(good)
            ok = ok and good
        sat.append(ok)
    cons = [c for ci, c in enumerate(counts) if pr.terms[ci].kind != OBJ_DIST]
    assert pr.constraint_counts(terms).tolist() == cons
    assert pr.satisfied(terms).tolist() == sat


def test_term_list_follows_action_constraints():
    sc, acts = sg.plain_problem()
    pr = Problem(sc, acts)
    assert [t.kind for t in pr.terms] == [KIN_POS, KIN_ROT, GRASP, CFREE_HOLD, JOINT_LIMIT,
                                          KIN_POS, KIN_ROT, STABLE_PLACE, CFREE_HOLD, CFREE_PLACE, JOINT_LIMIT]
    assert pr.D == 21
    sc2, acts2 = sg.packing_problem()
    assert Problem(sc2, acts2).D == 126


def test_invalid_skeletons_are_rejected():
    sc, _ = sg.packing_problem()
    with pytest.raises(ValueError):
        Problem(sc, [(1, 0, 0)])                      # place before pick
    with pytest.raises(ValueError):
        Problem(sc, [(0, 0, -1), (0, 1, -1)])         # pick while holding


# ------------------------------------------------------------------ Adam

def test_adam_first_step_closed_form():
    sc, acts = sg.plain_problem()
    pr = Problem(sc, acts)
    x = torch.tensor(sg.random_particles(sc, acts, 8, 17))
    _, g = pr.gradient(x)
    x1, m1, v1 = pr.adam_step(x, torch.zeros_like(x), torch.zeros_like(x), 1, g, 8)
    gh = g / 8
    expect = x - pr.learning_rates() * gh / (gh.abs() + 1e-8)
    assert torch.allclose(x1, expect, rtol=0, atol=1e-15)
    assert torch.allclose(m1, 0.1 * gh) and torch.allclose(v1, 0.001 * gh * gh)


def test_optimize_reports_satisfied_at_iteration_zero_for_witness():
    sc, acts, x = _scara_witness_scene()
    out = Problem(sc, acts).optimize(x, 3)
    assert out["first_iter"] == 0


def _replayed_checks(pr, X, n):
    """The optimiser's checks k = 0..n replayed one update at a time: states
    x_k, Eq. 3 flags and Eq. 2 costs."""
    xk, m, v = X.clone(), torch.zeros_like(X), torch.zeros_like(X)
    xs, S, C = [], [], []
    for k in range(n + 1):
        t = pr.term_values(xk)
        xs.append(xk.clone())
        S.append(pr.satisfied(t).numpy())
        C.append((t * pr.weights()).sum(1).numpy())
        if k < n:
            o = pr.optimize(xk, 1, m, v, t0=k)
            xk, m, v = o["x"], o["m"], o["v"]
    return xs, np.array(S).T, np.array(C).T


def test_best_record_is_the_lowest_cost_satisfying_check():
    """The best satisfying record of OptimizeParticles against its definition
    over a trajectory replayed update by update: the lowest-cost state among
    the checks where the particle satisfies Eq. 3 (the earliest of equal ones),
    none where it never does.  The batch (witness and small perturbations of
    it, one particle far off) has particles whose lowest check is neither their
    first nor their last satisfying one, and one that satisfies only at the
    check after the last update, so recording the first, the latest or
    skipping the final check each fails."""
    sc, acts, x = _scara_witness_scene()
    pr = Problem(sc, acts)
    rng = np.random.default_rng(0)
    X = x.repeat(25, 1).clone()
    X[1:24] += torch.tensor(rng.normal(0.0, 0.002, (23, X.shape[1])))
    X[24, 4:11] += 0.3                                # never satisfies
    n = 30
    out = pr.optimize(X, n)
    xs, S, C = _replayed_checks(pr, X, n)
    not_first = not_latest = only_final = never = 0
    for p in range(X.shape[0]):
        ks = np.nonzero(S[p])[0]
        if len(ks) == 0:
            never += 1
            assert int(out["best_iter"][p]) == -1 and math.isinf(float(out["best_cost"][p]))
            continue
        k = int(ks[np.argmin(C[p, ks])])
        not_first += k != ks[0]
        not_latest += k != ks[-1]
        only_final += len(ks) == 1 and ks[0] == n
        assert int(out["best_iter"][p]) == k, p
        assert float(out["best_cost"][p]) == C[p, k]
        assert torch.equal(out["best_x"][p], xs[k][p])
    assert not_first >= 3 and not_latest >= 3 and only_final >= 1 and never >= 1


def test_best_record_counts_checks_from_the_step_count():
    """Check indices of the record are the Adam step count at the check (t0 +
    k), as the first satisfying iteration of a continued run."""
    sc, acts, x = _scara_witness_scene()
    pr = Problem(sc, acts)
    out = pr.optimize(x, 2, t0=7)
    assert int(out["best_iter"][0]) == 7


def test_optimize_lowers_mean_cost():
    sc, acts = sg.plain_problem()
    pr = Problem(sc, acts)
    x = torch.tensor(philox.sample_uniform(pr, 64, 99))
    before = float(pr.total_cost(x).mean())
    out = pr.optimize(x, 40)
    assert float(out["cost"].mean()) < 0.8 * before


# ------------------------------------------------------------------ sampler

def test_philox_known_answers():
    for case in _gold("philox4x32_10_kat.json")["cases"]:
        ctr = [int(v, 16) for v in case["ctr"]]
        key = [int(v, 16) for v in case["key"]]
        out = philox.philox4x32_10(ctr, key)
        assert ["%08x" % int(w) for w in out] == case["out"]


def test_uniform_sampler_bounds_and_uniformity():
    from scipy.stats import kstest
    sc, acts = sg.packing_problem()
    pr = Problem(sc, acts)
    X = philox.sample_uniform(pr, 4000, 1234)
    for cfg in pr.configs:
        q = X[:, cfg["q_off"]:cfg["q_off"] + 7]
        assert (q >= -2.8).all() and (q < 2.8).all()
        assert kstest((q[:, 0] + 2.8) / 5.6, "uniform").pvalue > 1e-3
    terms = pr.term_values(torch.tensor(X[:256]))
    for ti, t in enumerate(pr.terms):
        if t.kind in (GRASP, STABLE_PLACE, JOINT_LIMIT):
            # grasp and joints are drawn inside their bounds; a placement's
            # centre is inside the region (its corners may stick out)
            if t.kind != STABLE_PLACE:
                assert float(terms[:, ti].max()) == 0.0


# ------------------------------------------------------------------ planted mistakes

def test_planted_mistakes_are_caught(monkeypatch):
    """Each plausible slip in the oracle makes at least one pin above fail."""
    orig_sdf, orig_dh, orig_grasp, orig_od = G.box_sdf, G.dh_transform, G.grasp_pose, G.obj_dist

    # 1. transposed obstacle rotation in the signed distance
    def sdf_transposed(c, center, R, half):
        return orig_sdf(c, center, R.transpose(-1, -2), half)
    monkeypatch.setattr(G, "box_sdf", sdf_transposed)
    assert _invariance_error()[0] > 1e-6 or _sdf_bruteforce_error()[0] > _sdf_bruteforce_error()[1]
    monkeypatch.setattr(G, "box_sdf", orig_sdf)

    # 2. DH factors in the wrong order (Rx before Tx)
    def dh_swapped(theta, d, a, alpha):
        theta = torch.as_tensor(theta, dtype=DT)
        z = torch.zeros_like(theta)
        return G.rot_z(theta) @ G.translation(z, z, z + d) @ G.rot_x(z + alpha) @ G.translation(z, z + a, z)
    monkeypatch.setattr(G, "dh_transform", dh_swapped)
    assert _fk_textbook_error() > 1e-6
    monkeypatch.setattr(G, "dh_transform", orig_dh)

    # 3. grasp without the top-down flip
    def grasp_noflip(gx, gy, gz, gyaw):
        return G.translation(gx, gy, gz) @ G.rot_z(gyaw)
    monkeypatch.setattr(G, "grasp_pose", grasp_noflip)
    assert _witness_max_hard_cost()[0] > 1e-3
    monkeypatch.setattr(G, "grasp_pose", orig_grasp)

    # 4. a dropped pair in the goal cost
    def od_dropped(pos):
        return orig_od(pos[..., :-1, :])
    monkeypatch.setattr(G, "obj_dist", od_dropped)
    g = _gold("geometry_hand_values.json")["obj_dist"]
    assert abs(float(G.obj_dist(torch.tensor(g["points"], dtype=DT))) - g["value"]) > 1e-3
    monkeypatch.setattr(G, "obj_dist", orig_od)

    # 5. containment measured in the world frame instead of the surface frame
    from oracle import problem as PM
    orig_cont = PM.Problem._containment

    def cont_world(self, b, s, p):
        sf = self.sc.surf.copy()
        saved = self.sc.surf
        sf[:, 2] = 0.0
        self.sc.surf = sf
        try:
            return orig_cont(self, b, s, p)
        finally:
            self.sc.surf = saved
    monkeypatch.setattr(PM.Problem, "_containment", cont_world)
    assert _invariance_error()[0] > 1e-6
    monkeypatch.setattr(PM.Problem, "_containment", orig_cont)

    # 6.-7. containment with the box's half extents swapped, or with a corner left out
    def cont_variant(swap, corners):
        def cont(self, b, s, p):
            cx, cy, syaw, hx, hy, _z = (float(v) for v in self.sc.surf[s])
            h = self.sc.box_half[b][[1, 0]] if swap else self.sc.box_half[b]
            cs, ss = math.cos(syaw), math.sin(syaw)
            c, si = torch.cos(p[:, 2]), torch.sin(p[:, 2])
            total = torch.zeros(p.shape[0], dtype=DT)
            for sx, sy in corners:
                wx = p[:, 0] + c * (sx * h[0]) - si * (sy * h[1]) - cx
                wy = p[:, 1] + si * (sx * h[0]) + c * (sy * h[1]) - cy
                u = torch.stack([cs * wx + ss * wy, -ss * wx + cs * wy], dim=-1)
                total = total + G.dist_from_bounds(u, torch.tensor([-hx, -hy], dtype=DT),
                                                   torch.tensor([hx, hy], dtype=DT))
            return total
        return cont
    four = [(-1.0, -1.0), (-1.0, 1.0), (1.0, -1.0), (1.0, 1.0)]
    assert _bounds_case_errors()[0] < 1e-12           # the rewritten form itself agrees
    monkeypatch.setattr(PM.Problem, "_containment", cont_variant(False, four))
    assert _bounds_case_errors()[0] < 1e-12
    monkeypatch.setattr(PM.Problem, "_containment", cont_variant(True, four))
    assert _bounds_case_errors()[0] > 1e-3
    for dropped in range(4):
        monkeypatch.setattr(PM.Problem, "_containment", cont_variant(False, four[:dropped] + four[dropped + 1:]))
        assert _bounds_case_errors()[0] > 1e-3
    monkeypatch.setattr(PM.Problem, "_containment", orig_cont)

    # 8. the top-down grasp's lower z bound taken as -h_z (the whole box) instead of h_z - 0.02
    orig_gb = PM.Problem._grasp_bounds

    def gb_whole_box(self, b):
        h = self.sc.box_half[b]
        return torch.tensor([-h[0], -h[1], -h[2]], dtype=DT), torch.tensor([h[0], h[1], h[2]], dtype=DT)
    monkeypatch.setattr(PM.Problem, "_grasp_bounds", gb_whole_box)
    assert _bounds_case_errors()[1] > 1e-3
    monkeypatch.setattr(PM.Problem, "_grasp_bounds", orig_gb)
