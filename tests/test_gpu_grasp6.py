"""6-DOF grasps through the C ABI (options grasp_dof = 6; Sec. VIII setup:
grasps are top-down 4-DOF or 6-DOF poses) against the FP64 oracle, with the
tolerances of tests/parity.py and the IK-sampler bar of tests/test_gpu_ik.py."""
import numpy as np
import pytest
import torch

import scenegen as sg
from oracle import ik, philox
from oracle.problem import Options, Problem
from tests.parity import compare_eval

from test_gpu_ik import _compare, _moved

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2411_11833_b300.build import build_library
    build_library()
    import paper_2411_11833_b300 as p
    torch.cuda.set_device(0)
    return p


@pytest.mark.parametrize("lanes,m,selfc", [(1, 0, 0), (2, 0, 0), (1, 1, 1)])
def test_eval_parity_with_six_dof_grasps(pkg, lanes, m, selfc):
    sc, acts = sg.robot_packing_problem(21002, n_boxes=2)
    pr = Problem(sc, acts, Options(grasp_dof=6, n_knots=m, self_collision=bool(selfc)))
    X = pr.interpolate_knots(philox.sample_uniform(pr, 70, 61))
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts, pkg.default_options(lanes=lanes, grasp_dof=6, n_knots=m, self_collision=selfc))
    D, _, kinds = scene.problem_info(pid)
    assert D == pr.D and kinds == [t.kind for t in pr.terms]
    out = scene.eval(pid, torch.tensor(np.ascontiguousarray(X.T), dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    scene.close()
    print(compare_eval(pr, X, *out, label=f"grasp6 L={lanes} knots={m} self={selfc}"))


def test_samplers_with_six_dof_grasps(pkg):
    sc, acts = sg.robot_packing_problem(21002, n_boxes=2)
    pr = Problem(sc, acts, Options(grasp_dof=6))
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts, pkg.default_options(grasp_dof=6))
    n, seed = 384, 23
    scene.sample(pid, n, seed)
    x = scene.get_particles(pid)[0].T.astype(np.float64)
    assert np.abs(x - philox.sample_uniform(pr, n, seed)).max() < 2e-6
    scene.sample(pid, n, seed, sampler=2)
    x = scene.get_particles(pid)[0].T.astype(np.float64)
    X0 = philox.sample_uniform(pr, n, seed)
    _compare(pr, x, ik.ik_configurations(pr, X0), ik.ik_configurations(pr, _moved(X0)))
    scene.close()


def test_adam_step_with_six_dof_grasps_matches_oracle(pkg):
    sc, acts = sg.robot_packing_problem(21003, n_boxes=2)
    pr = Problem(sc, acts, Options(grasp_dof=6))
    P = 80
    X = philox.sample_uniform(pr, P, 63)
    m0, v0 = sg.random_adam_state(P, pr.D, seed=64)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts, pkg.default_options(grasp_dof=6))
    scene.set_particles(pid, X.T.astype(np.float32), m0.T.astype(np.float32), v0.T.astype(np.float32), 2)
    scene.optimize(pid, 1)
    x1, m1, _, t1 = scene.get_particles(pid)
    scene.close()
    assert t1 == 3
    Xt = torch.tensor(X.astype(np.float32).astype(np.float64))
    _, g = pr.gradient(Xt)
    xr, mr, _ = pr.adam_step(Xt, torch.tensor(m0.astype(np.float32).astype(np.float64)),
                             torch.tensor(v0.astype(np.float32).astype(np.float64)), 3, g, P)
    keep = pr.kink_margin(Xt).numpy() > 1e-4
    assert keep.mean() > 0.5
    assert np.abs(m1.T - mr.numpy())[keep].max() <= 1e-3 * np.abs(mr.numpy()[keep]).max() + 1e-9
    step_g = (x1.T - X.astype(np.float32))[keep]
    step_r = (xr.numpy() - Xt.numpy())[keep]
    assert np.abs(step_g - step_r).max() <= 1e-3 * np.abs(step_r).max() + 2e-6


@pytest.mark.parametrize("with_g6", [True, False])
def test_one_launch_over_problems_with_different_optional_terms(pkg, with_g6):
    """Problems that need different kernel feature sets in one persistent
    launch (the launch takes the set that holds all of them: knots with 6-DOF
    grasps, or knots with 4-DOF grasps when no problem has 6-DOF grasps): each
    problem's costs still match the oracle, particle by particle."""
    from tests.parity import cost_ok
    sc, acts = sg.robot_packing_problem(21002, n_boxes=2)
    specs = [dict(n_knots=2), dict(), dict(self_collision=1)]
    if with_g6:
        specs.append(dict(grasp_dof=6))
    scene = pkg.Scene(sc)
    probs = []
    for i, o in enumerate(specs):
        pr = Problem(sc, acts, Options(n_knots=o.get("n_knots", 0), grasp_dof=o.get("grasp_dof", 4),
                                       self_collision=bool(o.get("self_collision", 0))))
        pid = scene.set_skeleton(acts, pkg.default_options(**o))
        X = pr.interpolate_knots(philox.sample_uniform(pr, 40 + 7 * i, 90 + i))
        scene.set_particles(pid, np.ascontiguousarray(X.T).astype(np.float32))
        probs.append((pid, pr, X))
    scene.optimize([p for p, _, _ in probs], 0)       # evaluation only, one launch
    for pid, pr, X in probs:
        q = scene.query(pid, X.shape[0])
        J = pr.total_cost(torch.tensor(X.astype(np.float32).astype(np.float64))).numpy()
        assert cost_ok(q["cost"].astype(np.float64), J).all(), (pid, np.abs(q["cost"] - J).max())
    scene.close()
