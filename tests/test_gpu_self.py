"""SelfCollision through the C ABI (options self_collision; the CFree
constraints' "does not cause robot self-collisions", tolerance 0) against the
FP64 oracle with the tolerances of tests/parity.py."""
import numpy as np
import pytest
import torch

import scenegen as sg
from oracle import philox
from oracle.problem import KNOT, SELF_COLLISION, Options, Problem
from tests.parity import compare_eval

from test_oracle_self import _planar_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2411_11833_b300.build import build_library
    build_library()
    import paper_2411_11833_b300 as p
    torch.cuda.set_device(0)
    return p


def _eval(pkg, sc, acts, X, **opts):
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts, pkg.default_options(**opts))
    out = scene.eval(pid, torch.tensor(np.ascontiguousarray(X.T), dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    kinds = scene.problem_info(pid)[2]
    scene.close()
    return out, kinds


@pytest.mark.parametrize("lanes,m", [(1, 0), (2, 0), (1, 1)])
def test_eval_parity_with_self_collision(pkg, lanes, m):
    sc, acts = sg.robot_packing_problem(21002, n_boxes=2)
    pr = Problem(sc, acts, Options(n_knots=m, self_collision=True))
    X = pr.interpolate_knots(philox.sample_uniform(pr, 70, 51))
    out, kinds = _eval(pkg, sc, acts, X, lanes=lanes, n_knots=m, self_collision=1)
    assert kinds == [t.kind for t in pr.terms]
    selfs = [i for i, t in enumerate(pr.terms) if t.kind == SELF_COLLISION]
    T = pr.term_values(torch.tensor(X)).numpy()
    assert (T[:, selfs] > 0).any()                           # some arms fold onto themselves
    print(compare_eval(pr, X, *out, label=f"self L={lanes} knots={m}"))


def test_folded_planar_arm_through_the_abi(pkg):
    sc = _planar_scene()
    acts = sg.pick_place_skeleton([0, 1])
    pr = Problem(sc, acts, Options(n_knots=1, self_collision=True))
    kn = next(c for c in pr.configs if c["kind"] == KNOT and c["box"] < 0)
    X = philox.sample_uniform(pr, 6, 1)
    X[:, kn["q_off"]:kn["q_off"] + 3] = [[0.0, 2.0944, 2.0944 + e] for e in (0.0, 0.01, 0.05, 0.1, 0.2, 0.6)]
    out, _ = _eval(pkg, sc, acts, X, n_knots=1, self_collision=1)
    compare_eval(pr, X, *out, label="planar")
    ci = pr.configs.index(kn)
    ti = next(i for i, t in enumerate(pr.terms) if t.kind == SELF_COLLISION and t.cfg == ci)
    assert out[1][ti].cpu().numpy()[0] > 0.09


def test_adam_step_with_self_collision_matches_oracle(pkg):
    sc, acts = sg.robot_packing_problem(21003, n_boxes=2)
    pr = Problem(sc, acts, Options(self_collision=True))
    P = 80
    X = philox.sample_uniform(pr, P, 53)
    m0, v0 = sg.random_adam_state(P, pr.D, seed=54)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts, pkg.default_options(self_collision=1))
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
