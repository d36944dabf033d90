"""Trajectory knots through the C ABI (options n_knots; Listing 1 MoveFree /
MoveHold: Motion, CFreeTraj(Hold), TrajLength; Sec. VIII knot points
initialised by linear interpolation) against the FP64 oracle, with the
tolerances of tests/parity.py."""
import numpy as np
import pytest
import torch

import scenegen as sg
from oracle import ik, philox
from oracle.problem import KNOT, TRAJ_LEN, Options, Problem
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


def _knotted(pr, P, seed, spread=0.3):
    """Uniform draws, knots interpolated and then moved off the line."""
    g = np.random.default_rng(seed)
    X = pr.interpolate_knots(philox.sample_uniform(pr, P, seed))
    for c in pr.configs:
        if c["kind"] == KNOT:
            X[:, c["q_off"]:c["q_off"] + pr.n] += g.normal(0, spread, (P, pr.n))
    return X


@pytest.mark.parametrize("lanes,m", [(1, 2), (2, 3), (1, 1)])
def test_eval_parity_with_knots(pkg, lanes, m):
    sc, acts = sg.robot_packing_problem(21002, n_boxes=2)
    pr = Problem(sc, acts, Options(n_knots=m))
    X = _knotted(pr, 75, 41)                                  # several tiles and a ragged tail
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts, pkg.default_options(lanes=lanes, n_knots=m))
    D, nt, kinds = scene.problem_info(pid)
    assert D == pr.D and kinds == [t.kind for t in pr.terms]
    out = scene.eval(pid, torch.tensor(np.ascontiguousarray(X.T), dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    scene.close()
    print(compare_eval(pr, X, *out, label=f"knots m={m} L={lanes}"))


def test_knots_start_on_the_line_between_their_configurations(pkg):
    sc, acts = sg.robot_packing_problem(21002, n_boxes=2)
    pr = Problem(sc, acts, Options(n_knots=2))
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts, pkg.default_options(n_knots=2))
    n, seed = 256, 17
    # uniform configurations: the knots are their interpolation, to FP32 rounding
    scene.sample(pid, n, seed)
    x = scene.get_particles(pid)[0].T.astype(np.float64)
    ref = pr.interpolate_knots(philox.sample_uniform(pr, n, seed))
    assert np.abs(x - ref).max() < 2e-6
    # IK configurations: the knots follow the solved ends
    scene.sample(pid, n, seed, sampler=2)
    x = scene.get_particles(pid)[0].T.astype(np.float64)
    X0 = philox.sample_uniform(pr, n, seed)
    _compare(pr, x, pr.interpolate_knots(ik.ik_configurations(pr, X0)),
             pr.interpolate_knots(ik.ik_configurations(pr, _moved(X0))))
    # and TrajLength of straight knots is the straight-line length
    tv = pr.term_values(torch.tensor(x)).numpy()
    for ti, t in enumerate(pr.terms):
        if t.kind == TRAJ_LEN:
            s = pr.segments[t.cfg]
            qa = x[:, pr.configs[s["start"]]["q_off"]:pr.configs[s["start"]]["q_off"] + pr.n]
            qb = x[:, pr.configs[s["end"]]["q_off"]:pr.configs[s["end"]]["q_off"] + pr.n]
            assert np.allclose(tv[:, ti], np.linalg.norm(qb - qa, axis=1), atol=1e-5)
    scene.close()


def test_adam_step_with_knots_matches_oracle(pkg):
    sc, acts = sg.robot_packing_problem(21003, n_boxes=2)
    pr = Problem(sc, acts, Options(n_knots=2))
    P = 90
    X = _knotted(pr, P, 43)
    m0, v0 = sg.random_adam_state(P, pr.D, seed=44)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts, pkg.default_options(n_knots=2))
    scene.set_particles(pid, X.T.astype(np.float32), m0.T.astype(np.float32), v0.T.astype(np.float32), 4)
    scene.optimize(pid, 1)
    x1, m1, _, t1 = scene.get_particles(pid)
    scene.close()
    assert t1 == 5
    Xt = torch.tensor(X.astype(np.float32).astype(np.float64))
    _, g = pr.gradient(Xt)
    xr, mr, _ = pr.adam_step(Xt, torch.tensor(m0.astype(np.float32).astype(np.float64)),
                             torch.tensor(v0.astype(np.float32).astype(np.float64)), 5, g, P)
    keep = pr.kink_margin(Xt).numpy() > 1e-4
    assert keep.mean() > 0.5
    assert np.abs(m1.T - mr.numpy())[keep].max() <= 1e-3 * np.abs(mr.numpy()[keep]).max() + 1e-9
    step_g = (x1.T - X.astype(np.float32))[keep]
    step_r = (xr.numpy() - Xt.numpy())[keep]
    assert np.abs(step_g - step_r).max() <= 1e-3 * np.abs(step_r).max() + 2e-6
