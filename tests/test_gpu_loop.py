"""The optimisation loop through the C ABI against the FP64 oracle: CUDA-graph
replay, the device-side stop on the first satisfying particle (graph and
tamp_optimize_steps), several problems in one persistent launch, odd cuboid
counts in the paired broad phase, and a caller-supplied allocator.

Multi-step trajectories follow the rule of tests/parity.py (check_trajectory).
"""
import dataclasses

import numpy as np
import pytest
import torch

import scenegen as sg
from oracle import philox
from oracle.problem import Problem
from tests.parity import (KINK_MARGIN, TRAJ_MARGIN, check_adam_step, check_trajectory, cost_ok, near_threshold,
                          oracle_run)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2411_11833_b300.build import build_library
    build_library()
    import paper_2411_11833_b300 as p
    torch.cuda.set_device(0)
    return p


def _counts_match(pr, x, counts):
    """Eq. 5 counts of the last check against the oracle's at the final iterate
    (a particle within 1e-5 of a tolerance may count either way)."""
    T = pr.term_values(torch.tensor(x.astype(np.float32).astype(np.float64)))
    ref = pr.constraint_counts(T).numpy()
    band = near_threshold(pr, T.numpy())
    assert np.abs(counts - ref).max() <= band.sum(), (counts, ref)


def test_graph_replay_matches_oracle(pkg):
    """4 captured chunks of 5 fused iterations against 20 oracle iterations."""
    sc, acts = sg.plain_problem(1001)
    pr = Problem(sc, acts)
    P = 150
    X = sg.random_particles(sc, acts, P, seed=21, spread=0.5).astype(np.float32).astype(np.float64)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    scene.set_particles(pid, X.T.astype(np.float32))
    g = pkg.Graph(scene, pid, 5, 4)
    steps = g.run()
    g.close()
    x, _, _, t = scene.get_particles(pid)
    q = scene.query(pid, P)
    scene.close()
    assert steps == 20 and t == 20
    out, margin = oracle_run(pr, X, 20)
    print(check_trajectory(pr, x.T, q["cost"], out, margin))
    assert q["first_iter"] == (out["first_iter"] if out["first_iter"] >= 0 else -1)
    _counts_match(pr, x.T, q["counts"])


def test_graph_stop_keeps_the_last_checks_counts(pkg):
    """After the stop, the skipped chunks leave the results of the last check."""
    from tests.test_oracle_pins import _scara_witness_scene
    sc, acts, x = _scara_witness_scene()
    pr = Problem(sc, acts)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    scene.set_particles(pid, np.repeat(x.numpy(), 3, axis=0).T.astype(np.float32))
    g = pkg.Graph(scene, pid, 5, 10, stop_on_first=True)
    steps = g.run()
    g.close()
    xs = scene.get_particles(pid)[0]
    q = scene.query(pid, 3)
    scene.close()
    assert steps == 5 and q["first_iter"] == 0
    assert q["counts"].max() > 0
    _counts_match(pr, xs.T, q["counts"])


def test_optimize_steps_stops_on_the_first_satisfying_particle(pkg):
    """tamp_optimize_steps(..., k): the constructed witness satisfies Eq. 3 at
    x_0, so only the first chunk of k iterations runs; its result is the
    oracle's k-step run."""
    from tests.test_oracle_pins import _scara_witness_scene
    sc, acts, x = _scara_witness_scene()
    pr = Problem(sc, acts)
    X = np.repeat(x.numpy(), 4, axis=0)
    X[1:, :4] += 0.002                       # grasps moved off the witness: not all particles satisfy
    X = X.astype(np.float32).astype(np.float64)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    scene.set_particles(pid, X.T.astype(np.float32))
    scene.optimize(pid, 100, stop_every=10)
    xs, _, _, t = scene.get_particles(pid)
    q = scene.query(pid, 4)
    scene.close()
    assert t == 10 and q["first_iter"] == 0
    out, margin = oracle_run(pr, X, 10)
    print(check_trajectory(pr, xs.T, q["cost"], out, margin, min_smooth=0.0))
    _counts_match(pr, xs.T, q["counts"])


def test_optimize_steps_stop_mode_without_a_solution_runs_every_chunk(pkg):
    """No particle satisfies within the budget: 23 steps in chunks 5, 5, 5, 5, 3;
    the trajectory and the last check's Eq. 5 counts are the oracle's."""
    sc, acts = sg.plain_problem(1001)
    pr = Problem(sc, acts)
    P = 96
    X = philox.sample_uniform(pr, P, 5).astype(np.float32).astype(np.float64)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    scene.set_particles(pid, X.T.astype(np.float32))
    scene.optimize(pid, 23, stop_every=5)
    xs, _, _, t = scene.get_particles(pid)
    q = scene.query(pid, P)
    scene.close()
    out, margin = oracle_run(pr, X, 23)
    assert out["first_iter"] < 0 and q["first_iter"] == -1
    assert t == 23
    print(check_trajectory(pr, xs.T, q["cost"], out, margin))
    _counts_match(pr, xs.T, q["counts"])


def test_batched_launch_takes_each_problems_oracle_adam_step(pkg):
    """Three skeletons of different lengths and batch sizes in one persistent
    launch, from a random Adam state: for every problem the gradient (read back
    from the first moment, m1 = b1 m0 + (1 - b1) g / N_b) matches the oracle's
    per particle, and every component's step matches within the bound that
    gradient tolerance implies for it."""
    sc, _ = sg.packing_problem(2001)
    skels = [sg.pick_place_skeleton([0]), sg.pick_place_skeleton([0, 1, 2]),
             sg.pick_place_skeleton(range(6), goal=True)]
    sizes = [100, 70, 45]
    t0 = 5
    scene = pkg.Scene(sc)
    opts = pkg.default_options(lanes=1)
    pids = [scene.set_skeleton(a, opts) for a in skels]
    state = []
    for pid, n, a in zip(pids, sizes, skels):
        pr = Problem(sc, a)
        X = sg.random_particles(sc, a, n, seed=300 + n, spread=0.5).astype(np.float32).astype(np.float64)
        m0, v0 = (s.astype(np.float32).astype(np.float64) for s in sg.random_adam_state(n, pr.D, seed=400 + n))
        scene.set_particles(pid, X.T.astype(np.float32), m0.T.astype(np.float32), v0.T.astype(np.float32), t0)
        state.append((pr, X, m0, v0))
    scene.optimize(pids, 1)
    for pid, (pr, X, m0, v0) in zip(pids, state):
        x1, m1, v1, t1 = scene.get_particles(pid)
        assert t1 == t0 + 1
        keep = pr.kink_margin(torch.tensor(X)).numpy() > KINK_MARGIN
        assert keep.mean() >= 0.6
        print(pid, check_adam_step(pr, X, m0, v0, t0, x1.T, m1.T, X.shape[0], keep))
    scene.close()


def test_batched_launch_matches_separate_launches_step_by_step(pkg):
    """The same three problems, six single-step launches each, batched and
    separate.  Each launch orders its float atomic additions differently, so a
    particle may part ways only at a step that starts near a kink (oracle
    margin below TRAJ_MARGIN); every other particle agrees to 1e-5 after each
    step, and the ones that parted are counted."""
    sc, _ = sg.packing_problem(2001)
    skels = [sg.pick_place_skeleton([0]), sg.pick_place_skeleton([0, 1, 2]),
             sg.pick_place_skeleton(range(6), goal=True)]
    sizes = [100, 70, 45]
    prs = [Problem(sc, a) for a in skels]
    opts = pkg.default_options(lanes=1)
    scenes = [pkg.Scene(sc), pkg.Scene(sc)]
    pids = [[s.set_skeleton(a, opts) for a in skels] for s in scenes]
    for s, ps in zip(scenes, pids):
        for pid, n, a in zip(ps, sizes, skels):
            s.set_particles(pid, sg.random_particles(sc, a, n, seed=100 + n, spread=0.5).T.astype(np.float32))
    alive = [np.ones(n, bool) for n in sizes]
    parted = 0
    for step in range(6):
        before = [scenes[0].get_particles(pid)[0].T.astype(np.float64) for pid in pids[0]]
        scenes[0].optimize(pids[0], 1)
        for pid in pids[1]:
            scenes[1].optimize(pid, 1)
        for i, pr in enumerate(prs):
            xb = scenes[0].get_particles(pids[0][i])[0].T
            xs = scenes[1].get_particles(pids[1][i])[0].T
            d = np.abs(xb - xs).max(axis=1)
            off = alive[i] & (d > 1e-5)
            if off.any():
                near = pr.kink_margin(torch.tensor(before[i][off])).numpy() < TRAJ_MARGIN
                assert near.all(), f"problem {i} step {step}: a particle away from kinks parted ({d[off].max():.2e})"
                parted += int(off.sum())
                alive[i] &= ~off
    for s in scenes:
        s.close()
    total = sum(sizes)
    print(f"{parted} of {total} particles parted at a step that started near a kink")
    assert parted <= 0.25 * total


@pytest.mark.parametrize("n_obs", [1, 3, 7])
@pytest.mark.parametrize("lanes", [1, 2])
def test_odd_cuboid_counts(pkg, n_obs, lanes):
    """The plain instantiation's broad phase tests cuboids two at a time and
    pads an odd count with a far-away record: costs, gradients and flags still
    match the oracle, and the broad phase passes exactly the pairs that the
    one-at-a-time broad phase of another instantiation passes."""
    from tests.parity import compare_eval
    sc, acts = sg.plain_problem(1001)
    rng = np.random.default_rng(n_obs)
    centres = np.stack([rng.uniform(-0.7, 0.7, n_obs), rng.uniform(-0.7, 0.7, n_obs), rng.uniform(0.1, 0.6, n_obs)], 1)
    rots = np.stack([sg._rz3(rng.uniform(-np.pi, np.pi)) for _ in range(n_obs)])
    half = rng.uniform(0.05, 0.2, (n_obs, 3))
    sc = dataclasses.replace(sc, obs_center=centres, obs_rot=rots, obs_half=half)
    pr = Problem(sc, acts)
    X = sg.random_particles(sc, acts, 90, seed=7 + n_obs)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts, pkg.default_options(lanes=lanes))
    out = scene.eval(pid, torch.tensor(np.ascontiguousarray(X.T), dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    print(compare_eval(pr, X, *out, label=f"{n_obs} cuboids L={lanes}"))
    # candidate counts of the paired (plain) and unpaired (self-collision) instantiations
    pid_self = scene.set_skeleton(acts, pkg.default_options(lanes=lanes, self_collision=1))
    counters = []
    for p in (pid, pid_self):
        scene.set_particles(p, X.T.astype(np.float32))
        scene.optimize(p, 0)
        counters.append(scene.work_counters(p))
    scene.close()
    assert counters[0][0] == counters[1][0] and counters[0][0] > 0, counters


def test_scene_on_a_caller_supplied_allocator(pkg):
    """A scene whose device memory comes from PyTorch's caching allocator
    (tamp_allocator callbacks) computes what a cudaMalloc scene computes, and
    gives every block back."""
    sc, acts = sg.packing_problem(2001)
    X = sg.random_particles(sc, acts, 200, seed=9).T.astype(np.float32)

    def run(torch_allocator):
        scene = pkg.Scene(sc, torch_allocator=torch_allocator)
        pid = scene.set_skeleton(acts)
        scene.set_particles(pid, X)
        scene.optimize(pid, 3)
        x = scene.get_particles(pid)[0]
        q = scene.query(pid, 200)
        g = pkg.Graph(scene, pid, 2, 2)
        g.run()
        g.close()
        live = dict(scene._alloc[2]) if torch_allocator else {}
        scene.close()
        return x, q, live, (scene._alloc[2] if torch_allocator else {})

    x0, q0, _, _ = run(False)
    x1, q1, live, after = run(True)
    assert len(live) > 0                     # the scene's buffers came from the callbacks
    assert len(after) == 0                   # ... and were all given back
    assert np.abs(x1 - x0).max() < 1e-4
    assert cost_ok(q1["cost"].astype(np.float64), q0["cost"].astype(np.float64)).mean() > 0.99
