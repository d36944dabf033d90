"""CUDA path vs FP64 oracle, element by element, through the C ABI."""
import math

import numpy as np
import pytest
import torch

import scenegen as sg
from oracle import philox
from oracle.problem import Options, Problem
from tests.parity import compare_eval, cost_ok, grad_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2411_11833_b300.build import build_library
    build_library()
    import paper_2411_11833_b300 as p
    torch.cuda.set_device(0)
    return p


def _dev(X):
    return torch.tensor(np.ascontiguousarray(X.T), dtype=torch.float32, device="cuda")


def _eval(pkg, sc, acts, X, lanes=0):
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts, pkg.default_options(lanes=lanes))
    out = scene.eval(pid, _dev(X))
    torch.cuda.synchronize()
    scene.close()
    return out


@pytest.mark.parametrize("lanes", [1, 2, 4, 8])
def test_eval_parity_plain(pkg, lanes):
    sc, acts = sg.plain_problem(1001)
    X = sg.random_particles(sc, acts, 203, seed=31)          # several tiles + a ragged tail
    res = compare_eval(Problem(sc, acts), X, *_eval(pkg, sc, acts, X, lanes), label=f"plain L={lanes}")
    print(res)


@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_eval_parity_packing(pkg, lanes):
    sc, acts = sg.packing_problem(2001)
    X = sg.random_particles(sc, acts, 77, seed=32)
    res = compare_eval(Problem(sc, acts), X, *_eval(pkg, sc, acts, X, lanes), label=f"packing L={lanes}")
    print(res)


@pytest.mark.parametrize("seed", [1002, 1003, 1004])
def test_eval_parity_other_plain_scenes(pkg, seed):
    sc, acts = sg.plain_problem(seed)
    X = sg.random_particles(sc, acts, 64, seed=seed)
    compare_eval(Problem(sc, acts), X, *_eval(pkg, sc, acts, X), label=f"plain seed {seed}")


def test_eval_single_particle_and_full_warp(pkg):
    sc, acts = sg.packing_problem(2002)
    for n in (1, 32, 33):
        X = sg.random_particles(sc, acts, n, seed=40 + n)
        compare_eval(Problem(sc, acts), X, *_eval(pkg, sc, acts, X, 2), label=f"n={n}")


def test_eval_stress_scene_sampled(pkg):
    """100-sphere arm, 64 cuboids, 12 boxes, 24 configurations."""
    sc, acts = sg.stress_problem(5001)
    X = sg.random_particles(sc, acts, 12, seed=51)
    compare_eval(Problem(sc, acts), X, *_eval(pkg, sc, acts, X, 1), label="stress")


def test_eval_full_size_packing_sampled(pkg):
    """4096 particles (the benchmark batch) evaluated in one launch; the oracle
    checks a sample of them one by one."""
    sc, acts = sg.packing_problem(2001)
    X = sg.random_particles(sc, acts, 4096, seed=33)
    cost, terms, flags, grad = _eval(pkg, sc, acts, X)
    idx = np.random.default_rng(0).choice(4096, 48, replace=False)
    compare_eval(Problem(sc, acts), X[idx], cost[idx], terms[:, idx], flags[idx], grad[:, idx], label="4096 sampled")


def test_uniform_sampler_matches_oracle_philox(pkg):
    sc, acts = sg.packing_problem(2001)
    pr = Problem(sc, acts)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    scene.sample(pid, 1000, seed=0x1234_5678_9ABC)
    x, m, v, t = scene.get_particles(pid)
    ref = philox.sample_uniform(pr, 1000, 0x1234_5678_9ABC)
    assert np.abs(x.T - ref).max() < 2e-6
    assert not m.any() and not v.any() and t == 0
    scene.close()


def test_adam_step_matches_oracle(pkg):
    sc, acts = sg.plain_problem(1001)
    pr = Problem(sc, acts)
    P = 150
    X = sg.random_particles(sc, acts, P, seed=61)
    m0, v0 = sg.random_adam_state(P, pr.D, seed=62)
    t0 = 7
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    scene.set_particles(pid, X.T.astype(np.float32), m0.T.astype(np.float32), v0.T.astype(np.float32), t0)
    scene.optimize(pid, 1)
    x1, m1, v1, t1 = scene.get_particles(pid)
    scene.close()
    assert t1 == t0 + 1
    Xt = torch.tensor(X.astype(np.float32).astype(np.float64))
    _, g = pr.gradient(Xt)
    xr, mr, vr = pr.adam_step(Xt, torch.tensor(m0.astype(np.float32).astype(np.float64)),
                              torch.tensor(v0.astype(np.float32).astype(np.float64)), t0 + 1, g, P)
    margin = pr.kink_margin(Xt).numpy()
    keep = margin > 1e-4
    dm = np.abs(m1.T - mr.numpy())[keep]
    assert dm.max() <= 1e-3 * np.abs(mr.numpy()[keep]).max() + 1e-9
    # the update is lr * m_hat / (sqrt(v_hat) + eps): compare the step taken
    step_g = (x1.T - X.astype(np.float32))[keep]
    step_r = (xr.numpy() - Xt.numpy())[keep]
    assert np.abs(step_g - step_r).max() <= 1e-3 * np.abs(step_r).max() + 2e-6


def test_first_satisfying_iteration_of_witness(pkg):
    from tests.test_oracle_pins import _scara_witness_scene
    sc, acts, x = _scara_witness_scene()
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    X = np.repeat(x.numpy(), 5, axis=0)
    scene.set_particles(pid, X.T.astype(np.float32))
    q0 = scene.query(pid, 5)               # the check at x_0 alone
    scene.optimize(pid, 3)
    q = scene.query(pid, 5)
    scene.close()
    assert q0["n_satisfied"] == 5 and q0["first_iter"] == 0
    assert q["first_iter"] == 0


def test_optimize_trajectory_tracks_oracle(pkg):
    """Ten fused Adam iterations from the same particles: FP32 vs FP64 paths
    stay together except where a particle crosses a kink (counted)."""
    sc, acts = sg.plain_problem(1001)
    pr = Problem(sc, acts)
    P = 64
    X = philox.sample_uniform(pr, P, 77)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    scene.set_particles(pid, X.T.astype(np.float32))
    scene.optimize(pid, 10)
    x10, _, _, t = scene.get_particles(pid)
    q = scene.query(pid, P)
    scene.close()
    out = pr.optimize(torch.tensor(X.astype(np.float32).astype(np.float64)), 10)
    d = np.abs(x10.T - out["x"].numpy()).max(axis=1)
    close = d < 1e-3
    assert t == 10
    assert close.mean() >= 0.8, f"only {close.mean():.2f} of trajectories agree"
    ok = cost_ok(q["cost"][close].astype(np.float64), out["cost"].numpy()[close]) | (np.abs(q["cost"][close] - out["cost"].numpy()[close]) < 1e-3)
    assert ok.all()


def test_counts_and_mask_match_oracle(pkg):
    sc, acts = sg.packing_problem(2001)
    pr = Problem(sc, acts)
    P = 300
    X = sg.random_particles(sc, acts, P, seed=71, spread=0.0)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    scene.set_particles(pid, X.T.astype(np.float32))
    q = scene.query(pid, P)
    scene.close()
    T = pr.term_values(torch.tensor(X.astype(np.float32).astype(np.float64)))
    counts = pr.constraint_counts(T).numpy()
    from tests.parity import near_threshold
    band = near_threshold(pr, T.numpy())
    assert np.abs(q["counts"] - counts).max() <= band.sum()
    assert ((q["mask"] != pr.satisfied(T).numpy()) & ~band).sum() == 0


def test_cost_autograd_function(pkg):
    sc, acts = sg.plain_problem(1001)
    pr = Problem(sc, acts)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    X = sg.random_particles(sc, acts, 50, seed=81)
    x = torch.tensor(X, dtype=torch.float32, device="cuda", requires_grad=True)
    CostFn = pkg.cost_fn()
    J = CostFn.apply(x, scene, pid)
    (J * torch.linspace(0.5, 1.5, 50, device="cuda")).sum().backward()
    scene.close()
    Jr, gr = pr.gradient(torch.tensor(X.astype(np.float32).astype(np.float64)))
    w = np.linspace(0.5, 1.5, 50)
    margin = pr.kink_margin(torch.tensor(X)).numpy() > 1e-4
    err, bound = grad_errors(x.grad.cpu().double().numpy()[margin], (gr.numpy() * w[:, None])[margin])
    assert (err <= bound).all()


def test_invalid_skeleton_rejected(pkg):
    sc, acts = sg.plain_problem(1001)
    scene = pkg.Scene(sc)
    with pytest.raises(pkg.TampError):
        scene.set_skeleton([(1, 0, 0)])
    with pytest.raises(pkg.TampError):
        scene.set_skeleton([(0, 5, -1)])
    scene.close()


def test_no_obstacles_no_other_boxes(pkg):
    sc, acts = sg.plain_problem(1001)
    import dataclasses
    sc0 = dataclasses.replace(sc, obs_center=np.zeros((0, 3)), obs_rot=np.zeros((0, 3, 3)), obs_half=np.zeros((0, 3)))
    X = sg.random_particles(sc0, acts, 40, seed=91)
    compare_eval(Problem(sc0, acts), X, *_eval(pkg, sc0, acts, X), label="empty environment")


def test_batched_launch_matches_separate_launches(pkg):
    """Skeletons of different lengths and batch sizes share one persistent
    launch; every tile is independent, so the result equals separate launches
    up to the order of float atomic additions (shared-variable gradients and
    contact sums are accumulated with shared-memory atomics): after 6 Adam steps
    nearly every component agrees to 1e-4 and costs agree to 1e-4 relative."""
    sc, _ = sg.packing_problem(2001)
    skels = [sg.pick_place_skeleton([0]), sg.pick_place_skeleton([0, 1, 2]),
             sg.pick_place_skeleton(range(6), goal=True)]
    sizes = [100, 70, 45]
    opts = pkg.default_options(lanes=1)

    def run(batched):
        scene = pkg.Scene(sc)
        pids = [scene.set_skeleton(a, opts) for a in skels]
        for pid, n, a in zip(pids, sizes, skels):
            X = sg.random_particles(sc, a, n, seed=100 + n, spread=0.5)
            scene.set_particles(pid, X.T.astype(np.float32))
        if batched:
            scene.optimize(pids, 6)
        else:
            for pid in pids:
                scene.optimize(pid, 6)
        out = [scene.get_particles(pid)[0] for pid in pids]
        qs = [scene.query(pid, n) for pid, n in zip(pids, sizes)]
        scene.close()
        return out, qs

    xb, qb = run(True)
    xs, qs = run(False)
    for a, b in zip(xb, xs):
        d = np.abs(a - b)
        assert (d < 1e-4).mean() > 0.99 and d.max() < 0.1
    for a, b in zip(qb, qs):
        close = np.abs(a["cost"] - b["cost"]) <= 1e-4 * np.maximum(np.abs(b["cost"]), 0.1)
        assert close.mean() > 0.95


def test_batched_problem_matches_oracle(pkg):
    """A short skeleton in a batched launch still matches the oracle."""
    sc, _ = sg.packing_problem(2001)
    acts = sg.pick_place_skeleton([0, 1])
    pr = Problem(sc, acts)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    other = scene.set_skeleton(sg.pick_place_skeleton(range(6), goal=True))
    X = sg.random_particles(sc, acts, 64, seed=5)
    scene.set_particles(pid, X.T.astype(np.float32))
    scene.sample(other, 200, seed=3)
    scene.optimize([other, pid], 0)              # evaluation only
    q = scene.query(pid, 64)
    scene.close()
    J = pr.total_cost(torch.tensor(X.astype(np.float32).astype(np.float64))).numpy()
    assert cost_ok(q["cost"].astype(np.float64), J).all()


def test_graph_replays_the_optimisation_loop(pkg):
    """4 captured chunks of 5 fused iterations == 20 iterations of tamp_optimize_steps
    (up to float-atomic reordering); the step count advances on the device."""
    sc, acts = sg.plain_problem(1001)
    X = sg.random_particles(sc, acts, 150, seed=21, spread=0.5).T.astype(np.float32)

    def run(graph):
        scene = pkg.Scene(sc)
        pid = scene.set_skeleton(acts)
        scene.set_particles(pid, X)
        if graph:
            g = pkg.Graph(scene, pid, 5, 4)
            steps = g.run()
            g.close()
        else:
            scene.optimize(pid, 20)
            steps = 20
        x, _, _, t = scene.get_particles(pid)
        q = scene.query(pid, 150)
        scene.close()
        return x, t, steps, q

    xg, tg, sg_, qg = run(True)
    xo, to, _, qo = run(False)
    assert sg_ == 20 and tg == 20 and to == 20
    d = np.abs(xg - xo)
    assert (d < 1e-4).mean() > 0.99
    assert qg["first_iter"] == qo["first_iter"]


def test_graph_stops_on_first_satisfying_particle(pkg):
    from tests.test_oracle_pins import _scara_witness_scene
    sc, acts, x = _scara_witness_scene()
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    scene.set_particles(pid, np.repeat(x.numpy(), 3, axis=0).T.astype(np.float32))
    g = pkg.Graph(scene, pid, 5, 10, stop_on_first=True)
    steps = g.run()
    q = scene.query(pid, 3)
    g.close()
    scene.close()
    assert steps == 5 and q["first_iter"] == 0


def test_stacking_skeleton_parity(pkg):
    """Obstructed stacking: blockers standing on B, A placed on B's top face."""
    sc, skels, _ = sg.stacking_problem(3002)
    acts = max(skels, key=len)
    X = sg.random_particles(sc, acts, 70, seed=8)
    compare_eval(Problem(sc, acts), X, *_eval(pkg, sc, acts, X), label="stacking")


def test_stacking_searches_run_end_to_end(pkg):
    from paper_2411_11833_b300.search import batched_search, sequential_search
    sc, skels, sizes = sg.stacking_problem(3001)
    small = [max(64, n // 32) for n in sizes]
    scene = pkg.Scene(sc)
    out = batched_search(scene, skels, small, steps_per_chunk=10, max_iterations=30, seed=1)
    assert out["iterations"] in (10, 20, 30)
    scene.close()
    scene = pkg.Scene(sc)
    out = sequential_search(scene, skels[:4], small[:4], steps_per_chunk=10, chunks_per_visit=1,
                            max_iterations=20, seed=1)
    assert out["solved"] or out["iterations"] == 4 * 20
    scene.close()


def test_stress_full_batch_adam_step_sampled(pkg):
    """The stress workload at its full batch (65536 particles, D = 252, 24
    configurations) in the launch shape the benchmark's tuner picks for it
    (2 lanes, 16 warps): one fused iteration, then 32 sampled particles checked
    against the oracle's gradient + Adam step one by one (those within 1e-4 of a
    kink of the 64-cuboid scene are left out and counted)."""
    sc, acts = sg.stress_problem(5001)
    pr = Problem(sc, acts)
    P = 65536
    X = sg.random_particles(sc, acts, P, seed=81, spread=0.5).astype(np.float32)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    scene.set_particles(pid, np.ascontiguousarray(X.T))
    scene.set_tuning(pid, 2, 16)
    scene.optimize(pid, 1)
    x1, m1, _, t1 = scene.get_particles(pid)
    scene.close()
    assert t1 == 1
    idx = np.random.default_rng(3).choice(P, 32, replace=False)
    Xs = torch.tensor(X[idx].astype(np.float64))
    _, g = pr.gradient(Xs)
    xr, mr, _ = pr.adam_step(Xs, torch.zeros_like(Xs), torch.zeros_like(Xs), 1, g, P)
    keep = pr.kink_margin(Xs).numpy() > 1e-4
    assert keep.sum() >= 8, keep.sum()
    dm = np.abs(m1.T[idx] - mr.numpy())[keep]
    assert dm.max() <= 1e-3 * np.abs(mr.numpy()[keep]).max() + 1e-12
    step_g = (x1.T[idx] - X[idx])[keep]
    step_r = (xr.numpy() - Xs.numpy())[keep]
    # first Adam step: -lr * g / (|g| + eps), so compare the steps' signs and sizes
    assert np.abs(step_g - step_r).max() <= 1e-3 * np.abs(step_r).max() + 2e-6


def test_packing_full_batch_two_launches_sampled(pkg):
    """The packing workload at the benchmark's batch (4096 particles) in its
    launch shape (1 lane, 16 warps): two launches of one fused iteration each,
    the second starting at Adam step 1 (bias corrections 1 / (1 - beta^2) from
    the step count carried over).  32 sampled particles are checked one by one:
    the first step against the oracle's gradient + Adam step from the initial
    batch, the second against the oracle's step from the GPU's own state after
    the first (particles within 1e-4 of a kink are left out)."""
    sc, acts = sg.packing_problem(2001)
    pr = Problem(sc, acts)
    P = 4096
    X = sg.random_particles(sc, acts, P, seed=82).astype(np.float32)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    scene.set_particles(pid, np.ascontiguousarray(X.T))
    scene.set_tuning(pid, 1, 16)
    scene.optimize(pid, 1)
    x1, m1, v1, t1 = scene.get_particles(pid)
    scene.optimize(pid, 1)
    x2, m2, v2, t2 = scene.get_particles(pid)
    scene.close()
    assert (t1, t2) == (1, 2)
    idx = np.random.default_rng(4).choice(P, 32, replace=False)

    def check(x0, m0, v0, t, x_gpu, m_gpu):
        xs = torch.tensor(x0[idx].astype(np.float64))
        keep = pr.kink_margin(xs).numpy() > 1e-4
        assert keep.sum() >= 8, keep.sum()
        _, g = pr.gradient(xs)
        xr, mr, _ = pr.adam_step(xs, torch.tensor(m0[idx].astype(np.float64)),
                                 torch.tensor(v0[idx].astype(np.float64)), t, g, P)
        dm = np.abs(m_gpu[idx] - mr.numpy())[keep]
        assert dm.max() <= 1e-3 * np.abs(mr.numpy()[keep]).max() + 1e-12
        step_g = (x_gpu[idx] - x0[idx])[keep]
        step_r = (xr.numpy() - xs.numpy())[keep]
        assert np.abs(step_g - step_r).max() <= 1e-3 * np.abs(step_r).max() + 2e-6

    zeros = np.zeros_like(X)
    check(X, zeros, zeros, 1, x1.T, m1.T)
    check(x1.T, m1.T, v1.T, 2, x2.T, m2.T)
