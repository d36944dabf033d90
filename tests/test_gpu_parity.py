"""CUDA path vs FP64 oracle, element by element, through the C ABI."""
import math

import numpy as np
import pytest
import torch

import scenegen as sg
from oracle import philox
from oracle.problem import Options, Problem
from tests.parity import check_adam_step, check_trajectory, compare_eval, cost_ok, grad_errors, oracle_run

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
    """100-sphere arm, 64 cuboids, 12 boxes, 24 configurations.  Contacts are
    dense here (about half the particles sit within 1e-4 of a kink), so the
    batch is large enough for the gradient comparison to keep 40 or more."""
    sc, acts = sg.stress_problem(5001)
    X = sg.random_particles(sc, acts, 96, seed=51, spread=0.0)
    res = compare_eval(Problem(sc, acts), X, *_eval(pkg, sc, acts, X, 1), label="stress", min_kept=0.4)
    assert res["kept"] >= 40, res
    print(res)


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
    X32 = X.astype(np.float32).astype(np.float64)
    keep = pr.kink_margin(torch.tensor(X32)).numpy() > 1e-4
    print(check_adam_step(pr, X32, m0.astype(np.float32).astype(np.float64), v0.astype(np.float32).astype(np.float64),
                          t0, x1.T, m1.T, P, keep))


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
    stay together except where a particle comes near a kink (counted; the
    rule of tests/parity.py check_trajectory)."""
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
    out, margin = oracle_run(pr, X.astype(np.float32).astype(np.float64), 10)
    assert t == 10
    print(check_trajectory(pr, x10.T, q["cost"], out, margin))


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
    xt = torch.tensor(X.astype(np.float32).astype(np.float64))
    T = pr.term_values(xt)
    counts = pr.constraint_counts(T).numpy()
    from tests.parity import near_threshold
    band = near_threshold(pr, T.numpy(), pr.kink_margin(xt).numpy())
    assert band.sum() < P // 2, f"{int(band.sum())} of {P} particles near a tolerance: the check would be vacuous"
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
    (2 lanes, 16 warps): one fused iteration, then 48 sampled particles checked
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
    idx = np.random.default_rng(3).choice(P, 48, replace=False)
    Xs = X[idx].astype(np.float64)
    keep = pr.kink_margin(torch.tensor(Xs)).numpy() > 1e-4
    assert keep.sum() >= 16, keep.sum()
    zeros = np.zeros_like(Xs)
    print(check_adam_step(pr, Xs, zeros, zeros, 0, x1.T[idx], m1.T[idx], P, keep))


def test_packing_full_batch_two_launches_sampled(pkg):
    """The packing workload at the benchmark's batch (4096 particles) in its
    launch shape (1 lane, 16 warps): two launches of one fused iteration each,
    the second starting at Adam step 1 (bias corrections 1 / (1 - beta^2) from
    the step count carried over).  48 sampled particles are checked one by one:
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
    idx = np.random.default_rng(4).choice(P, 48, replace=False)

    def check(x0, m0, v0, t0, x_gpu, m_gpu):
        xs = x0[idx].astype(np.float64)
        keep = pr.kink_margin(torch.tensor(xs)).numpy() > 1e-4
        assert keep.sum() >= 16, keep.sum()
        print(check_adam_step(pr, xs, m0[idx].astype(np.float64), v0[idx].astype(np.float64), t0, x_gpu[idx],
                              m_gpu[idx], P, keep))

    zeros = np.zeros_like(X)
    check(X, zeros, zeros, 0, x1.T, m1.T)
    check(x1.T, m1.T, v1.T, 1, x2.T, m2.T)
