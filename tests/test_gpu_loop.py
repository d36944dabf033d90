"""The optimisation loop through the C ABI against the FP64 oracle: CUDA-graph
replay, the device-side stop on the first satisfying particle (graph and
tamp_optimize_steps), several problems in one persistent launch, odd cuboid
counts in the paired broad phase, a caller-supplied allocator, and the
best-satisfying record (tamp_query_best).

Multi-step trajectories follow the rule of tests/parity.py (check_trajectory).
"""
import dataclasses

import numpy as np
import pytest
import torch

import scenegen as sg
from oracle import philox
from oracle.problem import Problem
from tests.parity import (KINK_MARGIN, TRAJ_MARGIN, check_adam_step, check_trajectory, cost_ok, cost_sum_bound,
                          near_threshold, oracle_run)

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
    xt = torch.tensor(x.astype(np.float32).astype(np.float64))
    T = pr.term_values(xt)
    ref = pr.constraint_counts(T).numpy()
    band = near_threshold(pr, T.numpy(), pr.kink_margin(xt).numpy())
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


def _check_best_valid(pr, best):
    """Every recorded state satisfies Eq. 3 in the oracle (a particle within 1e-5
    of a tolerance may fall either side) at the cost the record gives."""
    f = best["found"]
    if not f.any():
        return 0
    xb = best["particles"].T[f].astype(np.float64)
    T = pr.term_values(torch.tensor(xb))
    ok = pr.satisfied(T).numpy() | near_threshold(pr, T.numpy())
    assert ok.all(), f"{int((~ok).sum())} recorded states do not satisfy Eq. 3"
    cost = (T * pr.weights()).sum(1).numpy()
    bad = np.abs(best["cost"][f].astype(np.float64) - cost) > cost_sum_bound(pr, T.numpy())
    if bad.any():
        idx = np.nonzero(f)[0][bad]
        marg = pr.kink_margin(torch.tensor(xb[bad])).numpy()
        raise AssertionError(f"record costs differ from the oracle's at the recorded state: particles {idx[:6]}, "
                             f"gpu {best['cost'][idx[:6]]}, oracle {cost[bad][:6]}, checks {best['iter'][idx[:6]]}, "
                             f"kink margins {marg[:6]}, terms {T.numpy()[bad][:2]}")
    assert np.isinf(best["cost"][~f]).all() and (best["iter"][~f] == -1).all()
    return int(f.sum())


def test_best_record_is_the_lowest_cost_satisfying_check(pkg):
    """tamp_query_best against its definition on the run's own checks, each
    check pinned to the oracle.  200 particles (7 tiles, a ragged tail of 8)
    around the SCARA witness, whose satisfying checks come and go as Adam moves
    them, run 30 single-iteration calls (the record runs across calls); after
    each call the state x_k, the Eq. 3 mask and Eq. 2 costs of its last check
    are read back.  Every check must agree with the oracle evaluated at the same
    FP32 state (flags, except within 1e-5 of a tolerance; costs within the
    bound the per-term rule implies), and the record must be the state of the
    lowest-cost satisfying check (bit for bit), with its cost and index.

    Near satisfaction the FP32 and FP64 trajectories themselves part ways: a
    Kin error norm passing near zero turns a rounding difference d into a
    gradient direction change d/|e|, which the next step (about the learning
    rate) multiplies by lr/|e| (60 at |e| = 1.6e-4; measured: smooth-margin
    particles 1.4e-2 apart after 30 steps), so the record is checked on the
    run's own iterates rather than against the oracle's trajectory."""
    from tests.test_oracle_pins import _scara_witness_scene
    sc, acts, x = _scara_witness_scene()
    pr = Problem(sc, acts)
    P, n = 200, 30
    rng = np.random.default_rng(3)
    X = np.repeat(x.numpy(), P, axis=0)
    X[1:] += rng.normal(0.0, 0.002, (P - 1, X.shape[1]))
    X[-5:, 4:11] += 0.3                                # far off: never satisfy
    X = X.astype(np.float32).astype(np.float64)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts, pkg.default_options(keep_best=1))
    scene.set_particles(pid, X.T.astype(np.float32))
    xs, masks, costs = [], [], []
    for k in range(n + 1):
        if k:
            scene.optimize(pid, 1)
        q = scene.query(pid, P)                        # k = 0: the check of the batch as set
        xs.append(scene.get_particles(pid)[0].T.copy())
        masks.append(q["mask"])
        costs.append(q["cost"].astype(np.float64))
    best = scene.query_best(pid, P)
    scene.close()
    S, C = np.array(masks).T, np.array(costs).T       # [P, n + 1]
    near = np.zeros_like(S)
    for k in range(n + 1):
        T = pr.term_values(torch.tensor(xs[k].astype(np.float64)))
        near[:, k] = near_threshold(pr, T.numpy())
        ok = (pr.satisfied(T).numpy() == S[:, k]) | near[:, k]
        assert ok.all(), f"check {k}: Eq. 3 flags differ for particles {np.nonzero(~ok)[0][:8]}"
        c_ora = (T * pr.weights()).sum(1).numpy()
        assert (np.abs(C[:, k] - c_ora) <= cost_sum_bound(pr, T.numpy())).all(), f"check {k}: costs"
    assert _check_best_valid(pr, best) == best["n_found"]
    # a particle re-checked at the start of a call (same state as the last check
    # of the call before) may take the recheck's cost, equal up to the order of
    # its summed collision contributions; particles with a flag within 1e-5 of a
    # tolerance at some check are only checked for validity (above)
    strict = ~near.any(axis=1)
    assert np.array_equal(S.any(axis=1)[strict], best["found"][strict])
    n_sat_checks = 0
    for p in np.nonzero(strict & best["found"])[0]:
        ks = np.nonzero(S[p])[0]
        kg = int(best["iter"][p])
        assert kg in set(ks.tolist()), (p, kg, ks)
        tie = 1e-5 * max(abs(C[p, ks].min()), 1e-2)
        assert C[p, kg] <= C[p, ks].min() + tie, (p, kg, C[p, ks])
        assert abs(np.float64(best["cost"][p]) - C[p, kg]) <= tie
        assert np.array_equal(best["particles"][:, p], xs[kg][p].astype(np.float32)), p
        n_sat_checks += len(ks)
    print(dict(found=best["n_found"], strict=int(strict.sum()), satisfying_checks=n_sat_checks))
    assert strict.sum() >= P // 2 and best["n_found"] >= 100


def test_best_record_is_kept_only_where_asked(pkg):
    """Plain optimisation launches skip the record unless the problem's options
    ask for it (keep_best); the stop mode keeps it.  The same witness batch,
    which satisfies at its first check, in three problems of one scene."""
    from tests.test_oracle_pins import _scara_witness_scene
    sc, acts, x = _scara_witness_scene()
    X = np.repeat(x.numpy(), 8, axis=0).T.astype(np.float32)
    scene = pkg.Scene(sc)
    plain = scene.set_skeleton(acts)
    kept = scene.set_skeleton(acts, pkg.default_options(keep_best=1))
    stop = scene.set_skeleton(acts)
    for pid in (plain, kept, stop):
        scene.set_particles(pid, X)
    scene.optimize(plain, 5)
    scene.optimize(kept, 5)
    scene.optimize(stop, 5, stop_every=5)
    found = [scene.query_best(pid, 8, want_particles=False)["n_found"] for pid in (plain, kept, stop)]
    firsts = [scene.query(pid, 8)["first_iter"] for pid in (plain, kept, stop)]
    scene.close()
    assert firsts == [0, 0, 0]
    assert found[0] == 0 and found[1] == 8 and found[2] == 8


def test_stop_on_first_satisfying_keeps_the_satisfying_state(pkg):
    """After tamp_optimize_steps stops on the first satisfying particle, the
    particle that satisfied is in the record, even where the updates after its
    check moved it out of the feasible set (the witness does so after one
    update: Kin's gradient has unit size at zero error).  The record's earliest
    check is the first satisfying iteration, and each recorded state satisfies
    Eq. 3 in the oracle."""
    from tests.test_oracle_pins import _scara_witness_scene
    sc, acts, x = _scara_witness_scene()
    pr = Problem(sc, acts)
    X = np.repeat(x.numpy(), 40, axis=0)
    X[1:] += np.random.default_rng(4).normal(0.0, 0.002, (39, X.shape[1]))
    X = X.astype(np.float32).astype(np.float64)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    scene.set_particles(pid, X.T.astype(np.float32))
    scene.optimize(pid, 100, stop_every=10)
    t = scene.get_particles(pid)[3]
    q = scene.query(pid, 40)
    best = scene.query_best(pid, 40)
    scene.close()
    assert t == 10 and q["first_iter"] == 0
    assert best["n_found"] >= 1 and best["found"][0] and best["iter"][0] == 0
    assert best["iter"][best["found"]].min() == q["first_iter"]
    assert (best["iter"][best["found"]] <= t).all()
    # the witness, recorded at x_0, is the state that was set
    assert np.array_equal(best["particles"][:, 0], X[0].astype(np.float32))
    _check_best_valid(pr, best)


def test_graph_stop_keeps_the_satisfying_states_of_every_problem(pkg):
    """A CUDA graph stopping on the first satisfying particle, over two
    problems in one launch: the witness batch (perturbed copies of the SCARA
    witness, which satisfies at x_0) and the same skeleton from particles far
    from it (joints moved 0.3 rad: no particle satisfies in the 5 iterations
    that run).  The first problem's record holds its satisfying states, each
    satisfying Eq. 3 in the oracle, the witness at x_0 among them; the second's
    stays empty."""
    from tests.test_oracle_pins import _scara_witness_scene
    sc, acts, x = _scara_witness_scene()
    pr = Problem(sc, acts)
    X = np.repeat(x.numpy(), 40, axis=0)
    X[1:] += np.random.default_rng(5).normal(0.0, 0.002, (39, X.shape[1]))
    X = X.astype(np.float32).astype(np.float64)
    Y = X.copy()
    Y[:, 4:11] += 0.3
    scene = pkg.Scene(sc)
    p1, p2 = scene.set_skeleton(acts), scene.set_skeleton(acts)
    scene.set_particles(p1, X.T.astype(np.float32))
    scene.set_particles(p2, Y.T.astype(np.float32))
    g = pkg.Graph(scene, [p1, p2], 5, 10, stop_on_first=True)
    steps = g.run()
    g.close()
    b1, b2 = scene.query_best(p1, 40), scene.query_best(p2, 40)
    q1 = scene.query(p1, 40)
    scene.close()
    assert steps == 5 and q1["first_iter"] == 0
    assert b1["n_found"] >= 1 and b1["found"][0] and b1["iter"][0] == 0
    assert np.array_equal(b1["particles"][:, 0], X[0].astype(np.float32))
    assert b1["iter"][b1["found"]].min() == 0 and (b1["iter"][b1["found"]] <= steps).all()
    _check_best_valid(pr, b1)
    assert b2["n_found"] == 0


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
    gives every block back.  The two run side by side one step at a time; as
    with any two launches, a particle may part ways only at a step that starts
    near a kink (oracle margin below TRAJ_MARGIN), every other one agrees to
    1e-5 after each step, and the costs of those that never parted agree."""
    sc, acts = sg.packing_problem(2001)
    n = 200
    pr = Problem(sc, acts)
    X = sg.random_particles(sc, acts, n, seed=9).T.astype(np.float32)
    scenes = [pkg.Scene(sc), pkg.Scene(sc, torch_allocator=True)]
    pids = [s.set_skeleton(acts) for s in scenes]
    for s, pid in zip(scenes, pids):
        s.set_particles(pid, X)
    assert len(scenes[1]._alloc[2]) > 0      # the scene's buffers came from the callbacks
    alive = np.ones(n, bool)
    parted = 0
    for step in range(3):
        x0 = scenes[0].get_particles(pids[0])[0].T.astype(np.float64)
        for s, pid in zip(scenes, pids):
            s.optimize(pid, 1)
        d = np.abs(scenes[0].get_particles(pids[0])[0] - scenes[1].get_particles(pids[1])[0]).max(axis=0)
        off = alive & (d > 1e-5)
        if off.any():
            near = pr.kink_margin(torch.tensor(x0[off])).numpy() < TRAJ_MARGIN
            assert near.all(), f"step {step}: a particle away from kinks parted ({d[off].max():.2e})"
            parted += int(off.sum())
            alive &= ~off
    q = [s.query(pid, n) for s, pid in zip(scenes, pids)]
    assert cost_ok(q[1]["cost"].astype(np.float64), q[0]["cost"].astype(np.float64))[alive].all()
    assert parted <= 0.25 * n
    for s, pid in zip(scenes, pids):
        g = pkg.Graph(s, pid, 2, 2)
        g.run()
        g.close()
    live = dict(scenes[1]._alloc[2])
    for s in scenes:
        s.close()
    assert len(live) > 0 and len(scenes[1]._alloc[2]) == 0   # ... and were all given back
