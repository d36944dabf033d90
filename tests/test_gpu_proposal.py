"""Learned proposals through the C ABI vs the oracle (oracle/proposal.py,
oracle/mlp.py): the feature rows and training targets the library builds, and
the particles sampler 1 draws from a network's outputs."""
import math

import numpy as np
import pytest
import torch

import scenegen as sg
from oracle import mlp as om
from oracle import philox
from oracle import proposal as op
from oracle.problem import GRASP, STABLE_PLACE, Problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2411_11833_b300.build import build_library
    build_library()
    import paper_2411_11833_b300 as p
    torch.cuda.set_device(0)
    return p


def _wrap(a):
    return (a + math.pi) % (2 * math.pi) - math.pi


def _params(seed, out_scale=1.0):
    th = om.init_params(seed).numpy()
    g = np.random.default_rng(seed)
    o = 0
    for li, ((wr, wc), (bn,)) in enumerate(om.shapes()):
        o += wr * wc
        th[o:o + bn] = g.normal(0.0, 0.1 if li < 3 else out_scale, bn)
        o += bn
    return th.astype(np.float32)


@pytest.mark.parametrize("maker", [lambda: sg.plain_problem(1001), lambda: sg.packing_problem(2001),
                                   lambda: (lambda s: (s[0], s[1][-1]))(sg.stacking_problem(3001))])
def test_proposal_rows_match_oracle(pkg, maker):
    sc, acts = maker()
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    X = philox.sample_uniform(Problem(sc, acts), 64, 21).astype(np.float32)
    F, Y, M = scene.proposal_rows(pid, X.T)
    Fo, Yo, Mo = op.encode(sc, acts, X.astype(np.float64))
    assert scene.proposal_rows(pid) == len(op.action_rows(sc, acts))
    assert np.abs(F - Fo).max() < 1e-6
    assert np.array_equal(M, Mo)
    assert np.abs(Y - Yo).max() < 1e-5
    scene.close()


@pytest.mark.parametrize("maker", [lambda: sg.plain_problem(1002), lambda: sg.packing_problem(2003)])
def test_proposal_sampler_matches_oracle(pkg, maker):
    sc, acts = maker()
    pr = Problem(sc, acts)
    th = _params(17)
    net = pkg.Mlp(max_batch=64)
    net.set_params(th)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    scene.set_proposal(net)
    n, seed = 2000, 0xBEEF_0042
    scene.sample(pid, n, seed, sampler=1)
    x, m, v, t = scene.get_particles(pid)
    x = x.T.astype(np.float64)
    assert not m.any() and not v.any() and t == 0
    out = om.forward(torch.from_numpy(th).double(), torch.from_numpy(op.features(sc, acts))).numpy()
    ref = op.sample(sc, acts, out, n, seed)
    kinds = np.array(pr.kinds)
    q = kinds == "q"
    assert np.abs(x[:, q] - ref[:, q]).max() < 2e-6            # joints: the uniform sampler's
    pos = np.isin(kinds, ["gpos", "ppos"])
    assert np.abs(x[:, pos] - ref[:, pos]).max() < 1e-4
    yaw = np.isin(kinds, ["gyaw", "pyaw"])
    dy = np.abs(_wrap(x[:, yaw] - ref[:, yaw]))
    # atan2 of two slots is ill-conditioned only where both are near zero
    assert np.mean(dy < 1e-3) > 0.995 and np.median(dy) < 1e-5
    # the seeds differ from the uniform ones (the network is in use)
    U = philox.sample_uniform(pr, n, seed)
    assert np.abs(x[:, pos] - U[:, pos]).max() > 1e-3
    scene.close()
    net.close()


def test_proposal_sampler_needs_a_network(pkg):
    from paper_2411_11833_b300 import TampError
    sc, acts = sg.plain_problem(1001)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    with pytest.raises(TampError, match="STATE"):
        scene.sample(pid, 100, 1, sampler=1)
    scene.close()


def test_trained_proposals_gain_over_the_method_without_them(pkg, trained):
    """What the trained network adds, judged on held-out scenes of one robot.

    Training: the method itself (uniform grasps/placements, IK configurations,
    200 Adam steps) solves 128 plain Pick-Place scenes; up to 256 satisfying
    particles per scene become rows; the library's own tensor-core kernels fit
    the network.  Test: on 16 unseen scenes, 4096 particles drawn with the
    network's grasps and placements (then IK) against uniform ones (then IK),
    same seeds and tolerances; the measure is how many particles satisfy
    Eq. 3 straight after sampling, counted by the GPU check and re-judged by
    the FP64 oracle on a subset."""
    net, st, losses = trained
    assert st["particles"] >= 8000, st
    assert losses[-1][1] < losses[0][1] - 0.5, losses
    counts = {2: [], 3: []}
    oracle_rate = {2: [], 3: []}
    for k in range(16):
        sc, acts = sg.robot_plain_problem(20000 + k)
        pr = Problem(sc, acts)
        scene = pkg.Scene(sc)
        pid = scene.set_skeleton(acts)
        scene.set_proposal(net)
        for sampler in (2, 3):
            scene.sample(pid, 4096, 555 + k, sampler=sampler)
            scene.optimize(pid, 0)                      # the Eq. 3 check of the seeds
            q = scene.query(pid, 4096, want_particles=k < 4)
            counts[sampler].append(q["n_satisfied"])
            if k < 4:                                   # the FP64 oracle as the judge
                X = q["particles"][:, :512].T.astype(np.float64)
                ok = pr.satisfied(pr.term_values(torch.from_numpy(X))).numpy()
                oracle_rate[sampler].append(float(ok.mean()))
                gpu = q["mask"][:512]
                assert (ok != gpu).mean() < 0.01
        scene.set_proposal(None)
        scene.close()
    u, l = np.array(counts[2]), np.array(counts[3])
    print(f"\nproposal: harvest {st}; satisfying seeds of 4096 per held-out scene: uniform+IK mean {u.mean():.0f} "
          f"{u.tolist()}; learned+IK mean {l.mean():.0f} {l.tolist()}; oracle-judged rates uniform "
          f"{np.round(oracle_rate[2], 3).tolist()} learned {np.round(oracle_rate[3], 3).tolist()}")
    assert l.mean() > u.mean()


def test_learned_seeds_against_uniform_seeds_judged_by_the_oracle(pkg, trained):
    """The learned-proposal comparison without IK (the network proposes grasps
    and placements, joints stay uniform), on 32 held-out scenes: iterations to
    the first satisfying particle under the device-side stop (checks every 10
    iterations, at most 1000), and the FP64 oracle's judgement of the seeds
    themselves -- the share of seeds whose Grasp and StablePlace constraints
    (the terms that depend only on what the network proposes) hold."""
    net = trained[0]
    iters = {0: [], 1: []}
    held = {0: [], 1: []}
    for k in range(32):
        sc, acts = sg.robot_plain_problem(20000 + k)
        pr = Problem(sc, acts)
        own = [i for i, t in enumerate(pr.terms) if t.kind in (GRASP, STABLE_PLACE)]
        scene = pkg.Scene(sc)
        pid = scene.set_skeleton(acts)
        scene.set_proposal(net)
        for sampler in (0, 1):
            scene.sample(pid, 1024, 31 + k, sampler=sampler)
            X = scene.get_particles(pid)[0][:, :256].T.astype(np.float64)
            T = pr.term_values(torch.from_numpy(X)).numpy()
            held[sampler].append(float((T[:, own] <= pr.tolerances().numpy()[own]).all(axis=1).mean()))
            scene.optimize(pid, 1000, stop_every=10)
            f = scene.query(pid, 1024)["first_iter"]
            iters[sampler].append(f if f >= 0 else 1000)
        scene.set_proposal(None)
        scene.close()
    iu, il = np.array(iters[0]), np.array(iters[1])
    hu, hl = np.array(held[0]), np.array(held[1])
    print(f"\nlearned vs uniform seeds, 32 held-out scenes: iterations to first satisfying mean {il.mean():.0f} vs "
          f"{iu.mean():.0f}; oracle: Grasp and StablePlace hold for {hl.mean():.3f} vs {hu.mean():.3f} of seeds")
    assert hl.mean() > hu.mean()                     # the oracle prefers the network's seeds
    # both forms solve most scenes (over 256 held-out scenes: 96-97%); on 32 scenes, and with a network
    # whose training rounds differently from build to build, a few more may stay unsolved
    assert (il < 1000).mean() >= 0.8 and (iu < 1000).mean() >= 0.8


@pytest.fixture(scope="module")
def trained(pkg):
    """The network trained on what the method finds on 128 plain Pick-Place
    scenes of one robot (uniform grasps/placements, IK configurations, 200
    Adam steps), by the library's tensor-core kernels."""
    from paper_2411_11833_b300 import proposal
    train = [sg.robot_plain_problem(10000 + k) for k in range(128)]
    F, Y, M, st = proposal.harvest(train, n_particles=4096, iters=200, chunk=50, sampler=2,
                                   max_rows_per_problem=256)
    net, losses = proposal.train(F, Y, M, steps=1500, batch=4096, lr=1e-3, log_every=500)
    yield net, st, losses
    net.close()
