"""Pins of the trajectory knots in the FP64 oracle (Listing 1 MoveFree /
MoveHold with Motion, CFreeTraj(Hold) and TrajLength; Sec. VIII: knot points
initialised by linear interpolation) against closed forms, the configuration
terms they reuse, explicit bookkeeping and central finite differences (CPU)."""
import numpy as np
import torch

import scenegen as sg
from oracle import philox
from oracle.problem import (CFREE_HOLD, CFREE_TRAJ, JOINT_LIMIT, KNOT, PICK, PLACE, TRAJ_LEN, Options, Problem)

from test_oracle_pins import _fd_error

DT = torch.float64


def _problem(m=2, n_boxes=2, seed=21002):
    sc, acts = sg.robot_packing_problem(seed, n_boxes=n_boxes)
    return sc, acts, Problem(sc, acts, Options(n_knots=m))


def test_knots_sit_before_the_action_they_lead_to():
    sc, acts, pr = _problem(m=2)
    n = pr.n
    pick, place = ["gpos"] * 3 + ["gyaw"] + ["q"] * n, ["ppos"] * 2 + ["pyaw"] + ["q"] * n
    knots = ["q"] * (2 * n)
    assert pr.kinds == pick + knots + place + knots + pick + knots + place
    assert len(pr.segments) == 3
    assert [t.kind for t in pr.terms].count(TRAJ_LEN) == 3
    assert [t.kind for t in pr.terms].count(CFREE_TRAJ) == 6
    # MoveHold between a Pick and its Place holds the box and sees the other one;
    # MoveFree after the Place holds nothing and sees both boxes, the placed one
    # at its placement variable
    kn = [c for c in pr.configs if c["kind"] == KNOT]
    assert [c["box"] for c in kn] == [0, 0, -1, -1, 1, 1]
    assert [j for j, _ in kn[0]["env"]] == [1]
    assert [(j, src[0]) for j, src in kn[2]["env"]] == [(0, "var"), (1, "init")]
    # the costs are not constraints
    assert pr.constraint_mask().sum() == len(pr.terms) - 3 - 1


def test_straight_knots_give_the_straight_line_length():
    sc, acts, pr = _problem(m=3)
    X = pr.interpolate_knots(philox.sample_uniform(pr, 16, 3))
    tv = pr.term_values(torch.tensor(X)).numpy()
    for ti, t in enumerate(pr.terms):
        if t.kind != TRAJ_LEN:
            continue
        seg = pr.segments[t.cfg]
        qa = X[:, pr.configs[seg["start"]]["q_off"]:pr.configs[seg["start"]]["q_off"] + pr.n]
        qb = X[:, pr.configs[seg["end"]]["q_off"]:pr.configs[seg["end"]]["q_off"] + pr.n]
        assert np.allclose(tv[:, ti], np.linalg.norm(qb - qa, axis=1), rtol=0, atol=1e-12)
    # knots off the line make every motion strictly longer (triangle inequality)
    g = np.random.default_rng(1)
    Y = X.copy()
    for c in pr.configs:
        if c["kind"] == KNOT:
            Y[:, c["q_off"]:c["q_off"] + pr.n] += g.normal(0, 0.1, (16, pr.n))
    ty = pr.term_values(torch.tensor(Y)).numpy()
    lens = [ti for ti, t in enumerate(pr.terms) if t.kind == TRAJ_LEN]
    assert (ty[:, lens] > tv[:, lens] + 1e-9).all()


def test_a_holding_knot_at_the_pick_configuration_has_its_collision():
    # CFreeTrajHold at q = the Pick's q is the Pick's CFreeHold: the same arm,
    # the same held box at FK(q) G(g)^-1, the same environment
    sc, acts, pr = _problem(m=1)
    X = philox.sample_uniform(pr, 32, 5)
    pick = pr.configs[0]
    knot = next(c for c in pr.configs if c["kind"] == KNOT)
    X[:, knot["q_off"]:knot["q_off"] + pr.n] = X[:, pick["q_off"]:pick["q_off"] + pr.n]
    tv = pr.term_values(torch.tensor(X)).numpy()
    ci_k = pr.configs.index(knot)
    hold = next(ti for ti, t in enumerate(pr.terms) if t.kind == CFREE_HOLD and t.cfg == 0)
    traj = next(ti for ti, t in enumerate(pr.terms) if t.kind == CFREE_TRAJ and t.cfg == ci_k)
    assert np.array_equal(tv[:, traj], tv[:, hold])
    assert (tv[:, hold] > 0).any()


def test_knot_joint_limits_are_the_bound_distance():
    sc, acts, pr = _problem(m=1)
    X = pr.interpolate_knots(philox.sample_uniform(pr, 4, 6))
    knot = next(c for c in pr.configs if c["kind"] == KNOT)
    X[:, knot["q_off"] + 2] = sc.q_hi[2] + 0.1
    X[:, knot["q_off"] + 5] = sc.q_lo[5] - 0.2
    tv = pr.term_values(torch.tensor(X)).numpy()
    jl = next(ti for ti, t in enumerate(pr.terms) if t.kind == JOINT_LIMIT and t.cfg == pr.configs.index(knot))
    assert np.allclose(tv[:, jl], np.hypot(0.1, 0.2), rtol=0, atol=1e-12)


def test_gradient_with_knots_matches_central_differences():
    sc, acts, pr = _problem(m=2)
    g = np.random.default_rng(2)
    X = pr.interpolate_knots(philox.sample_uniform(pr, 24, 7))
    for c in pr.configs:
        if c["kind"] == KNOT:
            X[:, c["q_off"]:c["q_off"] + pr.n] += g.normal(0, 0.2, (24, pr.n))
    x = torch.tensor(X)
    x = x[pr.kink_margin(x) > 1e-4][:4]
    assert x.shape[0] >= 2
    assert _fd_error(pr, x) < 1e-6


def test_planted_mistakes_are_caught(monkeypatch):
    """Plausible slips in the knot terms make one of the pins above fail."""
    import pytest
    from oracle import problem as PM
    orig_len, orig_walk = PM.Problem._traj_length, PM.Problem._walk

    # 1. TrajLength without its last edge (the knots' end configuration dropped)
    def len_short(self, seg, x):
        w = self._waypoints(seg, x)[:-1]
        return sum(PM.G.norm(w[i + 1] - w[i]) for i in range(len(w) - 1))
    monkeypatch.setattr(PM.Problem, "_traj_length", len_short)
    with pytest.raises(AssertionError):
        test_straight_knots_give_the_straight_line_length()
    monkeypatch.setattr(PM.Problem, "_traj_length", orig_len)

    # 2. a MoveFree knot that does not see the box just placed
    def walk_blind(self):
        orig_walk(self)
        for c in self.configs:
            if c["kind"] == KNOT and c["box"] < 0:
                c["env"] = [(j, src) for j, src in c["env"] if src[0] == "init"]
    monkeypatch.setattr(PM.Problem, "_walk", walk_blind)
    with pytest.raises(AssertionError):
        test_knots_sit_before_the_action_they_lead_to()
    monkeypatch.setattr(PM.Problem, "_walk", orig_walk)
