"""Pins of the SelfCollision term in the FP64 oracle (the CFree constraints'
"does not cause robot self-collisions", tolerance 0 penetration: appendix
constraint definitions and tolerances) against a closed form on a folded
planar arm, the ignore rule, and central finite differences (CPU)."""
import dataclasses
import math

import numpy as np
import torch

import scenegen as sg
from oracle import philox
from oracle.problem import KNOT, SELF_COLLISION, Options, Problem

from test_oracle_pins import _fd_error


def _planar_scene():
    """Three revolute joints about z (alpha 0, d 0), links a = 0.3 m; one
    sphere (r 0.05) per link: link 1's at the base origin (local (-0.3, 0, 0)),
    link 2's at frame 2's origin, link 3's at frame 3's origin (the tip)."""
    sc, _ = sg.robot_packing_problem(21002, n_boxes=2)
    n = 3
    return dataclasses.replace(
        sc, dh_a=np.full(n, 0.3), dh_d=np.zeros(n), dh_alpha=np.zeros(n), dh_offset=np.zeros(n),
        q_lo=np.full(n, -2.8), q_hi=np.full(n, 2.8), base=np.eye(4), tool=np.eye(4),
        sphere_link=np.array([1, 2, 3], dtype=np.int32),
        sphere_xyzr=np.array([[-0.3, 0, 0, 0.05], [0, 0, 0, 0.05], [0, 0, 0, 0.05]]))


def _free_knot(pr):
    # a MoveFree knot (between Place 0 and Pick 1): the arm alone
    return next(c for c in pr.configs if c["kind"] == KNOT and c["box"] < 0)


def test_folded_planar_arm_penetration_is_the_closed_form():
    sc = _planar_scene()
    acts = sg.pick_place_skeleton([0, 1])
    pr = Problem(sc, acts, Options(n_knots=1, self_collision=True))
    # links 1 and 3 are two apart and apart at q = 0 (base origin vs (0.9, 0)): tested
    assert pr.self_links == {(3, 1)}
    kn = _free_knot(pr)
    ci = pr.configs.index(kn)
    ti = next(i for i, t in enumerate(pr.terms) if t.kind == SELF_COLLISION and t.cfg == ci)
    X = philox.sample_uniform(pr, 5, 1)
    eps = np.array([0.0, 0.01, 0.05, 0.2, 0.6])
    q2, q3 = 2 * math.pi / 3, 2 * math.pi / 3 + eps
    X[:, kn["q_off"]] = 0.0
    X[:, kn["q_off"] + 1] = q2
    X[:, kn["q_off"] + 2] = q3
    # the tip: 0.3 (1, 0) + 0.3 (cos q2, sin q2) + 0.3 (cos(q2 + q3), sin(q2 + q3)); link 1's sphere at 0
    tip = 0.3 * np.stack([1 + np.cos(q2) + np.cos(q2 + q3), np.sin(q2) + np.sin(q2 + q3)], 1)
    want = np.maximum(0.0, 0.1 - np.linalg.norm(tip, axis=1))
    got = pr.term_values(torch.tensor(X)).numpy()[:, ti]
    assert np.allclose(got, want, rtol=0, atol=1e-12)
    assert got[0] > 0.09 and got[-1] == 0.0


def test_no_self_collision_at_the_reference_configuration():
    # pairs that touch at q = 0 are not tested, the rest do not touch there
    sc, acts = sg.robot_packing_problem(21002, n_boxes=2)
    pr = Problem(sc, acts, Options(n_knots=1, self_collision=True))
    kn = _free_knot(pr)
    X = philox.sample_uniform(pr, 3, 2)
    X[:, kn["q_off"]:kn["q_off"] + pr.n] = 0.0
    ci = pr.configs.index(kn)
    ti = next(i for i, t in enumerate(pr.terms) if t.kind == SELF_COLLISION and t.cfg == ci)
    assert (pr.term_values(torch.tensor(X)).numpy()[:, ti] == 0.0).all()
    # adjacent links are never tested
    assert all(i - j >= 2 for i, j in pr.self_links)
    # uniform configurations do fold the arm onto itself
    tv = pr.term_values(torch.tensor(philox.sample_uniform(pr, 256, 3))).numpy()
    selfs = [i for i, t in enumerate(pr.terms) if t.kind == SELF_COLLISION]
    assert (tv[:, selfs] > 0).mean() > 0.05


def test_gradient_with_self_collision_matches_central_differences():
    sc, acts = sg.robot_packing_problem(21002, n_boxes=2)
    pr = Problem(sc, acts, Options(n_knots=1, self_collision=True))
    x = torch.tensor(philox.sample_uniform(pr, 96, 4))
    selfs = [i for i, t in enumerate(pr.terms) if t.kind == SELF_COLLISION]
    active = (pr.term_values(x).numpy()[:, selfs] > 0).any(axis=1)
    x = x[torch.as_tensor(active) & (pr.kink_margin(x) > 1e-4)][:4]
    assert x.shape[0] >= 2
    assert _fd_error(pr, x) < 1e-6


def test_planted_mistakes_are_caught(monkeypatch):
    """Plausible slips in SelfCollision make one of the pins above fail."""
    import pytest
    from oracle import problem as PM
    orig_pairs, orig_pen = PM.Problem._self_pairs, PM.Problem._self_penetration

    # 1. adjacent links counted, and links that touch at q = 0 not ignored
    def pairs_all(self):
        orig_pairs(self)
        links = np.asarray(self.sc.sphere_link)
        self.self_mask = links[:, None] > links[None, :]
    monkeypatch.setattr(PM.Problem, "_self_pairs", pairs_all)
    with pytest.raises(AssertionError):
        test_no_self_collision_at_the_reference_configuration()
    monkeypatch.setattr(PM.Problem, "_self_pairs", orig_pairs)

    # 2. one radius instead of the sum of the pair's radii
    def pen_one_radius(self, c, r):
        return orig_pen(self, c, r * 0.5) * 2.0
    monkeypatch.setattr(PM.Problem, "_self_penetration", pen_one_radius)
    with pytest.raises(AssertionError):
        test_folded_planar_arm_penetration_is_the_closed_form()
    monkeypatch.setattr(PM.Problem, "_self_penetration", orig_pen)
