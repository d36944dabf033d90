"""The packing scene built around an FP64 witness (tests/golden/packing_witness.json,
written by tests/golden/make_packing_witness.py from the oracle alone): the
stored scene is the packing workload's draw for its seed, and the witness
particle satisfies every constraint of Eq. 3 on the 6-box packing skeleton
(67 terms) -- a whole-particle pin of the oracle on the headline's kind of
problem, next to the construction's geometric facts checked here without the
oracle's terms (footprints inside the region and pairwise apart, top-down
grasps at the box centres)."""
import json
import math
import os

import numpy as np
import torch

import scenegen as sg
from oracle.problem import DT, PICK, PLACE, Problem

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "packing_witness.json")


def load_witness():
    d = json.load(open(GOLDEN))
    sc, acts = sg.packing_problem(d["scene_seed"])
    return d, sc, acts


def _corners(x, y, yaw, hx, hy):
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[x + c * a - s * b, y + s * a + c * b] for a, b in ((hx, hy), (-hx, hy), (-hx, -hy), (hx, -hy))])


def _separated(p, q):
    """Convex polygons p, q (corners in order) do not overlap (separating axis)."""
    for poly in (p, q):
        for i in range(len(poly)):
            e = poly[(i + 1) % len(poly)] - poly[i]
            n = np.array([-e[1], e[0]])
            a, b = p @ n, q @ n
            if a.max() <= b.min() or b.max() <= a.min():
                return True
    return False


def test_stored_scene_is_the_packing_workloads_draw():
    d, sc, acts = load_witness()
    for k, v in d["scene"].items():
        assert np.array_equal(np.asarray(getattr(sc, k), dtype=np.float64), np.asarray(v, dtype=np.float64)), k
    assert [list(a) for a in acts] == d["actions"]


def test_witness_satisfies_every_constraint():
    d, sc, acts = load_witness()
    pr = Problem(sc, acts)
    w = torch.tensor(np.array(d["witness"])[None], dtype=DT)
    with torch.no_grad():
        terms = pr.term_values(w)
    assert bool(pr.satisfied(terms)[0])
    assert np.allclose(terms[0].numpy(), d["witness_terms"], rtol=0, atol=1e-12)
    assert len(pr.terms) == 67 and pr.D == 126


def test_witness_construction_geometry():
    """The arrangement and grasps the witness was built from, checked directly:
    each placed box's footprint lies inside the target region by at least 4 mm,
    the footprints are pairwise apart, and every grasp is top-down at its box's
    centre, 1 cm below the top face (so containment, box-box collision and the
    grasp bound are 0 by geometry, not by the oracle's own functions)."""
    d, sc, acts = load_witness()
    pr = Problem(sc, acts)
    w = np.array(d["witness"])
    cx, cy, ryaw, rhx, rhy = sc.surf[0, :5]
    feet = []
    for cfg in pr.configs:
        b = cfg["box"]
        if cfg["kind"] == PICK:
            g = w[cfg["g_off"]:cfg["g_off"] + 4]
            assert g[0] == 0.0 and g[1] == 0.0 and abs(g[2] - (sc.box_half[b, 2] - 0.01)) < 1e-15
        elif cfg["kind"] == PLACE:
            po = cfg["target"][1]
            corners = _corners(w[po], w[po + 1], w[po + 2], sc.box_half[b, 0], sc.box_half[b, 1])
            c, s = math.cos(ryaw), math.sin(ryaw)
            local = (corners - [cx, cy]) @ np.array([[c, -s], [s, c]])    # rotate into the region frame
            assert (np.abs(local[:, 0]) <= rhx - 0.004).all() and (np.abs(local[:, 1]) <= rhy - 0.004).all()
            feet.append(corners)
    assert len(feet) == 6
    for i in range(6):
        for j in range(i + 1, 6):
            assert _separated(feet[i], feet[j]), (i, j)


def test_moving_a_box_off_the_arrangement_is_seen():
    """The witness's zeros are not the oracle missing contacts: a placement moved
    onto its row neighbour makes the placed boxes collide (CFreePlace above
    1 mm), one moved 0.3 m along the region's x axis (past its edge) breaks
    StablePlace."""
    from oracle.problem import CFREE_PLACE, STABLE_PLACE
    d, sc, acts = load_witness()
    pr = Problem(sc, acts)
    w = np.array(d["witness"])
    places = [c for c in pr.configs if c["kind"] == PLACE]
    a, b = places[0], places[1]                         # neighbours in the first row
    pa, pb = a["target"][1], b["target"][1]
    moved = w.copy()
    moved[pa:pa + 2] = 0.5 * (w[pa:pa + 2] + w[pb:pb + 2])
    with torch.no_grad():
        t = pr.term_values(torch.tensor(moved[None], dtype=DT))[0].numpy()
    kinds = np.array([x.kind for x in pr.terms])
    assert t[kinds == CFREE_PLACE].max() > 1e-3
    out = w.copy()
    cx, cy, ryaw = sc.surf[0, :3]
    out[pa] += 0.3 * math.cos(ryaw)                      # 0.3 m along the region's x: past its edge
    out[pa + 1] += 0.3 * math.sin(ryaw)
    with torch.no_grad():
        t = pr.term_values(torch.tensor(out[None], dtype=DT))[0].numpy()
    assert t[kinds == STABLE_PLACE].max() > 1e-3
