"""Writes tests/golden/packing_witness.json: a packing scene of the packing
workload's recipe (a random 7-DOF arm, 6 boxes with edges ~ U[0.04, 0.10] m, 8
cuboids, a 0.3 x 0.3 m target region, 6 Pick-Place pairs + the MinimizeObjDist
goal) built around an FP64 witness: a particle that satisfies every constraint
of Eq. 3 -- feasibility by construction.  Test infrastructure: it calls only the
oracle and the seeded scene generator, and its output is a stored input that
the tests and the benchmark read.

Per scene seed (2001, 2002, ...), with the scene drawn as the packing workload
draws it (scenegen.packing_problem):
  1. placements: the 6 boxes in 2 rows of 3 on the region's axes, each turned so
     that its shorter side lies along the rows, 5 mm apart and at least 5 mm
     inside the region (corner spheres sit inside the boxes, so boxes that do not
     overlap do not collide); a seed whose boxes do not fit is skipped;
  2. grasps: top-down at each box's centre, 1 cm below its top face;
  3. configurations: damped least squares (the oracle's IK step) from 256 joint
     seeds drawn within the limits, in skeleton order; a Pick's grasp yaw is
     free (as in the oracle's configuration sampler), a Place's placement yaw
     stays that of the arrangement (the full pose is the target);
  4. given the placements and grasps, the boxes are independent (a box's Pick
     and Place terms depend on its own grasp and configurations and on where the
     others stand, which the arrangement fixes): each box takes its grasp and
     configurations from a seed at which every one of its terms holds, and the
     particle so assembled must satisfy Eq. 3 by the oracle's check; a scene
     seed where some box has no such joint seed is skipped.

Usage: python tests/golden/make_packing_witness.py [first_seed] [n_seeds]
"""
from __future__ import annotations

import json
import math
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import scenegen as sg  # noqa: E402
from oracle import ik as oik  # noqa: E402
from oracle.problem import DT, PICK, PLACE, Problem  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "packing_witness.json")
GAP, MARGIN, RESTARTS, ITERS = 0.005, 0.005, 256, 128


def arrangement(sc):
    """(x, y, yaw) in the world for each box, or None if they do not fit."""
    cx, cy, ryaw, rhx, rhy = (float(v) for v in sc.surf[0, :5])
    half = sc.box_half
    n = half.shape[0]
    rows = [list(range(0, n // 2)), list(range(n // 2, n))]
    along = np.minimum(half[:, 0], half[:, 1])           # half extent along the row
    across = np.maximum(half[:, 0], half[:, 1])
    turned = half[:, 0] > half[:, 1]                      # box x along the region's y
    depth = [2.0 * max(across[i] for i in r) for r in rows]
    if depth[0] + depth[1] + GAP > 2.0 * (rhy - MARGIN):
        return None
    c, s = math.cos(ryaw), math.sin(ryaw)
    out = [None] * n
    ly = [-(GAP / 2 + depth[0] / 2), GAP / 2 + depth[1] / 2]
    for k, r in enumerate(rows):
        width = sum(2.0 * along[i] for i in r) + GAP * (len(r) - 1)
        if width > 2.0 * (rhx - MARGIN):
            return None
        lx = -width / 2
        for i in r:
            px = lx + along[i]
            lx += 2.0 * along[i] + GAP
            out[i] = (cx + c * px - s * ly[k], cy + s * px + c * ly[k], ryaw + (math.pi / 2 if turned[i] else 0.0))
    return out


def solve(sc, acts, seed):
    pr = Problem(sc, acts)
    place = arrangement(sc)
    if place is None:
        return None, pr, "boxes do not fit"
    rng = np.random.default_rng(seed)
    X = np.zeros((RESTARTS, pr.D))
    for cfg in pr.configs:
        b = cfg["box"]
        X[:, cfg["q_off"]:cfg["q_off"] + pr.n] = rng.uniform(sc.q_lo, sc.q_hi, (RESTARTS, pr.n))
        if cfg["kind"] == PICK:
            X[:, cfg["g_off"]:cfg["g_off"] + 4] = [0.0, 0.0, sc.box_half[b, 2] - 0.01, 0.0]
        elif cfg["kind"] == PLACE:
            po = cfg["target"][1]
            X[:, po:po + 3] = place[b]
    x = torch.tensor(X, dtype=DT)
    for cfg in pr.configs:
        target, yo = oik._target_fn(pr, cfg, x)
        qo = cfg["q_off"]
        q, y = x[:, qo:qo + pr.n].clone(), x[:, yo].clone()
        for _ in range(ITERS):
            q, y_new, _ = oik.dls_step(pr.arm, q, y, target, q_lo=sc.q_lo, q_hi=sc.q_hi)
            if cfg["kind"] == PICK:
                y = y_new
        x[:, qo:qo + pr.n] = q
        x[:, yo] = y
    with torch.no_grad():
        terms = pr.term_values(x).numpy()
    tol = pr.tolerances().numpy()
    cm = pr.constraint_mask().numpy()
    ok = (terms <= tol) | ~cm                             # [restarts, terms]
    w = x[0].numpy().copy()
    counts = []
    for b in range(sc.n_boxes):
        mine = np.array([t.box == b and cm[i] for i, t in enumerate(pr.terms)])
        good = np.flatnonzero(ok[:, mine].all(axis=1))
        counts.append(int(good.size))
        if good.size == 0:
            continue
        k = int(good[0])
        for cfg in pr.configs:
            if cfg["box"] != b:
                continue
            w[cfg["q_off"]:cfg["q_off"] + pr.n] = x[k, cfg["q_off"]:cfg["q_off"] + pr.n].numpy()
            if cfg["kind"] == PICK:
                w[cfg["g_off"]:cfg["g_off"] + 4] = x[k, cfg["g_off"]:cfg["g_off"] + 4].numpy()
    if min(counts) == 0:
        return None, pr, f"joint seeds satisfying each box's terms: {counts}"
    with torch.no_grad():
        sat = bool(pr.satisfied(pr.term_values(torch.tensor(w[None], dtype=DT)))[0])
    if not sat:
        return None, pr, f"assembled particle fails Eq. 3 (per-box seeds {counts})"
    return w, pr, f"joint seeds satisfying each box's terms: {counts}"


def main():
    first = int(sys.argv[1]) if len(sys.argv) > 1 else 2001
    count = int(sys.argv[2]) if len(sys.argv) > 2 else 200
    for seed in range(first, first + count):
        sc, acts = sg.packing_problem(seed)
        w, pr, note = solve(sc, acts, seed)
        print(seed, note, flush=True)
        if w is None:
            continue
        terms = pr.term_values(torch.tensor(w[None], dtype=DT))[0].numpy()
        data = {
            "recipe": "packing workload (scenegen.packing_problem) built around an FP64 witness; "
                      "tests/golden/make_packing_witness.py",
            "scene_seed": seed,
            "scene": {k: np.asarray(getattr(sc, k)).tolist() for k in
                      ("dh_a", "dh_d", "dh_alpha", "dh_offset", "q_lo", "q_hi", "base", "tool", "sphere_link",
                       "sphere_xyzr", "box_half", "box_init", "box_spheres", "obs_center", "obs_rot", "obs_half",
                       "surf")},
            "actions": [list(a) for a in acts],
            "witness": w.tolist(),
            "witness_terms": terms.tolist(),
            "note": note,
        }
        with open(OUT, "w") as f:
            json.dump(data, f)
        print("wrote", OUT, "scene seed", seed, flush=True)
        return
    raise SystemExit("no witness found")


if __name__ == "__main__":
    main()
