"""Learned particle proposals: feature rows, training targets, and the decoding
of network outputs into initial particles (oracle; test infrastructure only).

The paper lets particles be seeded by learned samplers instead of uniformly
(Sec. V-A, Sec. VIII) without fixing one.  This is the reading the library
implements, written out plainly:

* One row per Pick or Place action of a skeleton, in action order.  Its 48
  features describe what the action acts on, not the particle, so one network
  evaluation per row serves every particle of a batch:
    [0:3]   half extents of the action's box
    [3:8]   the box's initial pose: x, y, z, cos yaw, sin yaw
    [8:15]  the surface the box is placed on (a Place's own surface; for a Pick,
            the surface of the next Place of the same box, zeros if none):
            centre x, y, cos yaw, sin yaw, half x, half y, top z
    [15:17] one-hot action kind (Pick, Place)
    [17]    action index / number of actions
    [18]    1 if the skeleton has a goal action
    [19:27] DH a of joints 1..8 (zero past the arm's joints)
    [27:35] DH d, [35:43] DH alpha / (pi / 2), [43] joints / 8, [44:48] zero.
* Targets (16 slots; a mask selects the ones in use) in normalised units:
    Pick row  slots 0..4: g_x / h_x, g_y / h_y, (g_z - (h_z - 0.02)) / 0.01 - 1,
                          cos g_yaw, sin g_yaw        (the grasp bounds map to [-1, 1])
    Place row slots 5..8: u / H_x, v / H_y, cos p_yaw, sin p_yaw
                          ((u, v): placement centre in the surface frame)
* Sampling: network outputs give mean mu_k and log std s_k per slot;
  t_k = mu_k + exp(clamp(s_k, -8, 3)) xi_k with xi_k a standard normal drawn by
  Box-Muller from Philox4x32-10 at counter (i, 16 r + k, 1, 0) (particle i,
  row r): u1 = ((w0 >> 8) + 1) 2^-24, u2 = (w1 >> 8) 2^-24,
  xi = sqrt(-2 ln u1) cos(2 pi u2).  Decoding clamps the position slots to
  [-1, 1] (so seeds respect the grasp bounds and lie on the surface) and takes
  yaw = atan2(sin slot, cos slot).  Joint configurations keep the uniform
  sampler's values.
"""
from __future__ import annotations

import math

import numpy as np

from . import philox
from .problem import GOAL, KNOT, PICK, PLACE, Problem

NF, NT = 48, 16
LS_MIN, LS_MAX = -8.0, 3.0


def action_rows(sc, actions):
    """[(action index, kind, box, surface for the features, particle offset)]
    for every Pick and Place, in order."""
    pr = Problem(sc, actions)
    rows = []
    for cfg in pr.configs:
        if cfg["kind"] == KNOT:
            continue
        ai = cfg["action"]
        kind, b, s = actions[ai]
        if kind == PICK:
            nxt = [a for a in actions[ai + 1:] if a[0] == PLACE and a[1] == b]
            surf = nxt[0][2] if nxt else -1
            rows.append((ai, PICK, b, surf, cfg["g_off"]))
        else:
            rows.append((ai, PLACE, b, s, cfg["target"][1]))
    return rows


def features(sc, actions) -> np.ndarray:
    """Feature rows [R, 48] (float64; the library stores them as float32)."""
    rows = action_rows(sc, actions)
    n_act = len(actions)
    has_goal = any(a[0] == GOAL for a in actions)
    F = np.zeros((len(rows), NF))
    nj = len(sc.dh_a)
    for r, (ai, kind, b, s, _off) in enumerate(rows):
        f = F[r]
        f[0:3] = sc.box_half[b]
        x, y, z, yaw = sc.box_init[b]
        f[3:8] = [x, y, z, math.cos(yaw), math.sin(yaw)]
        if s >= 0:
            cx, cy, syaw, hx, hy, zt = sc.surf[s]
            f[8:15] = [cx, cy, math.cos(syaw), math.sin(syaw), hx, hy, zt]
        f[15 if kind == PICK else 16] = 1.0
        f[17] = ai / n_act
        f[18] = 1.0 if has_goal else 0.0
        f[19:19 + nj] = sc.dh_a
        f[27:27 + nj] = sc.dh_d
        f[35:35 + nj] = np.asarray(sc.dh_alpha) / (math.pi / 2)
        f[43] = nj / 8.0
    return F


def encode(sc, actions, X: np.ndarray):
    """Training rows from particles X [P, D]: features [P*R, 48], targets
    [P*R, 16], mask [P*R, 16]; row i*R + r is particle i, action row r."""
    rows = action_rows(sc, actions)
    F = features(sc, actions)
    P, R = X.shape[0], len(rows)
    Y = np.zeros((P, R, NT))
    M = np.zeros((P, R, NT))
    for r, (ai, kind, b, s, off) in enumerate(rows):
        if kind == PICK:
            hx, hy, hz = sc.box_half[b]
            Y[:, r, 0] = X[:, off] / hx
            Y[:, r, 1] = X[:, off + 1] / hy
            Y[:, r, 2] = (X[:, off + 2] - (hz - 0.02)) / 0.01 - 1.0
            Y[:, r, 3] = np.cos(X[:, off + 3])
            Y[:, r, 4] = np.sin(X[:, off + 3])
            M[:, r, 0:5] = 1.0
        else:
            cx, cy, syaw, hx, hy, _ = sc.surf[s]
            dx, dy = X[:, off] - cx, X[:, off + 1] - cy
            u = math.cos(syaw) * dx + math.sin(syaw) * dy
            v = -math.sin(syaw) * dx + math.cos(syaw) * dy
            Y[:, r, 5] = u / hx
            Y[:, r, 6] = v / hy
            Y[:, r, 7] = np.cos(X[:, off + 2])
            Y[:, r, 8] = np.sin(X[:, off + 2])
            M[:, r, 5:9] = 1.0
    return np.tile(F, (P, 1)), Y.reshape(P * R, NT), M.reshape(P * R, NT)


def normals(n_particles: int, row: int, slot: int, seed: int) -> np.ndarray:
    """Standard normals xi for every particle of one (row, slot), Box-Muller
    over Philox4x32-10 (counter (i, 16 row + slot, 1, 0))."""
    i = np.arange(n_particles, dtype=np.uint64)
    w = philox.philox4x32_10((i, 16 * row + slot, 1, 0), (seed & philox.MASK, (seed >> 32) & philox.MASK))
    u1 = ((w[0] >> np.uint64(8)).astype(np.float64) + 1.0) * 2.0 ** -24
    u2 = (w[1] >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def decode(sc, actions, out: np.ndarray, X: np.ndarray, xi) -> np.ndarray:
    """Overwrite the grasp and placement components of particles X [P, D] from
    network outputs out [R, 32] (mean slots 0..15, log std slots 16..31) and
    normals xi(row, slot) -> [P]."""
    X = X.copy()
    for r, (ai, kind, b, s, off) in enumerate(action_rows(sc, actions)):
        mu, ls = out[r, :NT], np.clip(out[r, NT:2 * NT], LS_MIN, LS_MAX)
        t = {k: mu[k] + math.exp(ls[k]) * xi(r, k) for k in ((0, 1, 2, 3, 4) if kind == PICK else (5, 6, 7, 8))}
        if kind == PICK:
            hx, hy, hz = sc.box_half[b]
            X[:, off] = hx * np.clip(t[0], -1.0, 1.0)
            X[:, off + 1] = hy * np.clip(t[1], -1.0, 1.0)
            X[:, off + 2] = hz - 0.02 + 0.01 * (np.clip(t[2], -1.0, 1.0) + 1.0)
            X[:, off + 3] = np.arctan2(t[4], t[3])
        else:
            cx, cy, syaw, hx, hy, _ = sc.surf[s]
            u = hx * np.clip(t[5], -1.0, 1.0)
            v = hy * np.clip(t[6], -1.0, 1.0)
            X[:, off] = cx + math.cos(syaw) * u - math.sin(syaw) * v
            X[:, off + 1] = cy + math.sin(syaw) * u + math.cos(syaw) * v
            X[:, off + 2] = np.arctan2(t[8], t[7])
    return X


def sample(sc, actions, out: np.ndarray, n_particles: int, seed: int) -> np.ndarray:
    """The proposal sampler: uniform joint configurations, grasps and
    placements decoded from the network outputs with Philox normals."""
    X = philox.sample_uniform(Problem(sc, actions), n_particles, seed)
    return decode(sc, actions, out, X, lambda r, k: normals(n_particles, r, k, seed))
