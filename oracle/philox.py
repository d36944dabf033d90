"""Philox4x32-10 and the uniform particle sampler (oracle; test infrastructure).

Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC 2011): a 128-bit counter and a 64-bit key go through 10 rounds; each
round multiplies counter words 0 and 2 by the constants 0xD2511F53 and 0xCD9E8D57
(keeping both 32-bit halves of the products) and mixes the halves with words 1
and 3 and the round key; the key is bumped by the Weyl constants 0x9E3779B9 and
0xBB67AE85 between rounds.

The sampler is the "Optimization" baseline's initialisation (Sec. VIII:
particles drawn uniformly within the variables' bounds): component c of
particle i of a problem draws the first output word of
Philox(counter = (i, c, 0, 0), key = (seed lo 32 bits, seed hi 32 bits)),
u = (word >> 8) * 2^-24 in [0, 1), and maps it onto the variable's range
(include/tamp.h, tamp_sample_particles).
"""
from __future__ import annotations

import math

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds on numpy uint64 arrays holding 32-bit words.

    ctr: 4 arrays (broadcastable), key: 2 arrays.  Returns 4 arrays of words.
    """
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & MASK for v in ctr)
    k0, k1 = (np.asarray(v, dtype=np.uint64) & MASK for v in key)
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = np.uint64(M0) * c0          # < 2^64: exact in uint64
        p1 = np.uint64(M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK, lo1, (hi0 ^ c3 ^ k1) & MASK, lo0
    return c0, c1, c2, c3


def uniform01(n_particles: int, component: int, seed: int) -> np.ndarray:
    """u in [0, 1) for every particle of one component (24-bit resolution)."""
    i = np.arange(n_particles, dtype=np.uint64)
    w = philox4x32_10((i, component, 0, 0), (seed & MASK, (seed >> 32) & MASK))[0]
    return (w >> np.uint64(8)).astype(np.float64) * (2.0 ** -24)


def sample_uniform(problem, n_particles: int, seed: int) -> np.ndarray:
    """Uniform initial particles [P, D] in FP64 for a ``problem.Problem``.

    q_j ~ U[lo_j, hi_j]; grasp x, y, z ~ U over the grasp bounds; any yaw ~
    U[-pi, pi); a placement draws (u, v) uniformly over the surface rectangle
    in its own frame and is rotated/translated into the world.
    """
    sc = problem.sc
    X = np.zeros((n_particles, problem.D))
    U = [uniform01(n_particles, c, seed) for c in range(problem.D)]
    n = problem.n
    for cfg in problem.configs:
        qo = cfg["q_off"]
        for j in range(n):
            X[:, qo + j] = sc.q_lo[j] + (sc.q_hi[j] - sc.q_lo[j]) * U[qo + j]
        b = cfg["box"]
        if cfg["kind"] == 2:      # a trajectory knot has only its configuration
            continue
        if cfg["kind"] == 0:      # Pick introduces the grasp variable
            go = cfg["g_off"]
            h = sc.box_half[b]
            lo = [-h[0], -h[1], h[2] - 0.02]
            hi = [h[0], h[1], h[2]]
            for j in range(3):
                X[:, go + j] = lo[j] + (hi[j] - lo[j]) * U[go + j]
            X[:, go + 3] = -math.pi + 2.0 * math.pi * U[go + 3]
            if problem.opts.grasp_dof == 6:
                # roll and pitch in [-pi/2, pi/2): from above to the side, never from below
                for j in (4, 5):
                    X[:, go + j] = -0.5 * math.pi + math.pi * U[go + j]
                lo = [-h[0], -h[1], -h[2]]
                for j in range(3):
                    X[:, go + j] = lo[j] + (hi[j] - lo[j]) * U[go + j]
        else:
            _, po, s = cfg["target"]
            cx, cy, syaw, hx, hy, _z = sc.surf[s]
            u = -hx + 2.0 * hx * U[po]
            v = -hy + 2.0 * hy * U[po + 1]
            X[:, po] = cx + math.cos(syaw) * u - math.sin(syaw) * v
            X[:, po + 1] = cy + math.sin(syaw) * u + math.cos(syaw) * v
            X[:, po + 2] = -math.pi + 2.0 * math.pi * U[po + 2]
    return X
