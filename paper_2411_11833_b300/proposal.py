"""Learned particle proposals: harvesting training rows from particles the
method itself satisfies, training the tensor-core network, and measuring
iterations to the first satisfying particle with and without it.

The paper seeds particles from learned samplers where it has them (Sec. V-A,
Sec. VIII) and leaves the sampler open; here it is the library's proposal
network (tamp_mlp_*, tamp_set_proposal, tamp_sample_particles sampler 1).
Everything runs through the C ABI; this module only loops and shuffles.
"""
from __future__ import annotations

import time

import numpy as np

from . import Graph, Mlp, Scene


def _solve(scene: Scene, pid: int, n: int, seed: int, sampler: int, iters: int, chunk: int, stop: bool):
    scene.sample(pid, n, seed, sampler=sampler)
    g = Graph(scene, pid, chunk, max(1, iters // chunk), stop_on_first=stop)
    ran = g.run()
    g.close()
    return ran


def harvest(problems, n_particles: int = 4096, iters: int = 1000, chunk: int = 50, seed: int = 1,
            max_rows_per_problem: int | None = None, sampler: int = 0):
    """Optimise each (scene, skeleton) from ``sampler`` seeds (never the
    network: the method without it) for ``iters`` iterations and turn the
    particles that then satisfy Eq. 3 into training rows.  Returns (features,
    targets, mask, stats)."""
    if sampler & 1:
        raise ValueError("harvest runs the method without the network")
    Fs, Ys, Ms = [], [], []
    stats = dict(problems=0, solved=0, particles=0, wall_s=0.0)
    t0 = time.perf_counter()
    for k, (sc, acts) in enumerate(problems):
        scene = Scene(sc)
        pid = scene.set_skeleton(acts)
        _solve(scene, pid, n_particles, seed + 7919 * k, sampler, iters, chunk, False)
        q = scene.query(pid, n_particles, want_particles=True)
        stats["problems"] += 1
        sel = np.flatnonzero(q["mask"])
        if sel.size:
            stats["solved"] += 1
            if max_rows_per_problem is not None:
                sel = sel[:max_rows_per_problem]
            stats["particles"] += int(sel.size)
            F, Y, M = scene.proposal_rows(pid, q["particles"][:, sel])
            Fs.append(F)
            Ys.append(Y)
            Ms.append(M)
        scene.close()
    stats["wall_s"] = time.perf_counter() - t0
    if not Fs:
        z = np.zeros((0, 48), np.float32)
        return z, np.zeros((0, 16), np.float32), np.zeros((0, 16), np.float32), stats
    return np.concatenate(Fs), np.concatenate(Ys), np.concatenate(Ms), stats


def train(F, Y, M, steps: int = 2000, batch: int = 4096, lr: float = 1e-3, seed: int = 0, net: Mlp | None = None,
          init=None, log_every: int = 0):
    """Adam on the Gaussian NLL of the harvested rows (tamp_mlp_train_step).
    Returns (network, losses)."""
    import torch
    g = np.random.default_rng(seed)
    n = F.shape[0]
    batch = min(batch, n)
    if net is None:
        net = Mlp(max_batch=batch)
        if init is None:
            init = _init_params(seed)
        net.set_params(init)
    Fd = torch.from_numpy(np.ascontiguousarray(F)).cuda()
    Yd = torch.from_numpy(np.ascontiguousarray(Y)).cuda()
    Md = torch.from_numpy(np.ascontiguousarray(M)).cuda()
    losses = []
    perm = torch.from_numpy(g.permutation(n)).cuda()
    pos = 0
    for it in range(steps):
        if pos + batch > n:
            perm = torch.from_numpy(g.permutation(n)).cuda()
            pos = 0
        idx = perm[pos:pos + batch]
        pos += batch
        want = log_every and (it % log_every == 0 or it == steps - 1)
        loss = net.train_step(Fd[idx].contiguous(), Yd[idx].contiguous(), Md[idx].contiguous(), lr, want_loss=bool(want))
        if want:
            losses.append((it, loss))
    torch.cuda.synchronize()
    return net, losses


def _init_params(seed: int) -> np.ndarray:
    """Uniform(+-1/sqrt(fan_in)) weights, zero biases (the usual dense-layer start)."""
    g = np.random.default_rng(seed)
    parts = []
    for (wr, wc), bn in (((256, 48), 256), ((256, 256), 256), ((256, 256), 256), ((32, 256), 32)):
        lim = 1.0 / np.sqrt(wc)
        parts.append(g.uniform(-lim, lim, wr * wc))
        parts.append(np.zeros(bn))
    return np.concatenate(parts).astype(np.float32)


def iterations_to_first(problems, net: Mlp | None, n_particles: int = 4096, iters: int = 1000, chunk: int = 25,
                        seed: int = 1000, ik: bool = False):
    """Per problem: the first iteration whose Eq. 3 check finds a satisfying
    particle (-1 if none within ``iters``), for uniform seeds and, if ``net``
    is given, for the network's proposals (same particle count, seeds and
    tolerances; with ``ik`` both then get IK configurations).  Also the wall
    time of each run."""
    out = []
    for k, (sc, acts) in enumerate(problems):
        scene = Scene(sc)
        pid = scene.set_skeleton(acts)
        row = {}
        base = 2 if ik else 0
        for name, sampler in (("uniform", base), ("learned", base | 1)):
            if sampler & 1:
                if net is None:
                    continue
                scene.set_proposal(net)
            t0 = time.perf_counter()
            _solve(scene, pid, n_particles, seed + 7919 * k, sampler, iters, chunk, True)
            q = scene.query(pid, n_particles)
            row[name] = dict(first_iter=q["first_iter"], wall_s=time.perf_counter() - t0)
        scene.set_proposal(None)
        scene.close()
        out.append(row)
    return out
