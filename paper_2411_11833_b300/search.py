"""Search over candidate plan skeletons (Algorithm 1) as a small host loop.

The skeleton candidates are given (the obstructed-stacking workload enumerates
them); everything continuous runs on the GPU through the C ABI.

* ``plan_heuristic`` -- Eq. 5: the mean over a skeleton's constraints of the
  number of particles satisfying each one, with a large negative penalty for a
  constraint no particle satisfies.
* ``sequential_search`` -- Algorithm 1 with one skeleton optimised at a time:
  Stage 1 initialises every candidate's particles and scores it with Eq. 5;
  Stage 2 repeatedly pops the best-scoring skeleton, optimises it for a few
  chunks (a CUDA graph that stops at the first satisfying particle), returns
  if a particle satisfies Eq. 3, and otherwise re-scores it and pushes it back.
* ``batched_search`` -- all candidates in one persistent launch per chunk,
  captured in one CUDA graph that stops as soon as any skeleton has a
  satisfying particle.
"""
from __future__ import annotations

import heapq
import time

import numpy as np


def plan_heuristic(counts, lambda_penalty: float) -> float:
    """Eq. 5: H = mean_c h(c), h(c) = n_satisfying(c) or Lambda_penalty if 0."""
    counts = np.asarray(counts, dtype=np.float64)
    if counts.size == 0:
        return 0.0
    return float(np.where(counts > 0, counts, lambda_penalty).mean())


class _Backend:
    """The calls the search makes, on a ``paper_2411_11833_b300.Scene``."""

    def __init__(self, scene):
        self.scene = scene

    def compile(self, actions, options):
        return self.scene.set_skeleton(actions, options)

    def sample(self, pid, n, seed):
        self.scene.sample(pid, n, seed)

    def check(self, pid, n):
        self.scene.optimize(pid, 0)
        return self.scene.query(pid, n)

    def query(self, pid, n):
        return self.scene.query(pid, n)

    def graph(self, pids, steps, chunks, stop_on_first):
        from . import Graph
        return Graph(self.scene, pids, steps, chunks, stop_on_first)


def _backend(scene):
    return scene if hasattr(scene, "graph") else _Backend(scene)


def sequential_search(scene, skeletons, sizes, steps_per_chunk: int = 50, chunks_per_visit: int = 2,
                      max_iterations: int = 1000, seed: int = 0, lambda_penalty: float = -1e4, options=None):
    """Algorithm 1, one skeleton at a time.  ``max_iterations`` bounds the
    iterations of any one skeleton.  Returns a dict: solved, skeleton (index),
    first_iter (iteration of that skeleton's first satisfying check), total
    iterations run over all skeletons, visits, wall_s."""
    be = _backend(scene)
    t0 = time.perf_counter()
    pids, graphs, heap, iters = [], [], [], []
    for i, (acts, n) in enumerate(zip(skeletons, sizes)):       # Stage 1
        pid = be.compile(acts, options)
        be.sample(pid, n, seed + 7919 * i)
        q = be.check(pid, n)
        if q["n_satisfied"] > 0:
            return dict(solved=True, skeleton=i, first_iter=0, iterations=0, visits=0,
                        wall_s=time.perf_counter() - t0)
        pids.append(pid)
        graphs.append(None)
        iters.append(0)
        heapq.heappush(heap, (-plan_heuristic(q["counts"], lambda_penalty), i))
    total, visits = 0, 0
    while heap:                                                   # Stage 2
        _, i = heapq.heappop(heap)
        visits += 1
        if graphs[i] is None:
            graphs[i] = be.graph([pids[i]], steps_per_chunk, chunks_per_visit, True)
        ran = graphs[i].run()
        total += ran
        iters[i] += ran
        q = be.query(pids[i], sizes[i])
        if q["n_satisfied"] > 0 or q["first_iter"] >= 0:
            return dict(solved=True, skeleton=i, first_iter=q["first_iter"], iterations=total, visits=visits,
                        wall_s=time.perf_counter() - t0)
        if iters[i] < max_iterations:
            heapq.heappush(heap, (-plan_heuristic(q["counts"], lambda_penalty), i))
    return dict(solved=False, skeleton=-1, first_iter=-1, iterations=total, visits=visits,
                wall_s=time.perf_counter() - t0)


def batched_search(scene, skeletons, sizes, steps_per_chunk: int = 50, max_iterations: int = 1000,
                   seed: int = 0, options=None):
    """Every candidate in one persistent launch per chunk, one CUDA graph that
    stops when any skeleton has a satisfying particle.  Returns a dict: solved,
    skeletons (indices with a satisfying particle), first_iter, iterations
    (per skeleton), wall_s."""
    be = _backend(scene)
    t0 = time.perf_counter()
    pids = []
    for i, (acts, n) in enumerate(zip(skeletons, sizes)):
        pid = be.compile(acts, options)
        be.sample(pid, n, seed + 7919 * i)
        pids.append(pid)
    g = be.graph(pids, steps_per_chunk, max(1, max_iterations // steps_per_chunk), True)
    ran = g.run()
    qs = [be.query(pid, n) for pid, n in zip(pids, sizes)]
    hits = [i for i, q in enumerate(qs) if q["first_iter"] >= 0]
    first = min((qs[i]["first_iter"] for i in hits), default=-1)
    return dict(solved=bool(hits), skeletons=hits, first_iter=first, iterations=ran,
                wall_s=time.perf_counter() - t0)
