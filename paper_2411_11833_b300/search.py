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

Both take two options of Sec. VI-VII:

* ``cache=True`` (reusing samples across skeletons): a skeleton's particles
  are initialised from the already sampled skeleton that shares the longest
  action prefix with it -- the same sub-CSP at the same particle components --
  through tamp_sample_particles_from, so the shared subgraph's samples are
  reused and only the rest is drawn and solved.
* ``prune=True`` (pruning plan skeletons with failed subgraphs): a constraint
  no particle satisfies after initialisation marks its subgraph as likely
  unsatisfiable (``constraint_signatures`` names the subgraph); skeletons that
  contain a marked subgraph are not sampled or optimised.  Every
  ``reinit_every`` visits (chunks, for the batched form) each marked subgraph is
  re-initialised on its own -- the skeleton prefix up to its action, freshly
  sampled -- and a subgraph that then has a satisfying particle is cleared and
  the skeletons it held back rejoin the search.
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


PICK, PLACE, GOAL = 0, 1, 2
_COSTS = (7, 9)                               # MinimizeObjDist, TrajLength: never constraints
_COLLISION_KINDS = (4, 5, 8)                  # CFreeHold, CFreePlace, CFreeTraj


def constraint_signatures(actions, term_kinds, term_actions):
    """For every constraint of a skeleton (its terms other than the costs,
    in constraint order), a hashable name of its constraint subgraph (Sec.
    VII): the term kind, the action (kind, box, surface), where the acted-on
    box stands before the action (initial pose, or on the surface an earlier
    Place put it) and, for the collision terms, where the other boxes stand
    (the moved ones are named; the rest are at their initial poses).
    Two skeletons whose constraints carry the same name pose the same
    constraint on variables drawn the same way, so a name that no particle
    satisfied in one skeleton is likely unsatisfiable in the other."""
    acts = [tuple(int(v) for v in a) for a in actions]
    state, before = {}, []
    for kind, box, surface in acts:
        before.append(dict(state))
        if kind == PLACE:
            state[box] = ("on", surface)
    sigs = []
    for k, a in zip(term_kinds, term_actions):
        if k in _COSTS:
            continue
        kind, box, surface = acts[a]
        st = before[a]
        where = ("on", surface) if kind == PLACE else st.get(box, "init")
        env = None
        if k in _COLLISION_KINDS:
            # the boxes moved so far and where they stand; every other box of
            # the scene is at its initial pose in every skeleton
            env = tuple(sorted((b, w) for b, w in st.items() if b != box))
        sigs.append((int(k), kind, box, surface if kind == PLACE else -1, where, env))
    return sigs


def _shared_prefix(a, b):
    k = 0
    while k < len(a) and k < len(b) and tuple(a[k]) == tuple(b[k]):
        k += 1
    return k


class _Backend:
    """The calls the search makes, on a ``paper_2411_11833_b300.Scene``;
    ``sampler`` is the tamp_sample_particles flag combination."""

    def __init__(self, scene, sampler: int = 0):
        self.scene = scene
        self.sampler = sampler

    def compile(self, actions, options):
        return self.scene.set_skeleton(actions, options)

    def sample(self, pid, n, seed, cache_from=None):
        return self.scene.sample(pid, n, seed, self.sampler, cache_from)

    def terms(self, pid):
        _, _, kinds = self.scene.problem_info(pid)
        return kinds, self.scene.term_actions(pid)

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


class _Candidates:
    """Initialisation of the candidate skeletons (Stage 1 of Algorithm 1) with
    the cache and prune options, and the re-initialisation of failed
    subgraphs, shared by both search forms."""

    def __init__(self, be, skeletons, sizes, seed, options, cache, prune):
        self.be, self.sk, self.sizes, self.seed, self.options = be, skeletons, sizes, seed, options
        self.cache, self.prune = cache, prune
        n = len(skeletons)
        self.pids, self.sigs, self.con_actions = [None] * n, [None] * n, [None] * n
        self.sampled = []           # initialised skeletons: the sources of cached samples
        self.failed = {}            # subgraph name -> the skeleton it failed in
        self.held = {}              # held-back skeleton -> the failed names it contains
        self.scratch = {}           # subgraph name -> (problem of its skeleton prefix, constraint index)
        self.rounds = 0             # re-initialisation rounds so far
        self.cached_components = 0  # components copied instead of drawn, over all skeletons

    def _compile(self, actions):
        pid = self.be.compile(actions, self.options)
        kinds, acts = self.be.terms(pid)
        return pid, constraint_signatures(actions, kinds, acts), [a for k, a in zip(kinds, acts) if k not in _COSTS]

    def initialise(self, i):
        """Compile and sample skeleton i and check its particles; None if a
        failed subgraph holds it back."""
        if self.pids[i] is None:
            if self.prune:
                self.pids[i], self.sigs[i], self.con_actions[i] = self._compile(self.sk[i])
            else:
                self.pids[i] = self.be.compile(self.sk[i], self.options)
        if self.prune:
            blocked = {s for s in self.sigs[i] if s in self.failed}
            if blocked:
                self.held[i] = blocked
                return None
        src, best = None, 0
        if self.cache:
            for j in self.sampled:
                k = _shared_prefix(self.sk[i], self.sk[j])
                if k > best and self.sizes[j] == self.sizes[i]:
                    best, src = k, self.pids[j]
        self.cached_components += self.be.sample(self.pids[i], self.sizes[i], self.seed + 7919 * i,
                                                  cache_from=src) or 0
        self.sampled.append(i)
        q = self.be.check(self.pids[i], self.sizes[i])
        if self.prune:
            for name, c in zip(self.sigs[i], q["counts"]):
                if c == 0:
                    self.failed.setdefault(name, i)
        return q

    def reinitialise(self):
        """Sample every failed subgraph afresh on its own -- the prefix of the
        skeleton it failed in, up to the constraint's action -- and clear the
        names that now have a satisfying particle.  Returns the held-back
        skeletons that no failed name holds any longer."""
        self.rounds += 1
        for name, i in list(self.failed.items()):
            if name not in self.scratch:
                a = self.con_actions[i][self.sigs[i].index(name)]
                pid, sigs, _ = self._compile(self.sk[i][:a + 1])
                self.scratch[name] = (pid, sigs.index(name))
            pid, c = self.scratch[name]
            self.be.sample(pid, self.sizes[i], self.seed + 104729 * self.rounds + 7919 * i)
            if self.be.check(pid, self.sizes[i])["counts"][c] > 0:
                del self.failed[name]
        free = [i for i, names in self.held.items() if not any(n in self.failed for n in names)]
        for i in free:
            del self.held[i]
        return sorted(free)


def sequential_search(scene, skeletons, sizes, steps_per_chunk: int = 50, chunks_per_visit: int = 2,
                      max_iterations: int = 1000, seed: int = 0, lambda_penalty: float = -1e4, options=None,
                      cache: bool = False, prune: bool = False, reinit_every: int = 8, max_reinit: int = 16):
    """Algorithm 1, one skeleton at a time.  ``max_iterations`` bounds the
    iterations of any one skeleton; with ``prune``, failed subgraphs are
    re-initialised every ``reinit_every`` visits (and whenever no skeleton is
    left to visit), at most ``max_reinit`` times.  Returns a dict: solved,
    skeleton (index), first_iter (iteration of that skeleton's first
    satisfying check), total iterations run over all skeletons, visits,
    held_back (skeletons a failed subgraph still held back), cached_components,
    wall_s."""
    be = _backend(scene)
    t0 = time.perf_counter()
    cand = _Candidates(be, skeletons, sizes, seed, options, cache, prune)
    n = len(skeletons)
    graphs, heap, iters = [None] * n, [], [0] * n
    total, visits = 0, 0

    def result(solved, i, first):
        return dict(solved=solved, skeleton=i, first_iter=first, iterations=total, visits=visits,
                    held_back=len(cand.held), cached_components=cand.cached_components,
                    wall_s=time.perf_counter() - t0)

    def admit(i):
        q = cand.initialise(i)
        if q is None:
            return False
        if q["n_satisfied"] > 0:
            return True
        heapq.heappush(heap, (-plan_heuristic(q["counts"], lambda_penalty), i))
        return False

    for i in range(n):                                            # Stage 1
        if admit(i):
            return result(True, i, 0)
    while heap or (cand.held and cand.rounds < max_reinit):       # Stage 2
        if cand.held and cand.rounds < max_reinit and (not heap or (visits and visits % reinit_every == 0)):
            for i in cand.reinitialise():
                if admit(i):
                    return result(True, i, 0)
            if not heap:
                continue
        _, i = heapq.heappop(heap)
        visits += 1
        if graphs[i] is None:
            graphs[i] = be.graph([cand.pids[i]], steps_per_chunk, chunks_per_visit, True)
        ran = graphs[i].run()
        total += ran
        iters[i] += ran
        q = be.query(cand.pids[i], sizes[i])
        if q["n_satisfied"] > 0 or q["first_iter"] >= 0:
            return result(True, i, q["first_iter"])
        if iters[i] < max_iterations:
            heapq.heappush(heap, (-plan_heuristic(q["counts"], lambda_penalty), i))
    return result(False, -1, -1)


def batched_search(scene, skeletons, sizes, steps_per_chunk: int = 50, max_iterations: int = 1000,
                   seed: int = 0, options=None, cache: bool = False, prune: bool = False, reinit_every: int = 8):
    """Every candidate in one persistent launch per chunk, one CUDA graph that
    stops when any skeleton has a satisfying particle.  With ``prune`` the
    launch holds only the skeletons no failed subgraph holds back, and every
    ``reinit_every`` chunks the failed subgraphs are re-initialised (the freed
    skeletons join the launch).  Returns a dict: solved, skeletons (indices
    with a satisfying particle), first_iter, iterations, held_back,
    cached_components, wall_s."""
    be = _backend(scene)
    t0 = time.perf_counter()
    cand = _Candidates(be, skeletons, sizes, seed, options, cache, prune)
    active, done = [], 0

    def result(hits, first):
        return dict(solved=bool(hits), skeletons=hits, first_iter=first, iterations=done, held_back=len(cand.held),
                    cached_components=cand.cached_components, wall_s=time.perf_counter() - t0)

    def admit(i):
        q = cand.initialise(i)
        if q is not None:
            active.append(i)
            return q["n_satisfied"] > 0
        return False

    hits = [i for i in range(len(skeletons)) if admit(i)]
    if hits:
        return result(hits, 0)
    chunks_left = max(1, max_iterations // steps_per_chunk)
    while chunks_left > 0 and (active or cand.held):
        seg = min(chunks_left, reinit_every) if cand.held else chunks_left
        if active:
            g = be.graph([cand.pids[i] for i in active], steps_per_chunk, seg, True)
            done += g.run()
            if hasattr(g, "close"):
                g.close()
            qs = {i: be.query(cand.pids[i], sizes[i]) for i in active}
            hits = [i for i in active if qs[i]["first_iter"] >= 0]
            if hits:
                return result(hits, min(qs[i]["first_iter"] for i in hits))
        chunks_left -= seg
        if cand.held:
            hits = [i for i in cand.reinitialise() if admit(i)]
            if hits:
                return result(hits, 0)
    return result([], -1)
