"""Host logic of the skeleton search (Algorithm 1, Eq. 5) on a scripted backend
(CPU only), plus the stacking workload's skeleton enumeration."""
import numpy as np
import pytest

import scenegen as sg
from oracle.problem import Problem
from paper_2411_11833_b300.search import (GOAL, PICK, PLACE, batched_search, constraint_signatures, plan_heuristic,
                                          sequential_search)


def test_plan_heuristic_is_eq5():
    # mean of counts, a zero count replaced by the penalty
    assert plan_heuristic([4, 0, 2], -100.0) == pytest.approx((4 - 100 + 2) / 3)
    assert plan_heuristic([3, 3], -1.0) == 3.0
    assert plan_heuristic([], -1.0) == 0.0


class FakeGraph:
    def __init__(self, be, pids, steps, chunks, stop):
        self.be, self.pids, self.steps, self.chunks, self.stop = be, pids, steps, chunks, stop

    def run(self):
        ran = 0
        for _ in range(self.chunks):
            ran += self.steps
            done = False
            for pid in self.pids:
                self.be.t[pid] += self.steps
                if self.be.t[pid] >= self.be.solve_at[pid] and self.be.first[pid] < 0:
                    self.be.first[pid] = self.be.solve_at[pid]
                    done = True
            if self.stop and done:
                break
        return ran


class FakeBackend:
    """Problem i becomes satisfiable after solve_at[i] iterations; its Eq. 5
    counts are scripted."""

    def __init__(self, solve_at, counts):
        self.solve_at, self.counts = solve_at, counts
        self.t, self.first, self.order = {}, {}, []

    def compile(self, acts, options):
        pid = len(self.t)
        self.t[pid], self.first[pid] = 0, -1
        return pid

    def sample(self, pid, n, seed, cache_from=None):
        pass

    def check(self, pid, n):
        return dict(n_satisfied=0, first_iter=-1, counts=self.counts[pid])

    def query(self, pid, n):
        self.order.append(pid)
        return dict(n_satisfied=int(self.first[pid] >= 0), first_iter=self.first[pid], counts=self.counts[pid])

    def graph(self, pids, steps, chunks, stop):
        return FakeGraph(self, pids, steps, chunks, stop)


def test_sequential_search_visits_best_heuristic_first():
    be = FakeBackend(solve_at=[10**9, 100, 60], counts=[[5, 5], [0, 9], [1, 1]])
    out = sequential_search(be, [[]] * 3, [8, 8, 8], steps_per_chunk=20, chunks_per_visit=1, max_iterations=400)
    # H = 5, (-1e4 + 9)/2, 1: problem 0 first, then 2 (solves at 60) before 1
    assert out["solved"] and out["skeleton"] == 2
    assert be.order[0] == 0 and 1 not in be.order


def test_sequential_search_gives_up_after_budget():
    be = FakeBackend(solve_at=[10**9], counts=[[1]])
    out = sequential_search(be, [[]], [8], steps_per_chunk=10, chunks_per_visit=2, max_iterations=100)
    assert not out["solved"] and out["iterations"] == 100


def test_batched_search_stops_at_first_solver():
    be = FakeBackend(solve_at=[300, 80, 10**9], counts=[[1], [1], [1]])
    out = batched_search(be, [[]] * 3, [8, 8, 8], steps_per_chunk=20, max_iterations=1000)
    assert out["solved"] and out["skeletons"] == [1] and out["first_iter"] == 80 and out["iterations"] == 80


def test_stacking_skeletons():
    sc, skels, sizes = sg.stacking_problem(3002)
    nb = sc.meta["n_blockers"]
    assert len(skels) == 16 and all(s in (1024, 2048, 4096, 8192) for s in sizes)
    lengths = sorted({len(a) for a in skels})
    assert lengths[0] == 2 and lengths[-1] <= 8
    for acts in skels:
        assert acts[-2:] == [(0, 0, -1), (1, 0, 0)]               # A onto B last
        pr = Problem(sc, acts)                                    # a valid CSP
        assert pr.D == sum(11 if k == 0 else 10 for k, _, _ in acts)
    # every blocker initially rests on B's top face
    assert np.allclose(sc.box_init[2:2 + nb, 2], sc.surf[0, 5] + sc.box_half[2:2 + nb, 2])


def test_stacking_blockers_occupy_every_placement_on_b():
    # the 0-blocker skeleton (Pick A, Place A on B) has no contained,
    # collision-free placement: the blockers' spheres cover B's top
    import torch
    from oracle import philox
    from oracle.problem import CFREE_PLACE, STABLE_PLACE
    for seed in (3001, 3002, 3009):
        sc, skels, _ = sg.stacking_problem(seed)
        pr = Problem(sc, skels[0])
        tv = pr.term_values(torch.tensor(philox.sample_uniform(pr, 1500, 5))).numpy()
        cp = [j for j, t in enumerate(pr.terms) if t.kind == CFREE_PLACE]
        st = [j for j, t in enumerate(pr.terms) if t.kind == STABLE_PLACE]
        inside = tv[:, st].sum(axis=1) <= 1e-3
        assert inside.sum() > 300
        assert not (inside & (tv[:, cp].sum(axis=1) <= 1e-3)).any()


# ---------------------------------------------------------------- Sec. VI-VII: caching and pruning

PICK_TERMS = [0, 1, 2, 4, 6]          # Kin pos, Kin rot, Grasp, CFreeHold, joint limits
PLACE_TERMS = [0, 1, 3, 4, 5, 6]      # Kin pos, Kin rot, StablePlace, CFreeHold, CFreePlace, joint limits


def _terms(acts):
    kinds, owner = [], []
    for a, (kind, _, _) in enumerate(acts):
        ks = PICK_TERMS if kind == PICK else (PLACE_TERMS if kind == PLACE else [7])
        kinds += ks
        owner += [a] * len(ks)
    return kinds, owner


def test_term_layout_of_the_fake_is_the_oracle_walk():
    sc, skels, _ = sg.stacking_problem(3001)
    for acts in skels[:4]:
        pr = Problem(sc, acts)
        assert _terms(acts) == ([t.kind for t in pr.terms], [t.action for t in pr.terms])


def test_constraint_names_follow_the_skeleton_state():
    sc, skels, _ = sg.stacking_problem(3001)
    names = [constraint_signatures(a, *_terms(a)) for a in skels]
    cons = [[(a, k) for k, a in zip(*_terms(s)) if k != 7] for s in skels]
    # a prefix of actions names its constraints alike in every skeleton that has it
    for i, a in enumerate(skels):
        for j, b in enumerate(skels):
            k = 0
            while k < min(len(a), len(b)) and tuple(a[k]) == tuple(b[k]):
                k += 1
            pa = [n for n, (act, _) in zip(names[i], cons[i]) if act < k]
            pb = [n for n, (act, _) in zip(names[j], cons[j]) if act < k]
            assert pa == pb
    # the final Place of A on B: moving the same blockers in another order gives
    # the same collision names, moving other blockers other ones
    def final_place_collision(i):
        last = len(skels[i]) - 1
        return {n for n, (act, kd) in zip(names[i], cons[i]) if act == last and kd in (4, 5)}
    by_set = {}
    for i, acts in enumerate(skels):
        moved = frozenset(b for kind, b, _ in acts[:-2] if kind == PICK)
        by_set.setdefault(moved, set()).add(frozenset(final_place_collision(i)))
    assert all(len(v) == 1 for v in by_set.values())
    assert len({next(iter(v)) for v in by_set.values()}) == len(by_set)
    # Kin of picking a box from its initial pose carries one name wherever it appears
    kin_pick = {}
    for i, acts in enumerate(skels):
        for n, (act, kd) in zip(names[i], cons[i]):
            if kd == 0 and acts[act][0] == PICK:
                kin_pick.setdefault(acts[act][1], set()).add(n)
    assert all(len(v) == 1 for v in kin_pick.values())


class SubgraphBackend:
    """Skeletons with the library's term layout; the Eq. 5 count of a
    constraint is scripted by its subgraph name: names in ``failing`` have no
    satisfying particle until they have been sampled ``failing[name]`` times
    (None: never).  Every problem becomes satisfiable after ``solve_at``
    iterations unless it contains a never-satisfiable name."""

    def __init__(self, failing, solve_at=40):
        self.failing, self.solve_at = dict(failing), solve_at
        self.acts, self.t, self.first, self.samples, self.cache_from = {}, {}, {}, {}, {}
        self.seen = {}

    def compile(self, acts, options):
        pid = len(self.acts)
        self.acts[pid] = [tuple(a) for a in acts]
        self.t[pid], self.first[pid] = 0, -1
        return pid

    def terms(self, pid):
        return _terms(self.acts[pid])

    def names(self, pid):
        return constraint_signatures(self.acts[pid], *self.terms(pid))

    def sample(self, pid, n, seed, cache_from=None):
        self.samples[pid] = self.samples.get(pid, 0) + 1
        self.cache_from[pid] = cache_from
        for name in self.names(pid):
            self.seen[name] = self.seen.get(name, 0) + 1
        return 0 if cache_from is None else 7

    def _counts(self, pid):
        out = []
        for name in self.names(pid):
            need = self.failing.get(name, 0)
            out.append(0 if need is None or self.seen.get(name, 0) <= need else 5)
        return out

    def check(self, pid, n):
        return dict(n_satisfied=0, first_iter=-1, counts=self._counts(pid))

    def query(self, pid, n):
        return dict(n_satisfied=int(self.first[pid] >= 0), first_iter=self.first[pid], counts=self._counts(pid))

    def graph(self, pids, steps, chunks, stop):
        be = self

        class G:
            def run(self):
                ran = 0
                for _ in range(chunks):
                    ran += steps
                    hit = False
                    for pid in pids:
                        be.t[pid] += steps
                        if be.t[pid] >= be.solve_at and 0 not in be._counts(pid) and be.first[pid] < 0:
                            be.first[pid] = be.t[pid]
                            hit = True
                    if stop and hit:
                        break
                return ran
        return G()


def _stack_skeletons():
    # boxes: A = 0, B = 1, blockers 2, 3 on B; surface 0 = B's top, 1 = table
    mv = lambda b: [(PICK, b, -1), (PLACE, b, 1)]
    fin = [(PICK, 0, -1), (PLACE, 0, 0)]
    return [fin, mv(2) + fin, mv(3) + fin, mv(2) + mv(3) + fin, mv(3) + mv(2) + fin]


def _final_place_names(acts):
    names = constraint_signatures(acts, *_terms(acts))
    kinds, owner = _terms(acts)
    cons = [(k, a) for k, a in zip(kinds, owner) if k != 7]
    return {n for n, (k, a) in zip(names, cons) if a == len(acts) - 1 and k == 5}


def test_pruning_holds_back_skeletons_with_a_failed_subgraph():
    skels = _stack_skeletons()
    # placing A on B fails while a blocker is still there
    failing = {n: None for acts in skels[:3] for n in _final_place_names(acts)}
    be = SubgraphBackend(failing)
    out = sequential_search(be, skels, [8] * 5, steps_per_chunk=20, chunks_per_visit=1, max_iterations=200,
                            prune=True, reinit_every=2, max_reinit=3)
    assert out["solved"] and out["skeleton"] in (3, 4)
    # skeletons 0-2 fail on their own final Place; none is held back (their names
    # differ: different blockers remain) -- and the two orders of moving both
    # blockers share every name, so both are tried
    assert out["held_back"] == 0
    # a later skeleton with an already failed name is never sampled
    be = SubgraphBackend(failing)
    out = sequential_search(be, skels + [[(PICK, 2, -1), (PLACE, 2, 1)] + [(PICK, 0, -1), (PLACE, 0, 0)]],
                            [8] * 6, steps_per_chunk=20, chunks_per_visit=1, max_iterations=200, prune=True,
                            reinit_every=2, max_reinit=3)
    assert 5 not in be.samples and out["held_back"] == 1


def test_reinitialised_subgraph_releases_held_back_skeletons():
    skels = _stack_skeletons()
    f = next(iter(_final_place_names(skels[1])))
    # the failed name of skeleton 1 passes from its third sampling on; skeleton 5
    # shares it and is held back until the re-initialisation clears it
    extra = [(PICK, 2, -1), (PLACE, 2, 1), (PICK, 0, -1), (PLACE, 0, 0)]
    be = SubgraphBackend({f: 2}, solve_at=10**9)
    out = sequential_search(be, skels[1:2] + [extra], [8, 8], steps_per_chunk=20, chunks_per_visit=1,
                            max_iterations=100, prune=True, reinit_every=1, max_reinit=4)
    assert not out["solved"]
    assert be.samples.get(1, 0) == 1 and out["held_back"] == 0
    # the re-initialisation sampled the failed subgraph on its own prefix problem
    assert any(be.acts[p] == [tuple(a) for a in skels[1]] for p in be.acts if p >= 2)
    # batched form: the freed skeleton joins the launch
    be = SubgraphBackend({f: 2}, solve_at=60)
    out = batched_search(be, skels[1:2] + [extra], [8, 8], steps_per_chunk=20, max_iterations=400, prune=True,
                         reinit_every=1)
    assert out["held_back"] == 0 and be.samples.get(1, 0) == 1


def test_cache_samples_from_the_longest_shared_prefix():
    skels = _stack_skeletons()
    be = SubgraphBackend({})
    out = sequential_search(be, skels, [8, 8, 8, 8, 4], steps_per_chunk=20, chunks_per_visit=1,
                            max_iterations=100, cache=True)
    # 0 first (nothing sampled), 1 and 2 share nothing with 0 (their first action
    # differs), 3 shares (Pick 2, Place 2) with 1, 4 shares (Pick 3, Place 3) with 2
    # but has another batch size
    assert be.cache_from[0] is None and be.cache_from[1] is None and be.cache_from[2] is None
    assert be.cache_from[3] == 1 and be.cache_from[4] is None
    assert out["cached_components"] == 7
