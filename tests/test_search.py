"""Host logic of the skeleton search (Algorithm 1, Eq. 5) on a scripted backend
(CPU only), plus the stacking workload's skeleton enumeration."""
import numpy as np
import pytest

import scenegen as sg
from oracle.problem import Problem
from paper_2411_11833_b300.search import batched_search, plan_heuristic, sequential_search


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

    def sample(self, pid, n, seed):
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
