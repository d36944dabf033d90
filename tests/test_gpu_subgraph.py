"""Subgraph caching and constraint identities through the C ABI (Sec. VI,
reusing samples across skeletons; Sec. VII, pruning skeletons with failed
subgraphs) against the FP64 oracle.

* tamp_term_actions names the action of every term exactly as the oracle's
  skeleton walk does.
* tamp_sample_particles_from copies the components of the shared action prefix
  bit for bit from the source batch and draws the rest as tamp_sample_particles
  would; its IK pass solves only the configurations after the prefix, compared
  with the oracle's sampler on the same draws (the IK tolerance of
  tests/test_gpu_ik.py).
"""
import numpy as np
import pytest
import torch

import scenegen as sg
from oracle import ik, philox
from oracle.problem import Problem

from test_gpu_ik import _compare, _moved

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2411_11833_b300.build import build_library
    build_library()
    import paper_2411_11833_b300 as p
    torch.cuda.set_device(0)
    return p


def test_term_actions_match_the_oracle(pkg):
    for maker in (lambda: sg.packing_problem(2001), lambda: sg.plain_problem(1001)):
        sc, acts = maker()
        scene = pkg.Scene(sc)
        pid = scene.set_skeleton(acts)
        assert scene.term_actions(pid) == [t.action for t in Problem(sc, acts).terms]
        scene.close()


def test_cached_prefix_sampling_matches_the_oracle(pkg):
    sc, _ = sg.robot_packing_problem(21001, n_boxes=3)
    acts1 = sg.pick_place_skeleton([0, 1, 2], goal=True)
    acts2 = sg.pick_place_skeleton([0, 2, 1], goal=True)     # shares (Pick 0, Place 0)
    acts3 = sg.pick_place_skeleton([1, 0, 2], goal=True)     # shares nothing
    pr2 = Problem(sc, acts2)
    k = pr2.configs[1]["q_off"] + pr2.n
    n = 512
    scene = pkg.Scene(sc)
    p1, p2, p3 = (scene.set_skeleton(a) for a in (acts1, acts2, acts3))
    scene.sample(p1, n, 11, sampler=2)
    assert scene.sample(p2, n, 12, sampler=2, cache_from=p1) == k
    x1 = scene.get_particles(p1)[0]
    x2 = scene.get_particles(p2)[0]
    assert np.array_equal(x2[:k], x1[:k])                    # [D][P]: the prefix rows, bit for bit
    X = philox.sample_uniform(pr2, n, 12)
    X[:, :k] = x1[:k].T.astype(np.float64)
    Xm = _moved(X)
    Xm[:, :k] = X[:, :k]                                      # the copied prefix is exact
    _compare(pr2, x2.T.astype(np.float64), ik.ik_configurations(pr2, X, keep=k), ik.ik_configurations(pr2, Xm, keep=k))
    # no shared prefix: exactly the plain sampler
    assert scene.sample(p3, n, 13, sampler=2, cache_from=p1) == 0
    x3 = scene.get_particles(p3)[0]
    scene.sample(p3, n, 13, sampler=2)
    assert np.array_equal(scene.get_particles(p3)[0], x3)
    # a source without a batch of the same size, or the problem itself, is refused
    with pytest.raises(pkg.TampError):
        scene.sample(p2, n // 2, 14, sampler=2, cache_from=p1)
    with pytest.raises(pkg.TampError):
        scene.sample(p2, n, 14, sampler=2, cache_from=p2)
    scene.close()


def test_search_holds_back_skeletons_with_an_unreachable_pick(pkg):
    """Box 1 stands 3 m away: no particle satisfies Kin of picking it (Eq. 5
    count 0 even with IK seeds), so after the first skeleton that picks it,
    every other skeleton that does is held back without being sampled, and
    the search solves with the reachable box."""
    from paper_2411_11833_b300 import search
    sc, _ = sg.robot_packing_problem(21001, n_boxes=2)
    sc.box_init = sc.box_init.copy()
    sc.box_init[1, :2] = (3.0, 3.0)
    far, near = sg.pick_place_skeleton([1]), sg.pick_place_skeleton([0])
    skels = [far, near, far + near, near + far]
    scene = pkg.Scene(sc)
    be = search._Backend(scene, sampler=2)
    sampled = []
    plain_sample = be.sample

    def sample(pid, n, seed, cache_from=None):
        sampled.append(pid)
        return plain_sample(pid, n, seed, cache_from)
    be.sample = sample
    out = search.batched_search(be, skels, [1024] * 4, steps_per_chunk=20, max_iterations=600, prune=True,
                                reinit_every=10)
    assert out["solved"] and set(out["skeletons"]) <= {1}
    # the first skeleton's failed name holds back the two others that pick box 1
    # (problems 0-3 are the skeletons; re-initialisation compiles prefix problems after them)
    assert out["held_back"] == 2 and {p for p in sampled if p < 4} == {0, 1}
    scene.close()
