"""The launch-shape autotuner (tamp_autotune, tamp_set_tuning) on the GPU:
trials leave the problems' state untouched, the tuned shape computes what any
other shape computes (up to the order of float atomic additions), and bad
shapes are refused."""
import numpy as np
import pytest
import torch

import scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2411_11833_b300.build import build_library
    build_library()
    import paper_2411_11833_b300 as p
    torch.cuda.set_device(0)
    return p


def test_autotune_keeps_state_and_matches_other_shapes(pkg):
    sc, acts = sg.packing_problem(2001)
    n = 700
    X = sg.random_particles(sc, acts, n, seed=5, spread=0.5).T.astype(np.float32)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    scene.set_particles(pid, X)
    scene.optimize(pid, 3)
    before = scene.get_particles(pid)
    L, W, ms = scene.autotune(pid, trial_steps=5)
    assert L in (1, 2, 4, 8) and 1 <= W <= 16 and ms > 0
    after = scene.get_particles(pid)
    for a, b in zip(before[:3], after[:3]):
        assert np.array_equal(a, b)
    assert before[3] == after[3]
    scene.optimize(pid, 6)                       # the tuned shape (options lanes = 0)
    xt = scene.get_particles(pid)[0]
    qt = scene.query(pid, n)
    # the same work with an explicit lane split and the default warps
    ref = pkg.Scene(sc)
    rid = ref.set_skeleton(acts, pkg.default_options(lanes=1 if L != 1 else 2))
    ref.set_particles(rid, X)
    ref.optimize(rid, 3)
    ref.optimize(rid, 6)
    xr = ref.get_particles(rid)[0]
    qr = ref.query(rid, n)
    d = np.abs(xt - xr)
    assert (d < 1e-4).mean() > 0.99 and d.max() < 0.1
    close = np.abs(qt["cost"] - qr["cost"]) <= 1e-4 * np.maximum(np.abs(qr["cost"]), 0.1)
    assert close.mean() > 0.95
    scene.close()
    ref.close()


def test_set_tuning_validates_and_clears(pkg):
    from paper_2411_11833_b300 import TampError
    sc, acts = sg.plain_problem(1001)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    with pytest.raises(TampError, match="STATE"):
        scene.set_tuning(pid, 1, 2)              # no batch yet
    scene.sample(pid, 256, 3)
    with pytest.raises(TampError):
        scene.set_tuning(pid, 3, 2)
    with pytest.raises(TampError):
        scene.set_tuning(pid, 1, 17)
    scene.set_tuning(pid, 4, 1)
    scene.optimize(pid, 2)
    scene.set_tuning(pid, 0, 0)                  # back to the library's heuristic
    scene.optimize(pid, 2)
    assert scene.get_particles(pid)[3] == 4
    scene.close()
