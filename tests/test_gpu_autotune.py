"""The launch-shape autotuner (tamp_autotune, tamp_set_tuning) on the GPU:
trials leave the problems' state untouched, the tuned shape computes what any
other shape computes (up to the order of float atomic additions), and bad
shapes are refused."""
import numpy as np
import pytest
import torch

import scenegen as sg
from tests.parity import check_adam_step

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
    # the tuned shape (options lanes = 0) against an explicit other lane split with the default warps,
    # from the same state, one step at a time: each launch orders its float atomic additions differently,
    # so a particle may part ways only at a step that starts near a kink (oracle margin below TRAJ_MARGIN);
    # every other particle agrees to 1e-5 after each step, and the ones that parted are counted
    from oracle.problem import Problem
    from tests.parity import TRAJ_MARGIN
    pr = Problem(sc, acts)
    ref = pkg.Scene(sc)
    rid = ref.set_skeleton(acts, pkg.default_options(lanes=1 if L != 1 else 2))
    ref.set_particles(rid, before[0], before[1], before[2], before[3])
    alive = np.ones(n, bool)
    parted = 0
    for step in range(6):
        x0 = scene.get_particles(pid)[0].T.astype(np.float64)
        scene.optimize(pid, 1)
        ref.optimize(rid, 1)
        d = np.abs(scene.get_particles(pid)[0] - ref.get_particles(rid)[0]).max(axis=0)
        off = alive & (d > 1e-5)
        if off.any():
            near = pr.kink_margin(torch.tensor(x0[off])).numpy() < TRAJ_MARGIN
            assert near.all(), f"step {step}: a particle away from kinks parted ({d[off].max():.2e})"
            parted += int(off.sum())
            alive &= ~off
    scene.close()
    ref.close()
    print(f"{parted} of {n} particles parted at a step that started near a kink")
    assert parted <= 0.25 * n


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


@pytest.mark.parametrize("lanes,warps", [(1, 16), (1, 5), (1, 1), (2, 7), (4, 16), (8, 3)])
def test_every_launch_shape_takes_the_oracle_adam_step(pkg, lanes, warps):
    """Whatever the lane split and however many warps share a configuration's
    two pieces (the work items pulled from the per-pass counter), one fused
    iteration equals the oracle's gradient + Adam step (packing problem, 12
    configurations, a ragged last tile)."""
    from oracle.problem import Problem
    sc, acts = sg.packing_problem(2002)
    pr = Problem(sc, acts)
    P = 45
    X = sg.random_particles(sc, acts, P, seed=71, spread=0.5)
    m0, v0 = sg.random_adam_state(P, pr.D, seed=72)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    scene.set_particles(pid, X.T.astype(np.float32), m0.T.astype(np.float32), v0.T.astype(np.float32), 3)
    scene.set_tuning(pid, lanes, warps)
    scene.optimize(pid, 1)
    x1, m1, _, t1 = scene.get_particles(pid)
    scene.close()
    assert t1 == 4
    X32, m32, v32 = (a.astype(np.float32).astype(np.float64) for a in (X, m0, v0))
    keep = pr.kink_margin(torch.tensor(X32)).numpy() > 1e-4
    assert keep.mean() > 0.5
    check_adam_step(pr, X32, m32, v32, 3, x1.T, m1.T, P, keep)


def test_adam_moments_in_global_memory_take_the_oracle_step(pkg):
    """A tile too large for shared memory at one lane with its Adam moments
    (the stress skeleton, D = 252, 8 warps) runs with the moments used in
    place in global memory; one fused iteration from non-zero moments still
    equals the oracle's step, and the moments it leaves are the oracle's."""
    from oracle.problem import Problem
    sc, acts = sg.stress_problem(5001)
    pr = Problem(sc, acts)
    P = 40
    X = sg.random_particles(sc, acts, P, seed=91, spread=0.5)
    m0, v0 = sg.random_adam_state(P, pr.D, seed=92)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    scene.set_particles(pid, X.T.astype(np.float32), m0.T.astype(np.float32), v0.T.astype(np.float32), 5)
    scene.set_tuning(pid, 1, 8)
    scene.optimize(pid, 1)
    x1, m1, v1, t1 = scene.get_particles(pid)
    scene.close()
    assert t1 == 6
    X32, m32, v32 = (a.astype(np.float32).astype(np.float64) for a in (X, m0, v0))
    keep = pr.kink_margin(torch.tensor(X32)).numpy() > 1e-4
    assert keep.sum() >= 8
    check_adam_step(pr, X32, m32, v32, 5, x1.T, m1.T, P, keep)
    # the second moment left in global memory: v1 = b2 v0 + (1 - b2) (g / N_b)^2, where a gradient error
    # |dg_c| <= b (the particle's gradient bound) moves it by (1 - b2) (2 |g_c| + b) b / N_b^2, plus FP32 rounding
    _, g = pr.gradient(torch.tensor(X32))
    g = g.numpy()
    b = (1e-3 * np.maximum(np.linalg.norm(g, axis=1), 1e-2))[:, None]
    vr = pr.opts.beta2 * v32 + (1.0 - pr.opts.beta2) * (g / P) ** 2
    lim = (1.0 - pr.opts.beta2) * (2.0 * np.abs(g) + b) * b / P ** 2 + 2.0 ** -22 * vr
    assert (np.abs(v1.T - vr) <= lim)[keep].all()


def test_fp32_peak_probe_is_near_the_unit_count_peak(pkg):
    """The FFMA-chain probe behind the roofline denominator: its rate is of
    the order of SMs x 128 lanes x 2 FLOP x clock (it may run below the
    maximum clock under the power cap, never far above)."""
    import ctypes
    from paper_2411_11833_b300 import _native, flops
    tf, ms = ctypes.c_double(), ctypes.c_double()
    assert _native.load().tamp_measure_fp32_peak(0, ctypes.byref(tf), ctypes.byref(ms)) == 0
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = flops.fp32_peak_tflops(sms, 2032.0)
    assert 0.4 * nominal < tf.value < 1.05 * nominal, (tf.value, nominal)
