"""The IK configuration sampler (TAMP_SAMPLE_IK) through the C ABI vs the FP64
oracle (oracle/ik.py) on the same uniform draws.

The sampler is an iteration of 64 damped-least-squares steps with a clipped
step and joint limits.  Near a clip or a limit it is sensitive to its inputs
in any precision: the FP64 oracle itself, rerun from inputs moved by one FP32
rounding (a relative 2^-24), ends more than 1e-6 away on 16-44% of particles
and more than 1e-3 away on up to 1.2%.  The bar therefore has two parts:
among the particles whose FP64 run is stable under that perturbation (it moves
by at most 1e-6), at least 99% end within 1e-3 rad / m of the oracle on every
component the sampler writes (measured: 99.7-100%); over all particles at
least 97% do (measured: 97.5-99.8%), the rest being counted; and the share of
particles whose Kin terms the sampler satisfied (judged by the oracle's Kin
terms) agrees within 3 points.
"""
import numpy as np
import pytest
import torch

import scenegen as sg
from oracle import ik, philox
from oracle import mlp as om
from oracle import proposal as op
from oracle.problem import KIN_POS, KIN_ROT, Problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2411_11833_b300.build import build_library
    build_library()
    import paper_2411_11833_b300 as p
    torch.cuda.set_device(0)
    return p


def _wrap(a):
    return (a + np.pi) % (2 * np.pi) - np.pi


def _kin_ok(pr, X):
    tv = pr.term_values(torch.tensor(X)).numpy()
    kin = [j for j, t in enumerate(pr.terms) if t.kind in (KIN_POS, KIN_ROT)]
    return (tv[:, kin] <= np.array([5e-3 if pr.terms[j].kind == KIN_POS else 0.05 for j in kin])).all(axis=1)


def _max_diff(pr, a, b):
    kinds = np.array(pr.kinds)
    d = np.abs(a - b)
    yaw = np.isin(kinds, ["gyaw", "pyaw"])
    d[:, yaw] = np.abs(_wrap(a[:, yaw] - b[:, yaw]))
    return d.max(axis=1)


def _compare(pr, x, ref, ref_moved):
    """x: the kernel's configurations; ref: the oracle's from the same draws;
    ref_moved: the oracle's from the draws moved by one FP32 rounding."""
    d = _max_diff(pr, x, ref)
    stable = _max_diff(pr, ref_moved, ref) <= 1e-6
    assert stable.mean() >= 0.5, stable.mean()
    assert (d[stable] <= 1e-3).mean() >= 0.99, (d[stable] <= 1e-3).mean()
    assert (d <= 1e-3).mean() >= 0.97, (d <= 1e-3).mean()
    ok_g, ok_o = _kin_ok(pr, x), _kin_ok(pr, ref)
    assert abs(ok_g.mean() - ok_o.mean()) <= 0.03, (ok_g.mean(), ok_o.mean())
    print(f"\nIK: {int((d > 1e-3).sum())} of {len(d)} particles beyond 1e-3, "
          f"{int((d[stable] > 1e-3).sum())} of {int(stable.sum())} stable ones")
    return ok_g.mean()


def _moved(X, seed=0):
    """The draws moved by one FP32 rounding (relative 2^-24, random sign)."""
    return X * (1.0 + np.random.default_rng(seed).choice([-1.0, 1.0], X.shape) * 2.0 ** -24)


@pytest.mark.parametrize("maker,n", [(lambda: sg.robot_plain_problem(20001), 512),
                                     (lambda: sg.plain_problem(1001), 512),
                                     (lambda: sg.robot_packing_problem(21001, n_boxes=3), 256)])
def test_ik_sampler_matches_oracle(pkg, maker, n):
    sc, acts = maker()
    pr = Problem(sc, acts)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    seed = 0x5EED_0001
    scene.sample(pid, n, seed, sampler=2)
    x = scene.get_particles(pid)[0].T.astype(np.float64)
    X0 = philox.sample_uniform(pr, n, seed)
    rate = _compare(pr, x, ik.ik_configurations(pr, X0), ik.ik_configurations(pr, _moved(X0)))
    print(f"\nIK sampler: {sc.name} Kin satisfied after sampling {rate:.3f}")
    scene.close()


def test_learned_then_ik_matches_oracle(pkg):
    sc, acts = sg.robot_plain_problem(20002)
    pr = Problem(sc, acts)
    th = om.init_params(4).numpy().astype(np.float32)
    net = pkg.Mlp(max_batch=64)
    net.set_params(th)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    scene.set_proposal(net)
    n, seed = 512, 77
    scene.sample(pid, n, seed, sampler=3)
    x = scene.get_particles(pid)[0].T.astype(np.float64)
    out = om.forward(torch.from_numpy(th).double(), torch.from_numpy(op.features(sc, acts))).numpy()
    X0 = op.sample(sc, acts, out, n, seed)
    _compare(pr, x, ik.ik_configurations(pr, X0), ik.ik_configurations(pr, _moved(X0)))
    scene.close()
    net.close()
