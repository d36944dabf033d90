"""Pins of the proposal rows (oracle/proposal.py) against what the definitions
fix: encode/decode round trips, the bounds every decoded seed keeps, the normal
generator's distribution, the feature rows' structure (CPU only)."""
import math

import numpy as np
import pytest
from scipy import stats

import scenegen as sg
from oracle import philox
from oracle import proposal as op
from oracle.problem import Problem


def _wrap(a):
    return (a + math.pi) % (2 * math.pi) - math.pi


@pytest.mark.parametrize("maker", [lambda: sg.plain_problem(1001), lambda: sg.packing_problem(2002)])
def test_decode_inverts_encode_at_zero_noise(maker):
    sc, acts = maker()
    pr = Problem(sc, acts)
    X = philox.sample_uniform(pr, 40, seed=5)
    rows = op.action_rows(sc, acts)
    R = len(rows)
    _, Y, _ = op.encode(sc, acts, X)
    Y = Y.reshape(40, R, op.NT)
    for i in range(40):
        out = np.zeros((R, 2 * op.NT))
        out[:, :op.NT] = Y[i]
        Xi = op.decode(sc, acts, out, X[i:i + 1], lambda r, k: np.zeros(1))
        d = Xi[0] - X[i]
        yaw = [c for c, k in enumerate(pr.kinds) if k in ("gyaw", "pyaw")]
        d[yaw] = _wrap(d[yaw])
        assert np.abs(d).max() < 1e-12


def test_grasp_bounds_map_to_unit_interval():
    sc, acts = sg.plain_problem(1001)
    pr = Problem(sc, acts)
    hx, hy, hz = sc.box_half[0]
    X = np.zeros((2, pr.D))
    X[0, 0:4] = [hx, hy, hz, 0.0]
    X[1, 0:4] = [-hx, -hy, hz - 0.02, math.pi / 2]
    cx, cy = sc.surf[0, 0], sc.surf[0, 1]
    po = op.action_rows(sc, acts)[1][4]
    X[:, po:po + 3] = [cx, cy, 0.0]
    _, Y, M = op.encode(sc, acts, X)
    assert np.allclose(Y[0, :5], [1, 1, 1, 1, 0]) and np.allclose(Y[2, :5], [-1, -1, -1, 0, 1])
    assert np.allclose(Y[1, 5:9], [0, 0, 1, 0])
    assert M[0].tolist() == [1] * 5 + [0] * 11 and M[1].tolist() == [0] * 5 + [1] * 4 + [0] * 7


def test_decoded_seeds_keep_the_bounds_whatever_the_network_says():
    sc, acts = sg.packing_problem(2001)
    pr = Problem(sc, acts)
    rows = op.action_rows(sc, acts)
    g = np.random.default_rng(0)
    out = g.normal(0, 3, (len(rows), 2 * op.NT))
    X = op.sample(sc, acts, out, 500, seed=9)
    for (_, kind, b, s, off) in rows:
        if kind == 0:
            hx, hy, hz = sc.box_half[b]
            assert (np.abs(X[:, off]) <= hx + 1e-12).all() and (np.abs(X[:, off + 1]) <= hy + 1e-12).all()
            assert ((X[:, off + 2] >= hz - 0.02 - 1e-12) & (X[:, off + 2] <= hz + 1e-12)).all()
            assert (np.abs(X[:, off + 3]) <= math.pi).all()
        else:
            cx, cy, syaw, hx, hy, _ = sc.surf[s]
            dx, dy = X[:, off] - cx, X[:, off + 1] - cy
            u = math.cos(syaw) * dx + math.sin(syaw) * dy
            v = -math.sin(syaw) * dx + math.cos(syaw) * dy
            assert (np.abs(u) <= hx + 1e-9).all() and (np.abs(v) <= hy + 1e-9).all()
    # joint configurations are the uniform sampler's
    U = philox.sample_uniform(pr, 500, 9)
    q = [c for c, k in enumerate(pr.kinds) if k == "q"]
    assert np.array_equal(X[:, q], U[:, q])


def test_box_muller_normals_are_standard_normal():
    xi = op.normals(20000, 3, 7, seed=12345)
    assert np.isfinite(xi).all()
    assert stats.kstest(xi, "norm").pvalue > 1e-3
    assert abs(xi.mean()) < 0.03 and abs(xi.var() - 1) < 0.05
    # different rows / slots are different streams
    assert np.corrcoef(xi, op.normals(20000, 3, 8, seed=12345))[0, 1] < 0.05


def test_zero_mean_small_sigma_seeds_sit_at_the_centre():
    sc, acts = sg.plain_problem(1003)
    rows = op.action_rows(sc, acts)
    out = np.zeros((len(rows), 2 * op.NT))
    out[:, op.NT:] = op.LS_MIN                     # sigma = e^-8
    out[:, 3] = 1.0                                # grasp yaw 0
    out[:, 7] = 1.0                                # placement yaw 0
    X = op.sample(sc, acts, out, 64, seed=3)
    hz = sc.box_half[0, 2]
    assert np.allclose(X[:, 0:3], [[0, 0, hz - 0.01]], atol=2e-3)
    po = rows[1][4]
    assert np.allclose(X[:, po:po + 2], sc.surf[0, :2], atol=2e-3)
    assert np.abs(X[:, [3, po + 2]]).max() < 2e-3


def test_feature_rows_follow_the_skeleton():
    sc, skels, _ = sg.stacking_problem(3001)
    acts = skels[-1]
    rows = op.action_rows(sc, acts)
    F = op.features(sc, acts)
    assert len(rows) == sum(1 for a in acts if a[0] in (0, 1)) == F.shape[0]
    nj = len(sc.dh_a)
    for r, (ai, kind, b, s, _) in enumerate(rows):
        assert F[r, 15 + kind] == 1 and F[r, 16 - kind] == 0
        assert np.allclose(F[r, 0:3], sc.box_half[b])
        assert F[r, 17] == pytest.approx(ai / len(acts))
        # a Pick row sees where its box goes next
        place = [a for a in acts[ai:] if a[0] == 1 and a[1] == b][0]
        assert s == place[2]
        assert np.allclose(F[r, 8:10], sc.surf[s, :2]) and F[r, 14] == sc.surf[s, 5]
        assert np.allclose(F[r, 19:19 + nj], sc.dh_a) and (F[r, 19 + nj:27] == 0).all()
        assert (F[r, 44:] == 0).all()
