"""The packing witness scene through the C ABI (tests/golden/packing_witness.json,
built from the oracle alone): Eq. 3 at the benchmark's batch on particles that
satisfy every constraint, and evaluation parity with the oracle around them,
where the checks fall on both sides of the tolerances."""
import numpy as np
import pytest
import torch

from oracle.problem import Problem
from tests.parity import compare_eval
from tests.test_witness_scene import load_witness

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2411_11833_b300.build import build_library
    build_library()
    import paper_2411_11833_b300 as p
    torch.cuda.set_device(0)
    return p


def test_every_copy_of_the_witness_satisfies_at_full_batch(pkg):
    """4096 copies of the witness (the packing workload's batch, 128 tiles):
    the Eq. 3 check passes for every one, the first satisfying check is the
    first, the Eq. 5 counts are the full batch for every constraint, and the
    best-satisfying record holds each copy at that check."""
    d, sc, acts = load_witness()
    P = 4096
    w32 = np.array(d["witness"], dtype=np.float32)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts, pkg.default_options(keep_best=1))
    scene.set_particles(pid, np.repeat(w32[:, None], P, axis=1))
    q = scene.query(pid, P)
    b = scene.query_best(pid, P)
    scene.close()
    assert q["n_satisfied"] == P and q["first_iter"] == 0
    assert (q["counts"] == P).all()
    assert b["n_found"] == P and (b["iter"] == 0).all()
    assert np.array_equal(b["particles"], np.repeat(w32[:, None], P, axis=1))


def test_evaluation_parity_around_the_witness(pkg):
    """300 particles (the witness and perturbations of it from 0.1 mm to 3 cm /
    mrad to 30 mrad: 10 tiles, a ragged tail of 12) through tamp_eval against
    the oracle: costs, terms, Eq. 3 flags and gradients by the rules of
    tests/parity.py, with particles on both sides of the tolerances."""
    d, sc, acts = load_witness()
    pr = Problem(sc, acts)
    w = np.array(d["witness"])
    rng = np.random.default_rng(11)
    P = 300
    scale = np.geomspace(1e-4, 3e-2, P)[:, None]
    X = (w[None] + scale * rng.normal(size=(P, w.size)))
    X[0] = w
    X = X.astype(np.float32).astype(np.float64)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    out = scene.eval(pid, torch.tensor(np.ascontiguousarray(X.T), dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    scene.close()
    res = compare_eval(pr, X, *out, label="packing witness", min_kept=0.3)
    print(res)
    flags = out[2].cpu().numpy().astype(bool)
    assert flags[0] and 0 < flags.sum() < P        # satisfying and violating particles both present
