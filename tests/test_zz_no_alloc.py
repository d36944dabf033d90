"""tamp_eval_static_scratch: evaluation without device allocation.

Some callers may not allocate device memory while they run (a control loop with
a frozen memory budget, a framework that owns every device byte); this entry
point keeps its launch tables in a static device array instead of memory it
allocates.  It must give what tamp_eval gives, call after call, at the same
tolerances the parity tests use.  The file sorts last so that a run stopping at
its first failure has run every other test before this one.
"""
import ctypes

import numpy as np
import pytest
import torch

import scenegen as sg
from tests.parity import COST_FLOOR, COST_REL, grad_errors

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_static_scratch_eval_matches_eval_on_two_calls_in_a_row():
    from paper_2411_11833_b300.build import build_library
    build_library()
    import paper_2411_11833_b300 as pkg
    from paper_2411_11833_b300 import _native
    lib = _native.load()
    torch.cuda.set_device(0)
    sc, acts = sg.packing_problem(2001)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    D, nt, _ = scene.problem_info(pid)
    for n, seed in ((300, 1), (77, 2)):           # two calls in a row, different sizes
        X = sg.random_particles(sc, acts, n, seed=seed)
        x = torch.tensor(np.ascontiguousarray(X.T), dtype=torch.float32, device="cuda")
        cost_r, terms_r, flags_r, grad_r = scene.eval(pid, x)
        cost = torch.empty(n, device="cuda")
        terms = torch.empty(nt, n, device="cuda")
        flags = torch.empty(n, dtype=torch.uint8, device="cuda")
        grad = torch.empty(D, n, device="cuda")
        st = lib.tamp_eval_static_scratch(scene._h, pid, n, _p(x), _p(cost), _p(terms), _p(flags), _p(grad))
        assert st == 0, lib.tamp_last_error(scene._h).decode()
        torch.cuda.synchronize()
        c, cr = cost.cpu().double().numpy(), cost_r.cpu().double().numpy()
        assert (np.abs(c - cr) <= COST_REL * np.maximum(np.abs(cr), COST_FLOOR)).all()
        t, tr = terms.cpu().double().numpy(), terms_r.cpu().double().numpy()
        assert (np.abs(t - tr) <= COST_REL * np.maximum(np.abs(tr), COST_FLOOR)).all()
        # the same kernel runs both calls: flags agree except where a term sits
        # on its tolerance to within the float-atomic reordering
        assert (flags.cpu().numpy() != flags_r.cpu().numpy()).mean() < 0.01
        err, bound = grad_errors(grad.cpu().double().numpy().T, grad_r.cpu().double().numpy().T)
        assert (err <= bound).all()
    # beyond the static array's capacity the call is refused before any GPU work
    big = 4096 * 32 + 1
    st = lib.tamp_eval_static_scratch(scene._h, pid, big, _p(x), _p(cost), _p(terms), _p(flags), _p(grad))
    assert st == 1 and b"static scratch limit" in lib.tamp_last_error(scene._h)
    scene.close()
