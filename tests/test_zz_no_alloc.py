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


_FIRST_CALL_ON_A_SIDE_STREAM = r"""
import ctypes, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
import scenegen as sg
import paper_2411_11833_b300 as pkg
from paper_2411_11833_b300 import _native
from tests.parity import COST_FLOOR, COST_REL
lib = _native.load()
torch.cuda.set_device(0)
side = torch.cuda.Stream()
with torch.cuda.stream(side):                     # the scene's stream is this non-blocking side stream
    sc, acts = sg.packing_problem(2001)
    scene = pkg.Scene(sc)
    pid = scene.set_skeleton(acts)
    D, nt, _ = scene.problem_info(pid)
    n = 2000                                       # 63 tiles: a stale work-item list would show
    X = sg.random_particles(sc, acts, n, seed=3)
    x = torch.tensor(np.ascontiguousarray(X.T), dtype=torch.float32, device="cuda")
    cost = torch.full((n,), float("nan"), device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    st = lib.tamp_eval_static_scratch(scene._h, pid, n, p(x), p(cost), None, None, None)
    assert st == 0, lib.tamp_last_error(scene._h).decode()
    cost_r = scene.eval(pid, x)[0]
side.synchronize()
c, cr = cost.cpu().double().numpy(), cost_r.cpu().double().numpy()
assert np.isfinite(c).all(), "some tiles were never evaluated"
assert (np.abs(c - cr) <= COST_REL * np.maximum(np.abs(cr), COST_FLOOR)).all()
scene.close()
print("first call on a side stream ok")
"""


def test_static_scratch_first_call_on_a_side_stream():
    # The array is set up by the first call in a process, so this runs in a
    # fresh one whose first call is issued on a non-default stream.
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = subprocess.run([sys.executable, "-c", _FIRST_CALL_ON_A_SIDE_STREAM, root], capture_output=True,
                         text=True, timeout=600, cwd=root)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "first call on a side stream ok" in res.stdout
