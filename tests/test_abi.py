"""The C ABI library loads and exports every entry point include/tamp.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(tamp_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2411_11833_b300.build import build_library
    build_library()
    from paper_2411_11833_b300 import _native
    return _native.load()


def test_header_declares_the_boundary_calls():
    names = _declared()
    for n in ("tamp_create_scene", "tamp_set_skeleton", "tamp_sample_particles", "tamp_optimize_steps",
              "tamp_query_satisfied", "tamp_eval"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2411_11833_b300 import _native
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in _native.SIGNATURES, f"binding lacks {name}"


def test_default_options_are_the_papers(lib):
    import paper_2411_11833_b300 as pkg
    o = pkg.default_options()
    # ... and the readings for the knot terms (CFreeTraj as the other collisions,
    # TrajLength 0.01); no knots by default
    # and self-collision (1.0, 0 penetration); no knots, no self-collision by default
    assert list(o.w) == pytest.approx([1.0, 5.0, 1.0, 2.0, 1.0, 1.0, 1.0, 0.25, 1.0, 0.01, 1.0])
    assert list(o.tol)[:7] == pytest.approx([5e-3, 0.05, 1e-3, 1e-3, 1e-3, 1e-3, 0.0])
    assert o.tol[8] == pytest.approx(1e-3) and o.tol[10] == 0.0
    assert o.n_knots == 0 and o.self_collision == 0 and o.grasp_dof == 4
    assert o.beta1 == pytest.approx(0.9) and o.beta2 == pytest.approx(0.999)


def test_null_arguments_are_rejected_without_a_device(lib):
    h = ctypes.c_void_p()
    assert lib.tamp_create_scene(None, 0, None, None, ctypes.byref(h)) == 1
    # an allocator must give both callbacks: refused before the description is read or a device touched
    from paper_2411_11833_b300 import _native
    half = _native.Allocator(_native.ALLOC_FN(lambda n, d, s, c: None), _native.FREE_FN(), None)
    desc = _native.SceneDesc()
    assert lib.tamp_create_scene(ctypes.byref(desc), 0, None, ctypes.byref(half), ctypes.byref(h)) == 1
    assert not h.value
    assert lib.tamp_destroy_scene(None) == 1
    assert lib.tamp_optimize_steps(None, None, 0, 1, 0) == 1
