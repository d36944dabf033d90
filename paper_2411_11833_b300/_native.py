"""ctypes declarations of libtamp.so (include/tamp.h).  Marshalling only."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libtamp.so")

N_TERM_KINDS = 11
c_double_p = ctypes.POINTER(ctypes.c_double)
c_float_p = ctypes.POINTER(ctypes.c_float)
c_int_p = ctypes.POINTER(ctypes.c_int)


class SceneDesc(ctypes.Structure):
    _fields_ = [
        ("n_joints", ctypes.c_int),
        ("dh_a", c_double_p), ("dh_d", c_double_p), ("dh_alpha", c_double_p), ("dh_offset", c_double_p),
        ("q_lo", c_double_p), ("q_hi", c_double_p),
        ("base", ctypes.c_double * 16), ("tool", ctypes.c_double * 16),
        ("n_spheres", ctypes.c_int), ("sphere_link", c_int_p), ("sphere_xyzr", c_double_p),
        ("n_boxes", ctypes.c_int), ("box_half", c_double_p), ("box_init", c_double_p),
        ("spheres_per_box", ctypes.c_int), ("box_spheres", c_double_p),
        ("n_obs", ctypes.c_int), ("obs_center", c_double_p), ("obs_rot", c_double_p), ("obs_half", c_double_p),
        ("n_surf", ctypes.c_int), ("surf", c_double_p),
    ]


class Action(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("box", ctypes.c_int), ("surface", ctypes.c_int)]


class Options(ctypes.Structure):
    _fields_ = [
        ("w", ctypes.c_float * N_TERM_KINDS), ("tol", ctypes.c_float * N_TERM_KINDS),
        ("lr_joint", ctypes.c_float), ("lr_pos", ctypes.c_float), ("lr_yaw", ctypes.c_float),
        ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
        ("optimize_grasp", ctypes.c_int), ("scale_by_batch", ctypes.c_int), ("lanes", ctypes.c_int),
        ("n_knots", ctypes.c_int), ("self_collision", ctypes.c_int), ("grasp_dof", ctypes.c_int),
        ("keep_best", ctypes.c_int),
    ]


# tamp_allocator: the callbacks' C types and the struct
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


# every symbol include/tamp.h declares, with its ctypes signature
SIGNATURES = {
    "tamp_default_options": (None, [ctypes.POINTER(Options)]),
    "tamp_create_scene": (ctypes.c_int, [ctypes.POINTER(SceneDesc), ctypes.c_int, ctypes.c_void_p,
                                         ctypes.POINTER(Allocator), ctypes.POINTER(ctypes.c_void_p)]),
    "tamp_destroy_scene": (ctypes.c_int, [ctypes.c_void_p]),
    "tamp_set_skeleton": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Action), ctypes.c_int,
                                         ctypes.POINTER(Options), c_int_p]),
    "tamp_problem_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_int_p, c_int_p, c_int_p]),
    "tamp_sample_particles": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                             ctypes.c_int]),
    "tamp_sample_particles_from": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                                  ctypes.c_int, ctypes.c_int, c_int_p]),
    "tamp_term_actions": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_int_p]),
    "tamp_set_particles": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "tamp_get_particles": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, c_int_p, ctypes.c_int]),
    "tamp_optimize_steps": (ctypes.c_int, [ctypes.c_void_p, c_int_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "tamp_query_satisfied": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, c_int_p, c_int_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tamp_query_best": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, c_int_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "tamp_eval": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tamp_eval_static_scratch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tamp_work_counters": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]),
    "tamp_graph_create": (ctypes.c_int, [ctypes.c_void_p, c_int_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "tamp_graph_run": (ctypes.c_int, [ctypes.c_void_p, c_int_p]),
    "tamp_graph_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "tamp_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "tamp_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "tamp_mlp_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "tamp_mlp_param_count": (ctypes.c_int, []),
    "tamp_mlp_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "tamp_mlp_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "tamp_mlp_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "tamp_mlp_gradient": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int, ctypes.c_void_p, c_float_p]),
    "tamp_mlp_train_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int, ctypes.c_float, c_float_p]),
    "tamp_mlp_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "tamp_set_proposal": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "tamp_autotune": (ctypes.c_int, [ctypes.c_void_p, c_int_p, ctypes.c_int, ctypes.c_int, c_int_p, c_int_p, c_float_p]),
    "tamp_set_tuning": (ctypes.c_int, [ctypes.c_void_p, c_int_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "tamp_measure_fp32_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double)]),
    "tamp_proposal_rows": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, c_int_p]),
}

STATUS = {0: "TAMP_OK", 1: "TAMP_ERR_INVALID_ARG", 2: "TAMP_ERR_STATE", 3: "TAMP_ERR_OOM",
          4: "TAMP_ERR_CUDA", 5: "TAMP_ERR_TIMEOUT", 6: "TAMP_ERR_DEVICE_CHECK"}

_lib = None


def load(path: str = LIB_PATH):
    """Load libtamp.so; raises if it is missing (there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libtamp.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class TampError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
