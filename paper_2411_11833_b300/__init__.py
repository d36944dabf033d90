"""B300-native particle optimisation for differentiable task-and-motion planning.

Python binding of libtamp.so (include/tamp.h): argument marshalling only; every
step of the hot path runs in the library's CUDA kernels.  PyTorch supplies device
memory and the current stream.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native
from ._native import Action, Options, SceneDesc, TampError

# term kinds that are costs, never constraints (Eq. 3): MinimizeObjDist, TrajLength
COST_TERM_KINDS = (7, 9)

PICK, PLACE, GOAL = 0, 1, 2
TERM_NAMES = ["kin_pos", "kin_rot", "grasp", "stable_place", "cfree_hold", "cfree_place", "joint_limit",
              "obj_dist"]


def default_options(**overrides) -> Options:
    o = Options()
    _native.load().tamp_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_native.c_double_p)


def _torch():
    import torch
    return torch


def _torch_allocator():
    """tamp_allocator callbacks on PyTorch's caching allocator.  Returns the
    struct and a record of the live blocks (the callbacks must outlive the
    scene, so the Scene keeps both)."""
    torch = _torch()
    live = {}

    def alloc(nbytes, device, stream, _ctx):
        try:
            ptr = torch.cuda.caching_allocator_alloc(int(nbytes), device=int(device), stream=int(stream or 0))
        except RuntimeError:
            return None
        live[ptr] = int(nbytes)
        return ptr

    def free(ptr, _device, _stream, _ctx):
        if ptr:
            live.pop(ptr, None)
            torch.cuda.caching_allocator_delete(ptr)

    cb = (_native.ALLOC_FN(alloc), _native.FREE_FN(free))
    return _native.Allocator(cb[0], cb[1], None), cb, live


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


class Scene:
    """A scene on one device; owns its problems (compiled skeletons)."""

    def __init__(self, sc, device: int = 0, stream=None, torch_allocator: bool = False):
        """``torch_allocator``: back every device buffer of the scene with
        PyTorch's caching allocator (tamp_allocator callbacks) instead of
        cudaMalloc."""
        lib = _native.load()
        self._lib = lib
        torch = _torch()
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self._alloc = _torch_allocator() if torch_allocator else None
        keep = {}

        def arr(name, dtype=np.float64):
            a = np.ascontiguousarray(np.asarray(getattr(sc, name), dtype=dtype))
            keep[name] = a
            return a

        d = SceneDesc()
        d.n_joints = int(len(sc.dh_a))
        d.dh_a, d.dh_d = _dptr(arr("dh_a")), _dptr(arr("dh_d"))
        d.dh_alpha, d.dh_offset = _dptr(arr("dh_alpha")), _dptr(arr("dh_offset"))
        d.q_lo, d.q_hi = _dptr(arr("q_lo")), _dptr(arr("q_hi"))
        d.base[:] = [float(v) for v in np.asarray(sc.base, dtype=np.float64).ravel()]
        d.tool[:] = [float(v) for v in np.asarray(sc.tool, dtype=np.float64).ravel()]
        links = arr("sphere_link", np.int32)
        d.n_spheres = int(links.shape[0])
        d.sphere_link = links.ctypes.data_as(_native.c_int_p)
        d.sphere_xyzr = _dptr(arr("sphere_xyzr"))
        d.n_boxes = int(np.asarray(sc.box_half).shape[0])
        d.box_half, d.box_init = _dptr(arr("box_half")), _dptr(arr("box_init"))
        bs = arr("box_spheres")
        d.spheres_per_box = int(bs.shape[1]) if bs.ndim == 3 else 1
        d.box_spheres = _dptr(bs)
        d.n_obs = int(np.asarray(sc.obs_center).shape[0])
        d.obs_center, d.obs_rot, d.obs_half = _dptr(arr("obs_center")), _dptr(arr("obs_rot")), _dptr(arr("obs_half"))
        d.n_surf = int(np.asarray(sc.surf).shape[0])
        d.surf = _dptr(arr("surf"))
        h = ctypes.c_void_p()
        alloc = ctypes.byref(self._alloc[0]) if self._alloc else None
        st = lib.tamp_create_scene(ctypes.byref(d), int(device), ctypes.c_void_p(stream), alloc, ctypes.byref(h))
        if st != 0:
            raise TampError(st, "tamp_create_scene rejected the scene description")
        self._h = h
        self.device = device
        self._sizes = {}          # batch size per problem (host bookkeeping)
        self.shape = dict(n_joints=d.n_joints, n_spheres=d.n_spheres, n_boxes=d.n_boxes,
                          spheres_per_box=d.spheres_per_box, n_obs=d.n_obs, n_surf=d.n_surf)

    # -------------------------------------------------------------- helpers
    def _check(self, st):
        if st != 0:
            raise TampError(st, self._lib.tamp_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.tamp_destroy_scene(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- C ABI
    def set_skeleton(self, actions, options: Options | None = None) -> int:
        arr = (Action * len(actions))(*[Action(int(k), int(b), int(s)) for k, b, s in actions])
        pid = ctypes.c_int()
        opt = ctypes.byref(options) if options is not None else None
        self._check(self._lib.tamp_set_skeleton(self._h, arr, len(actions), opt, ctypes.byref(pid)))
        return pid.value

    def problem_info(self, pid: int):
        D, nt = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.tamp_problem_info(self._h, pid, ctypes.byref(D), ctypes.byref(nt), None))
        kinds = (ctypes.c_int * nt.value)()
        self._check(self._lib.tamp_problem_info(self._h, pid, ctypes.byref(D), ctypes.byref(nt), kinds))
        return D.value, nt.value, list(kinds)

    def sample(self, pid: int, n: int, seed: int, sampler: int = 0, cache_from: int | None = None):
        """tamp_sample_particles; with ``cache_from`` (another problem id)
        tamp_sample_particles_from, copying the components of the action prefix
        the two skeletons share from that problem's batch.  Returns the number
        of components copied (0 without ``cache_from``)."""
        shared = ctypes.c_int(0)
        if cache_from is None:
            self._check(self._lib.tamp_sample_particles(self._h, pid, int(n), ctypes.c_uint64(seed), int(sampler)))
        else:
            self._check(self._lib.tamp_sample_particles_from(self._h, pid, int(n), ctypes.c_uint64(seed),
                                                             int(sampler), int(cache_from), ctypes.byref(shared)))
        self._sizes[pid] = int(n)
        return shared.value

    def term_actions(self, pid: int):
        """tamp_term_actions: the skeleton action that introduced each term."""
        _, nt, _ = self.problem_info(pid)
        out = (ctypes.c_int * nt)()
        self._check(self._lib.tamp_term_actions(self._h, pid, out))
        return list(out)

    def set_particles(self, pid: int, x, m=None, v=None, t0: int = 0):
        """x, m, v: [D][P] float32, numpy (host) or torch CUDA tensors (device)."""
        torch = _torch()
        on_dev = isinstance(x, torch.Tensor) and x.is_cuda
        keep = []

        def p(a):
            if a is None:
                return None
            if on_dev:
                a = a.contiguous()
                keep.append(a)
                return ctypes.c_void_p(a.data_ptr())
            a = np.ascontiguousarray(a, dtype=np.float32)
            keep.append(a)
            return ctypes.c_void_p(a.ctypes.data)

        n = int(x.shape[1])
        self._check(self._lib.tamp_set_particles(self._h, pid, n, p(x), p(m), p(v), int(t0), int(on_dev)))
        self._sizes[pid] = n
        if on_dev:
            torch.cuda.current_stream(self.device).synchronize()

    def get_particles(self, pid: int):
        D, _, _ = self.problem_info(pid)
        x = np.zeros((D, self._n(pid)), np.float32)
        m, v = np.zeros_like(x), np.zeros_like(x)
        t = ctypes.c_int()
        self._check(self._lib.tamp_get_particles(self._h, pid, ctypes.c_void_p(x.ctypes.data),
                                                 ctypes.c_void_p(m.ctypes.data), ctypes.c_void_p(v.ctypes.data),
                                                 ctypes.byref(t), 0))
        return x, m, v, t.value

    def _n(self, pid):
        return self._sizes[pid]

    def optimize(self, pids, n_steps: int, stop_every: int = 0):
        """tamp_optimize_steps; ``stop_every`` = k > 0 stops at the end of the
        first chunk of k iterations in which a satisfying particle was found."""
        if isinstance(pids, int):
            pids = [pids]
        arr = (ctypes.c_int * len(pids))(*pids)
        self._check(self._lib.tamp_optimize_steps(self._h, arr, len(pids), int(n_steps), int(stop_every)))

    def query(self, pid: int, n: int, want_particles: bool = False):
        D, nt, kinds = self.problem_info(pid)
        ncon = sum(1 for k in kinds if k not in COST_TERM_KINDS)
        mask = np.zeros(n, np.uint8)
        cost = np.zeros(n, np.float32)
        counts = np.zeros(max(ncon, 1), np.int32)
        parts = np.zeros((D, n), np.float32) if want_particles else None
        ns, first = ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.tamp_query_satisfied(
            self._h, pid, ctypes.c_void_p(mask.ctypes.data), ctypes.byref(ns), ctypes.byref(first),
            None if parts is None else ctypes.c_void_p(parts.ctypes.data), ctypes.c_void_p(cost.ctypes.data),
            ctypes.c_void_p(counts.ctypes.data)))
        return dict(mask=mask.astype(bool), n_satisfied=ns.value, first_iter=first.value, cost=cost,
                    counts=counts[:ncon], particles=parts)

    def query_best(self, pid: int, n: int, want_particles: bool = True):
        """tamp_query_best: each particle's lowest-cost state among the Eq. 3
        checks it satisfied since the batch was set."""
        D, _, _ = self.problem_info(pid)
        found = np.zeros(n, np.uint8)
        cost = np.zeros(n, np.float32)
        it = np.zeros(n, np.int32)
        parts = np.zeros((D, n), np.float32) if want_particles else None
        nf = ctypes.c_int()
        self._check(self._lib.tamp_query_best(
            self._h, pid, ctypes.c_void_p(found.ctypes.data), ctypes.byref(nf),
            None if parts is None else ctypes.c_void_p(parts.ctypes.data), ctypes.c_void_p(cost.ctypes.data),
            ctypes.c_void_p(it.ctypes.data)))
        return dict(found=found.astype(bool), n_found=nf.value, cost=cost, iter=it, particles=parts)

    def set_proposal(self, net):
        """Attach a proposal network (``Mlp``) for ``sample(..., sampler=1)``; None detaches."""
        self._proposal = net                      # keep it alive while attached
        self._check(self._lib.tamp_set_proposal(self._h, None if net is None else net._h))

    def proposal_rows(self, pid: int, X=None):
        """Training rows of particles X [D][n] (host float32): (features
        [n*R, 48], targets [n*R, 16], mask [n*R, 16]); with X None, R."""
        R = ctypes.c_int()
        if X is None:
            self._check(self._lib.tamp_proposal_rows(self._h, pid, 0, None, None, None, None, ctypes.byref(R)))
            return R.value
        X = np.ascontiguousarray(X, dtype=np.float32)
        n = int(X.shape[1])
        self._check(self._lib.tamp_proposal_rows(self._h, pid, 0, None, None, None, None, ctypes.byref(R)))
        F = np.zeros((n * R.value, 48), np.float32)
        Y = np.zeros((n * R.value, 16), np.float32)
        M = np.zeros((n * R.value, 16), np.float32)
        self._check(self._lib.tamp_proposal_rows(self._h, pid, n, ctypes.c_void_p(X.ctypes.data),
                                                 ctypes.c_void_p(F.ctypes.data), ctypes.c_void_p(Y.ctypes.data),
                                                 ctypes.c_void_p(M.ctypes.data), ctypes.byref(R)))
        return F, Y, M

    def autotune(self, pids, trial_steps: int = 10):
        """Time the launch shapes for these problems' current batches and keep
        the fastest (tamp_autotune).  Returns (lanes, warps, ms)."""
        if isinstance(pids, int):
            pids = [pids]
        arr = (ctypes.c_int * len(pids))(*pids)
        L, W, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        self._check(self._lib.tamp_autotune(self._h, arr, len(pids), int(trial_steps), ctypes.byref(L),
                                            ctypes.byref(W), ctypes.byref(ms)))
        return L.value, W.value, ms.value

    def set_tuning(self, pids, lanes: int, warps: int):
        if isinstance(pids, int):
            pids = [pids]
        arr = (ctypes.c_int * len(pids))(*pids)
        self._check(self._lib.tamp_set_tuning(self._h, arr, len(pids), int(lanes), int(warps)))

    def work_counters(self, pid: int):
        """(cuboid, box) broad-phase candidates resolved exactly since the batch was set."""
        out = (ctypes.c_uint64 * 2)()
        self._check(self._lib.tamp_work_counters(self._h, pid, out))
        return int(out[0]), int(out[1])

    def eval(self, pid: int, x, want_terms=True, want_grad=True):
        """Evaluate a device batch x [D][n] (float32 CUDA tensor).  Returns
        (cost [n], terms [n_terms][n], flags [n] uint8, grad [D][n])."""
        torch = _torch()
        D, nt, _ = self.problem_info(pid)
        assert x.is_cuda and x.dtype == torch.float32 and x.shape[0] == D
        x = x.contiguous()
        n = int(x.shape[1])
        cost = torch.empty(n, dtype=torch.float32, device=x.device)
        terms = torch.empty(nt, n, dtype=torch.float32, device=x.device) if want_terms else None
        flags = torch.empty(n, dtype=torch.uint8, device=x.device)
        grad = torch.empty(D, n, dtype=torch.float32, device=x.device) if want_grad else None
        self._check(self._lib.tamp_eval(self._h, pid, n, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(cost.data_ptr()),
                                        ctypes.c_void_p(_ptr(terms)) if terms is not None else None,
                                        ctypes.c_void_p(flags.data_ptr()),
                                        ctypes.c_void_p(_ptr(grad)) if grad is not None else None))
        return cost, terms, flags, grad


class Graph:
    """CUDA graph of chunked optimisation with an optional device-side stop on
    the first satisfying particle (tamp_graph_*)."""

    def __init__(self, scene: Scene, pids, steps_per_chunk: int, n_chunks: int, stop_on_first: bool = False):
        if isinstance(pids, int):
            pids = [pids]
        self.scene = scene
        arr = (ctypes.c_int * len(pids))(*pids)
        h = ctypes.c_void_p()
        scene._check(scene._lib.tamp_graph_create(scene._h, arr, len(pids), int(steps_per_chunk), int(n_chunks),
                                                  int(bool(stop_on_first)), ctypes.byref(h)))
        self._h = h

    def run(self) -> int:
        """Replay and wait; returns the number of iterations run."""
        steps = ctypes.c_int()
        self.scene._check(self.scene._lib.tamp_graph_run(self._h, ctypes.byref(steps)))
        return steps.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.scene._lib.tamp_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cost_fn():
    """torch.autograd.Function over the fused cost + adjoint kernel: forward
    returns the Eq. 2 cost of every particle; backward returns dJ/dx from the
    hand-written reverse sweep (computed in the same launch)."""
    torch = _torch()

    class CostFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x, scene: Scene, pid: int):
            # x: [P, D] float32 CUDA; the library works on [D][P]
            xt = x.detach().t().contiguous()
            cost, _, _, grad = scene.eval(pid, xt, want_terms=False, want_grad=True)
            ctx.save_for_backward(grad.t())
            return cost

        @staticmethod
        def backward(ctx, gout):
            (grad,) = ctx.saved_tensors
            return gout[:, None] * grad, None, None

    return CostFn


class Mlp:
    """Proposal network on the tensor cores (tamp_mlp_*): 48 -> 256 -> 256 ->
    256 -> 32, BF16 weights and activations, FP32 accumulation, Adam on FP32
    master weights, Gaussian NLL.  Batches are float32 CUDA tensors, row-major."""

    IN, OUT, NTGT = 48, 32, 16

    def __init__(self, max_batch: int, device: int = 0, stream=None):
        lib = _native.load()
        self._lib = lib
        torch = _torch()
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        h = ctypes.c_void_p()
        st = lib.tamp_mlp_create(int(device), ctypes.c_void_p(stream), int(max_batch), ctypes.byref(h))
        if st != 0:
            raise TampError(st, "tamp_mlp_create failed")
        self._h = h
        self.device = device
        self.max_batch = int(max_batch)
        self.n_params = int(lib.tamp_mlp_param_count())

    def _check(self, st):
        if st != 0:
            raise TampError(st, self._lib.tamp_mlp_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.tamp_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        a = np.ascontiguousarray(np.asarray(theta, dtype=np.float32))
        self._check(self._lib.tamp_mlp_set_params(self._h, ctypes.c_void_p(a.ctypes.data), int(a.size)))

    def get_params(self) -> np.ndarray:
        a = np.zeros(self.n_params, np.float32)
        self._check(self._lib.tamp_mlp_get_params(self._h, ctypes.c_void_p(a.ctypes.data), int(a.size)))
        return a

    def forward(self, x):
        torch = _torch()
        x = x.contiguous()
        out = torch.empty(x.shape[0], self.OUT, dtype=torch.float32, device=x.device)
        self._check(self._lib.tamp_mlp_forward(self._h, ctypes.c_void_p(x.data_ptr()), int(x.shape[0]),
                                               ctypes.c_void_p(out.data_ptr())))
        return out

    def gradient(self, x, y, mask):
        torch = _torch()
        x, y, mask = x.contiguous(), y.contiguous(), mask.contiguous()
        g = torch.empty(self.n_params, dtype=torch.float32, device=x.device)
        loss = ctypes.c_float()
        self._check(self._lib.tamp_mlp_gradient(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                                ctypes.c_void_p(mask.data_ptr()), int(x.shape[0]),
                                                ctypes.c_void_p(g.data_ptr()), ctypes.byref(loss)))
        return loss.value, g

    def train_step(self, x, y, mask, lr: float, want_loss: bool = True):
        loss = ctypes.c_float()
        self._check(self._lib.tamp_mlp_train_step(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                                  ctypes.c_void_p(mask.data_ptr()), int(x.shape[0]), float(lr),
                                                  ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None
