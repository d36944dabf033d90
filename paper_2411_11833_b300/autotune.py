"""Persistent cache of tuned launch shapes (tamp_autotune / tamp_set_tuning).

The library's autotuner times the launch shapes of the persistent kernel for a
set of problems and keeps the fastest in the scene.  This module keeps those
choices across processes in a JSON file keyed by the GPU (name, SM count) and a
signature of the work -- the scene's sizes and each problem's particle
dimension, term kinds and batch size -- so a later run on the same kind of GPU
and workload installs the shape without timing it again.
"""
from __future__ import annotations

import hashlib
import json
import os


def default_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "tamp_b300", "autotune.json")


def signature(shape: dict, problems) -> str:
    """problems: [(D, term_kinds, batch size)] in launch order."""
    blob = json.dumps({"scene": shape, "problems": [[int(D), list(map(int, kinds)), int(P)]
                                                   for D, kinds, P in problems]}, sort_keys=True)
    return hashlib.sha256(blob.encode()).hexdigest()[:24]


def gpu_key(name: str, sm_count: int) -> str:
    return f"{name}|{int(sm_count)}"


def load(path: str) -> dict:
    try:
        with open(path) as fh:
            data = json.load(fh)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store(path: str, data: dict) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(scene, pids, sizes, trial_steps: int = 10, path: str | None = None, gpu=None):
    """Install the cached shape for (GPU, work) or time one and cache it.
    ``sizes``: the batch size of each problem (as sampled).  Returns
    dict(lanes, warps, ms, cached)."""
    if isinstance(pids, int):
        pids, sizes = [pids], [sizes]
    path = path or default_path()
    if gpu is None:
        import torch
        props = torch.cuda.get_device_properties(scene.device)
        gpu = (props.name, props.multi_processor_count)
    probs = []
    for pid, P in zip(pids, sizes):
        D, _, kinds = scene.problem_info(pid)
        probs.append((D, kinds, P))
    key = f"{gpu_key(*gpu)}|{signature(scene.shape, probs)}"
    data = load(path)
    if key in data:
        ent = data[key]
        scene.set_tuning(pids, ent["lanes"], ent["warps"])
        return dict(ent, cached=True)
    L, W, ms = scene.autotune(pids, trial_steps)
    data = load(path)
    data[key] = {"lanes": L, "warps": W, "ms": ms, "trial_steps": trial_steps}
    store(path, data)
    return dict(lanes=L, warps=W, ms=ms, trial_steps=trial_steps, cached=False)
