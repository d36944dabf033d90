"""Comparison rules of the CUDA path against the FP64 oracle.

Tolerances (FP32 kernel vs FP64 oracle):
  * term values and Eq. 2 totals: |gpu - ora| <= 1e-4 * max(|ora|, 0.1).  The
    floor 0.1 (m or rad) gives an absolute 1e-5: FP32 unit roundoff (6e-8) times
    the workspace scale (~1 m) times the depth of the kinematic chain and the
    sums over sphere pairs (~100 roundings) is ~6e-6.
  * gradients, per particle: ||g_gpu - g_ora|| <= 1e-3 * max(||g_ora||, 1e-2),
    for particles whose kink margin (oracle ``kink_margin``) is above
    KINK_MARGIN; the others are counted and reported.
  * Eq. 3 flags: identical, except particles with some constraint within 1e-5
    of its tolerance (counted).
"""
from __future__ import annotations

import numpy as np
import torch

COST_REL, COST_FLOOR = 1e-4, 0.1
GRAD_REL, GRAD_FLOOR = 1e-3, 1e-2
KINK_MARGIN = 1e-4
FLAG_BAND = 1e-5


def cost_ok(gpu: np.ndarray, ora: np.ndarray) -> np.ndarray:
    return np.abs(gpu - ora) <= COST_REL * np.maximum(np.abs(ora), COST_FLOOR)


def grad_errors(gpu: np.ndarray, ora: np.ndarray):
    """Per-particle (error, bound) for [P, D] gradients."""
    err = np.linalg.norm(gpu - ora, axis=1)
    bound = GRAD_REL * np.maximum(np.linalg.norm(ora, axis=1), GRAD_FLOOR)
    return err, bound


def near_threshold(problem, terms_ora: np.ndarray) -> np.ndarray:
    tol = problem.tolerances().numpy()
    cm = problem.constraint_mask().numpy()
    return (np.abs(terms_ora[:, cm] - tol[cm]) <= FLAG_BAND).any(axis=1)


def compare_eval(problem, X: np.ndarray, cost, terms, flags, grad, label=""):
    """Full comparison of a tamp_eval result with the oracle on the same X [P, D].

    Returns a dict of counts; raises AssertionError with details on a violation."""
    Xt = torch.tensor(X, dtype=torch.float64)
    with torch.no_grad():
        T_ora = problem.term_values(Xt).numpy()
    J_ora, g_ora = problem.gradient(Xt)
    J_ora, g_ora = J_ora.numpy(), g_ora.numpy()
    margin = problem.kink_margin(Xt).numpy()
    cost = cost.detach().cpu().double().numpy()
    terms = terms.detach().cpu().double().numpy().T
    flags = flags.detach().cpu().numpy().astype(bool)
    grad = grad.detach().cpu().double().numpy().T

    bad_t = ~cost_ok(terms, T_ora)
    if bad_t.any():
        p, t = np.argwhere(bad_t)[0]
        raise AssertionError(f"{label}: term {t} of particle {p}: gpu {terms[p, t]!r} oracle {T_ora[p, t]!r} "
                             f"({int(bad_t.sum())} bad of {bad_t.size})")
    bad_c = ~cost_ok(cost, J_ora)
    assert not bad_c.any(), f"{label}: cost {cost[bad_c][:4]} vs {J_ora[bad_c][:4]}"

    err, bound = grad_errors(grad, g_ora)
    keep = margin > KINK_MARGIN
    bad_g = (err > bound) & keep
    if bad_g.any():
        p = int(np.argmax(np.where(keep, err / bound, 0)))
        d = np.abs(grad[p] - g_ora[p])
        c = int(np.argmax(d))
        raise AssertionError(f"{label}: gradient of particle {p}: err {err[p]:.3e} > {bound[p]:.3e} "
                             f"(worst component {c}: gpu {grad[p, c]!r} oracle {g_ora[p, c]!r}; margin {margin[p]:.2e}; "
                             f"{int(bad_g.sum())} bad of {int(keep.sum())})")

    ora_flags = problem.satisfied(torch.tensor(T_ora)).numpy()
    band = near_threshold(problem, T_ora)
    bad_f = (flags != ora_flags) & ~band
    assert not bad_f.any(), f"{label}: Eq. 3 flags differ for particles {np.nonzero(bad_f)[0][:8]}"
    return dict(n=len(X), kink_excluded=int((~keep).sum()), flag_band=int(band.sum()),
                satisfied=int(ora_flags.sum()), max_rel_grad=float(np.max(np.where(keep, err / bound, 0))) * GRAD_REL)
