"""Comparison rules of the CUDA path against the FP64 oracle.

Tolerances (FP32 kernel vs FP64 oracle):
  * term values: |gpu - ora| <= 1e-4 * max(|ora|, floor), floor 1e-2 (m or
    rad: an absolute 1e-6 near zero), except the terms computed from positions
    that FP32 forward kinematics carries through the whole chain -- the Kin pose
    errors, CFreeHold, CFreeTraj, SelfCollision -- floor 5e-2 (absolute 5e-6:
    0.1% of the 5 mm Kin tolerance, 0.5% of the 1 mm collision tolerance).
    Those positions hold a roughly constant absolute rounding of about 1e-6
    (a few ulps of a metre-scale chain), however small the error or the
    penetration they feed, and a collision sum adds one such rounding per
    active sphere pair (measured: 2.5e-6 on a CFreeHold sum of 0.0166 m,
    particles around the packing witness); every other term's rounding scales
    with its value.  Measured over the plain, packing, stress, stacking, knot,
    self-collision and 6-DOF workloads, away from satisfaction: the largest
    error is 0.22 of the 1e-2-floor bound (a collision sum, 3.2e-6 absolute at
    0.15 m), every other term kind at most 0.07 of it.
  * Eq. 2 totals: within the weighted sum of their terms' bounds (the per-term
    rule and the triangle inequality: cost_sum_bound), since near satisfaction
    several weighted Kin terms sit near zero at once (measured: 1.07e-6 at a
    total of 8e-3 with rotation errors of 5e-5 and 8e-4 rad, weight 5).
  * gradients, per particle: ||g_gpu - g_ora|| <= 1e-3 * max(||g_ora||, 1e-2),
    for particles whose kink margin (oracle ``kink_margin``) is above
    KINK_MARGIN; the others are counted and reported.
  * Eq. 3 flags: identical, except particles with some constraint within 1e-5
    of its tolerance, or, at a zero tolerance, with the quantity behind an
    exact zero within 1e-5 of switching on (near_threshold; counted).
  * multi-step trajectories: FP32 and FP64 iterates can part ways only where a
    particle comes within the FP32 rounding band of a point at which a cost's
    derivative jumps (a penetration switching on, a bound crossed, a norm at
    zero: the oracle's ``kink_margin``).  A particle whose margin stays above
    TRAJ_MARGIN at every iterate of the oracle's run must end within TRAJ_TOL
    of the oracle's iterate (measured: at most 5.4e-6 after 20 Adam steps,
    from FP32 rounding of x, about 1e-7 per step); the others are counted.
    The rule holds for batches away from satisfaction: a norm that passes
    near zero (a Kin error at a satisfying state) turns a difference d into a
    gradient direction change d/|e|, which the next step multiplies by about
    lr/|e|, so near-satisfying particles part ways even with margins well
    above TRAJ_MARGIN (1.4e-2 apart after 30 steps at margins of 1e-4); runs
    that follow such particles compare each check at the CUDA path's own
    iterates instead.
  * the gradient comparison must keep at least MIN_KEPT of a batch of 16 or more
    particles (a caller may lower it for scenes dense in contacts, with more
    particles), so that it never rests on a handful of them.
"""
from __future__ import annotations

import numpy as np
import torch

COST_REL, COST_FLOOR, FK_FLOOR = 1e-4, 1e-2, 5e-2
GRAD_REL, GRAD_FLOOR = 1e-3, 1e-2
# term kinds computed from forward-kinematics positions (oracle/problem.py):
# KIN_POS, KIN_ROT, CFREE_HOLD, CFREE_TRAJ, SELF_COLLISION
FK_KINDS = (0, 1, 4, 8, 10)
KINK_MARGIN = 1e-4
FLAG_BAND = 1e-5
MIN_KEPT = 0.6
TRAJ_MARGIN, TRAJ_TOL = 1e-6, 5e-5


def cost_ok(gpu: np.ndarray, ora: np.ndarray) -> np.ndarray:
    return np.abs(gpu - ora) <= COST_REL * np.maximum(np.abs(ora), COST_FLOOR)


def term_bounds(problem, terms_ora: np.ndarray) -> np.ndarray:
    """Per-term bounds [P, n_terms]: 1e-4 max(|T|, floor), the floor 5e-2 for
    the terms computed from forward-kinematics positions and 1e-2 for every
    other term (see the module notes)."""
    fk = np.array([t.kind in FK_KINDS for t in problem.terms])
    floor = np.where(fk, FK_FLOOR, COST_FLOOR)
    return COST_REL * np.maximum(np.abs(terms_ora), floor)


def cost_sum_bound(problem, terms_ora: np.ndarray) -> np.ndarray:
    """Bound on an Eq. 2 total that the per-term rule implies: the weighted sum
    of the terms' bounds (triangle inequality)."""
    w = problem.weights().numpy()
    return (w * term_bounds(problem, terms_ora)).sum(axis=1)


def grad_errors(gpu: np.ndarray, ora: np.ndarray):
    """Per-particle (error, bound) for [P, D] gradients."""
    err = np.linalg.norm(gpu - ora, axis=1)
    bound = GRAD_REL * np.maximum(np.linalg.norm(ora, axis=1), GRAD_FLOOR)
    return err, bound


def near_threshold(problem, terms_ora: np.ndarray, margin: np.ndarray | None = None) -> np.ndarray:
    """Particles whose Eq. 3 flag FP32 may decide differently from FP64: a
    constraint term within 1e-5 of a positive tolerance, or, for a zero
    tolerance (joint limits, self-collision), a term in (0, 1e-5].  A term that
    is exactly 0 at a zero tolerance is decided alike in both precisions unless
    the quantity behind it (a joint against its limit, a sphere pair's gap) is
    within 1e-5 of switching on: ``margin`` (the oracle's kink margin, which
    measures those distances among others), when given, marks such particles
    too.  (Counting every exact zero as near would mark every particle of
    every skeleton -- joint limits are 0 inside the limits -- and leave no
    flag to compare.)"""
    tol = problem.tolerances().numpy()
    cm = problem.constraint_mask().numpy()
    t, e = terms_ora[:, cm], tol[cm]
    pos = e > 0
    near = ((np.abs(t - e) <= FLAG_BAND) & pos).any(axis=1) | ((t > 0) & (t <= FLAG_BAND) & ~pos).any(axis=1)
    if margin is not None:
        near = near | (margin <= FLAG_BAND)
    return near


def compare_eval(problem, X: np.ndarray, cost, terms, flags, grad, label="", min_kept=MIN_KEPT):
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

    bad_t = np.abs(terms - T_ora) > term_bounds(problem, T_ora)
    if bad_t.any():
        p, t = np.argwhere(bad_t)[0]
        raise AssertionError(f"{label}: term {t} of particle {p}: gpu {terms[p, t]!r} oracle {T_ora[p, t]!r} "
                             f"({int(bad_t.sum())} bad of {bad_t.size})")
    bad_c = np.abs(cost - J_ora) > cost_sum_bound(problem, T_ora)
    assert not bad_c.any(), f"{label}: cost {cost[bad_c][:4]} vs {J_ora[bad_c][:4]}"

    err, bound = grad_errors(grad, g_ora)
    keep = margin > KINK_MARGIN
    if len(X) >= 16:
        assert keep.mean() >= min_kept, (f"{label}: the gradient comparison keeps only {int(keep.sum())} of "
                                         f"{len(X)} particles")
    bad_g = (err > bound) & keep
    if bad_g.any():
        p = int(np.argmax(np.where(keep, err / bound, 0)))
        d = np.abs(grad[p] - g_ora[p])
        c = int(np.argmax(d))
        raise AssertionError(f"{label}: gradient of particle {p}: err {err[p]:.3e} > {bound[p]:.3e} "
                             f"(worst component {c}: gpu {grad[p, c]!r} oracle {g_ora[p, c]!r}; margin {margin[p]:.2e}; "
                             f"{int(bad_g.sum())} bad of {int(keep.sum())})")

    ora_flags = problem.satisfied(torch.tensor(T_ora)).numpy()
    band = near_threshold(problem, T_ora, margin)
    bad_f = (flags != ora_flags) & ~band
    assert not bad_f.any(), f"{label}: Eq. 3 flags differ for particles {np.nonzero(bad_f)[0][:8]}"
    return dict(n=len(X), kept=int(keep.sum()), kink_excluded=int((~keep).sum()), flag_band=int(band.sum()),
                satisfied=int(ora_flags.sum()), max_rel_grad=float(np.max(np.where(keep, err / bound, 0))) * GRAD_REL)


def oracle_run(problem, X: np.ndarray, n_steps: int):
    """The oracle's n-step run (Problem.optimize from zero moments) and, per
    particle, the smallest kink margin met at its iterates x_0 .. x_n."""
    out = problem.optimize(torch.tensor(X), n_steps)
    x = torch.tensor(X)
    m, v = torch.zeros_like(x), torch.zeros_like(x)
    margin = problem.kink_margin(x).numpy()
    for t in range(n_steps):
        _, g = problem.gradient(x)
        x, m, v = problem.adam_step(x, m, v, t + 1, g, x.shape[0])
        margin = np.minimum(margin, problem.kink_margin(x).numpy())
    assert torch.equal(x, out["x"])            # the same steps as Problem.optimize
    return out, margin


def check_trajectory(problem, x_gpu: np.ndarray, cost_gpu: np.ndarray, out, margin, min_smooth=0.5):
    """x_gpu [P, D] and cost_gpu [P] after the run against oracle_run's result."""
    smooth = margin > TRAJ_MARGIN
    d = np.abs(x_gpu - out["x"].numpy()).max(axis=1)
    assert smooth.mean() >= min_smooth, f"only {int(smooth.sum())} of {len(smooth)} trajectories stay off kinks"
    bad = smooth & (d > TRAJ_TOL)
    assert not bad.any(), f"{int(bad.sum())} smooth trajectories left the oracle's (worst {d[smooth].max():.2e})"
    assert cost_ok(cost_gpu.astype(np.float64), out["cost"].numpy())[smooth].all()
    return dict(smooth=int(smooth.sum()), of=len(smooth), worst=float(d[smooth].max()) if smooth.any() else 0.0,
                parted=int((d > TRAJ_TOL).sum()))


def check_adam_step(problem, X, m0, v0, t0: int, x1, m1, n_batch: int, keep):
    """One fused Adam step from (X, m0, v0) at step count t0 (all [P, D],
    FP32-representable) against the oracle's.  The kernel's gradient is read
    back from the first moment (m1 = b1 m0 + (1 - b1) g / N_b) and must match
    the oracle's per particle; each component's step must match within what
    that gradient bound implies for it: a gradient error dg moves the step by
    lr (1 - b1) dg / N_b / (1 - b1^t) / (sqrt(v_hat) + eps), plus the FP32
    rounding of x (the step is read as x1 - x0).  Particles near a kink
    (keep False) are left out.  Returns the largest error/bound ratios."""
    Xt = torch.tensor(X)
    _, g = problem.gradient(Xt)
    g = g.numpy()
    o = problem.opts
    b1, t = o.beta1, t0 + 1
    gsc = n_batch if o.scale_by_batch else 1.0
    g_gpu = (m1.astype(np.float64) - b1 * m0) / (1.0 - b1) * gsc
    err, bound = grad_errors(g_gpu, g)
    # m1 is FP32: its rounding, scaled back to a gradient, widens the bound
    bound = bound + 2.0 ** -23 * (np.abs(m1) + b1 * np.abs(m0)).max(axis=1) / (1.0 - b1) * gsc * np.sqrt(X.shape[1])
    assert (err <= bound)[keep].all(), f"gradient err {np.max(err[keep] / bound[keep]):.2f} x its bound"
    xr, mr, vr = problem.adam_step(Xt, torch.tensor(m0), torch.tensor(v0), t, torch.tensor(g), n_batch)
    lr = problem.learning_rates().numpy()
    vhat = vr.numpy() / (1.0 - o.beta2 ** t)
    dstep = lr * (1.0 - b1) * bound[:, None] / gsc / (1.0 - b1 ** t) / (np.sqrt(vhat) + o.eps)
    step_r = xr.numpy() - X
    lim = 2.0 * dstep + 1e-4 * np.abs(step_r) + 4.0 * 2.0 ** -24 * np.maximum(np.abs(X), 1.0)
    dx = np.abs((x1.astype(np.float64) - X) - step_r)
    assert (dx <= lim)[keep].all(), f"step err {np.max((dx / lim)[keep]):.2f} x its bound"
    return dict(grad=float(np.max(err[keep] / bound[keep])), step=float(np.max((dx / lim)[keep])))
