"""FP64 CPU oracle for the particle-optimisation hot path (TEST INFRASTRUCTURE).

This package is the plain, slow, obviously-correct statement of what the CUDA path
computes, written from the paper (arXiv 2411.11833, Sec. V "Parallelized
Constraint Satisfaction", Eq. 1-5, the action definitions of Listing 1 and the
appendix's problem formulation, the example cost functions of the appendix
listing, the appendix's cost weights and tolerances) and from Kingma & Ba (Adam).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import it.  It shares no code with the CUDA path (``paper_2411_11833_b300``) and
never imports it; both take their inputs from ``scenegen``.

Modules:
  geometry  -- poses, DH forward kinematics, signed distances, the appendix's
               bound-distance / object-distance / pose-error costs
  problem   -- skeleton -> CSP (variables, constraints, costs), Eq. 2 / 3 / 5,
               gradients (reverse-mode autodiff of the plain definitions, as the
               paper does), Adam, the optimisation loop, kink margins
  philox    -- Philox4x32-10 counter-based generator and the uniform sampler
  mlp       -- the proposal network's forward/backward in FP64
"""
