"""FP64 CPU oracle of the PNCG-IPC gel-pad frame solve (test infrastructure).

This package is the plain, slow, obviously-correct reference that the CUDA
library is checked against. It is test infrastructure only: the tests, the
smoke check and the benchmark's CPU-baseline leg may import it; the product
library never does, and the two share no code.

Everything is numpy float64, vectorised over elements / pairs only (each
element's arithmetic is the textbook definition). Second directional
derivatives along a line (the p^T H p of the step-size rule and the
Newton check) are taken with the truncated Taylor arithmetic of
``oracle.taylor``, so they do not depend on any hand-derived Hessian formula.

Modules
  geometry   -- rest shape (Dm^-1, volume), lumped mass, surface primitives,
                marker mappings (barycentric, kNN-IDW), indenter placement
  taylor     -- second-order forward-mode arithmetic (value, d/dt, d2/dt2)
  energy     -- the incremental potential of Eq. (ipc_energy): inertia,
                Neo-Hookean elasticity, log-barrier over PT / EE pairs,
                lagged friction with the mollifier of Eq. (friction_mollifier)
  broadphase -- the candidate-pair set (inflated-AABB predicate) and a
                brute-force exact-distance pair set
  solver     -- the per-frame PNCG iteration of Eq. (dk_direction) and
                Eq. (step_size), indenter advance, markers, Newton check
  adjoint    -- implicit-function gradient of a marker loss

Parity status: every function is pinned by tests under ``tests/`` (closed
forms, finite differences, brute force, invariants) except the numerical
conventions the paper does not fix (barrier stiffness, friction epsilon,
stopping rule, indenter advance schedule), which are shared conventions and
are "parity unpinned" against the paper itself.
"""
