"""Plain FP64 CPU oracle for the PFEM element operator and its solvers.

TEST INFRASTRUCTURE ONLY. tests/, __graft_entry__.smoke() and bench.py's CPU baseline /
reference arm may import it; nothing in the product package does. It shares no code with
the CUDA path: the only module both sides use is pfem_inputs (seeded input generation).

Modules:
  fem    element geometry, linear and Neo-Hookean constitutive laws, global assembly,
         external force, masked operator, energy.
  solve  Jacobi-PCG and Newton-Raphson with load steps, plus sparse direct solves.

Every function is pinned by tests/test_oracle_*.py against closed forms, invariants,
finite differences, manufactured solutions or library routines.
"""

from . import fem, solve  # noqa: F401
