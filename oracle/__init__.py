"""Plain FP64 CPU oracle of the leapfrog wave path and its derivatives.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline may import this package; the CUDA library and its binding never do,
and this package never imports them.  It is deliberately slow and obvious:
element-by-element FE assembly, one scipy sparse product per step, the
derivative recursions written out as derived from App. A of the paper.

Modules:
  fem   - P1 stiffness, lumped eps-mass, first-order absorbing-boundary matrix,
          CFL bound.
  wave  - forward traces, tangent (directional derivative), adjoint gradient,
          restriction to a coarse nested level.
  projected - the time inner products of Sec. II ("Projected data"), the
          projected data and the weights of its Jacobian transpose.
  inversion - the TV-regularised iteration, coarse-to-fine steps and
          compression of Sec. II, dense on tiny problems.
  approx_jacobian - the paper's approximate Jacobian (auxiliary sources,
          Green's functions by reciprocity, coarse-mass multigrid variant).
  mixed - the first-order leapfrog with element fluxes and the split-field
          perfectly matched layer of App. A.

Every function here is pinned by tests against facts that do not come from
the oracle itself (tests/test_oracle_pins.py): exact discrete energy balance,
the closed-form leapfrog evolution of a Dirichlet eigenmode, the straight-ray
travel time, complex-step and central finite differences, reciprocity, and
the source's mass balance.
"""
from . import approx_jacobian, fem, inversion, mixed, projected, wave  # noqa: F401
