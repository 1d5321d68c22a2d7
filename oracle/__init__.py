"""FP64 CPU oracle for the BART forward-model hot path (test infrastructure only).

This package is the slow, plain statement of what the GPU library computes.  It
exists to check the CUDA path and nothing else: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it.
It shares no code with the CUDA path (the seeded input generators in
``workloads`` hold none of the method's arithmetic) and never takes an input or
expected value from it.

Every function follows a passage of Harrington et al. (2022), "An Open-Source
Bayesian Atmospheric Radiative Transfer (BART) Code: I" (arXiv:2104.12522),
cited by section and equation.  Where the paper defers to its companion papers
(line strengths, widths, the emission and transit integrals, the T(P)
parameterisation), the oracle takes the reading stated in its docstring.

Pins (tests/test_oracle_*.py) tie each function to something other than itself:
closed forms, limits, invariants, brute-force quadrature, textbook constants
and values the paper prints (tests/golden/).  The steps between the grid and
the radiative transfer (temperature interpolation, abundances, mass opacity)
are pinned through the composed emission and transit paths
(tests/test_oracle_composed.py); the T(P) profile by the radiative-equilibrium
relations it solves.  The MLP is pinned by finite differences and closed
forms, the samplers by sampling known Gaussian targets and by their
stationary acceptance rates, App. C's content error by the retrieval table
of Sec. 6.3.
tests/oracle_mutation.py plants one mistake at a time in a copy of this
package and reports any that no pin notices.  Nothing here is "parity
unpinned".
"""
