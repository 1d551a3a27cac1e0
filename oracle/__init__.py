"""Plain FP64 CPU oracle for HOTRG on the 2D generalized XY model (q = 2).

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
restatement of the method that the CUDA library is checked against.  Only the
test suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
leg of ``bench.py`` may import it.  The product path (the C-ABI library and its
Python binding) never imports, calls or links anything here, and this package
never imports the product package: the two share no code.

Contents (each function cites the passage of the thesis it follows):
  bessel      own modified Bessel I_n(x) by its power series (§3.2, §3.3)
  gxy         Fourier coefficients a_n (Eq. 3.4), site tensor (Eq. 3.6 / 3.15),
              impurity tensors (Eq. 3.20, 3.21), the 2D Ising tensor (pin only)
  hotrg       one HOTRG step (§2.4.1: Eq. 2.11, 2.12, the eps_1/eps_2 rule,
              Eq. 2.15, 2.16) and the full run with ln Z / N accumulation
  exact       brute-force small lattices, direct numerical integration,
              Onsager's closed form, the high-temperature series (pins)
  observables f, C_V (Eq. 3.17), m and m1 via impurity tensors (Eq. 3.19-3.21),
              chi by finite differences (Eq. 3.18)

Parity status: every function has a pin in ``tests/test_oracle_*.py`` except
the susceptibility field values (h-bar, delta), which the thesis does not
print; the finite-difference formula itself is pinned by a second route
(derivative of ln Z), but the specific field values are "parity unpinned".
"""

from .bessel import bessel_i  # noqa: F401
from .gxy import (  # noqa: F401
    fourier_coefficients,
    field_factor,
    site_tensor,
    ising_tensor,
    leg_charges,
)
from .hotrg import hotrg_step, hotrg_run, StepRecord, RunResult  # noqa: F401
