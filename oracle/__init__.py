"""FP64 CPU oracle of the simwave finite-difference acoustic solver (arXiv 2201.05278).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py may import, call, link or run anything in this
package.  The product library (paper_2201_05278_b300) never imports it and
shares no code, header, table or constant generator with it.

Contents (paper section / equation):
  fd.py       FD weights from polynomial exactness (Eq. 9-10), stable dt (Eq. 8)
  source.py   Kaiser-windowed sinc source/receiver weights (Eq. 11-12)
  wavelet.py  Ricker wavelet (Sec. 2.4)
  damping.py  absorbing-layer profile eta = alpha d^p (Eq. 4)
  oracle.c    leapfrog loop of Eq. 7 with ghost nodes and face conditions
  solver.py   forward(): setup + call into oracle.c
  adjoint.py  exact discrete adjoint of the same recurrence and the misfit
              gradient w.r.t. velocity (beyond the paper: its FWI use)

Pins: every function is checked against something other than itself in
tests/test_oracle_*.py (closed forms, textbook values, the paper's printed
time-step counts, analytic Green's functions, convergence orders, exact
discrete eigenmodes, reciprocity, manufactured solutions).  Parity of the
variable-density term at boundaries depends on the reading that ln(rho) ghosts
mirror even; the manufactured-solution test pins its interior order.
"""
from .fd import critical_dt, first_derivative_weights, second_derivative_weights, stencil_abs_sum
from .source import KAISER_B, bessel_i0, kaiser_window, point_windows, sinc, weights_1d
from .wavelet import ricker, ricker_samples
from .damping import distance_to_interior, eta_field
from .solver import BC_DIRICHLET, BC_NEUMANN, BC_NONE, forward, run_raw

__all__ = [
    "critical_dt", "first_derivative_weights", "second_derivative_weights", "stencil_abs_sum",
    "KAISER_B", "bessel_i0", "kaiser_window", "point_windows", "sinc", "weights_1d",
    "ricker", "ricker_samples", "distance_to_interior", "eta_field",
    "BC_DIRICHLET", "BC_NEUMANN", "BC_NONE", "forward", "run_raw",
]
