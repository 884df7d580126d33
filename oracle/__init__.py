"""CPU FP64 oracle for the N-1 contingency screen (test infrastructure).

This package is the slow, plainly written reference that the CUDA path is
checked against.  It is test infrastructure only: the test-suite, the smoke
check and the CPU-baseline leg of the benchmark may import it; the library
itself never does, and it shares no code with the library.

What it computes, and where the paper defines it:

* ``powerflow``  -- the bus power mismatch of eqs. (1)-(3) (Sec. II.C), the
  fast-decoupled matrices B' and B'' of eqs. (4)-(5) (Sec. III.B), branch
  flows, and the fast-decoupled power flow itself.  Every linear system is
  solved *directly*: each contingency matrix is re-formed and fully
  factorised, the "LUD" method the paper compares against (Sec. I, Sec. V,
  Table I).  The fixed point is the exact AC power-flow solution of the
  post-outage, re-dispatched network, which is also the fixed point of the
  preconditioned iteration.
* ``islands``    -- islanding detection by graph traversal (Sec. IV.C).
* ``redispatch`` -- proportional re-dispatch of an island's net injection
  over the main island's generators (Sec. IV.C).
* ``factor``     -- incomplete Cholesky on a given sparsity pattern (the
  base-case preconditioner of Sec. IV.B, eq. (6)) and the triangular solves
  that apply it.
* ``screen``     -- the N-1 loop over all single-branch outages (Sec. IV.A),
  run across host processes.
* ``adjoint``    -- loss and gradients of a smooth overload penalty summed
  over N-1 scenarios of the P-theta (DC) model, by one adjoint solve per
  scenario; pinned by finite differences.
* ``dc``         -- the N-1 quick screen of the P-theta equation alone (DC
  model, Sec. IV.A), re-formed and solved directly per scenario; pinned by
  radial closed forms and line-outage distribution factors.

Parity status of each function is stated in its docstring; the one function
the paper gives no formula for (the re-dispatch weights) says
"parity unpinned".
"""
from . import adjoint, dc, factor, islands, powerflow, redispatch, screen  # noqa: F401
from .powerflow import (STATUS_DIVERGED, STATUS_ISLAND_NO_GEN, STATUS_MAXITER,
                        STATUS_OK)

__all__ = ["adjoint", "dc", "factor", "islands", "powerflow", "redispatch", "screen",
           "STATUS_OK", "STATUS_MAXITER", "STATUS_DIVERGED",
           "STATUS_ISLAND_NO_GEN"]
