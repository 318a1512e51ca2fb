"""CPU FP64 oracle for the space-time IgA monodomain / Rogers-McCulloch solver.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, independent
definition of what the CUDA path computes: it assembles the sparse space-time
matrices element by element with Gauss quadrature and solves them with a direct
sparse solver (Sec. 2-3 of the paper).  It shares no code with the CUDA path;
only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
it.

Pins (tests/test_oracle_*.py) tie it to what the paper and the mathematics fix:
partition of unity and linear precision of the B-splines, textbook 1D mass and
stiffness rows, the W_t + W_t^T identity, the Kronecker structure of A and
A-hat, the tau invariant, the w elimination, the rest state, the low-rank
tolerance, convergence rates against closed-form solutions and the spatially
uniform ODE limit.  Parity is unpinned for the full nonlinear Spline-Upwind
wave runs, which only the oracle itself defines.

`supg` holds the comparison method of Sec. 4.2 (C^0 time splines, SUPG and
shock capturing), pinned by exact reproduction of a solution in its discrete
space and by its convergence rate; its constants h/(2p+1) and c h^2/4 are
the paper's definitions and are parity unpinned.

For problems too large to assemble, `rows` evaluates selected rows of the
operators and of the load vector over the supports of their test functions.
That uses the same tables and Gauss rule as the assembly, and the rows equal
the assembled ones on small meshes (tests/test_oracle_rows.py).
"""

from .solve import Oracle  # noqa: F401
from .spacetime import SpaceTime  # noqa: F401
