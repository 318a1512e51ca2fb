"""Parity at the 2D workload's full size: p = 3, 128 x 128 spatial x 256 time
elements, 4.43 M unknowns, the benchmark's problem and launch configuration.

The oracle cannot assemble this system, so it computes sampled rows one by
one, integrating over the support of each test function (oracle/rows.py).
The rows are at the corners of space-time, inside the stimulus at t = 0, and
at random.  Checked on them:
  * the load vector f (1e-12 relative);
  * the FP64 and FP32 operators at a seeded linearization (1e-12 / 2e-5);
  * the FP64 preconditioner, through the residual A-hat z - r (1e-9);
  * the mixed-precision solve, through the residual f - A x.  Every row of it
    is bounded by the residual norm, which the solve brings below
    1e-8 ||f||.
The operator is the Galerkin one.  The SU term needs Theta-hat from maxima
over all Gauss points and a global SVD, which the oracle cannot form at this
size; it is checked on the smaller meshes of test_gpu_parity.py.  With or
without it, the same kernels run at the same launch shapes: the SU term only
changes the values of the time bands.
"""

import numpy as np
import pytest

import workloads as W
from oracle.spacetime import SpaceTime
from tests import sampled_rows as SR
from tests.gpu_helpers import dev, empty, host, library, ptr, stream, torch_cuda

pytestmark = pytest.mark.gpu


def test_full_size_sampled_rows():
    torch_cuda()
    P = library()
    desc = W.config("c2_aniso_2d")
    desc.update(stabilization="galerkin", precision="mixed")
    st = SpaceTime(desc)
    n = st.N_dof
    rows = SR.sample_rows(st, desc, seed=5)
    inp = SR.linearization_inputs(n)
    s = P.Solver(desc, stream())
    assert s.dims["N_dof"] == n
    f = empty(n)
    s.rhs(ptr(f))
    fh = host(f)
    f_rows = SR.check_rhs(st, desc, rows, fh)
    du, dw = dev(inp["u"]), dev(inp["w"])
    s.ionic(ptr(du), ptr(dw))
    dx, dy = dev(inp["x"]), empty(n)
    s.apply(ptr(dx), ptr(dy), P.ST_FP64)
    SR.check_apply(st, desc, rows, inp, host(dy), 1e-12)
    dx32, dy32 = dev(inp["x"], np.float32), empty(n, "float32")
    s.apply(ptr(dx32), ptr(dy32), P.ST_MIXED)
    SR.check_apply(st, desc, rows, inp, host(dy32), 2e-5)
    dr, dz = dev(inp["r"]), empty(n)
    s.precond(ptr(dr), ptr(dz), P.ST_FP64)
    SR.check_precond(st, desc, rows, inp, host(dz), 1e-9)
    dsol = empty(n)
    out = s.linsolve(ptr(f), ptr(dsol))
    assert out["rel_res"] <= 1e-8
    SR.check_solution(st, desc, rows, inp, f_rows, np.linalg.norm(fh), host(dsol), 1e-8)
    s.close()


def test_newton_workload_full_size():
    """The Newton workload at its full size (2D, p = 2, 16 x 16 x 32 elements,
    10,692 unknowns, FP64): three nonlinear steps from u = w = 0 on both sides,
    against the oracle's assembled solves.  The SU ranks of the three steps
    are 1, 1 and 2; the oracle's tails at the cut are 0.03 to 0.12 and 1.26
    to 100 of the tolerance, far from a tie."""
    torch_cuda()
    from oracle import Oracle
    P = library()
    desc = W.config("c1_newton_2d")
    desc.update(max_fp=3, delta=0.0, rtol=1e-13, gmres_m=80)
    o = Oracle(desc)
    u_ref, w_ref, hist = o.solve(max_fp=3)
    s = P.Solver(desc, stream())
    u, w = empty(o.st.N_dof), empty(o.st.N_dof)
    st = s.solve(ptr(u), ptr(w), allow_unconverged=True)
    assert st["fp_iters"] == 3
    assert st["rank"] == hist[-1]["rank"]
    for got, ref in ((host(u), u_ref), (host(w), w_ref)):
        assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()
    s.close()
