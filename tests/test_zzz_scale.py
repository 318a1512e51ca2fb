"""GPU tests at wide and full sizes (this module runs after the others).

* Wide x axes, for which the fused x pass needs more than 48 KB of dynamic
  shared memory: every instance of that kernel must have its own opt-in,
  whatever order the instances first run in.
* The workloads at their full sizes: the 2D problem of the benchmark (p = 3,
  128 x 128 x 256 elements, 4.43 M unknowns), the Newton problem (10,692
  unknowns), and the 3D problem (p = 2, 64^3 x 128 elements, 37.1 M unknowns,
  105 GB on the device).  The oracle cannot assemble the large ones. For them
  it computes sampled rows one by one, integrating over the support of each
  test function (oracle/rows.py); the rows are at the corners of space-time,
  inside the stimulus at t = 0, and at random.  Checked on them:
    - the load vector f (1e-12 relative);
    - the FP64 and FP32 operators at a seeded linearization (1e-12 / 2e-5);
    - the FP64 preconditioner, through the residual A-hat z - r (5e-8 of
      max |r|, which the 1e-10 forward tolerance of the small meshes implies);
    - the mixed-precision solve, through the residual f - A x.  Every row of it
      is bounded by the residual norm, which the solve brings below
      1e-8 ||f||.
  These checks use the Galerkin operator.
* The largest workload (3D, p = 3, 96^3 x 192 elements), in the lean form:
  f, both operators and the preconditioner on sampled rows.
* Both operator forms (time bands stored per Gauss point, or the lean form)
  on the 2D and 3D problems.
* The 2D problem again with its SU term, at a smooth seeded linearization (an
  excitation front, workloads.wave_fields): the oracle evaluates the residual
  one time element at a time (oracle/streamed.py) and forms Theta-hat, its
  maxima and denominator, and the truncated SVD of Eq. (tol) at full size.
  Checked: the maxima and denominator, every entry of Theta-hat, the rank and
  the singular values, and sampled rows of both operators with the low-rank
  SU term.
"""

import numpy as np
import pytest

import workloads as W
from oracle import Oracle
from oracle.spacetime import SpaceTime
from oracle import rows as OR
from oracle import streamed as S
from oracle.stabilization import low_rank, tau_solve
from tests import sampled_rows as SR
from tests.gpu_helpers import dev, empty, host, library, ptr, rel, stream, torch_cuda

pytestmark = pytest.mark.gpu


def small_problem(c):
    desc = W.base_desc(d=c["d"], p=c["p"], n_el=c["n_el"], n_el_t=c["n_el_t"], T=8.0, C_m=1.0,
                       D=[2e-2, 1e-2, 5e-3][:c["d"]],
                       source=dict(kind="stim", boxes=[W.stim_box([0.0] * c["d"], [0.35] * c["d"], 0.0, 1.5, 1.0)]))
    desc.update(W.DIMENSIONAL_RM)
    return desc


def test_apply_wide_x_every_fused_instance():
    """p = 3 (band slices by bulk copy), then p = 2 with Q_x a multiple of 4
    (bulk copy) and not (plain loads), in one process; the operators against
    the oracle as in test_gpu_parity.py."""
    torch_cuda()
    P = library()
    for c in (dict(d=2, p=3, n_el=[120, 2], n_el_t=3), dict(d=2, p=2, n_el=[196, 2], n_el_t=3),
              dict(d=2, p=2, n_el=[194, 2], n_el_t=3)):
        desc = small_problem(c)
        o = Oracle(desc)
        u, w, hist = o.solve(max_fp=2, record=True)
        u, w = hist[-1]["u"], hist[-1]["w"]
        A, _ = o.linearization(u, w, "picard")
        s = P.Solver(desc, stream())
        du, dw = dev(u), dev(w)
        s.ionic(ptr(du), ptr(dw))
        x = W.random_vector(o.st.N_dof, seed=5)
        dx, dy = dev(x), empty(o.st.N_dof)
        s.apply(ptr(dx), ptr(dy), P.ST_FP64)
        assert rel(host(dy), A @ x) < 1e-12, c
        dx32, dy32 = dev(x, np.float32), empty(o.st.N_dof, "float32")
        s.apply(ptr(dx32), ptr(dy32), P.ST_MIXED)
        assert rel(host(dy32), A @ x) < 2e-5, c
        s.close()


def test_wide_x_solves_in_one_process():
    """Solves in the order that a serving stream met them: a p = 3 request
    first, then p = 2 requests whose fused x pass of the FP64 operator needs
    more than 48 KB of shared memory (224 threads, Q_x not a multiple of 4 and
    a multiple of 4).  With one opt-in per element type the p = 2 solves
    failed with a CUDA error.  One fixed-point step each, small in y and time."""
    P = library()
    torch_cuda()
    base = W.serving_requests(n_req=1, seed=21)[0]["desc"]
    for p, nx in ((3, 120), (2, 194), (2, 216)):
        desc = dict(base, p=p, n_el=[nx, 8], n_el_t=8, max_fp=1, gmres_m=60)
        n = W.n_dofs(desc)
        s = P.Solver(desc, stream())
        u, w = empty(n), empty(n)
        st = s.solve(ptr(u), ptr(w), allow_unconverged=True)
        assert st["fp_iters"] == 1, (p, nx)
        assert np.all(np.isfinite(host(u))) and np.abs(host(u)).max() > 0.0, (p, nx)
        s.close()


def test_newton_workload_full_size():
    """The Newton workload at its full size (2D, p = 2, 16 x 16 x 32 elements,
    10,692 unknowns, FP64): three nonlinear steps from u = w = 0 on both sides,
    against the oracle's assembled solves.  The SU ranks of the three steps
    are 1, 1 and 2; the oracle's tails at the cut are 0.03 to 0.12 and 1.26
    to 100 of the tolerance, far from a tie."""
    torch_cuda()
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
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
    s.close()


def sampled_rows_at_full_size(name, form="auto", solve=True, **over):
    torch = torch_cuda()
    P = library()
    desc = W.config(name)
    desc.update(stabilization="galerkin", precision="mixed", operator_form=form, **over)
    torch.cuda.empty_cache()
    free, _total = torch.cuda.mem_get_info()
    need = P.footprint(desc) + 8 * 8 * W.n_dofs(desc)   # the handle and the test's own vectors
    if free < need:
        pytest.skip(f"{name} needs {need / 1e9:.0f} GB of device memory, {free / 1e9:.0f} GB free")
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
    del dy
    dx32, dy32 = dev(inp["x"], np.float32), empty(n, "float32")
    s.apply(ptr(dx32), ptr(dy32), P.ST_MIXED)
    SR.check_apply(st, desc, rows, inp, host(dy32), 2e-5)
    del dx, dx32, dy32
    dr, dz = dev(inp["r"]), empty(n)
    s.precond(ptr(dr), ptr(dz), P.ST_FP64)
    SR.check_precond(st, desc, rows, inp, host(dz), SR.PRECOND_RESIDUAL_TOL)
    del dr, dz
    if not solve:
        s.close()
        return
    dsol = empty(n)
    out = s.linsolve(ptr(f), ptr(dsol))
    assert out["rel_res"] <= 1e-8
    SR.check_solution(st, desc, rows, inp, f_rows, np.linalg.norm(fh), host(dsol), 1e-8)
    s.close()


@pytest.mark.parametrize("form", ["bands", "lean"])
def test_2d_workload_full_size_sampled_rows(form):
    sampled_rows_at_full_size("c2_aniso_2d", form)


@pytest.mark.parametrize("form", ["bands", "lean"])
def test_3d_workload_full_size_sampled_rows(form):
    sampled_rows_at_full_size("c3_cube_3d", form)


def test_c5_workload_full_size_sampled_rows():
    """The largest workload (3D, p = 3, 96^3 x 192 elements, 188 M unknowns),
    which only the lean form fits on one GB300: f, both operators and the
    preconditioner on sampled rows (the solve is timed by the benchmark)."""
    sampled_rows_at_full_size("c5_cube_3d", "lean", solve=False, gmres_m=40)


def test_2d_workload_full_size_su():
    torch = torch_cuda()
    P = library()
    desc = W.config("c2_aniso_2d")
    desc.update(precision="mixed")
    torch.cuda.empty_cache()
    free, _total = torch.cuda.mem_get_info()
    need = P.footprint(desc) + 8 * 8 * W.n_dofs(desc)
    if free < need:
        pytest.skip(f"needs {need / 1e9:.0f} GB of device memory, {free / 1e9:.0f} GB free")
    st = SpaceTime(desc)
    n = st.N_dof
    u, w = W.wave_fields(desc)
    th, info = S.theta_hat(st, desc, u, w, desc["suppext"])
    eps = desc["eps_theta"]
    U, sv, V = low_rank(th, eps)
    R = len(sv)
    # no tie at the cut: the tails around it stay clear of eps ||Theta||_F
    allsv = np.linalg.svd(th, compute_uv=False)
    fro = np.sqrt(np.sum(allsv ** 2))
    tail = np.sqrt(np.concatenate([np.cumsum((allsv ** 2)[::-1])[::-1], [0.0]]))
    assert R >= 2 and tail[R - 1] > (1 + 1e-4) * eps * fro and tail[R] < (1 - 1e-4) * eps * fro
    rows = SR.sample_rows(st, desc, seed=5)
    _, tau_q = tau_solve(st)
    terms = OR.picard_galerkin_terms(st, desc, u, w) + S.su_terms(st, desc, tau_q, U, sv, V)
    x = W.random_vector(n, seed=13)
    ref = OR.apply_rows(st, terms, rows, x)
    for form in ("bands", "lean"):
        s = P.Solver(dict(desc, operator_form=form), stream())
        du, dw = dev(u), dev(w)
        g = s.ionic(ptr(du), ptr(dw))
        for key in ("u_max", "ut_max", "r_max", "den"):
            assert abs(g[key] - info[key]) <= 1e-12 * info[key], (form, key, g[key], info[key])
        assert g["rank"] == R
        thg = np.array(s.get("theta_hat", n)).reshape(st.N_t, st.N_s)
        assert np.abs(thg - th).max() <= 1e-12
        assert rel(np.array(s.get("lowrank_s", R)), sv) <= 1e-10
        dx, dy = dev(x), empty(n)
        s.apply(ptr(dx), ptr(dy), P.ST_FP64)
        y = host(dy)
        assert np.abs(y[rows] - ref).max() <= 1e-12 * np.abs(y).max(), form
        dx32, dy32 = dev(x, np.float32), empty(n, "float32")
        s.apply(ptr(dx32), ptr(dy32), P.ST_MIXED)
        y32 = host(dy32)
        assert np.abs(y32[rows] - ref).max() <= 2e-5 * np.abs(y32).max(), form
        s.close()
        del du, dw, dx, dy, dx32, dy32
