"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Every test builds the same problem on both sides from the same seeded inputs
(workloads) and compares element by element.  Tolerances: 1e-10 relative for
FP64 results; FP32 results within a bound derived from single precision;
mixed-precision solves within 1e-8 relative residual measured by the oracle.
"""

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import workloads as W
from oracle import Oracle
from tests.gpu_helpers import library, dev, empty, host, ptr, stream, rel

pytestmark = pytest.mark.gpu

CASES = [
    dict(d=1, p=2, n_el=[7], n_el_t=9),
    dict(d=1, p=3, n_el=[5], n_el_t=6),
    dict(d=2, p=2, n_el=[5, 4], n_el_t=6),
    dict(d=2, p=3, n_el=[4, 5], n_el_t=5),
    dict(d=3, p=2, n_el=[3, 4, 3], n_el_t=4),
    dict(d=2, p=1, n_el=[6, 5], n_el_t=7),
    dict(d=1, p=4, n_el=[6], n_el_t=7),
]
IDS = [f"d{c['d']}p{c['p']}" for c in CASES]


def problem(c, **over):
    desc = W.base_desc(d=c["d"], p=c["p"], n_el=c["n_el"], n_el_t=c["n_el_t"], T=8.0, C_m=1.0,
                       D=[2e-2, 1e-2, 5e-3][:c["d"]],
                       source=dict(kind="stim", boxes=[W.stim_box([0.0] * c["d"], [0.35] * c["d"], 0.0, 1.5, 1.0)]))
    desc.update(W.DIMENSIONAL_RM)
    desc.update(over)
    return desc


def band_of(Mdense, p):
    n = Mdense.shape[0]
    out = np.zeros((n, 2 * p + 1))
    for i in range(n):
        for k in range(2 * p + 1):
            j = i - p + k
            if 0 <= j < n:
                out[i, k] = Mdense[i, j]
    return out


@pytest.fixture(scope="module")
def P():
    return library()


def solver(P, desc):
    return P.Solver(desc, stream())


def iterate(o, k):
    """(u^k, w^k) of the oracle's own nonlinear loop (inputs for the linearization tests)."""
    u, w, hist = o.solve(max_fp=k, record=True)
    return hist[-1]["u"], hist[-1]["w"]


@pytest.mark.parametrize("c", CASES, ids=IDS)
def test_setup_1d_data(P, c):
    desc = problem(c)
    o = Oracle(desc)
    s = solver(P, desc)
    st = o.st
    p = c["p"]
    m = st.matrices_1d()
    nb = sum(2 * st.n[l] for l in range(c["d"])) + 2 * st.N_t
    got = np.array(s.get("bands_1d", nb * (2 * p + 1)))
    exp = []
    for l in range(c["d"]):
        exp.append(band_of(m[f"M{l}"], p).ravel())
        exp.append(band_of(m[f"K{l}"], p).ravel())
    exp.append(band_of(m["Mt"], p).ravel())
    exp.append(band_of(m["Wt"], p).ravel())
    exp = np.concatenate(exp)
    assert rel(got, exp) < 1e-13
    tau = np.array(s.get("tau_q", p * st.n_el_t * (p + 1)))
    exp_tau = np.concatenate([t.ravel() for t in o.tau_q])
    assert np.abs(tau - exp_tau).max() <= 1e-11 * max(1.0, np.abs(exp_tau).max())
    # generalized eigenvalues of (D_ll K_l, M_l)
    lam = np.array(s.get("fd_eig", sum(st.n)))
    off = 0
    for l in range(c["d"]):
        ref = sla.eigh(desc["D"][l] * m[f"K{l}"], m[f"M{l}"], eigvals_only=True)
        got_l = np.sort(lam[off:off + st.n[l]])
        assert np.abs(got_l - ref).max() <= 1e-12 * np.abs(ref).max()
        off += st.n[l]
    s.close()


@pytest.mark.parametrize("c", CASES, ids=IDS)
def test_rhs(P, c):
    desc = problem(c)
    o = Oracle(desc)
    s = solver(P, desc)
    f = empty(o.st.N_dof)
    s.rhs(ptr(f))
    assert rel(host(f), o.F) < 1e-13
    s.close()


# (case, operator form): the band form everywhere, the lean form where it applies (d >= 2)
FORM_CASES = [(c, f) for c in CASES for f in ("bands", "lean") if f == "bands" or c["d"] >= 2]
FORM_IDS = [f"d{c['d']}p{c['p']}-{f}" for c, f in FORM_CASES]


@pytest.mark.parametrize("c,form", FORM_CASES, ids=FORM_IDS)
@pytest.mark.parametrize("kind", ["picard", "newton"])
def test_linearization_and_apply(P, c, form, kind):
    desc = problem(c, nonlinear=kind, operator_form=form)
    o = Oracle(desc)
    u, w = iterate(o, 2)
    A, info = o.linearization(u, w, kind)
    s = solver(P, desc)
    du, dw = dev(u), dev(w)
    ginfo = s.ionic(ptr(du), ptr(dw))
    # Theta-hat and the low-rank step
    th = np.array(s.get("theta_hat", o.st.N_dof)).reshape(o.st.N_t, o.st.N_s)
    assert np.abs(th - info["theta_hat"]).max() < 1e-12
    assert ginfo["rank"] == len(info["s"])
    assert abs(ginfo["den"] - info["den"]) <= 1e-12 * info["den"]
    # FP64 operator
    x = W.random_vector(o.st.N_dof, seed=5)
    dx, dy = dev(x), empty(o.st.N_dof)
    s.apply(ptr(dx), ptr(dy), P.ST_FP64)
    ref = A @ x
    assert rel(host(dy), ref) < 1e-12
    # FP32 operator
    dx32, dy32 = dev(x, np.float32), empty(o.st.N_dof, "float32")
    s.apply(ptr(dx32), ptr(dy32), P.ST_MIXED)
    assert rel(host(dy32), ref) < 2e-5
    s.close()


# x extents that put the last element of the lean kernel's row in lanes
# 0 .. p-2 of a warp (33, 34 with p = 3) or last in a warp (64 with p = 2)
TAIL_CASES = [dict(d=2, p=3, n_el=[33, 2], n_el_t=4), dict(d=2, p=3, n_el=[34, 2], n_el_t=4),
              dict(d=2, p=2, n_el=[64, 2], n_el_t=4)]


@pytest.mark.parametrize("c", TAIL_CASES, ids=[f"p{c['p']}-nx{c['n_el'][0]}" for c in TAIL_CASES])
def test_lean_trailing_coefficients(P, c):
    """The lean form gives each x element one thread, and the thread of the
    last element also writes the p coefficients after it, taking the
    contributions of the elements before it from the previous warp's exchange
    slots when they sit there: both operators against the assembled matrix."""
    desc = problem(c, operator_form="lean")
    o = Oracle(desc)
    u, w = iterate(o, 2)
    A, info = o.linearization(u, w, "picard")
    s = solver(P, desc)
    du, dw = dev(u), dev(w)
    ginfo = s.ionic(ptr(du), ptr(dw))
    assert ginfo["rank"] == len(info["s"])
    x = W.random_vector(o.st.N_dof, seed=5)
    ref = A @ x
    dx, dy = dev(x), empty(o.st.N_dof)
    s.apply(ptr(dx), ptr(dy), P.ST_FP64)
    assert rel(host(dy), ref) < 1e-12
    dx32, dy32 = dev(x, np.float32), empty(o.st.N_dof, "float32")
    s.apply(ptr(dx32), ptr(dy32), P.ST_MIXED)
    assert rel(host(dy32), ref) < 2e-5
    s.close()


@pytest.mark.parametrize("form", ["bands", "lean"])
def test_lowrank_long_time(P, form):
    """A Gram matrix larger than one batch of Lanczos steps (N_t = 61 against
    24), so the leading Ritz pairs must pass the residual test before the rank
    is taken: rank, Theta-hat and the FP64 operator as in the cases above."""
    c = dict(d=2, p=2, n_el=[8, 8], n_el_t=60)
    desc = problem(c, operator_form=form)
    o = Oracle(desc)
    u, w = iterate(o, 2)
    A, info = o.linearization(u, w, "picard")
    s = solver(P, desc)
    du, dw = dev(u), dev(w)
    ginfo = s.ionic(ptr(du), ptr(dw))
    assert ginfo["rank"] == len(info["s"]) and ginfo["rank"] >= 1
    x = W.random_vector(o.st.N_dof, seed=5)
    dx, dy = dev(x), empty(o.st.N_dof)
    s.apply(ptr(dx), ptr(dy), P.ST_FP64)
    assert rel(host(dy), A @ x) < 1e-12
    s.close()


@pytest.mark.parametrize("form", ["bands", "lean"])
@pytest.mark.parametrize("kind", ["picard", "newton"])
def test_apply_tiny_mesh(P, form, kind):
    """A 2D mesh of 1 x 2 elements with p = 1 (6 coefficients per time slice, 3
    time functions): one 32-column strip far wider than the plane, time bands
    cut at both ends.  FP64 and FP32 operator as in the cases above."""
    c = dict(d=2, p=1, n_el=[1, 2], n_el_t=3)
    desc = problem(c, nonlinear=kind, operator_form=form)
    o = Oracle(desc)
    u, w = iterate(o, 2)
    A, _ = o.linearization(u, w, kind)
    s = solver(P, desc)
    du, dw = dev(u), dev(w)
    s.ionic(ptr(du), ptr(dw))
    x = W.random_vector(o.st.N_dof, seed=5)
    dx, dy = dev(x), empty(o.st.N_dof)
    s.apply(ptr(dx), ptr(dy), P.ST_FP64)
    assert rel(host(dy), A @ x) < 1e-12
    dx32, dy32 = dev(x, np.float32), empty(o.st.N_dof, "float32")
    s.apply(ptr(dx32), ptr(dy32), P.ST_MIXED)
    assert rel(host(dy32), A @ x) < 2e-5
    s.close()


@pytest.mark.parametrize("c", CASES, ids=IDS)
def test_precond(P, c):
    desc = problem(c)
    o = Oracle(desc)
    Ah = o.precond_matrix().tocsc()
    s = solver(P, desc)
    r = W.random_vector(o.st.N_dof, seed=9)
    ref = spla.spsolve(Ah, r)
    dr, dz = dev(r), empty(o.st.N_dof)
    s.precond(ptr(dr), ptr(dz), P.ST_FP64)
    assert rel(host(dz), ref) < 1e-10
    dr32, dz32 = dev(r, np.float32), empty(o.st.N_dof, "float32")
    s.precond(ptr(dr32), ptr(dz32), P.ST_MIXED)
    # FP32 path: transforms with TF32 inputs on the tensor cores (unit roundoff
    # 2^-11 per rounded input, four transforms) and FP32 time solves
    assert rel(host(dz32), ref) < 1e-2
    s.close()


@pytest.mark.parametrize("c", CASES[:5], ids=IDS[:5])
def test_wupdate(P, c):
    desc = problem(c, b=0.05, d_e=1.3)
    o = Oracle(desc)
    u = W.random_vector(o.st.N_dof, seed=13)
    ref = o.w_update(u)
    s = solver(P, desc)
    du, dw = dev(u), empty(o.st.N_dof)
    s.wupdate(ptr(du), ptr(dw))
    assert rel(host(dw), ref) < 1e-12
    s.close()


SOLVE_CASES = [(c, f, i) for c in CASES[:5] for f, i in (("bands", "auto"), ("lean", "fp32"), ("lean", "df"))
               if f == "bands" or c["d"] >= 2]
SOLVE_IDS = [f"d{c['d']}p{c['p']}-{f}-{i}" for c, f, i in SOLVE_CASES]


@pytest.mark.parametrize("c,form,inner", SOLVE_CASES, ids=SOLVE_IDS)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_linsolve(P, c, form, inner, precision):
    """FP64 solves to 1e-13 against the oracle's direct solve (1e-10); mixed
    solves, with the inner operator in FP32 or in double-float, to an oracle
    residual of 1e-8."""
    desc = problem(c, precision=precision, rtol=1e-13 if precision == "fp64" else 1e-8, gmres_m=60,
                   operator_form=form, inner_op=inner)
    o = Oracle(desc)
    u, w = iterate(o, 2)
    A, _ = o.linearization(u, w)
    ref = spla.spsolve(A.tocsc(), o.F)
    s = solver(P, desc)
    du, dw = dev(u), dev(w)          # keep the device buffers alive during the calls
    s.ionic(ptr(du), ptr(dw))
    f = empty(o.st.N_dof)
    s.rhs(ptr(f))
    x = dev(u)
    st = s.linsolve(ptr(f), ptr(x))
    xs = host(x)
    res = np.linalg.norm(o.F - A @ xs) / np.linalg.norm(o.F)
    if precision == "fp64":
        assert rel(xs, ref) < 1e-10
        assert st["rel_res"] <= 1e-13
    else:
        assert res <= 1e-8
    s.close()


NL_CASES = [(c, f) for c in CASES[:5] for f in ("bands", "lean") if f == "bands" or c["d"] >= 2]


@pytest.mark.parametrize("c,form", NL_CASES, ids=[f"d{c['d']}p{c['p']}-{f}" for c, f in NL_CASES])
@pytest.mark.parametrize("kind", ["picard", "newton"])
def test_nonlinear_iterations(P, c, form, kind):
    """Three nonlinear steps from u = w = 0 on both sides (FP64, tight inner solves)."""
    desc = problem(c, nonlinear=kind, max_fp=3, delta=0.0, rtol=1e-13, gmres_m=80, operator_form=form)
    o = Oracle(desc)
    u_ref, w_ref, _ = o.solve(max_fp=3)
    s = solver(P, desc)
    u, w = empty(o.st.N_dof), empty(o.st.N_dof)
    st = s.solve(ptr(u), ptr(w), allow_unconverged=True)
    assert st["fp_iters"] == 3
    assert rel(host(u), u_ref) < 1e-10
    assert rel(host(w), w_ref) < 1e-10
    s.close()


LR_CASES = [(c, f) for c in (CASES[0], CASES[2], CASES[3], CASES[4]) for f in ("bands", "lean")
            if f == "bands" or c["d"] >= 2]


@pytest.mark.parametrize("c,form", LR_CASES, ids=[f"d{c['d']}p{c['p']}-{f}" for c, f in LR_CASES])
@pytest.mark.parametrize("kind", ["picard", "newton"])
@pytest.mark.parametrize("eps", [1e-2, 1e-4])
def test_lowrank_reaction(P, c, form, kind, eps):
    """The low-rank reaction coefficient (reading A7): its rank and singular
    values, and both operators, against the oracle's (the coefficient's
    Greville values truncated at eps_reaction and interpolated)."""
    from oracle import model
    from oracle.stabilization import greville_values
    desc = problem(c, nonlinear=kind, operator_form=form, eps_reaction=eps)
    o = Oracle(desc)
    u, w = iterate(o, 2)
    A, info = o.linearization(u, w, kind)
    sc = info["sc"]
    R = len(sc)
    # no tie at the cut
    ug, wg = greville_values(o.st, u), greville_values(o.st, w)
    C = model.jacobian_coef(desc, ug, wg) if kind == "newton" else model.reaction_coef(desc, ug, wg)
    sv = np.linalg.svd(C, compute_uv=False)
    fro = np.sqrt(np.sum(sv ** 2))
    tail = np.sqrt(np.concatenate([np.cumsum((sv ** 2)[::-1])[::-1], [0.0]]))
    assert tail[R - 1] > (1 + 1e-6) * eps * fro and tail[R] < (1 - 1e-6) * eps * fro
    s = solver(P, desc)
    du, dw = dev(u), dev(w)
    ginfo = s.ionic(ptr(du), ptr(dw))
    assert ginfo["rank_reaction"] == R
    assert rel(np.array(s.get("reaction_s", R)), sc) < 1e-10
    x = W.random_vector(o.st.N_dof, seed=5)
    dx, dy = dev(x), empty(o.st.N_dof)
    s.apply(ptr(dx), ptr(dy), P.ST_FP64)
    assert rel(host(dy), A @ x) < 1e-12
    dx32, dy32 = dev(x, np.float32), empty(o.st.N_dof, "float32")
    s.apply(ptr(dx32), ptr(dy32), P.ST_MIXED)
    assert rel(host(dy32), A @ x) < 2e-5
    s.close()
