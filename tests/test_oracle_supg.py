"""Pins of the oracle's comparison method of Sec. 4.2: C^0-in-time splines with
SUPG and shock capturing (oracle/supg.py)."""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import Oracle
from oracle import supg
from oracle.bspline import bspline_all
from oracle.spacetime import c0_time_knots


@pytest.mark.parametrize("p,n_el", [(1, 4), (2, 5), (3, 4), (4, 3)])
def test_c0_time_basis(p, n_el):
    """Every interior breakpoint repeated p times: p n_el + 1 functions (p n_el
    once the first is removed), a partition of unity whose derivatives sum to
    zero, and at each interior breakpoint exactly one function equal to 1 (the
    basis interpolates there, which is what C^0 means)."""
    kn = c0_time_knots(n_el, p)
    n = len(kn) - p - 1
    assert n - 1 == p * n_el
    rng = np.random.Generator(np.random.PCG64(1))
    x = rng.uniform(0.0, 1.0, 50)
    assert np.abs(bspline_all(kn, p, x).sum(axis=1) - 1.0).max() < 1e-14
    assert np.abs(bspline_all(kn, p, x, 1).sum(axis=1)).max() < 1e-11
    br = np.linspace(0.0, 1.0, n_el + 1)[1:-1]
    v = bspline_all(kn, p, br)
    for row in v:
        assert np.sum(np.abs(row - 1.0) < 1e-14) == 1
        assert np.sum(np.abs(row) > 1e-14) == 1


def _q(x):
    """3x^2 - 2x^3: zero slope at both ends of [0, 1] (Neumann), cubic."""
    return 3 * x * x - 2 * x ** 3, 6 - 12 * x


def discrete_problem(d, p=3):
    """Linear heat problem (c1 = c2 = 0) on C^0 time splines with SUPG + shock
    capturing, whose exact solution u = t^2 prod_l q(x_l) lies in the discrete
    space (degree 3 in space, 2 in time), with the load at the Gauss points from
    that solution."""
    desc = W.base_desc(d=d, p=p, n_el=[4, 3][:d], n_el_t=3, T=2.0, D=[3e-2, 1e-2][:d], C_m=1.3,
                       time_continuity="c0", stabilization="supg_sc", c1=0.0, c2=0.0)
    o = Oracle(desc)
    st = o.st
    t = st.time_points()[:, None, :, None]
    xs = [x[None, :, None, :] for x in st.xs]
    qs = [_q(x) for x in xs]
    prod = np.ones_like(xs[0])
    for qv, _ in qs:
        prod = prod * qv
    ue = t * t * prod
    f = desc["C_m"] * 2 * t * prod
    for l in range(d):
        other = np.ones_like(xs[0])
        for m in range(d):
            if m != l:
                other = other * qs[m][0]
        f = f - desc["D"][l] * t * t * qs[l][1] * other
    shape = (st.n_el_t, st.N_el_s, st.nq_t, st.nq_s)
    o.f_q = f * np.ones(shape)
    o.F = st.load(o.f_q) + supg.supg_load(st, o.f_q)
    # coefficients of the exact solution: its L2 projection (exact, since it
    # lies in the space)
    M = st.assemble(st.mass_terms(st.const(1.0)))
    c = spla.spsolve(M.tocsc(), st.load(ue * np.ones(shape)))
    return o, c


@pytest.mark.parametrize("d", [1, 2])
def test_discrete_space_solution_is_reproduced(d):
    """SUPG is residual-based and the shock-capturing coefficient is |R| / den:
    for a solution in the discrete space the residual vanishes at every Gauss
    point, so the stabilized system, linearized at that solution, returns it."""
    o, c = discrete_problem(d)
    A, info = o.linearization(c, np.zeros_like(c))
    assert np.abs(info["R"]).max() < 1e-10 * np.abs(o.f_q).max()
    x = spla.spsolve(A.tocsc(), o.F)
    assert np.abs(x - c).max() < 1e-10 * np.abs(c).max()


def test_a_dropped_supg_load_or_a_flipped_laplacian_is_caught(monkeypatch):
    """The reproduction pin fails when the f part of SUPG is left off the
    right-hand side, or when the diffusion term of SUPG has the wrong sign."""
    o, c = discrete_problem(1)
    st = o.st
    F_plain = st.load(o.f_q)
    A, _ = o.linearization(c, np.zeros_like(c))
    x = spla.spsolve(A.tocsc(), F_plain)
    assert np.abs(x - c).max() > 1e-6 * np.abs(c).max()

    orig = supg.supg_terms

    def flipped(st_, C_m, D, cr_q):
        return orig(st_, C_m, [-v for v in D], cr_q)

    monkeypatch.setattr(supg, "supg_terms", flipped)
    A, _ = o.linearization(c, np.zeros_like(c))
    x = spla.spsolve(A.tocsc(), o.F)
    assert np.abs(x - c).max() > 1e-6 * np.abs(c).max()


def test_heat_mms_converges_at_the_optimal_rate():
    """Linear heat, u = cos(pi x) sin t (reading A13), on C^0 time splines with
    SUPG + shock capturing, iterated to its fixed point: the L2 error falls at
    about p + 1 per halving of the mesh."""
    p = 2
    errs = []
    for ne in (4, 8, 16):
        desc = W.base_desc(d=1, p=p, n_el=[ne], n_el_t=ne, T=1.0, D=[1.0], C_m=1.0, c1=0.0, c2=0.0,
                           time_continuity="c0", stabilization="supg_sc", source=dict(kind="heat_mms"),
                           alpha=1.0, delta=1e-13, max_fp=30)
        o = Oracle(desc)
        u, w, hist = o.solve()
        assert hist[-1]["diff"] <= 1e-12
        err, nrm = o.l2_error(u)
        errs.append(err / nrm)
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert rates[-1] > p + 0.5, (errs, rates)
