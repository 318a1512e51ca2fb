"""Pins of the oracle's solver (Sec. 3.1 fixed point, Eq. lin_sys_L, Sec. 4.1)
against closed forms, the exact w elimination, the rest state and the ODE
limit of a spatially uniform stimulus."""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import Oracle
import workloads as W


def test_w_elimination_matches_kronecker_formula():
    """w = vec(M_s^-1 G (W_t + b d_e M_t)^-T) with g = vec(G) (Sec. 3.2)."""
    desc = W.base_desc(d=2, p=2, n_el=[3, 4], n_el_t=5, T=3.0, b=0.05, d_e=1.3)
    o = Oracle(desc)
    u = W.random_vector(o.st.N_dof, seed=11)
    w1 = o.w_update(u)
    m = o.st.matrices_1d()
    Ms = np.kron(m["M1"], m["M0"])
    At = m["Wt"] + desc["b"] * desc["d_e"] * m["Mt"]
    g = o.w_rhs(u)
    G = g.reshape(o.st.N_t, o.st.N_s).T                  # columns = time index
    X = np.linalg.solve(Ms, G) @ np.linalg.inv(At).T
    w2 = X.T.reshape(-1)
    assert np.abs(w1 - w2).max() < 1e-12 * np.abs(w2).max()
    # g = b (M_t x M_s) u exactly, since u lies in the discrete space
    assert np.abs(g - desc["b"] * np.kron(m["Mt"], Ms) @ u).max() < 1e-14


@pytest.mark.parametrize("kind", ["picard", "newton"])
@pytest.mark.parametrize("stab", ["galerkin", "su"])
def test_rest_state(kind, stab):
    desc = W.base_desc(d=2, p=2, n_el=[3, 3], n_el_t=4, T=5.0, nonlinear=kind, stabilization=stab)
    o = Oracle(desc)
    u, w, hist = o.solve()
    assert np.all(u == 0.0) and np.all(w == 0.0)
    info = o.ionic(u, w)
    assert np.all(info["theta_hat"] == 0.0) and np.all(info["R"] == 0.0)
    assert len(hist) == 1 and hist[0]["rank"] == 0


def _rk4_rm(desc, f_amp, times, dt=1e-3):
    """Pointwise Rogers-McCulloch dynamics C_m u' = f - c1 u(u-a)(u-1) - c2 u w,
    w' = b (u - d_e w), u(0) = w(0) = 0, by classical RK4."""
    a, b, c1, c2, de, Cm = (desc[k] for k in ("a", "b", "c1", "c2", "d_e", "C_m"))

    def rhs(y):
        u, w = y
        return np.array([(f_amp - c1 * u * (u - a) * (u - 1) - c2 * u * w) / Cm, b * (u - de * w)])

    out = []
    y = np.zeros(2)
    t = 0.0
    for tt in np.sort(times):
        while t < tt - 1e-15:
            h = min(dt, tt - t)
            k1 = rhs(y); k2 = rhs(y + 0.5 * h * k1); k3 = rhs(y + 0.5 * h * k2); k4 = rhs(y + h * k3)
            y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
            t += h
        out.append(y[0])
    return np.array(out)


@pytest.mark.parametrize("p", [2, 3])
def test_uniform_stimulus_reduces_to_rm_ode(p):
    """f constant in space: the solution is constant in space (partition of
    unity), and the space-time Galerkin solution converges to the RM ODE."""
    T, amp = 20.0, 0.3
    errs = []
    for n_el_t in (8, 16, 32):
        desc = W.base_desc(d=1, p=p, n_el=[3], n_el_t=n_el_t, T=T, D=[1e-3], stabilization="galerkin",
                           delta=1e-12, max_fp=400,
                           source=dict(kind="stim", boxes=[W.stim_box([0.0], [1.0], 0.0, 2 * T, amp)]))
        o = Oracle(desc)
        u, w, hist = o.solve()
        assert hist[-1]["diff"] <= 1e-12
        U = u.reshape(o.st.N_t, o.st.N_s)
        assert np.abs(U - U[:, :1]).max() < 1e-10
        uq = o.st.field(u)[:, 0, :, 0]                      # (n_el_t, nq_t) at x-element 0, point 0
        tq = o.st.time_points()
        ref = _rk4_rm(desc, amp, tq.reshape(-1)).reshape(tq.shape)
        errs.append(np.sqrt(np.sum(o.st.tdir.wq * (uq - ref) ** 2)))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    assert errs[-1] < 1e-3
    assert rates[-1] > p + 0.5


@pytest.mark.slow
@pytest.mark.parametrize("p", [2, 3])
def test_heat_mms_convergence_rate(p):
    """Linear heat equation (c1 = c2 = 0), Galerkin: L2 error decays like h^(p+1)."""
    errs = []
    for ne in (4, 8, 16):
        desc = W.config("heat_mms_2d")
        desc.update(p=p, n_el=[ne, ne], n_el_t=ne)
        o = Oracle(desc)
        A, _ = o.linearization(np.zeros(o.st.N_dof), np.zeros(o.st.N_dof))
        u = spla.spsolve(A.tocsc(), o.F)
        e, n = o.l2_error(u)
        errs.append(e / n)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > p + 1 - 0.15


@pytest.mark.slow
@pytest.mark.parametrize("p", [2, 3])
def test_e1_su_optimal_order(p):
    """Smooth 1D test of Sec. 4.1 with SU: optimal order p+1 in L2."""
    errs = []
    for ne in (8, 16, 32):
        desc = W.config("e1_mms_1d")
        desc.update(p=p, n_el=[ne], n_el_t=ne, delta=1e-12, max_fp=300)
        o = Oracle(desc)
        u, _, hist = o.solve()
        assert hist[-1]["diff"] <= 1e-12
        e, n = o.l2_error(u)
        errs.append(e / n)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > p + 1 - 0.35
    assert errs[-1] < (2e-4 if p == 2 else 5e-6)


def test_newton_and_picard_reach_the_same_solution():
    """Both iterations have the same fixed point (Galerkin, no theta)."""
    base = W.base_desc(d=1, p=2, n_el=[6], n_el_t=8, T=6.0, D=[1e-2], stabilization="galerkin",
                       delta=1e-12, max_fp=500,
                       source=dict(kind="stim", boxes=[W.stim_box([0.0], [0.3], 0.0, 1.0, 0.5)]))
    sols = []
    for kind in ("picard", "newton"):
        desc = dict(base, nonlinear=kind)
        u, w, hist = Oracle(desc).solve()
        assert hist[-1]["diff"] <= 1e-12
        sols.append((u, w))
    assert np.abs(sols[0][0] - sols[1][0]).max() < 1e-9
    assert np.abs(sols[0][1] - sols[1][1]).max() < 1e-9


def test_newton_residual_vanishes_at_solution():
    """At a converged Newton iterate, f - A_lin u - S u - int I_ion(u, w) v = 0."""
    desc = W.base_desc(d=1, p=2, n_el=[5], n_el_t=6, T=4.0, D=[1e-2], stabilization="galerkin",
                       nonlinear="newton", delta=1e-13, max_fp=100,
                       source=dict(kind="stim", boxes=[W.stim_box([0.0], [0.4], 0.0, 1.0, 0.7)]))
    o = Oracle(desc)
    u, w, hist = o.solve()
    w_fix = o.w_update(u)
    r = o.F - o.operator(o.st.const(0.0)) @ u - o.ionic_load(u, w_fix)
    assert np.abs(r).max() < 1e-10 * np.abs(o.F).max()


def test_jacobian_coef_is_the_u_derivative_of_the_ionic_current():
    """C_J (the Newton coefficient of the u-equation) is d/du of
    I_ion(u, w) = c1 u (u - a)(u - 1) + c2 u w of eq. 3.1.  Checked three
    ways that do not retype the formula: a centred difference of I_ion at
    random (u, w); the slopes of the cubic at its three roots 0, a and 1,
    which are the products of the differences to the other two roots; and
    the w-dependence, d/dw of C_J = c2 = d/dw of I_ion / u."""
    from oracle import model
    desc = W.base_desc()
    desc.update(W.DIMENSIONAL_RM)
    a, c1, c2 = desc["a"], desc["c1"], desc["c2"]
    rng = np.random.Generator(np.random.PCG64(3))
    u = rng.uniform(-0.5, 1.5, 200)
    w = rng.uniform(-0.2, 1.0, 200)
    h = 1e-5
    fd = (model.ionic_current(desc, u + h, w) - model.ionic_current(desc, u - h, w)) / (2 * h)
    cj = model.jacobian_coef(desc, u, w)
    # the centred difference of a cubic is exact up to c1 h^2 and rounding
    assert np.abs(cj - fd).max() <= c1 * h * h + 1e-8 * np.abs(cj).max()
    for root, slope in ((0.0, (0.0 - a) * (0.0 - 1.0)), (a, (a - 0.0) * (a - 1.0)), (1.0, (1.0 - 0.0) * (1.0 - a))):
        wz = np.zeros(1)
        assert abs(model.jacobian_coef(desc, np.array([root]), wz)[0] - c1 * slope) <= 1e-13 * c1
        assert abs(model.ionic_current(desc, np.array([root]), wz)[0]) <= 1e-15 * c1
    dw = (model.jacobian_coef(desc, u, w + 0.25) - model.jacobian_coef(desc, u, w)) / 0.25
    assert np.abs(dw - c2).max() <= 1e-12 * c2
    # C_J = C_r + u dC_r/du: the Picard coefficient is I_ion / u
    nz = np.abs(u) > 1e-3
    assert np.abs(model.reaction_coef(desc, u, w)[nz] * u[nz] - model.ionic_current(desc, u, w)[nz]).max() < 1e-12


def _newton_errors(monkeypatch=None, coef=None):
    """Distances max|u_k - u*| of the oracle's Newton iterates to its converged
    solution, on a 1D Galerkin problem with w held at zero (so the u-equation
    is the whole system and Newton on it is exact Newton)."""
    from oracle import model
    desc = W.base_desc(d=1, p=2, n_el=[6], n_el_t=8, T=6.0, D=[1e-2], stabilization="galerkin",
                       nonlinear="newton", fix_w_zero=True, delta=0.0,
                       source=dict(kind="stim", boxes=[W.stim_box([0.0], [0.4], 0.0, 1.0, 0.6)]))
    if coef is not None:
        monkeypatch.setattr(model, "jacobian_coef", coef)
    _, _, hist = Oracle(desc).solve(max_fp=12, record=True)
    us = [np.zeros_like(hist[0]["u"])] + [h["u"] for h in hist]
    ref = us[-1]
    return np.array([np.abs(x - ref).max() for x in us[:-1]])


def test_newton_converges_quadratically(monkeypatch):
    """With the true derivative the error squares each step once it is small:
    e_{k+1} <= K e_k^2 with one K over the last steps before round-off, and
    the contraction e_{k+1}/e_k falls towards zero.  A coefficient with a
    term dropped (the c1 a part of C_J, a plausible slip) still converges to
    the same solution, but only linearly: the same test rejects it."""
    e = _newton_errors()
    live = [k for k in range(len(e) - 1) if e[k + 1] > 1e-12 and e[k] < 1e-1]
    assert len(live) >= 2, e
    ratio2 = [e[k + 1] / e[k] ** 2 for k in live]
    assert max(ratio2) < 50.0, e
    assert e[live[-1] + 1] / e[live[-1]] < 1e-2, e

    from oracle import model
    true = model.jacobian_coef

    def dropped(desc, u, w):
        return true(desc, u, w) - desc["c1"] * desc["a"]

    bad = _newton_errors(monkeypatch, dropped)
    live_b = [k for k in range(len(bad) - 1) if bad[k + 1] > 1e-12 and bad[k] < 1e-1]
    assert live_b, bad
    assert max(bad[k + 1] / bad[k] ** 2 for k in live_b) > 50.0 or \
        bad[live_b[-1] + 1] / bad[live_b[-1]] >= 1e-2, bad
