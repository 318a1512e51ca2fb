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
