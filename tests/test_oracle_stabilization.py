"""Pins of the oracle's Spline-Upwind ingredients (Sec. 3): tau (Eq. tau), the
residual and Theta-hat (Eq. theta_ce_u, Eq. suppext), the low-rank step (Eq. tol)
and the (d+1)-linear interpolation of theta."""

import numpy as np
import pytest

from oracle import Oracle, SpaceTime
from oracle.bspline import bspline_all, greville
from oracle.stabilization import tau_solve, low_rank, interpolate_at_gauss, theta_hat
import workloads as W


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("n_el_t,clustered", [(2, False), (4, False), (9, False), (9, True), (16, True)])
def test_tau_makes_time_block_lower_triangular(p, n_el_t, clustered):
    breaks_t = W.clustered_breaks(n_el_t, [0.5], p, T=3.0) if clustered else None
    st = SpaceTime(W.base_desc(d=1, p=p, n_el=[2], n_el_t=n_el_t, T=3.0, breaks_t=breaks_t))
    _, tau_q = tau_solve(st)
    m = st.matrices_1d()
    td = st.tdir
    S = 0
    for k in range(1, p + 1):
        Bk = td.vals[k].reshape(-1, td.n)[:, 1:]
        w = td.wq.reshape(-1) * tau_q[k - 1].reshape(-1)
        S = S + (Bk * w[:, None]).T @ Bk
    Mx = m["Wt"] + S
    assert np.abs(np.triu(Mx, 1)).max() <= 1e-12 * np.abs(Mx).max()
    # the diagonal stays positive: C_m d_t u + SU term is invertible by forward substitution
    assert np.all(np.diag(Mx) > 0)


def _fields_linear_in_time(st, beta, kappa):
    """Coefficients of u = beta t x^2 and w = kappa t (d = 1, p >= 2): time by the
    Greville (linear precision) identity, space by interpolation at the Greville points."""
    dr = st.sdirs[0]
    g = greville(dr.knots, dr.p)
    cx2 = np.linalg.solve(bspline_all(dr.knots, dr.p, g), g ** 2)
    ct = st.tdir.greville[1:]
    u = beta * np.kron(ct, cx2)
    w = kappa * np.kron(ct, np.ones(st.N_s))
    return u, w


@pytest.mark.parametrize("p", [2, 3])
def test_residual_closed_form(p):
    desc = W.base_desc(d=1, p=p, n_el=[5], n_el_t=4, T=2.0, C_m=1.3, D=[0.07],
                       source=dict(kind="stim", boxes=[W.stim_box([0.2], [0.6], 0.5, 1.5, 0.8)]))
    o = Oracle(desc)
    beta, kappa = 0.9, -0.4
    u, w = _fields_linear_in_time(o.st, beta, kappa)
    fl = o.fields(u, w)
    R = o.residual_q(fl)
    t = o.st.time_points()[:, None, :, None]
    x = o.st.xs[0][None, :, None, :]
    uu = beta * t * x ** 2
    ww = kappa * t
    f = 0.8 * ((x >= 0.2) & (x <= 0.6)) * ((t >= 0.5) & (t < 1.5))
    Rex = (1.3 * beta * x ** 2 - 0.07 * 2 * beta * t
           + desc["c1"] * uu * (uu - desc["a"]) * (uu - 1) + desc["c2"] * uu * ww - f)
    assert np.abs(R - Rex).max() < 1e-12
    assert np.abs(fl["u"] - uu).max() < 1e-13


@pytest.mark.parametrize("mode", ["literal", "symmetric"])
def test_theta_hat_windows_by_coordinates(mode):
    """Recompute every numerator from the knot coordinates of Eq. (suppext)."""
    p = 2
    desc = W.base_desc(d=2, p=p, n_el=[4, 3], n_el_t=5, T=2.0, suppext=mode)
    st = SpaceTime(desc)
    rng = np.random.Generator(np.random.PCG64(7))
    R = rng.standard_normal((st.n_el_t, st.N_el_s, st.nq_t, st.nq_s))
    u = rng.standard_normal(R.shape)
    ut = rng.standard_normal(R.shape)
    th, info = theta_hat(st, R, u, ut, 1.0, mode)
    den = np.abs(u).max() / st.T + np.abs(ut).max()
    emax = np.abs(R).max(axis=(2, 3)).reshape(st.n_el_t, 3, 4)

    def interval(knots, i1):   # 1-based basis index -> open interval of Eq. (suppext)
        lo = knots[max(i1 - p, 1) - 1]
        hi_idx = i1 + p + 1 if mode == "literal" else i1 + 2 * p + 1
        hi = knots[min(hi_idx, len(knots)) - 1]
        return lo, hi

    def spans_in(dr, lo, hi):
        mids = 0.5 * (dr.br[:-1] + dr.br[1:])
        return np.nonzero((mids > lo) & (mids < hi))[0]

    kt = st.tdir.knots            # parametric knots of the time direction
    for it in range(st.N_t):
        et = spans_in(type("D", (), {"br": st.tdir.br})(), *interval(kt, it + 2))
        for iy in range(st.n[1]):
            ey = spans_in(st.sdirs[1], *interval(st.sdirs[1].knots, iy + 1))
            for ix in range(st.n[0]):
                ex = spans_in(st.sdirs[0], *interval(st.sdirs[0].knots, ix + 1))
                num = emax[np.ix_(et, ey, ex)].max()
                assert th[it, ix + st.n[0] * iy] == pytest.approx(min(num / den, 1.0), rel=1e-15)


def test_theta_hat_zero_denominator_rule():
    st = SpaceTime(W.base_desc(d=1, p=2, n_el=[8], n_el_t=8, T=1.0))
    z = np.zeros((st.n_el_t, st.N_el_s, st.nq_t, st.nq_s))
    th, _ = theta_hat(st, z, z, z, 1.0)
    assert np.all(th == 0.0)
    R = z.copy()
    R[0, 0, 0, 0] = 1e-3
    th, _ = theta_hat(st, R, z, z, 1.0)
    assert th.max() == 1.0 and th.min() == 0.0


def test_low_rank_tolerance_and_minimality():
    rng = np.random.Generator(np.random.PCG64(3))
    A = rng.uniform(0, 1, (12, 4)) @ rng.uniform(0, 1, (4, 30)) + 0.05 * rng.uniform(0, 1, (12, 30))
    fro = np.linalg.norm(A)
    for eps in (0.3, 0.1, 0.03, 0.01, 1e-3):
        U, s, V = low_rank(A, eps)
        R = len(s)
        assert np.linalg.norm(A - (U * s) @ V.T) <= eps * fro * (1 + 1e-12)
        if R > 1:
            U1, s1, V1 = U[:, :R - 1], s[:R - 1], V[:, :R - 1]
            assert np.linalg.norm(A - (U1 * s1) @ V1.T) > eps * fro
        assert np.allclose(U.T @ U, np.eye(R), atol=1e-12)
        assert np.allclose(V.T @ V, np.eye(R), atol=1e-12)
    U, s, V = low_rank(A, 0.0)
    assert np.abs((U * s) @ V.T - A).max() < 1e-13
    U, s, V = low_rank(np.zeros((5, 7)), 0.1)
    assert len(s) == 0


@pytest.mark.parametrize("d", [1, 2, 3])
def test_interpolation_reproduces_affine_and_nodal_values(d):
    desc = W.base_desc(d=d, p=2, n_el=[3, 2, 2][:d], n_el_t=4, T=3.0)
    st = SpaceTime(desc)
    gt = st.tdir.greville[1:]
    gs = [dr.greville for dr in st.sdirs]
    coef = [0.3, -1.2, 0.7]
    # f(x, t) = 0.5 + 0.25 t + sum_l coef_l x_l (affine, reproduced by (d+1)-linear interp)
    grid = np.meshgrid(gt, *[gs[l] for l in range(d - 1, -1, -1)], indexing="ij")
    tab = 0.5 + 0.25 * grid[0]
    for l in range(d):
        tab = tab + coef[l] * grid[d - l]
    out = interpolate_at_gauss(st, tab.reshape(st.N_t, st.N_s))
    t = st.time_points()[:, None, :, None]
    ex = 0.5 + 0.25 * np.maximum(t, gt[0])  # constant continuation before the first node
    for l in range(d):
        ex = ex + coef[l] * st.xs[l][None, :, None, :]
    assert np.abs(out - ex).max() < 1e-13
