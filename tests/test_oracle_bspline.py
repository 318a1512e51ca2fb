"""Pins of the oracle's univariate spline layer (Sec. 2) against textbook facts."""

import os
from fractions import Fraction

import numpy as np
import pytest

from oracle.bspline import bspline_all, open_uniform_knots, greville, Direction
from oracle.spacetime import SpaceTime
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("n_el", [1, 3, 7])
def test_partition_of_unity_and_linear_precision(p, n_el):
    kn = open_uniform_knots(n_el, p)
    x = np.linspace(0.0, 1.0, 57)
    B = bspline_all(kn, p, x)
    assert B.shape == (len(x), n_el + p)
    assert np.abs(B.sum(axis=1) - 1.0).max() < 1e-14
    assert B.min() >= 0.0
    # sum_i gamma_i b_i(x) = x
    assert np.abs(B @ greville(kn, p) - x).max() < 1e-14
    for k in range(1, p + 1):
        Bk = bspline_all(kn, p, x, k)
        assert np.abs(Bk.sum(axis=1)).max() < 1e-10
    # derivative of the linear reproduction is 1
    B1 = bspline_all(kn, p, x, 1)
    assert np.abs(B1 @ greville(kn, p) - 1.0).max() < 1e-12


@pytest.mark.parametrize("p", [2, 3])
def test_derivative_against_finite_difference(p):
    kn = open_uniform_knots(5, p)
    x = np.array([0.13, 0.41, 0.77, 0.93])
    eps = 1e-6
    for k in range(1, p + 1):
        lo = bspline_all(kn, p, x - eps, k - 1)
        hi = bspline_all(kn, p, x + eps, k - 1)
        fd = (hi - lo) / (2 * eps)
        assert np.abs(fd - bspline_all(kn, p, x, k)).max() < 1e-5 * max(1.0, np.abs(fd).max())


@pytest.mark.parametrize("p", [2, 3])
def test_greville_values(p):
    kn = open_uniform_knots(4, p)
    g = greville(kn, p)
    assert g[0] == 0.0 and g[-1] == 1.0
    assert np.all(np.diff(g) > 0)
    if p == 2:
        assert np.allclose(g, [0.0, 0.125, 0.375, 0.625, 0.875, 1.0])


def _golden_rows():
    rows = {}
    with open(os.path.join(GOLDEN, "cardinal_rows.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            p, kind, scale = int(parts[0]), parts[1], parts[2]
            rows[(p, kind)] = (scale, np.array([float(Fraction(s)) for s in parts[3:]]))
    return rows


@pytest.mark.parametrize("p", [2, 3])
def test_interior_rows_match_cardinal_closed_form(p):
    n_el = 12
    h = 1.0 / n_el
    dr = Direction(n_el, p)
    B0 = dr.vals[0].reshape(-1, dr.n)
    B1 = dr.vals[1].reshape(-1, dr.n)
    w = dr.wq.reshape(-1)
    M = (B0 * w[:, None]).T @ B0
    K = (B1 * w[:, None]).T @ B1
    rows = _golden_rows()
    for i in range(2 * p, n_el - p):
        sl = slice(i - p, i + p + 1)
        assert np.allclose(M[i, sl], h * rows[(p, "mass")][1], rtol=0, atol=1e-15)
        assert np.allclose(K[i, sl], rows[(p, "stiff")][1] / h, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("p", [2, 3])
def test_mass_row_sums_and_stiffness_kernel(p):
    st = SpaceTime(W.base_desc(d=1, p=p, n_el=[6], n_el_t=5, T=2.5))
    m = st.matrices_1d()
    kn = st.sdirs[0].knots
    n = st.n[0]
    expect = np.array([(kn[i + p + 1] - kn[i]) / (p + 1) for i in range(n)])
    assert np.abs(m["M0"].sum(axis=1) - expect).max() < 1e-15
    assert np.abs(m["K0"] @ np.ones(n)).max() < 1e-12
    # time mass in physical units: T * parametric row sums (first function removed)
    ktt = st.tdir.knots
    full = np.array([(ktt[i + p + 1] - ktt[i]) / (p + 1) for i in range(st.n_t)]) * st.T
    # row sums over X_t miss the column of b_1
    B0 = st.tdir.vals[0].reshape(-1, st.n_t)
    wq = st.tdir.wq.reshape(-1)
    col_b1 = (B0[:, 1:] * wq[:, None]).T @ B0[:, 0]
    assert np.abs(m["Mt"].sum(axis=1) + col_b1 - full[1:]).max() < 1e-14


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_non_uniform_knots_partition_of_unity_and_linear_precision(p):
    """The same identities on clustered breakpoints (the non-uniform meshes the
    boundary accepts), and mass rows summing to the support lengths / (p+1)."""
    from oracle.spacetime import open_knots
    br = W.clustered_breaks(11, [0.3, 0.7], p)
    kn = open_knots(br, p)
    x = np.linspace(0.0, 1.0, 101)
    B = bspline_all(kn, p, x)
    assert np.abs(B.sum(axis=1) - 1.0).max() < 1e-13
    assert np.abs(B @ greville(kn, p) - x).max() < 1e-13
    d = Direction(11, p, knots=kn)
    M = (d.vals[0].reshape(-1, d.n) * d.wq.reshape(-1)[:, None]).T @ d.vals[0].reshape(-1, d.n)
    supp = np.array([kn[i + p + 1] - kn[i] for i in range(d.n)])
    assert np.abs(M.sum(axis=1) - supp / (p + 1)).max() < 1e-14
