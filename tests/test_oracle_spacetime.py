"""Pins of the oracle's space-time assembly against the Kronecker identities of
Sec. 3.1 (the discrete system) and Sec. 3.2 (the preconditioner), and the
W_t + W_t^T identity that follows from removing b_1 (Sec. 2)."""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import Oracle, SpaceTime
from oracle.stabilization import tau_solve
import workloads as W


def kron_list(mats):
    out = sp.csr_matrix(mats[0])
    for m in mats[1:]:
        out = sp.kron(out, sp.csr_matrix(m), format="csr")
    return out


def spatial(m, d, which):
    """Spatial Kronecker product M_d x ... x M_1 with `which` replacing direction l."""
    mats = []
    for l in range(d - 1, -1, -1):
        mats.append(m[which.get(l, f"M{l}")] if isinstance(which, dict) else m[f"M{l}"])
    return kron_list(mats)


CASES = [(1, 2, [5], 4), (1, 3, [4], 5), (2, 2, [3, 4], 4), (2, 3, [3, 2], 3), (3, 2, [2, 3, 2], 3)]


@pytest.mark.parametrize("d,p,n_el,n_el_t", CASES)
def test_linear_part_is_kronecker(d, p, n_el, n_el_t):
    desc = W.base_desc(d=d, p=p, n_el=n_el, n_el_t=n_el_t, T=3.0, C_m=1.7,
                       D=[1e-3, 2.5e-4, 7e-4][:d])
    st = SpaceTime(desc)
    m = st.matrices_1d()
    Ms = spatial(m, d, {})
    Ks = sum(desc["D"][l] * spatial(m, d, {l: f"K{l}"}) for l in range(d))
    kron = desc["C_m"] * sp.kron(m["Wt"], Ms) + sp.kron(m["Mt"], Ks)
    A = st.assemble(st.linear_terms(desc["C_m"], desc["D"]))
    assert abs(A - kron).max() <= 1e-14 * abs(kron).max()
    # constant reaction coefficient: c (M_t x M_s)
    R = st.assemble(st.mass_terms(st.const(0.37)))
    assert abs(R - 0.37 * sp.kron(m["Mt"], Ms)).max() < 1e-15


@pytest.mark.parametrize("d,p,n_el,n_el_t", CASES)
def test_preconditioner_is_kronecker(d, p, n_el, n_el_t):
    desc = W.base_desc(d=d, p=p, n_el=n_el, n_el_t=n_el_t, T=2.0, C_m=1.3,
                       D=[2e-3, 5e-4, 1e-3][:d])
    o = Oracle(desc)
    m = o.st.matrices_1d()
    for unit in (False, True):
        Dp = [1.0] * d if unit else desc["D"]
        Ms = spatial(m, d, {})
        Ks = sum(Dp[l] * spatial(m, d, {l: f"K{l}"}) for l in range(d))
        kron = desc["C_m"] * sp.kron(m["Wt"], Ms) + sp.kron(m["Mt"], Ks + desc["a"] * desc["c1"] * Ms)
        Ah = o.precond_matrix(unit_D=unit)
        assert abs(Ah - kron).max() <= 1e-14 * abs(kron).max()


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("n_el_t", [1, 2, 6])
def test_wt_plus_transpose(p, n_el_t):
    st = SpaceTime(W.base_desc(d=1, p=p, n_el=[2], n_el_t=n_el_t, T=4.0))
    Wt = st.matrices_1d()["Wt"]
    N = Wt.shape[0]
    E = np.zeros((N, N))
    E[-1, -1] = 1.0
    assert np.abs(Wt + Wt.T - E).max() < 1e-13


@pytest.mark.parametrize("d,p", [(1, 2), (2, 3)])
def test_su_term_with_unit_theta_is_kronecker(d, p):
    desc = W.base_desc(d=d, p=p, n_el=[3] * d, n_el_t=5, T=2.0, C_m=1.1)
    st = SpaceTime(desc)
    _, tau_q = tau_solve(st)
    m = st.matrices_1d()
    td = st.tdir
    S = 0
    for k in range(1, p + 1):
        Bk = td.vals[k].reshape(-1, td.n)[:, 1:]
        w = td.wq.reshape(-1) * tau_q[k - 1].reshape(-1)
        S = S + (Bk * w[:, None]).T @ Bk
    Ms = spatial(m, d, {})
    kron = desc["C_m"] * sp.kron(S, Ms)
    A = st.assemble(st.su_terms(desc["C_m"], tau_q, st.const(1.0)))
    assert abs(A - kron).max() <= 1e-13 * abs(kron).max()


def test_load_vector_of_separable_box():
    """f = chi_box(x) chi_[t0,t1)(t) tested against B_i is the product of 1D loads."""
    desc = W.base_desc(d=2, p=2, n_el=[4, 5], n_el_t=4, T=2.0,
                       source=dict(kind="stim", boxes=[W.stim_box([0.1, 0.3], [0.55, 0.8], 0.2, 1.3, 2.0)]))
    o = Oracle(desc)
    st = o.st
    loads = []
    for l, dr in enumerate(st.sdirs):
        x = dr.xq
        ind = ((x >= [0.1, 0.3][l]) & (x <= [0.55, 0.8][l])).astype(float)
        loads.append(np.einsum('eq,eqi->i', dr.wq * ind, dr.vals[0]))
    t = st.tdir.xq
    indt = ((t >= 0.2) & (t < 1.3)).astype(float)
    lt = np.einsum('eq,eqi->i', st.tdir.wq * indt, st.tdir.vals[0])[1:]
    expect = 2.0 * np.kron(lt, np.kron(loads[1], loads[0]))
    assert np.abs(o.F - expect).max() < 1e-15
